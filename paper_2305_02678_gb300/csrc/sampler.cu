// Importance sampling with the neural proxy density (Sec. 4.3, Appendix A).
//
// One query per thread: latent fetch as for the BRDF, the sampler MLP
// 11 -> 32 -> 32 -> 32 -> 9 (ReLU hidden layers, FP32 weights staged in shared
// memory), the output activations, then either the mixture density of the
// query's wo or one sample of wo with its density.  Sampler weights are laid
// out per layer as W (out x in) then b (out).
#include <cuda_runtime.h>

#include "common.cuh"

namespace nam {

namespace {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kAlphaMin = 1e-3f;
constexpr float kRhoMax = 0.99f;

__device__ __forceinline__ float qtanh(float x) {
  const float a = fabsf(x);
  return a >= 2.0f ? copysignf(1.0f, x) : x * (1.0f - 0.25f * a);
}
__device__ __forceinline__ float qsinh(float x) { return x * (1.0f + 0.5f * fabsf(x)); }

struct Proxy {
  float wd, mdx, mdy, ws, ax, ay, rho, msx, msy;
};

__device__ __forceinline__ Proxy activate(const float o[9]) {
  Proxy p;
  const float mx = fmaxf(o[0], o[3]);
  const float ed = expf(o[0] - mx), es = expf(o[3] - mx);
  const float inv = 1.0f / (ed + es);
  p.wd = ed * inv;
  p.ws = es * inv;
  p.mdx = qsinh(o[1]);
  p.mdy = qsinh(o[2]);
  p.ax = kAlphaMin + (1.0f - kAlphaMin) * 0.5f * (qtanh(o[4]) + 1.0f);
  p.ay = kAlphaMin + (1.0f - kAlphaMin) * 0.5f * (qtanh(o[5]) + 1.0f);
  p.rho = kRhoMax * qtanh(o[6]);
  p.msx = qsinh(o[7]);
  p.msy = qsinh(o[8]);
  return p;
}

// Half-vector density of the specular lobe: D_std(v / |v|) det(M^-1) / |v|^3,
// v = M^-1 h, D_std(w) = max(0, w_z) / pi.
__device__ __forceinline__ float pdf_half(const Proxy& p, float hx, float hy, float hz) {
  const float s = sqrtf(1.0f - p.rho * p.rho);
  const float vx = (hx + p.msx * hz) / p.ax;
  const float vy = (hy + p.msy * hz - p.ay * p.rho * vx) / (p.ay * s);
  const float vz = hz;
  const float vl2 = vx * vx + vy * vy + vz * vz;
  if (!(vz > 0.0f)) return 0.0f;
  // D_std(v/|v|) / |v|^3 = (vz / |v|) / pi / |v|^3 = vz / (pi |v|^4)
  return vz / (kPi * vl2 * vl2 * p.ax * p.ay * s);
}

__device__ __forceinline__ float pdf_full(const Proxy& p, const float wi[3], const float wo[3]) {
  const float ndx = -p.mdx, ndy = -p.mdy;
  const float ndl = rsqrtf(ndx * ndx + ndy * ndy + 1.0f);
  const float c = (wo[0] * ndx + wo[1] * ndy + wo[2]) * ndl;
  const float pd = c > 0.0f ? c / kPi : 0.0f;
  float hx = wi[0] + wo[0], hy = wi[1] + wo[1], hz = wi[2] + wo[2];
  const float hl2 = hx * hx + hy * hy + hz * hz;
  float ps = 0.0f;
  if (hl2 > 0.0f) {
    const float ih = rsqrtf(hl2);
    hx *= ih; hy *= ih; hz *= ih;
    const float oh = fabsf(wo[0] * hx + wo[1] * hy + wo[2] * hz);
    if (oh > 0.0f) ps = pdf_half(p, hx, hy, hz) / (4.0f * oh);
  }
  return p.wd * pd + p.ws * ps;
}

__device__ __forceinline__ void sample_dir(const Proxy& p, const float wi[3], float u0, float u1, float u2,
                                           float wo[3]) {
  const float r = sqrtf(u0);
  float sn, cs;
  sincospif(2.0f * u1, &sn, &cs);
  const float lx = r * cs, ly = r * sn, lz = sqrtf(fmaxf(1.0f - u0, 0.0f));
  if (u2 < p.wd) {
    // cosine lobe around n_d, frame from n_d by Duff et al.'s basis
    float n0 = -p.mdx, n1 = -p.mdy, n2 = 1.0f;
    const float il = rsqrtf(n0 * n0 + n1 * n1 + 1.0f);
    n0 *= il; n1 *= il; n2 *= il;
    const float sg = copysignf(1.0f, n2);
    const float a = -1.0f / (sg + n2);
    const float b = n0 * n1 * a;
    const float t0 = 1.0f + sg * n0 * n0 * a, t1 = sg * b, t2 = -sg * n0;
    const float b0 = n1 * t2 - n2 * t1, b1 = n2 * t0 - n0 * t2, b2 = n0 * t1 - n1 * t0;
    wo[0] = t0 * lx + b0 * ly + n0 * lz;
    wo[1] = t1 * lx + b1 * ly + n1 * lz;
    wo[2] = t2 * lx + b2 * ly + n2 * lz;
  } else {
    const float s = sqrtf(1.0f - p.rho * p.rho);
    float hx = p.ax * lx - p.msx * lz;
    float hy = p.ay * p.rho * lx + p.ay * s * ly - p.msy * lz;
    float hz = lz;
    const float ih = rsqrtf(hx * hx + hy * hy + hz * hz);
    hx *= ih; hy *= ih; hz *= ih;
    const float d = wi[0] * hx + wi[1] * hy + wi[2] * hz;
    wo[0] = 2.0f * d * hx - wi[0];
    wo[1] = 2.0f * d * hy - wi[1];
    wo[2] = 2.0f * d * hz - wi[2];
  }
}

template <bool F16>
__global__ void __launch_bounds__(128) sampler_kernel(const LaunchCommon L, const float* __restrict__ weights,
                                                      int mode, const float* __restrict__ u,
                                                      float* __restrict__ wo_out, float* __restrict__ pdf_out) {
  __shared__ __align__(16) float S[kSamplerFloats];
  for (int i = threadIdx.x; i < kSamplerFloats; i += blockDim.x) S[i] = weights[i];
  __syncthreads();
  const float* W1 = S;
  const float* b1 = W1 + 11 * 32;
  const float* W2 = b1 + 32;
  const float* b2 = W2 + 32 * 32;
  const float* W3 = b2 + 32;
  const float* b3 = W3 + 32 * 32;
  const float* W4 = b3 + 32;
  const float* b4 = W4 + 9 * 32;
  const QueryPtrs& q = L.q;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x) {
    float x[11];
    const float xi = q.xi ? q.xi[i] : 0.0f;
    fetch_latent<F16>(L.pyr, L.pyr0, q.u[i], q.v[i], q.lod[i], xi, x);
    const float wi[3] = {q.wix[i], q.wiy[i], q.wiz[i]};
    x[8] = wi[0];
    x[9] = wi[1];
    x[10] = wi[2];
    float h[32], g[32];
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
      float s = b1[j];
#pragma unroll
      for (int k = 0; k < 11; ++k) s = fmaf(W1[j * 11 + k], x[k], s);
      h[j] = fmaxf(s, 0.0f);
    }
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
      float s = b2[j];
#pragma unroll
      for (int k = 0; k < 32; ++k) s = fmaf(W2[j * 32 + k], h[k], s);
      g[j] = fmaxf(s, 0.0f);
    }
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
      float s = b3[j];
#pragma unroll
      for (int k = 0; k < 32; ++k) s = fmaf(W3[j * 32 + k], g[k], s);
      h[j] = fmaxf(s, 0.0f);
    }
    float o[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      float s = b4[j];
#pragma unroll
      for (int k = 0; k < 32; ++k) s = fmaf(W4[j * 32 + k], h[k], s);
      o[j] = s;
    }
    const Proxy p = activate(o);
    if (mode == 0) {
      const float wo[3] = {q.wox[i], q.woy[i], q.woz[i]};
      pdf_out[i] = pdf_full(p, wi, wo);
    } else {
      float wo[3];
      sample_dir(p, wi, u[3 * i], u[3 * i + 1], u[3 * i + 2], wo);
      wo_out[3 * i] = wo[0];
      wo_out[3 * i + 1] = wo[1];
      wo_out[3 * i + 2] = wo[2];
      if (pdf_out) pdf_out[i] = pdf_full(p, wi, wo);
    }
  }
}

}  // namespace

template <bool F16>
static int launch_sampler_one(const LaunchCommon& L, const float* sampler, int mode, const float* u, float* wo_out,
                              float* pdf_out, cudaStream_t s) {
  auto k = sampler_kernel<F16>;
  static std::atomic<int> occ{0};  // per instantiation (one GPU model)
  if (occ.load() == 0) occ.store(blocks_per_sm((const void*)k, 128, 0, 16));
  const int64_t blocks = (L.n + 127) / 128;
  const int64_t cap = (int64_t)occ.load() * L.num_sms;
  const int grid = (int)(blocks < cap ? blocks : cap);
  k<<<grid, 128, 0, s>>>(L, sampler, mode, u, wo_out, pdf_out);
  return (int)cudaGetLastError();
}

int launch_sampler(const LaunchCommon& L, const float* sampler, int mode, const float* u, float* wo_out,
                   float* pdf_out, void* stream) {
  if (L.n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  return L.pyr.f16 ? launch_sampler_one<true>(L, sampler, mode, u, wo_out, pdf_out, s)
                   : launch_sampler_one<false>(L, sampler, mode, u, wo_out, pdf_out, s);
}

}  // namespace nam
