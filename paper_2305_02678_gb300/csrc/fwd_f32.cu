// Plain FP32 evaluation: one query per thread, MLP weights staged in shared
// memory, FP32 FMA on CUDA cores.  This is the "divergent" per-thread form
// of the decoder (Sec. 7.1: whole network per thread, unrolled FMAs) and the
// FP32 reference point the reduced-precision tensor-core path is compared to.
#include <cuda_runtime.h>

#include "common.cuh"

namespace nam {

int64_t n_params_of(const Shape& s) {
  int64_t n = frame_params_of(s.frame);
  n += (int64_t)s.in * s.H + s.H;
  for (int i = 1; i < s.NH; ++i) n += (int64_t)s.H * s.H + s.H;
  n += 3 * s.H + 3;
  return n;
}

// Shared-memory image of the parameters, rows padded for 16-byte loads.
// FK: frame form (0 none, 1 MLP 8-16-6, 2 the paper's linear 8 -> 12);
// INP: decoder input row length (14 inputs padded to 16, or 20).
template <int H, int NH, int FK, int INP>
struct SmemF32 {
  float fW1[FK == 2 ? 12 * 8 : 16 * 8];  // FK 1: Wf1 [16][8]; FK 2: Wf [12][8]
  float fb1[16];
  float fW2[6 * 16];
  float fb2[8];
  float W1[H * INP];        // [H][INP], inputs past the decoder's width are zero
  float b1[H];
  float Wh[NH - 1][H * H];  // hidden -> hidden
  float bh[NH - 1][H];
  float WoT[H * 4];         // output weights transposed [H][4]
  float bo[4];
};

template <int H, int NH, int FK, int INP>
__device__ void load_params_f32(SmemF32<H, NH, FK, INP>& S, const float* __restrict__ p, int in) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (FK == 1) {
    for (int i = tid; i < 128; i += nt) S.fW1[i] = p[i];
    for (int i = tid; i < 16; i += nt) S.fb1[i] = p[128 + i];
    for (int i = tid; i < 96; i += nt) S.fW2[i] = p[144 + i];
    for (int i = tid; i < 8; i += nt) S.fb2[i] = i < 6 ? p[240 + i] : 0.0f;
    p += 246;
  } else if (FK == 2) {
    for (int i = tid; i < 96; i += nt) S.fW1[i] = p[i];
    for (int i = tid; i < 16; i += nt) S.fb1[i] = i < 12 ? p[96 + i] : 0.0f;
    p += 108;
  }
  for (int i = tid; i < H * INP; i += nt) {
    int j = i / INP, k = i % INP;
    S.W1[i] = k < in ? p[j * in + k] : 0.0f;
  }
  p += in * H;
  for (int i = tid; i < H; i += nt) S.b1[i] = p[i];
  p += H;
  for (int l = 0; l < NH - 1; ++l) {
    for (int i = tid; i < H * H; i += nt) S.Wh[l][i] = p[i];
    p += H * H;
    for (int i = tid; i < H; i += nt) S.bh[l][i] = p[i];
    p += H;
  }
  for (int i = tid; i < H * 4; i += nt) {
    int j = i >> 2, c = i & 3;
    S.WoT[i] = c < 3 ? p[c * H + j] : 0.0f;
  }
  p += 3 * H;
  for (int i = tid; i < 4; i += nt) S.bo[i] = i < 3 ? p[i] : 0.0f;
}

template <int H>
__device__ __forceinline__ float dot_row(const float* __restrict__ row, const float* h) {
  const float4* r4 = reinterpret_cast<const float4*>(row);
  float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
  for (int k = 0; k < H / 4; ++k) {
    float4 w = r4[k];
    s0 = fmaf(w.x, h[4 * k + 0], s0);
    s1 = fmaf(w.y, h[4 * k + 1], s1);
    s0 = fmaf(w.z, h[4 * k + 2], s0);
    s1 = fmaf(w.w, h[4 * k + 3], s1);
  }
  return s0 + s1;
}

template <int H, int NH, int FK, bool F16>
__global__ void __launch_bounds__(128) eval_f32_kernel(LaunchCommon L) {
  constexpr int INP = FK == 2 ? 20 : 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemF32<H, NH, FK, INP>& S = *reinterpret_cast<SmemF32<H, NH, FK, INP>*>(smem_raw);
  load_params_f32<H, NH, FK, INP>(S, reinterpret_cast<const float*>(L.w0), FK == 2 ? 20 : 14);
  __syncthreads();
  const QueryPtrs& q = L.q;
  const bool cosine = (L.flags & NAM_OUT_COSINE) != 0;
  const bool calib = L.amax != nullptr;
  float am0 = 0.0f, am1 = 0.0f, am2 = 0.0f;  // calibration: max |layer input|
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float z[8];
    const float xi = q.xi ? q.xi[i] : 0.0f;
    fetch_latent<F16>(L.pyr, L.pyr0, q.u[i], q.v[i], q.lod[i], xi, z);
    const float wix = q.wix[i], wiy = q.wiy[i], wiz = q.wiz[i];
    const float wox = q.wox[i], woy = q.woy[i], woz = q.woz[i];
    float x[INP];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = z[c];
    if constexpr (FK == 1) {
      float hf[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float s = S.fb1[j];
#pragma unroll
        for (int c = 0; c < 8; ++c) s = fmaf(S.fW1[j * 8 + c], z[c], s);
        hf[j] = fmaxf(s, 0.0f);
      }
      float r[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) r[j] = S.fb2[j] + dot_row<16>(&S.fW2[j * 16], hf);
      Frame F = build_frame(r);
      to_local(F, wix, wiy, wiz, x + 8);
      to_local(F, wox, woy, woz, x + 11);
    } else if constexpr (FK == 2) {
      float r[12];
#pragma unroll
      for (int j = 0; j < 12; ++j) {
        float s = S.fb1[j];
#pragma unroll
        for (int c = 0; c < 8; ++c) s = fmaf(S.fW1[j * 8 + c], z[c], s);
        r[j] = s;
      }
      Frame F1 = paper_frame(r), F2 = paper_frame(r + 6);
      to_local(F1, wix, wiy, wiz, x + 8);
      to_local(F2, wix, wiy, wiz, x + 11);
      to_local(F1, wox, woy, woz, x + 14);
      to_local(F2, wox, woy, woz, x + 17);
    } else {
      x[8] = wix; x[9] = wiy; x[10] = wiz;
      x[11] = wox; x[12] = woy; x[13] = woz;
    }
    if constexpr (FK != 2) {
      x[14] = 0.0f;
      x[15] = 0.0f;
    }
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) h1[j] = fmaxf(S.b1[j] + dot_row<INP>(&S.W1[j * INP], x), 0.0f);
    if (calib) {
#pragma unroll
      for (int c = 0; c < INP; ++c) am0 = fmaxf(am0, fabsf(x[c]));
#pragma unroll
      for (int j = 0; j < H; ++j) am1 = fmaxf(am1, h1[j]);
    }
    float y0 = S.bo[0], y1 = S.bo[1], y2 = S.bo[2];
    if (NH == 2) {
#pragma unroll 4
      for (int j = 0; j < H; ++j) {
        float s = fmaxf(S.bh[0][j] + dot_row<H>(&S.Wh[0][j * H], h1), 0.0f);
        am2 = fmaxf(am2, s);
        float4 wo = reinterpret_cast<const float4*>(S.WoT)[j];
        y0 = fmaf(wo.x, s, y0);
        y1 = fmaf(wo.y, s, y1);
        y2 = fmaf(wo.z, s, y2);
      }
    } else {
      float h2[H];
#pragma unroll 4
      for (int j = 0; j < H; ++j) h2[j] = fmaxf(S.bh[0][j] + dot_row<H>(&S.Wh[0][j * H], h1), 0.0f);
#pragma unroll 4
      for (int j = 0; j < H; ++j) {
        float s = fmaxf(S.bh[NH - 2][j] + dot_row<H>(&S.Wh[NH - 2][j * H], h2), 0.0f);
        float4 wo = reinterpret_cast<const float4*>(S.WoT)[j];
        y0 = fmaf(wo.x, s, y0);
        y1 = fmaf(wo.y, s, y1);
        y2 = fmaf(wo.z, s, y2);
      }
    }
    if (cosine) {
      float c = fmaxf(wiz, 0.0f);
      y0 *= c; y1 *= c; y2 *= c;
    }
    if (L.rgb) {
      L.rgb[3 * i + 0] = y0;
      L.rgb[3 * i + 1] = y1;
      L.rgb[3 * i + 2] = y2;
    }
  }
  if (calib) {
    // non-negative floats order like their bit patterns: integer atomic max
    for (int o = 16; o > 0; o >>= 1) {
      am0 = fmaxf(am0, __shfl_xor_sync(0xffffffffu, am0, o));
      am1 = fmaxf(am1, __shfl_xor_sync(0xffffffffu, am1, o));
      am2 = fmaxf(am2, __shfl_xor_sync(0xffffffffu, am2, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(reinterpret_cast<int*>(L.amax) + 0, __float_as_int(am0));
      atomicMax(reinterpret_cast<int*>(L.amax) + 1, __float_as_int(am1));
      atomicMax(reinterpret_cast<int*>(L.amax) + 2, __float_as_int(am2));
    }
  }
}

template <int H, int NH, int FK, bool F16>
static int launch_one(const LaunchCommon& L, cudaStream_t s) {
  auto k = eval_f32_kernel<H, NH, FK, F16>;
  const int smem = (int)sizeof(SmemF32<H, NH, FK, FK == 2 ? 20 : 16>);
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> occ{0};  // per instantiation (one GPU model)
  once_per_device(configured, [&] {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    occ.store(blocks_per_sm((const void*)k, 128, smem, 16));
  });
  int64_t blocks = (L.n + 127) / 128;
  int64_t cap = (int64_t)occ.load() * L.num_sms;
  int grid = (int)(blocks < cap ? blocks : cap);
  if (grid < 1) grid = 1;
  k<<<grid, 128, smem, s>>>(L);
  return (int)cudaGetLastError();
}

template <int H, int NH>
static int dispatch_frame(const LaunchCommon& L, cudaStream_t s) {
  const bool f16 = L.pyr.f16;
  switch (L.shape.frame) {
    case 1: return f16 ? launch_one<H, NH, 1, true>(L, s) : launch_one<H, NH, 1, false>(L, s);
    case 2: return f16 ? launch_one<H, NH, 2, true>(L, s) : launch_one<H, NH, 2, false>(L, s);
    default: return f16 ? launch_one<H, NH, 0, true>(L, s) : launch_one<H, NH, 0, false>(L, s);
  }
}

int launch_eval_f32(const LaunchCommon& L, void* stream) {
  if (L.n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const Shape& sh = L.shape;
  if (sh.NH == 2) {
    if (sh.H == 16) return dispatch_frame<16, 2>(L, s);
    if (sh.H == 32) return dispatch_frame<32, 2>(L, s);
    if (sh.H == 64) return dispatch_frame<64, 2>(L, s);
  }
  if (sh.NH == 3 && sh.H == 64) return dispatch_frame<64, 3>(L, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace nam
