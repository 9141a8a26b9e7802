// Importance sampling with the neural proxy density (Sec. 4.3, Appendix A).
//
// Per query: latent fetch as for the BRDF, the sampler MLP 11 -> 32 -> 32 ->
// 32 -> 9 (ReLU hidden layers), the output activations, then either the
// mixture density of the query's wo or one sample of wo with its density.
// Sampler weights (FP32 masters) are laid out per layer as W (out x in) then
// b (out).
//
// The MLP runs on the tensor cores at FP32 accuracy, tiles of 128 queries
// per warpgroup as in the evaluation kernel (thread r = query r = TMEM lane
// r).  Each weight is split into two binary16 values, W = W_hi + W_lo, and
// each layer input into x = x_hi + x_lo (hi: x with its 13 low mantissa bits
// cleared, exact in binary16); one MMA over [x_hi | x_lo | 1 1] x [W_hi |
// W_hi | b_hi b_lo] and one over x_hi x W_lo give W x + b up to the dropped
// W_lo x_lo term, a relative 2^-22.  The proxy's activations, density and
// sampling run per thread in FP32.
#include <cuda_runtime.h>

#include "eval_tc.cuh"

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


// ---------------------------------------------------------------------------
// weight blob: MMA B operands in the canonical no-swizzle K-major layout
// (element (row, k) at (k / 8) * R * 16 + row * 16 + (k % 8) * 2 for an R-row
// block), rows = outputs:
//   A1 32 x 32  [W1_hi (11) b1_hi 0 0 0 0 | W1_hi (11) b1_lo 0 0 0 0]
//   L1 32 x 16  [W1_lo (11) 0 ...]
//   A2, A3 32 x 80  [W_hi (32) | W_hi (32) | b_hi b_lo 0 ...]
//   L2, L3 32 x 32  W_lo
//   A4, L4 as A2, L2 with 16 rows (9 used)
// ---------------------------------------------------------------------------
constexpr int kSA1 = 0, kSL1 = 2048, kSA2 = 3072, kSL2 = 8192, kSA3 = 10240, kSL3 = 15360, kSA4 = 17408,
              kSL4 = 19968, kSamplerBlobBytes = 20992;

// TMEM columns of one warpgroup: the accumulator [0, 32), the A operand
// [32, 72): (x_hi, x_lo) of layer 1 in [32, 48); (h_hi, h_lo, 1 1 0 ...) of
// the later layers in [32, 72), the constant pair (1, 1) at column 64 written
// once.
constexpr int kSD = 0, kSA = 32, kSCols = 72;
constexpr int kSamplerNwg = 5;

template <bool F16P, int NWG>
struct SamplerSmem {
  static constexpr int STG_OFF = kSamplerBlobBytes;
  static constexpr int STG = F16P ? kStageBytes : 0;
  static constexpr int BAR_OFF = STG_OFF + NWG * STG;
  static constexpr int BYTES = BAR_OFF + NWG * 8 + 8 + 16;
};

template <bool F16P, int NWG>
__global__ void __launch_bounds__(NWG * 128, 1)
    sampler_tc_kernel(const LaunchCommon L, const uint8_t* __restrict__ blob, int mode, const float* __restrict__ u,
                      float* __restrict__ wo_out, float* __restrict__ pdf_out) {
  using S = SamplerSmem<F16P, NWG>;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, wg = tid >> 7, r = tid & 127, warp = tid >> 5;
  const uint32_t aW = ptx::smem_u32(smem);
  const uint32_t stg = ptx::smem_u32(smem + S::STG_OFF + wg * S::STG) + r * 16;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);
  const uint32_t bar_m = ptx::smem_u32(&bars[wg]);
  const uint32_t bar_w = ptx::smem_u32(&bars[NWG]);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::BAR_OFF + NWG * 8 + 8);
  const uint32_t bar_id = 1 + wg;

  if (r == 0) {
    ptx::mbar_init(bar_m, 1);
    if (tid == 0) ptx::mbar_init(bar_w, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tB = tmem + wg * kSCols;
  const uint32_t tBl = tB + ((uint32_t)((warp & 3) * 32) << 16);

  const int64_t ntiles = (L.n + 127) / 128;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t c_begin = (int64_t)blockIdx.x * per;
  const int64_t c_end = c_begin + per < ntiles ? c_begin + per : ntiles;

  uint32_t ph_m = 0;
  bool bad = false, mma_pending = false, w_pending = false;
  if (tid == 0 && c_begin < c_end) {
    ptx::fence_proxy_async();
    ptx::mbar_arrive_expect_tx(bar_w, kSamplerBlobBytes);
    ptx::bulk_g2s(aW, blob, kSamplerBlobBytes, bar_w);
    w_pending = true;
  }
  {
    // the constant pair (1, 1) that meets the bias columns (b_hi, b_lo)
    uint32_t one[8] = {0x3C003C00u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    ptx::tmem_st8(tBl + kSA + 32, one);
  }
  constexpr uint32_t ID32 = ptx::idesc_f16(128, 32);
  constexpr uint32_t ID16 = ptx::idesc_f16(128, 16);

  auto stage_issue = [&](auto issue) -> bool {
    ptx::tmem_st_wait();
    ptx::tc_fence_before();
    if (ptx::bar_red_or(bar_id, 128, bad)) {
      bad = true;
      return false;
    }
    if (r == 0) {
      ptx::tc_fence_after();
      issue();
      ptx::mma_commit(bar_m);
    }
    mma_pending = true;
    return true;
  };
  auto stage_wait = [&]() {
    bad |= !ptx::mbar_wait(bar_m, ph_m, L.timeout_ns);
    ph_m ^= 1;
    if (!bad) mma_pending = false;
    ptx::tc_fence_after();
  };
  // ReLU of the 32 accumulator columns, split into (h_hi, h_lo), 16 at a time
  auto hidden_operand = [&]() {
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 16) {
      uint32_t acc[16];
      ptx::tmem_ld16(tBl + kSD + c0, acc);
      ptx::tmem_ld_wait();
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) split_pair<true>(f32_of(acc[2 * j]), f32_of(acc[2 * j + 1]), hi[j], lo[j]);
      ptx::tmem_st8(tBl + kSA + c0 / 2, hi);
      ptx::tmem_st8(tBl + kSA + 16 + c0 / 2, lo);
    }
  };
  // one hidden or output layer: [h_hi | h_lo | 1 1] x [W_hi | W_hi | b], then h_hi x W_lo
  auto layer_mmas = [&](int a_off, int l_off, int rows, uint32_t id) {
    const uint32_t lbo = (uint32_t)rows * 16, step = (uint32_t)rows * 32;
#pragma unroll
    for (int s = 0; s < 5; ++s)
      ptx::mma_f16_ts(tB + kSD, tB + kSA + 8 * s, ptx::sdesc(aW + a_off + s * step, lbo, 128), id, s > 0 ? 1u : 0u);
#pragma unroll
    for (int s = 0; s < 2; ++s)
      ptx::mma_f16_ts(tB + kSD, tB + kSA + 8 * s, ptx::sdesc(aW + l_off + s * step, lbo, 128), id, 1u);
  };

  int64_t c = c_begin + wg;
  QF q_nxt{};
  bool w_ready = false;
  float zr[8];  // filtered latent of the tile about to start (FP16 pyramids)
  if (c < c_end) {
    const int64_t i0 = c * 128 + r;
    const QF q0 = load_qf(L.q, i0 < L.n ? i0 : L.n - 1);
    if (F16P) {
      fetch_issue(L.pyr, reinterpret_cast<const uint8_t*>(L.pyr0), q0, stg);
      fetch_finish(stg, zr);
    }
    if (c + NWG < c_end) {
      const int64_t i1 = (c + NWG) * 128 + r;
      q_nxt = load_qf(L.q, i1 < L.n ? i1 : L.n - 1);
    }
  }
  for (; c < c_end; c += NWG) {
    const bool has_next = c + NWG < c_end, has_next2 = c + 2 * NWG < c_end;
    const int64_t i_raw = c * 128 + r;
    const bool valid = i_raw < L.n;
    const int64_t i = valid ? i_raw : L.n - 1;
    const float wi[3] = {ptx::ld_nc_pinned(L.q.wix + i), ptx::ld_nc_pinned(L.q.wiy + i),
                         ptx::ld_nc_pinned(L.q.wiz + i)};
    if (!w_ready) {
      bad |= !ptx::mbar_wait(bar_w, 0, L.timeout_ns);
      if (!bad && tid == 0) w_pending = false;
      w_ready = true;
    }
    // ---- layer 1 input (z, wi, 1) as (hi, lo) ------------------------------
    float x[16];
    if (F16P) {
      // filtered while the previous tile's last layer ran
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = zr[k];
    } else {
      const QF q0 = load_qf(L.q, i);
      fetch_latent<false>(L.pyr, L.pyr0, q0.u, q0.v, q0.lod, q0.xi, x);
    }
    x[8] = wi[0];
    x[9] = wi[1];
    x[10] = wi[2];
    x[11] = 1.0f;
    x[12] = x[13] = x[14] = x[15] = 0.0f;
    {
      uint32_t v[16];
#pragma unroll
      for (int j = 0; j < 8; ++j) split_pair<false>(x[2 * j], x[2 * j + 1], v[j], v[8 + j]);
      v[8 + 5] = (v[8 + 5] & 0x0000FFFFu) | 0x3C000000u;  // lo block: the 1 meets b1_lo
      ptx::tmem_st16(tBl + kSA, v);
    }
    if (!stage_issue([&] {
#pragma unroll
          for (int s = 0; s < 2; ++s)
            ptx::mma_f16_ts(tB + kSD, tB + kSA + 8 * s, ptx::sdesc(aW + kSA1 + s * 1024, 512, 128), ID32,
                            s > 0 ? 1u : 0u);
          ptx::mma_f16_ts(tB + kSD, tB + kSA, ptx::sdesc(aW + kSL1, 512, 128), ID32, 1u);
        }))
      break;
    // the next tile's texel gathers while layer 1 runs
    QF q_nxt2{};
    if (F16P && has_next) fetch_issue(L.pyr, reinterpret_cast<const uint8_t*>(L.pyr0), q_nxt, stg);
    if (has_next2) {
      const int64_t i2 = (c + 2 * NWG) * 128 + r;
      q_nxt2 = load_qf(L.q, i2 < L.n ? i2 : L.n - 1);
    }
    stage_wait();
    // ---- layers 2, 3 (32 -> 32) and 4 (32 -> 9) -----------------------------
    hidden_operand();
    if (!stage_issue([&] { layer_mmas(kSA2, kSL2, 32, ID32); })) break;
    stage_wait();
    hidden_operand();
    if (!stage_issue([&] { layer_mmas(kSA3, kSL3, 32, ID32); })) break;
    stage_wait();
    hidden_operand();
    if (!stage_issue([&] { layer_mmas(kSA4, kSL4, 16, ID16); })) break;
    // the next tile's filter, while the last layer runs
    if (F16P && has_next) fetch_finish(stg, zr);
    stage_wait();
    // ---- proxy parameters, density or sample --------------------------------
    float o[9];
    {
      uint32_t acc[16];
      ptx::tmem_ld16(tBl + kSD, acc);
      ptx::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 9; ++j) o[j] = f32_of(acc[j]);
    }
    ptx::tc_fence_before();
    if (valid) {
      const Proxy p = activate(o);
      if (mode == 0) {
        const float wo[3] = {L.q.wox[i], L.q.woy[i], L.q.woz[i]};
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
    q_nxt = q_nxt2;
  }

  // ---- teardown (as in the evaluation kernel) --------------------------------
  ptx::cp_async_wait_all();
  bool drained = true;
  if (r == 0 && mma_pending) drained &= ptx::mbar_wait(bar_m, ph_m ^ 1, ptx::kDrainTimeoutNs);
  if (tid == 0 && w_pending) drained &= ptx::mbar_wait(bar_w, 0, ptx::kDrainTimeoutNs);
  if (bad) record_error(L.err, DEVERR_WAIT_TIMEOUT);
  if (!drained) record_error(L.err, DEVERR_DRAIN_TIMEOUT);
  ptx::tc_fence_before();
  const bool all_drained = __syncthreads_and(drained ? 1 : 0) != 0;
  if (warp == 0 && all_drained) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

}  // namespace

size_t sampler_blob_bytes() { return (size_t)kSamplerBlobBytes; }

// x = hi + lo in binary16: hi = x with its 13 low mantissa bits cleared
// (rounded to binary16, exact over its normal range), lo = the rest rounded
// to binary16.
static void split_f16(float x, __half& hi, __half& lo) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b &= 0xFFFFE000u;
  float t;
  std::memcpy(&t, &b, 4);
  hi = __float2half_rn(t);
  lo = __float2half_rn(x - __half2float(hi));
}

static void put_half(uint8_t* base, int R, int row, int k, __half h) {
  std::memcpy(base + (k / 8) * (R * 16) + row * 16 + (k % 8) * 2, &h, 2);
}

int pack_sampler_blob(const float* w, uint8_t* out) {
  for (int i = 0; i < kSamplerFloats; ++i)
    if (!(std::fabs(w[i]) < 32768.0f)) return -1;  // beyond the binary16 split
  std::memset(out, 0, kSamplerBlobBytes);
  const float* W1 = w;
  const float* b1 = W1 + 11 * 32;
  __half hi, lo;
  for (int j = 0; j < 32; ++j) {
    for (int k = 0; k < 11; ++k) {
      split_f16(W1[j * 11 + k], hi, lo);
      put_half(out + kSA1, 32, j, k, hi);
      put_half(out + kSA1, 32, j, 16 + k, hi);
      put_half(out + kSL1, 32, j, k, lo);
    }
    split_f16(b1[j], hi, lo);
    put_half(out + kSA1, 32, j, 11, hi);
    put_half(out + kSA1, 32, j, 27, lo);
  }
  // layers 2..4: W (rows x 32) then b
  const float* p = b1 + 32;
  const int a_off[3] = {kSA2, kSA3, kSA4}, l_off[3] = {kSL2, kSL3, kSL4}, rows[3] = {32, 32, 9};
  for (int l = 0; l < 3; ++l) {
    const int R = l < 2 ? 32 : 16;
    const float* W = p;
    const float* b = W + rows[l] * 32;
    for (int j = 0; j < rows[l]; ++j) {
      for (int k = 0; k < 32; ++k) {
        split_f16(W[j * 32 + k], hi, lo);
        put_half(out + a_off[l], R, j, k, hi);
        put_half(out + a_off[l], R, j, 32 + k, hi);
        put_half(out + l_off[l], R, j, k, lo);
      }
      split_f16(b[j], hi, lo);
      put_half(out + a_off[l], R, j, 64, hi);
      put_half(out + a_off[l], R, j, 65, lo);
    }
    p = b + rows[l];
  }
  return 0;
}

template <bool F16P>
static int launch_sampler_tc(const LaunchCommon& L, const void* blob, int mode, const float* u, float* wo_out,
                             float* pdf_out, cudaStream_t s) {
  constexpr int NWG = kSamplerNwg;
  using S = SamplerSmem<F16P, NWG>;
  static_assert(S::BYTES <= 227 * 1024, "shared memory");
  static_assert(NWG * kSCols <= 512, "TMEM columns");
  auto k = sampler_tc_kernel<F16P, NWG>;
  static std::atomic<uint64_t> configured{0};
  once_per_device(configured, [&] {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
    const int pct = (S::BYTES + 1024) * 100 / (228 * 1024) + 1;
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  });
  const int64_t ntiles = (L.n + 127) / 128;
  const int64_t want = (ntiles + NWG - 1) / NWG;
  const int grid = (int)(want < L.num_sms ? want : L.num_sms);
  k<<<grid, NWG * 128, S::BYTES, s>>>(L, reinterpret_cast<const uint8_t*>(blob), mode, u, wo_out, pdf_out);
  return (int)cudaGetLastError();
}

int launch_sampler(const LaunchCommon& L, const void* blob, int mode, const float* u, float* wo_out,
                   float* pdf_out, void* stream) {
  if (L.n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  return L.pyr.f16 ? launch_sampler_tc<true>(L, blob, mode, u, wo_out, pdf_out, s)
                   : launch_sampler_tc<false>(L, blob, mode, u, wo_out, pdf_out, s);
}

}  // namespace nam
