// FP16 tensor-core evaluation of the neural BRDF on sm_103a (tcgen05 + TMEM),
// pipelined over 128-query tiles.
//
// One CTA per SM with NWG warpgroups; a warpgroup owns a tile of 128 queries
// at a time (thread r = query r = TMEM lane r) and takes it through five MMA
// stages on its own TMEM columns:
//   1. latent z (Sec. 4.1, trilinear or stochastic filtering of the pyramid,
//      FP32 filter) -> MMA 1: the frame layer (Sec. 4.2) and the z part of
//      decoder layer 1 share their input, so one MMA of N = 16 + H computes
//      both;
//   2. the frame MLP's second layer (8 -> 16 -> 6 form);
//   3. frame build (Gram-Schmidt, b = n x t) and the direction transform
//      (Eq. 4) in FP32 registers -> MMA 3 adds the direction part of decoder
//      layer 1 and its bias onto MMA 1's accumulator;
//   4. hidden layers (ReLU, FP16 operands);
//   5. output layer, RGB store (x max(0, wi.z) if asked, Eq. 1).
// Precision: FP16 weights (post-training quantised, Sec. 5.2), FP32
// accumulation.  z, the transformed directions, the frame MLP's hidden layer
// and the decoder's last hidden layer (every hidden layer for H < 64) enter
// the MMA as two FP16 halves (x = hi + lo, hi = x with its 13 low mantissa
// bits cleared, exact in FP16; lo = x - hi, rounded), i.e. at ~22-bit
// accuracy; the other hidden layers are rounded to FP16 once.  (The two narrow layers in FP32 on the FMA pipes
// instead of the tensor core measured slower: their SIMT instructions cost
// more than the MMA round trips they save.)
// Latency hiding: the texel gathers of the next tile go to shared memory with
// cp.async while the current tile's first MMA runs, and (single-material
// launches) are filtered while its output MMA runs, z of the next tile then
// waiting in registers; each warpgroup's tile is independent of the others'.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nam {

// ---------------------------------------------------------------------------
// weight blob: MMA B operands (rows = N = outputs, K = inputs), canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices: element (row, k)
// at (k / 8) * (R * 16) + row * 16 + (k % 8) * 2 for an R-row block)
// ---------------------------------------------------------------------------
struct F16Lay {
  int NF;     // frame rows in the first MMA: 16 (frame forms 1, 2) or 0
  int N1;     // first MMA's N: H rows of decoder layer 1 (z inputs), then NF
  int ND;     // direction inputs of decoder layer 1: 6, or 12 (paper form)
  int KD;     // K of the direction block: (dir hi, dir lo, 1, 0 ...)
  int B1;     // N1 x 16: [W(z) | W(z)] for the operand (z hi, z lo)
  int B1B;    // 16 x 16: frame-layer bias in column 0 (A = constant block)
  int BF2;    // form 1: 16 x 32: [Wf2 | Wf2] (6 rows used)
  int BD;     // H x KD: [W(dirs) | W(dirs) | b1 | 0 ..]
  int BH;     // NH - 1 blocks of H x (H + 16): [W | b 0 ..]
  int BO;     // 16 x H: Wo (3 or 6 rows used)
  int SB;     // FP32 biases (binary16-rounded values) added in the
              // epilogues: frame MLP layer 2 at [16, 22), output at [24, 30)
  int BYTES;
};

__host__ __device__ constexpr F16Lay f16_lay(int H, int FK, int NH) {
  F16Lay o{};
  o.NF = FK ? 16 : 0;
  o.N1 = H + o.NF;
  o.ND = FK == 2 ? 12 : 6;
  o.KD = FK == 2 ? 32 : 16;
  o.B1 = 0;
  o.B1B = o.B1 + o.N1 * 16 * 2;
  o.BF2 = o.B1B + (FK ? 16 * 16 * 2 : 0);
  o.BD = o.BF2 + (FK == 1 ? 16 * 32 * 2 : 0);
  o.BH = o.BD + H * o.KD * 2;
  o.BO = o.BH + (NH - 1) * H * (H + 16) * 2;
  o.SB = o.BO + 16 * H * 2;
  o.BYTES = o.SB + 32 * 4;
  return o;
}

static inline bool f16_supported(const Shape& s) {
  const bool hidden_ok = (s.NH == 2 && (s.H == 16 || s.H == 32 || s.H == 64)) || (s.NH == 3 && s.H == 64);
  return hidden_ok && s.frame >= 0 && s.frame <= 2 && (s.out == 3 || s.out == 6);
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float f32_of(uint32_t x) { return __uint_as_float(x); }

// x = hi + lo with hi = x whose 13 low mantissa bits are cleared (at most 11
// significant bits: exact in binary16 over its normal range) and lo = x - hi
// (exact in FP32, then rounded to binary16: |error| <= 2^-21 |x|).  hi and lo
// carry the sign of x, so with RELU both halves of a negative x become +0.
template <bool RELU>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const float ta = __uint_as_float(__float_as_uint(a) & 0xFFFFE000u);
  const float tb = __uint_as_float(__float_as_uint(b) & 0xFFFFE000u);
  const float2 d = ptx::sub2(make_float2(a, b), make_float2(ta, tb));
  if (RELU) {
    hi = ptx::pack_h2_relu(ta, tb);
    lo = ptx::pack_h2_relu(d.x, d.y);
  } else {
    hi = ptx::pack_h2(ta, tb);
    lo = ptx::pack_h2(d.x, d.y);
  }
}

// The fetch-side query fields, loaded two tiles ahead of their use.
struct QF {
  float u, v, lod, xi;
};
__device__ __forceinline__ QF load_qf(const QueryPtrs& q, int64_t i) {
  QF x;
  x.u = ptx::ld_nc_pinned(q.u + i);
  x.v = ptx::ld_nc_pinned(q.v + i);
  x.lod = ptx::ld_nc_pinned(q.lod + i);
  x.xi = q.xi ? ptx::ld_nc_pinned(q.xi + i) : 0.0f;
  return x;
}

// A tile: up to 128 consecutive queries of one material.
struct TileRef {
  int64_t start;
  int count, mat;
};
__device__ __forceinline__ TileRef tile_at(const LaunchCommon& L, int64_t c) {
  TileRef t;
  if (L.chunks) {
    const Chunk ch = L.chunks[c];
    t.start = ch.start;
    t.count = ch.count;
    t.mat = ch.material;
  } else {
    t.start = c * 128;
    t.count = (int)((L.n - t.start) < 128 ? (L.n - t.start) : 128);
    t.mat = 0;
  }
  return t;
}

// Per-warpgroup staging of one tile's latent fetch in shared memory: tap k of
// row r at k * 2048 + r * 16 (8 binary16 channels), the eight tap weights
// at 16384 + j * 2048 + r * 16 (two float4).  Each thread reads back only
// what it wrote itself.
constexpr int kStageBytes = 16384 + 4096;

// Bilinear taps of level l (Sec. 4.1; texel centres at (i + 1/2) / W):
// issues the four 16-byte copies into slots dst + k * 2048 (zero-filled and
// not read when `load` is false) and writes the weights wl * (bilinear
// weight) to w[0..3].  `fast` (warp-uniform): power-of-two wrap with every
// lane's |u W0|, |v H0| < 2^22, where X = u W is exact and the continuous
// coordinate x = X - 1/2 is exact except for X in (-1/2, 1/2) (fraction moved
// by at most 2^-25); otherwise the exact general addressing of tap_axis.
__device__ __forceinline__ void level_issue(const PyrDesc& P, const uint8_t* pyr, int l, float u, float v,
                                            bool fast, float wl, bool load, uint32_t dst, float* w) {
  const int W = P.w[l], H = P.h[l];
  int x0, x1, y0, y1;
  float fx, fy;
  if (fast) {
    const float xs = u * (float)W - 0.5f, ys = v * (float)H - 0.5f;
    const float xf = floorf(xs), yf = floorf(ys);
    fx = xs - xf;
    fy = ys - yf;
    const int kx = (int)xf, ky = (int)yf;
    x0 = kx & (W - 1);
    x1 = (kx + 1) & (W - 1);
    y0 = ky & (H - 1);
    y1 = (ky + 1) & (H - 1);
  } else {
    tap_axis(P, u, W, x0, x1, fx);
    tap_axis(P, v, H, y0, y1, fy);
  }
  const uint32_t base = (uint32_t)P.off[l];
  const uint32_t r0 = base + (uint32_t)y0 * (uint32_t)W, r1 = base + (uint32_t)y1 * (uint32_t)W;
  const float gx = 1.0f - fx, gy = 1.0f - fy;
  const float a = gy * wl, b = fy * wl;
  w[0] = gx * a;
  w[1] = fx * a;
  w[2] = gx * b;
  w[3] = fx * b;
  const uint32_t sz = load ? 16u : 0u;
  ptx::cp_async16(dst, pyr + (size_t)(r0 + x0) * 16, sz);
  ptx::cp_async16(dst + 2048, pyr + (size_t)(r0 + x1) * 16, sz);
  ptx::cp_async16(dst + 4096, pyr + (size_t)(r1 + x0) * 16, sz);
  ptx::cp_async16(dst + 6144, pyr + (size_t)(r1 + x1) * 16, sz);
}

// Start the latent fetch of one query into its staging slots (FP16 pyramid).
// Trilinear: levels l0 (weight 1 - t) and l1 (weight t; not read when t = 0);
// stochastic: level l1 if xi < t else l0, weight 1 (Sec. 4.1).
__device__ __forceinline__ void fetch_issue(const PyrDesc& P, const uint8_t* pyr, const QF& q, uint32_t stg) {
  const float l = fminf(fmaxf(q.lod, 0.0f), (float)(P.levels - 1));  // NaN -> 0
  const float fl = floorf(l);
  const int l0 = (int)fl;
  const int l1 = min(l0 + 1, P.levels - 1);
  const float t = l - fl;
  int la = l0, lb = l1;
  float wa = 1.0f - t, wb = t;
  if (P.filter == NAM_FILTER_STOCHASTIC) {
    la = q.xi < t ? l1 : l0;
    wa = 1.0f;
    wb = 0.0f;
  }
  // the whole warp takes the general path if any lane needs it (huge or
  // non-finite coordinates), so that the common case has no divergence
  const bool in_range = fabsf(q.u * (float)P.w[0]) < 4194304.0f && fabsf(q.v * (float)P.h[0]) < 4194304.0f;
  const bool fast = P.pow2 && P.address == NAM_ADDRESS_WRAP && __all_sync(0xffffffffu, in_range);
  float w[8];
  level_issue(P, pyr, la, q.u, q.v, fast, wa, true, stg, w);
  level_issue(P, pyr, lb, q.u, q.v, fast, wb, wb != 0.0f, stg + 8192, w + 4);
  ptx::st_shared_v4(stg + 16384, __float_as_uint(w[0]), __float_as_uint(w[1]), __float_as_uint(w[2]),
                    __float_as_uint(w[3]));
  ptx::st_shared_v4(stg + 16384 + 2048, __float_as_uint(w[4]), __float_as_uint(w[5]), __float_as_uint(w[6]),
                    __float_as_uint(w[7]));
  ptx::cp_async_commit();
}

// Wait for this thread's copies and filter: z = sum_k w_k texel_k in FP32.
__device__ __forceinline__ void fetch_finish(uint32_t stg, float z[8]) {
  ptx::cp_async_wait_all();
  const uint4 wa = ptx::ld_shared_v4(stg + 16384), wb = ptx::ld_shared_v4(stg + 16384 + 2048);
  const float w[8] = {f32_of(wa.x), f32_of(wa.y), f32_of(wa.z), f32_of(wa.w),
                      f32_of(wb.x), f32_of(wb.y), f32_of(wb.z), f32_of(wb.w)};
  float2 acc[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint4 t = ptx::ld_shared_v4(stg + k * 2048);
    const __half2* h = reinterpret_cast<const __half2*>(&t);
    const float2 wk = make_float2(w[k], w[k]);
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = ptx::fma2(wk, __half22float2(h[c]), acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    z[2 * c] = acc[c].x;
    z[2 * c + 1] = acc[c].y;
  }
}

// ---------------------------------------------------------------------------
// kernel
// ---------------------------------------------------------------------------
// A launch that mixes materials keeps this many weight slots per CTA, shared
// by its warpgroups: a warpgroup whose tile needs a material finds it in a
// slot, or loads it into a slot no warpgroup is using.
constexpr int kMultiSlots = 2;

// Shared memory: constant block (1.0 in column 0 of every row) and zero block
// (the A operand of the bias steps), the weight slots (one, or kMultiSlots
// when a launch mixes materials), each warpgroup's fetch staging (FP16
// pyramids), the mbarriers (one per warpgroup for its MMAs, one per slot for
// its loads), the TMEM address, then the slot table: per slot its material,
// users and load count, a lock, and one word per warpgroup to broadcast the
// slot its leader acquired.
template <int H, int FK, int NH, bool F16P, bool MULTI, int NWG>
struct F16Smem {
  static constexpr F16Lay Y = f16_lay(H, FK, NH);
  static constexpr int SLOTS = MULTI ? kMultiSlots : 1;
  static constexpr int BLOB_AL = (Y.BYTES + 127) / 128 * 128;
  static constexpr int W_OFF = 4096;
  static constexpr int STG_OFF = W_OFF + SLOTS * BLOB_AL;
  static constexpr int STG = F16P ? kStageBytes : 0;
  static constexpr int BAR_OFF = STG_OFF + NWG * STG;
  static constexpr int TSLOT_OFF = (BAR_OFF + 8 * (NWG + SLOTS) + 15) / 16 * 16;
  static constexpr int TAB_OFF = TSLOT_OFF + 16;
  static constexpr int BYTES = (TAB_OFF + 4 * (3 * SLOTS + 1 + NWG) + 15) / 16 * 16;
};

// A lock word in shared memory, taken with a time limit (false: not taken).
__device__ __forceinline__ bool smem_lock(int* l, uint64_t t0, uint64_t timeout_ns) {
  while (atomicCAS(l, 0, 1) != 0) {
    if (ptx::globaltimer() - t0 > timeout_ns) return false;
    __nanosleep(64);
  }
  __threadfence_block();
  return true;
}
__device__ __forceinline__ void smem_unlock(int* l) {
  __threadfence_block();
  atomicExch(l, 0);
}

// TMEM columns of one warpgroup (H + 32):
//   [0, H)        decoder accumulator (layer 1, hidden layers); later the low
//                 halves of the last hidden layer's operand
//   [H, H + 16)   frame-layer accumulator; later the hidden-layer operand
//                 [H, H + H/2) (FP16 pairs)
//   [H+16, H+32)  operands of the frame MLP's second layer, z, directions
//   output accumulator: [32, 48) for H = 64, else [H + 16, H + 32)
template <int H>
struct F16Cols {
  static constexpr int COLS = H + 32;
  static constexpr int D = 0, F = H, A = H + 16, HID = H, LO = 0, OUT = H == 64 ? 32 : H + 16;
};

template <int H, int FK, int NH, bool F16P, bool MULTI, int NWG, bool P8>
__global__ void __launch_bounds__(NWG * 128, 1) eval_f16_kernel(const LaunchCommon L) {
  using S = F16Smem<H, FK, NH, F16P, MULTI, NWG>;
  using C = F16Cols<H>;
  constexpr F16Lay Y = S::Y;
  constexpr int ND = Y.ND;
  extern __shared__ __align__(1024) uint8_t smem[];

  const int tid = threadIdx.x, wg = tid >> 7, r = tid & 127, warp = tid >> 5;
  const uint32_t aConst = ptx::smem_u32(smem);
  uint32_t aW = ptx::smem_u32(smem + S::W_OFF);  // the weight slot this warpgroup reads
  const uint32_t stg = ptx::smem_u32(smem + S::STG_OFF + wg * S::STG) + r * 16;  // this row's slot 0
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);
  const uint32_t bar_m = ptx::smem_u32(&bars[wg]);
  const uint32_t bar_w = ptx::smem_u32(&bars[NWG]);  // slot 0's loads
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::TSLOT_OFF);
  // slot table (mixed-material launches)
  volatile int* slot_mat = reinterpret_cast<volatile int*>(smem + S::TAB_OFF);
  volatile int* slot_users = slot_mat + S::SLOTS;
  volatile int* slot_loads = slot_users + S::SLOTS;
  int* slot_lock = const_cast<int*>(slot_loads + S::SLOTS);
  volatile int* wg_word = slot_loads + S::SLOTS + 1;
  const uint32_t bar_id = 1 + wg;  // named barrier of this warpgroup

  if (r == 0) ptx::mbar_init(bar_m, 1);
  if (tid == 0) {
    for (int k = 0; k < S::SLOTS; ++k) {
      ptx::mbar_init(ptx::smem_u32(&bars[NWG + k]), 1);
      slot_mat[k] = -1;
      slot_users[k] = 0;
      slot_loads[k] = 0;
    }
    *slot_lock = 0;
  }
  if (r == 0) ptx::fence_mbar_init();
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), 512);
    ptx::tmem_relinquish();
  }
  if (tid < 128) {
    ptx::st_shared_v4(aConst + tid * 16, 0x3C00u, 0u, 0u, 0u);
    ptx::st_shared_v4(aConst + 2048 + tid * 16, 0u, 0u, 0u, 0u);
  }
  ptx::fence_proxy_async();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tB = tmem + wg * C::COLS;                      // MMA addresses (lane 0)
  const uint32_t tBl = tB + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lanes

  int64_t ntiles = L.chunks ? (int64_t)L.n_chunks : (L.n + 127) / 128;
  if (L.n_chunks_dev) {
    const int64_t d = *L.n_chunks_dev;  // written by an earlier launch on this stream
    ntiles = d < 0 ? 0 : d < ntiles ? d : ntiles;
  }
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t c_begin = (int64_t)blockIdx.x * per;
  const int64_t c_end = c_begin + per < ntiles ? c_begin + per : ntiles;

  uint32_t ph_m = 0;
  bool bad = false, mma_pending = false, w_pending = false;
  int cur_mat = -1, my_slot = -1;
  const bool cosine = (L.flags & NAM_OUT_COSINE) != 0;

  // single material: one copy of the weights for the whole CTA
  if (!MULTI) {
    if (tid == 0 && c_begin < c_end) {
      ptx::fence_proxy_async();
      ptx::mbar_arrive_expect_tx(bar_w, Y.BYTES);
      ptx::bulk_g2s(aW, L.w0, Y.BYTES, bar_w);
      w_pending = true;  // drained by thread 0 at teardown if needed
    }
  }

  constexpr uint32_t ID16 = ptx::idesc_f16(128, 16);
  constexpr uint32_t ID_H = ptx::idesc_f16(128, H);
  constexpr uint32_t ID_N1 = ptx::idesc_f16(128, Y.N1);

  // Make this warpgroup's TMEM writes visible to the tensor core, agree on
  // the error state, let one thread issue `issue` and commit it.  False (for
  // every thread of the warpgroup) if a wait of any thread ran out.
  auto stage_issue = [&](auto issue) -> bool {
    ptx::tmem_st_wait();
    ptx::tc_fence_before();
    if (ptx::bar_red_or(bar_id, 128, bad)) {
      bad = true;  // some thread's wait ran out: the whole warpgroup stops
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

  // the query behind row k of the chunk table (binned launches read the
  // caller's arrays through the binning permutation)
  auto src = [&](int64_t k) -> int64_t {
    if constexpr (MULTI) {
      if (L.gather) return (int64_t)__ldg(L.gather + k);
    }
    return k;
  };
  auto pyr_for = [&](const TileRef& t) -> const uint8_t* {
    return reinterpret_cast<const uint8_t*>(MULTI ? L.mats.pyramid[t.mat] : L.pyr0);
  };

  int64_t c = c_begin + wg;
  TileRef cur{}, nxt{};
  QF q_nxt{};
  // single-material launches filter the next tile while the output MMA runs
  // (mixed-material launches, short of registers, filter at the tile's start)
  constexpr bool SHADOW = F16P && !MULTI;
  float zr[8];  // filtered latent of the tile about to start (SHADOW)
  if (c < c_end) {
    cur = tile_at(L, c);
    if (F16P && cur.count > 0) {
      const QF q0 = load_qf(L.q, src(cur.start + (r < cur.count ? r : 0)));
      fetch_issue(L.pyr, pyr_for(cur), q0, stg);
      if (SHADOW) fetch_finish(stg, zr);
    }
    if (c + NWG < c_end) {
      nxt = tile_at(L, c + NWG);
      if (nxt.count > 0) q_nxt = load_qf(L.q, src(nxt.start + (r < nxt.count ? r : 0)));
    }
  }
  for (; c < c_end; c += NWG) {
    const bool has_next = c + NWG < c_end;
    const bool has_next2 = c + 2 * NWG < c_end;
    TileRef nxt2{};
    QF q_nxt2{};
    if (cur.count <= 0) {
      // an empty slot of a chunk table (count is uniform over the warpgroup)
      if (F16P && has_next && nxt.count > 0) {
        fetch_issue(L.pyr, pyr_for(nxt), q_nxt, stg);
        if (SHADOW) fetch_finish(stg, zr);
      }
      if (has_next2) {
        nxt2 = tile_at(L, c + 2 * NWG);
        if (nxt2.count > 0) q_nxt2 = load_qf(L.q, src(nxt2.start + (r < nxt2.count ? r : 0)));
      }
      cur = nxt;
      nxt = nxt2;
      q_nxt = q_nxt2;
      continue;
    }
    const bool valid = r < cur.count;
    const int64_t i = src(cur.start + (valid ? r : 0));
    // directions (used after the frame stages) and the masked-pass material
    // (issued here, ahead of the fetch and MMA 1, and kept here: a load the
    // compiler sinks to its first use would expose its full latency)
    const float wix = ptx::ld_nc_pinned(L.q.wix + i), wiy = ptx::ld_nc_pinned(L.q.wiy + i);
    const float wiz = ptx::ld_nc_pinned(L.q.wiz + i), wox = ptx::ld_nc_pinned(L.q.wox + i);
    const float woy = ptx::ld_nc_pinned(L.q.woy + i), woz = ptx::ld_nc_pinned(L.q.woz + i);
    const int32_t row_mat = L.row_ids ? __ldg(L.row_ids + i) : cur.mat;

    // weights: the CTA's copy (single material), or this warpgroup's,
    // restaged when the material changes (no MMA of the warpgroup in flight)
    if (MULTI) {
      if (cur.mat != cur_mat) {
        // no MMA of this warpgroup is in flight: its leader gives up its
        // slot and takes one holding the tile's material, or loads the
        // material into a slot no warpgroup uses (waiting, with the time
        // limit, while every slot is in use)
        if (ptx::bar_red_or(bar_id, 128, bad)) {
          bad = true;
          break;
        }
        if (r == 0) {
          const uint64_t t0 = ptx::globaltimer();
          int sl = -1, gen = 0;
          bool load = false, ok = smem_lock(slot_lock, t0, L.timeout_ns);
          if (ok && my_slot >= 0) slot_users[my_slot] = slot_users[my_slot] - 1;
          while (ok) {
            for (int k = 0; k < S::SLOTS && sl < 0; ++k)
              if (slot_mat[k] == cur.mat) {
                sl = k;
                slot_users[k] = slot_users[k] + 1;
                gen = slot_loads[k];
              }
            for (int k = 0; k < S::SLOTS && sl < 0; ++k)
              if (slot_users[k] == 0) {
                sl = k;
                load = true;
                slot_mat[k] = cur.mat;
                slot_users[k] = 1;
                gen = slot_loads[k] + 1;
                slot_loads[k] = gen;
              }
            smem_unlock(slot_lock);
            if (sl >= 0) break;
            __nanosleep(256);
            ok = smem_lock(slot_lock, t0, L.timeout_ns);
          }
          if (load) {
            const uint32_t bar = ptx::smem_u32(&bars[NWG + sl]);
            ptx::fence_proxy_async();
            ptx::mbar_arrive_expect_tx(bar, Y.BYTES);
            ptx::bulk_g2s(ptx::smem_u32(smem + S::W_OFF + sl * S::BLOB_AL), L.mats.weights[cur.mat], Y.BYTES,
                          bar);
          }
          wg_word[wg] = sl >= 0 ? (sl | (gen << 8)) : -1;
          my_slot = sl;
        }
        // broadcast the slot (a failed acquire stops the warpgroup)
        if (ptx::bar_red_or(bar_id, 128, false)) {
          bad = true;
          break;
        }
        const int word = wg_word[wg];
        if (word < 0) {
          bad = true;
          break;
        }
        const int sl = word & 0xFF, gen = word >> 8;
        aW = ptx::smem_u32(smem + S::W_OFF + sl * S::BLOB_AL);
        bad |= !ptx::mbar_wait(ptx::smem_u32(&bars[NWG + sl]), (uint32_t)(gen - 1) & 1u, L.timeout_ns);
        cur_mat = cur.mat;
      }
    } else if (cur_mat < 0) {
      bad |= !ptx::mbar_wait(bar_w, 0, L.timeout_ns);
      if (!bad && tid == 0) w_pending = false;
      cur_mat = 0;
    }

    // ---- 1. latent z, split into FP16 halves -> MMA 1 ---------------------
    float z[8];
    if (SHADOW) {
      // filtered while the previous tile's output MMA ran
#pragma unroll
      for (int k = 0; k < 8; ++k) z[k] = zr[k];
    } else if (F16P) {
      fetch_finish(stg, z);
    } else {
      QF q0 = load_qf(L.q, i);
      fetch_latent<false>(L.pyr, pyr_for(cur), q0.u, q0.v, q0.lod, q0.xi, z);
    }
    {
      uint32_t v[8];
      split_pair<false>(z[0], z[1], v[0], v[4]);
      split_pair<false>(z[2], z[3], v[1], v[5]);
      split_pair<false>(z[4], z[5], v[2], v[6]);
      split_pair<false>(z[6], z[7], v[3], v[7]);
      ptx::tmem_st8(tBl + C::A + 8, v);  // (z hi, z lo)
    }
    if (!stage_issue([&] {
          ptx::mma_f16_ts(tB + C::D, tB + C::A + 8, ptx::sdesc(aW + Y.B1, Y.N1 * 16, 128), ID_N1, 0);
          if (FK)
            ptx::mma_f16(tB + C::F, ptx::sdesc(aConst, 2048, 128), ptx::sdesc(aW + Y.B1B, 256, 128), ID16, 1);
        }))
      break;

    // ---- the next tile's texel gathers, while MMA 1 runs ----------------
    if (F16P && has_next && nxt.count > 0) fetch_issue(L.pyr, pyr_for(nxt), q_nxt, stg);
    if (has_next2) {
      nxt2 = tile_at(L, c + 2 * NWG);
      if (nxt2.count > 0) q_nxt2 = load_qf(L.q, src(nxt2.start + (r < nxt2.count ? r : 0)));
    }
    stage_wait();

    // ---- 2.-3. frame, transformed directions -> MMA 3 -------------------
    float d[12];
    if (FK == 1) {
      {
        uint32_t acc[16];
        ptx::tmem_ld16(tBl + C::F, acc);
        ptx::tmem_ld_wait();
        uint32_t v[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) split_pair<true>(f32_of(acc[2 * j]), f32_of(acc[2 * j + 1]), v[j], v[8 + j]);
        ptx::tmem_st16(tBl + C::A, v);  // (h hi, h lo)
      }
      if (!stage_issue([&] {
            ptx::mma_f16_ts(tB + C::F, tB + C::A, ptx::sdesc(aW + Y.BF2, 256, 128), ID16, 0);
            ptx::mma_f16_ts(tB + C::F, tB + C::A + 8, ptx::sdesc(aW + Y.BF2 + 512, 256, 128), ID16, 1);
          }))
        break;
      stage_wait();
      uint32_t acc[8];
      ptx::tmem_ld8(tBl + C::F, acc);
      ptx::tmem_ld_wait();
      const uint4 b0 = ptx::ld_shared_v4(aW + Y.SB + 64), b1 = ptx::ld_shared_v4(aW + Y.SB + 80);
      const float rr[6] = {f32_of(acc[0]) + f32_of(b0.x), f32_of(acc[1]) + f32_of(b0.y), f32_of(acc[2]) + f32_of(b0.z),
                           f32_of(acc[3]) + f32_of(b0.w), f32_of(acc[4]) + f32_of(b1.x), f32_of(acc[5]) + f32_of(b1.y)};
      const Frame F = build_frame(rr);
      to_local(F, wix, wiy, wiz, d);
      to_local(F, wox, woy, woz, d + 3);
    } else if (FK == 2) {
      uint32_t acc[16];
      ptx::tmem_ld16(tBl + C::F, acc);
      ptx::tmem_ld_wait();
      float rr[12];
#pragma unroll
      for (int j = 0; j < 12; ++j) rr[j] = f32_of(acc[j]);
      const Frame F1 = paper_frame(rr), F2 = paper_frame(rr + 6);
      to_local(F1, wix, wiy, wiz, d);
      to_local(F2, wix, wiy, wiz, d + 3);
      to_local(F1, wox, woy, woz, d + 6);
      to_local(F2, wox, woy, woz, d + 9);
    } else {
      d[0] = wix; d[1] = wiy; d[2] = wiz;
      d[3] = wox; d[4] = woy; d[5] = woz;
    }
    {
      // (d hi, d lo, 1, 0 ...): the 1 meets layer 1's bias column
      if (ND == 6) {
        uint32_t v[8];
        split_pair<false>(d[0], d[1], v[0], v[3]);
        split_pair<false>(d[2], d[3], v[1], v[4]);
        split_pair<false>(d[4], d[5], v[2], v[5]);
        v[6] = 0x00003C00u;
        v[7] = 0u;
        ptx::tmem_st8(tBl + C::A + 8, v);
      } else {
        uint32_t v[16];
#pragma unroll
        for (int j = 0; j < 6; ++j) split_pair<false>(d[2 * j], d[2 * j + 1], v[j], v[6 + j]);
        v[12] = 0x00003C00u;
        v[13] = v[14] = v[15] = 0u;
        ptx::tmem_st16(tBl + C::A, v);
      }
    }
    if (!stage_issue([&] {
          if (ND == 6) {
            ptx::mma_f16_ts(tB + C::D, tB + C::A + 8, ptx::sdesc(aW + Y.BD, H * 16, 128), ID_H, 1);
          } else {
            ptx::mma_f16_ts(tB + C::D, tB + C::A, ptx::sdesc(aW + Y.BD, H * 16, 128), ID_H, 1);
            ptx::mma_f16_ts(tB + C::D, tB + C::A + 8, ptx::sdesc(aW + Y.BD + 2 * H * 16, H * 16, 128), ID_H, 1);
          }
        }))
      break;
    stage_wait();

    // ---- 4. hidden layers: ReLU, FP16 -> next layer ----------------------
    // H = 64: rounded to FP16 once; narrower decoders, where one rounded
    // layer already takes a large share of the FP16 error budget, keep (hi,
    // lo) halves here too (lo in the operand columns [H + 16, H + 16 + H/2)).
    // FP8 (P8): each hidden -> hidden layer has E4M3 weights (codes of
    // W / s_w); its input x enters as two E4M3 code sets of x / s_a, hi =
    // E4M3(x / s_a) and lo = E4M3(x / s_a - hi), in [H, H + H/4) and
    // [H + H/4, H + H/2) (four codes per column), so that the accumulator
    // holds sum (hi + lo) code_w = (pre-activation - b) / c, c = s_a s_w; the
    // next epilogue restores c D + b in FP32.
    constexpr bool SPLIT_HID = H < 64 && !P8;
    constexpr int NC = H < 32 ? H : 32;
    constexpr uint32_t ID8_H = ptx::idesc_e4m3(128, H);
    bool ok = true;
    // (multiplier, bias) that turn the accumulator into the pre-activation
    // of the layer that wrote it: (1, 0) after an FP16 layer (bias in the MMA)
    float pre_c = 1.0f;
    uint32_t pre_b = 0;  // shared-memory address of the FP32 bias, 0: none
#pragma unroll
    for (int layer = 0; layer < NH - 1; ++layer) {
      const int boff = Y.BH + layer * H * (H + 16) * 2;
      if constexpr (P8) {
        const float inv_sa = reinterpret_cast<const float*>(smem + (aW - aConst) + Y.SB)[2 * layer];
#pragma unroll
        for (int c0 = 0; c0 < H; c0 += 16) {
          uint32_t acc[16];
          ptx::tmem_ld16(tBl + C::D + c0, acc);
          ptx::tmem_ld_wait();
          float t[16];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 b = pre_b ? ptx::ld_shared_v4(pre_b + 4 * (c0 + 4 * q)) : make_uint4(0u, 0u, 0u, 0u);
            const float2 t01 = ptx::fma2(make_float2(f32_of(acc[4 * q]), f32_of(acc[4 * q + 1])),
                                         make_float2(pre_c, pre_c), make_float2(f32_of(b.x), f32_of(b.y)));
            const float2 t23 = ptx::fma2(make_float2(f32_of(acc[4 * q + 2]), f32_of(acc[4 * q + 3])),
                                         make_float2(pre_c, pre_c), make_float2(f32_of(b.z), f32_of(b.w)));
            t[4 * q] = fmaxf(t01.x, 0.0f) * inv_sa;
            t[4 * q + 1] = fmaxf(t01.y, 0.0f) * inv_sa;
            t[4 * q + 2] = fmaxf(t23.x, 0.0f) * inv_sa;
            t[4 * q + 3] = fmaxf(t23.y, 0.0f) * inv_sa;
          }
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t h2[2], l2[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float x0 = t[4 * q + 2 * e], x1 = t[4 * q + 2 * e + 1];
              h2[e] = ptx::pack_e4m3x2(x0, x1);
              const float2 hv = ptx::unpack_e4m3x2(h2[e]);
              const float2 d = ptx::sub2(make_float2(x0, x1), hv);
              l2[e] = ptx::pack_e4m3x2(d.x, d.y);
            }
            hi[q] = h2[0] | (h2[1] << 16);
            lo[q] = l2[0] | (l2[1] << 16);
          }
          ptx::tmem_st4(tBl + C::HID + c0 / 4, hi);
          ptx::tmem_st4(tBl + C::HID + H / 4 + c0 / 4, lo);
        }
        if (!stage_issue([&] {
#pragma unroll
              for (int s = 0; s < (2 * H) / 32; ++s)
                ptx::mma_f8_ts(tB + C::D, tB + C::HID + 8 * s, ptx::sdesc(aW + boff + s * 2 * H * 16, H * 16, 128),
                               ID8_H, s > 0 ? 1u : 0u);
            })) {
          ok = false;
          break;
        }
        pre_c = reinterpret_cast<const float*>(smem + (aW - aConst) + Y.SB)[2 * layer + 1];
        pre_b = aW + boff + 2 * H * H;
      } else if constexpr (SPLIT_HID) {
#pragma unroll
        for (int c0 = 0; c0 < H; c0 += 16) {
          uint32_t acc[16];
          ptx::tmem_ld16(tBl + C::D + c0, acc);
          ptx::tmem_ld_wait();
          uint32_t hi[8], lo[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) split_pair<true>(f32_of(acc[2 * j]), f32_of(acc[2 * j + 1]), hi[j], lo[j]);
          ptx::tmem_st8(tBl + C::HID + c0 / 2, hi);
          ptx::tmem_st8(tBl + C::A + c0 / 2, lo);
        }
      } else {
#pragma unroll
        for (int c0 = 0; c0 < H; c0 += NC) {
          uint32_t acc[NC];
          if constexpr (NC == 32) ptx::tmem_ld32(tBl + C::D + c0, acc);
          else ptx::tmem_ld16(tBl + C::D + c0, acc);
          ptx::tmem_ld_wait();
          uint32_t pk[NC / 2];
#pragma unroll
          for (int j = 0; j < NC / 2; ++j) pk[j] = ptx::pack_h2_relu(f32_of(acc[2 * j]), f32_of(acc[2 * j + 1]));
          if constexpr (NC == 32) ptx::tmem_st16(tBl + C::HID + c0 / 2, pk);
          else ptx::tmem_st8(tBl + C::HID + c0 / 2, pk);
        }
      }
      if constexpr (!P8) {
        if (!stage_issue([&] {
#pragma unroll
              for (int s = 0; s < H / 16; ++s)
                ptx::mma_f16_ts(tB + C::D, tB + C::HID + 8 * s, ptx::sdesc(aW + boff + s * 2 * H * 16, H * 16, 128),
                                ID_H, s > 0 ? 1u : 0u);
              if constexpr (SPLIT_HID) {
#pragma unroll
                for (int s = 0; s < H / 16; ++s)
                  ptx::mma_f16_ts(tB + C::D, tB + C::A + 8 * s, ptx::sdesc(aW + boff + s * 2 * H * 16, H * 16, 128),
                                  ID_H, 1u);
              }
              ptx::mma_f16(tB + C::D, ptx::sdesc(aConst, 2048, 128),
                           ptx::sdesc(aW + boff + (H / 8) * H * 16, H * 16, 128), ID_H, 1u);
            })) {
          ok = false;
          break;
        }
      }
      stage_wait();
    }
    if (!ok) break;

    // ---- 5. last hidden layer as (hi, lo) FP16 halves -> output layer ------
#pragma unroll
    for (int c0 = 0; c0 < H; c0 += 16) {
      uint32_t acc[16];
      ptx::tmem_ld16(tBl + C::D + c0, acc);
      ptx::tmem_ld_wait();
      if constexpr (P8) {
        // the last hidden layer was an E4M3 layer: pre-activation = c D + b
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 b = ptx::ld_shared_v4(pre_b + 4 * (c0 + 4 * q));
          const float2 t01 = ptx::fma2(make_float2(f32_of(acc[4 * q]), f32_of(acc[4 * q + 1])),
                                       make_float2(pre_c, pre_c), make_float2(f32_of(b.x), f32_of(b.y)));
          const float2 t23 = ptx::fma2(make_float2(f32_of(acc[4 * q + 2]), f32_of(acc[4 * q + 3])),
                                       make_float2(pre_c, pre_c), make_float2(f32_of(b.z), f32_of(b.w)));
          acc[4 * q] = __float_as_uint(t01.x);
          acc[4 * q + 1] = __float_as_uint(t01.y);
          acc[4 * q + 2] = __float_as_uint(t23.x);
          acc[4 * q + 3] = __float_as_uint(t23.y);
        }
      }
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) split_pair<true>(f32_of(acc[2 * j]), f32_of(acc[2 * j + 1]), hi[j], lo[j]);
      // lo overwrites columns [c0/2, c0/2 + 8) of the accumulator, already read
      ptx::tmem_st8(tBl + C::HID + c0 / 2, hi);
      ptx::tmem_st8(tBl + C::LO + c0 / 2, lo);
    }
    if (!stage_issue([&] {
#pragma unroll
          for (int s = 0; s < H / 16; ++s)
            ptx::mma_f16_ts(tB + C::OUT, tB + C::HID + 8 * s, ptx::sdesc(aW + Y.BO + s * 512, 256, 128), ID16,
                            s > 0 ? 1u : 0u);
#pragma unroll
          for (int s = 0; s < H / 16; ++s)
            ptx::mma_f16_ts(tB + C::OUT, tB + C::LO + 8 * s, ptx::sdesc(aW + Y.BO + s * 512, 256, 128), ID16, 1u);
        }))
      break;
    // the next tile's filter, while the output MMA runs
    if (SHADOW && has_next && nxt.count > 0) fetch_finish(stg, zr);
    stage_wait();

    // ---- output ---------------------------------------------------------------
    {
      uint32_t acc[4];
      ptx::tmem_ld4(tBl + C::OUT, acc);
      ptx::tmem_ld_wait();
      const uint4 bo = ptx::ld_shared_v4(aW + Y.SB + 96);  // output bias
      float y0 = f32_of(acc[0]) + f32_of(bo.x), y1 = f32_of(acc[1]) + f32_of(bo.y),
            y2 = f32_of(acc[2]) + f32_of(bo.z);
      const bool store = valid && row_mat == cur.mat;
      if (L.albedo) {
        // albedo head: output columns 3..5 (no cosine factor)
        uint32_t acc2[4];
        ptx::tmem_ld4(tBl + C::OUT + 4, acc2);
        ptx::tmem_ld_wait();
        const uint4 bo2 = ptx::ld_shared_v4(aW + Y.SB + 112);
        if (store) {
          L.albedo[3 * i + 0] = f32_of(acc[3]) + f32_of(bo.w);
          L.albedo[3 * i + 1] = f32_of(acc2[0]) + f32_of(bo2.x);
          L.albedo[3 * i + 2] = f32_of(acc2[1]) + f32_of(bo2.y);
        }
      }
      if (cosine) {
        const float cz = fmaxf(wiz, 0.0f);
        y0 *= cz;
        y1 *= cz;
        y2 *= cz;
      }
      if (store) {
        L.rgb[3 * i + 0] = y0;
        L.rgb[3 * i + 1] = y1;
        L.rgb[3 * i + 2] = y2;
      }
    }
    ptx::tc_fence_before();
    cur = nxt;
    nxt = nxt2;
    q_nxt = q_nxt2;
  }

  // ---- teardown -------------------------------------------------------------
  // No cp.async may land in shared memory after the CTA exits; MMAs and bulk
  // copies still in flight after a wait gave up are waited for with the fixed
  // drain limit, and TMEM is freed only if they all completed.
  // a warpgroup leaving its loop gives up its weight slot
  if (MULTI && r == 0 && my_slot >= 0 && smem_lock(slot_lock, ptx::globaltimer(), L.timeout_ns)) {
    slot_users[my_slot] = slot_users[my_slot] - 1;
    smem_unlock(slot_lock);
  }
  ptx::cp_async_wait_all();
  bool drained = true;
  if (r == 0 && mma_pending) drained &= ptx::mbar_wait(bar_m, ph_m ^ 1, ptx::kDrainTimeoutNs);
  if (!MULTI && tid == 0 && w_pending) drained &= ptx::mbar_wait(bar_w, 0, ptx::kDrainTimeoutNs);
  if (MULTI) {
    __syncthreads();  // every warpgroup has left its loop: no slot is loaded after this
    if (tid == 0)
      for (int k = 0; k < S::SLOTS; ++k)
        if (slot_loads[k] > 0)
          drained &= ptx::mbar_wait(ptx::smem_u32(&bars[NWG + k]), (uint32_t)(slot_loads[k] - 1) & 1u,
                                    ptx::kDrainTimeoutNs);
  }
  if (bad) record_error(L.err, DEVERR_WAIT_TIMEOUT);
  if (!drained) record_error(L.err, DEVERR_DRAIN_TIMEOUT);
  ptx::tc_fence_before();
  const bool all_drained = __syncthreads_and(drained ? 1 : 0) != 0;
  if (warp == 0 && all_drained) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------
// Warpgroups per CTA (one CTA per SM): 640 threads at <= 96 registers; TMEM
// 5 x (H + 32) <= 480 of 512 columns.
constexpr int kF16Nwg = 5;

template <int H, int FK, int NH, bool F16P, bool MULTI>
constexpr int f16_nwg() {
  // five warpgroups where the shared memory allows (the largest blobs with
  // their staging leave room for four)
  return F16Smem<H, FK, NH, F16P, MULTI, kF16Nwg>::BYTES <= 227 * 1024 ? kF16Nwg : kF16Nwg - 1;
}

template <int H, int FK, int NH, bool F16P, bool MULTI, bool P8>
static int launch_f16_one(const LaunchCommon& L, cudaStream_t s) {
  constexpr int NWG = f16_nwg<H, FK, NH, F16P, MULTI>();
  using S = F16Smem<H, FK, NH, F16P, MULTI, NWG>;
  static_assert(S::BYTES <= 227 * 1024, "shared memory");
  static_assert(NWG * F16Cols<H>::COLS <= 512, "TMEM columns");
  auto k = eval_f16_kernel<H, FK, NH, F16P, MULTI, NWG, P8>;
  static std::atomic<uint64_t> configured{0};
  once_per_device(configured, [&] {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
    // the smallest carveout that holds the CTA: the rest of the SM's
    // L1/shared storage caches the texel gathers
    const int pct = (S::BYTES + 1024) * 100 / (228 * 1024) + 1;
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  });
  const int64_t ntiles = L.chunks ? (int64_t)L.n_chunks : (L.n + 127) / 128;
  if (ntiles == 0) return 0;
  const int64_t want = (ntiles + NWG - 1) / NWG;
  const int grid = (int)(want < L.num_sms ? want : L.num_sms);
  k<<<grid, NWG * 128, S::BYTES, s>>>(L);
  return (int)cudaGetLastError();
}

template <int H, int FK, int NH, bool P8>
static int f16_pick(const LaunchCommon& L, cudaStream_t s) {
  const bool f16 = L.pyr.f16 != 0, multi = L.chunks != nullptr;
  if (f16)
    return multi ? launch_f16_one<H, FK, NH, true, true, P8>(L, s) : launch_f16_one<H, FK, NH, true, false, P8>(L, s);
  return multi ? launch_f16_one<H, FK, NH, false, true, P8>(L, s) : launch_f16_one<H, FK, NH, false, false, P8>(L, s);
}

template <int H, int NH, bool P8>
static int f16_frame(const LaunchCommon& L, cudaStream_t s) {
  switch (L.shape.frame) {
    case 0: return f16_pick<H, 0, NH, P8>(L, s);
    case 1: return f16_pick<H, 1, NH, P8>(L, s);
    case 2: return f16_pick<H, 2, NH, P8>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace nam
