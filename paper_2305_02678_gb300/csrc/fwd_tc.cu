// Tensor-core evaluation of the neural BRDF on sm_103a (tcgen05 + TMEM).
//
// One CTA of 128 threads owns a tile of up to 128 queries at a time; thread r
// is query r of the tile and TMEM lane r.  Per tile:
//   1. coalesced planar query loads, latent fetch (16-byte texel gathers,
//      FP32 filter) -> z                                     (Sec. 4.1)
//   2. frame MLP 8 -> 16 -> 6 on the tensor core with each FP16 operand
//      split into a high and a low half (z = z_hi + z_lo), so the frame has
//      FP32 accuracy; FP32 bias + ReLU between the layers    (Sec. 4.2)
//   3. frame build (Gram-Schmidt, b = n x t) and the direction transform in
//      FP32 registers: each thread holds its own query's TMEM row, so the
//      six frame outputs need no cross-lane exchange          (Eq. 4)
//   4. decoder layers 14 -> H -> H -> 3: FP16 operands, FP32 accumulation in
//      TMEM; the bias rides in the MMA as a constant-1 input column; ReLU and
//      the FP16 rounding of the next layer's operand are one cvt.relu.f16x2
//   5. RGB store (x max(0, wi.z) if requested)
// MLP weights (and the frame biases) are staged once per CTA, or again when a
// multi-material launch switches material, with one bulk TMA copy of a blob
// that the host laid out in the MMA operand order at material creation.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nam {

// ---------------------------------------------------------------------------
// layouts
// ---------------------------------------------------------------------------
// Canonical no-swizzle K-major FP16 layout of an R x K operand: element
// (row, k) at byte (k / 8) * (R * 16) + row * 16 + (k % 8) * 2, i.e. 8-row x
// 16-byte core matrices, LBO = R * 16 (next core matrix along K), SBO = 128
// (next 8 rows).
__host__ __device__ constexpr int kmajor_off(int R, int row, int k) {
  return (k / 8) * (R * 16) + row * 16 + (k % 8) * 2;
}

template <int H, bool FRAME>
struct TcLayout {
  // A operand blocks (128 rows x 8 fp16 each): data blocks [0, KB), then a
  // block whose first column is 1.0 (bias input) and an all-zero block.
  static constexpr int KB = (H / 8) > 4 ? (H / 8) : 4;
  static constexpr int A_BYTES = (KB + 2) * 2048;
  // weight blob: every bias rides in the MMA as the weight of the constant-1
  // input column (one extra K step of 16)
  static constexpr int B_F1 = 0;                          // 16 x 32: [Wf1 | Wf1 | bf1 0..]
  static constexpr int B_F2 = FRAME ? 1024 : 0;           // 16 x 48: [Wf2 | Wf2 | bf2 0..]
  static constexpr int B_L1 = FRAME ? 2560 : 0;           // H x 16: [W1 | b1 0]
  static constexpr int B_L2 = B_L1 + H * 16 * 2;          // H x (H + 16)
  static constexpr int B_LO = B_L2 + H * (H + 16) * 2;    // 16 x (H + 16)
  static constexpr int BLOB = B_LO + 16 * (H + 16) * 2;
  static constexpr int BLOB_ALIGNED = (BLOB + 127) / 128 * 128;
  static constexpr int SMEM = BLOB_ALIGNED + A_BYTES + 64;
};

size_t tc_blob_bytes(const Shape& s, int precision) {
  if (precision != NAM_PREC_F16 || s.NH != 2) return 0;
  if (s.frame) {
    if (s.H == 16) return TcLayout<16, true>::BLOB;
    if (s.H == 32) return TcLayout<32, true>::BLOB;
    if (s.H == 64) return TcLayout<64, true>::BLOB;
  } else {
    if (s.H == 16) return TcLayout<16, false>::BLOB;
    if (s.H == 32) return TcLayout<32, false>::BLOB;
    if (s.H == 64) return TcLayout<64, false>::BLOB;
  }
  return 0;
}

static void put_h(uint8_t* base, int R, int row, int k, float v) {
  __half h = __float2half_rn(v);
  std::memcpy(base + kmajor_off(R, row, k), &h, 2);
}

// Lay out the FP16-quantised weights as MMA B operands (N rows = outputs,
// K = inputs, K-major), each layer's bias in the extra input column that
// meets the constant-1 column of the A operand.  The frame layers take their
// FP16 operand in two halves (high part, residual), so their weights appear
// twice along K.
int pack_tc_blob(const Shape& s, int precision, const float* frame, const float* dec, const float* /*act_scale*/,
                 uint8_t* out, float* /*weight_scales_out*/) {
  if (precision != NAM_PREC_F16) return -1;
  const size_t bytes = tc_blob_bytes(s, precision);
  if (!bytes) return -1;
  std::memset(out, 0, bytes);
  const int H = s.H;
  const int B_L1 = s.frame ? 2560 : 0;
  const int B_L2 = B_L1 + H * 16 * 2;
  const int B_LO = B_L2 + H * (H + 16) * 2;
  if (s.frame) {
    const float* Wf1 = frame;            // [16][8]
    const float* bf1 = Wf1 + 128;        // [16]
    const float* Wf2 = bf1 + 16;         // [6][16]
    const float* bf2 = Wf2 + 96;         // [6]
    for (int n = 0; n < 16; ++n) {
      for (int k = 0; k < 16; ++k) put_h(out + 0, 16, n, k, Wf1[n * 8 + (k & 7)]);
      put_h(out + 0, 16, n, 16, bf1[n]);
    }
    for (int n = 0; n < 6; ++n) {
      for (int k = 0; k < 32; ++k) put_h(out + 1024, 16, n, k, Wf2[n * 16 + (k & 15)]);
      put_h(out + 1024, 16, n, 32, bf2[n]);
    }
  }
  const float* W1 = dec;                 // [H][14]
  const float* b1 = W1 + 14 * H;
  const float* W2 = b1 + H;              // [H][H]
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;              // [3][H]
  const float* b3 = W3 + 3 * H;
  for (int n = 0; n < H; ++n) {
    for (int k = 0; k < 14; ++k) put_h(out + B_L1, H, n, k, W1[n * 14 + k]);
    put_h(out + B_L1, H, n, 14, b1[n]);
  }
  for (int n = 0; n < H; ++n) {
    for (int k = 0; k < H; ++k) put_h(out + B_L2, H, n, k, W2[n * H + k]);
    put_h(out + B_L2, H, n, H, b2[n]);
  }
  for (int n = 0; n < 3; ++n) {
    for (int k = 0; k < H; ++k) put_h(out + B_LO, 16, n, k, W3[n * H + k]);
    put_h(out + B_LO, 16, n, H, b3[n]);
  }
  return 0;
}

// ---------------------------------------------------------------------------
// kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ float u2f(uint32_t x) { return __uint_as_float(x); }

// Split two FP32 values into binary16 high parts and binary16 residuals.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  hi = ptx::pack_h2(a, b);
  __half2 h = *reinterpret_cast<__half2*>(&hi);
  float2 f = __half22float2(h);
  lo = ptx::pack_h2(a - f.x, b - f.y);
}

// One query's inputs, loaded a tile ahead of its use.
struct QueryIn {
  float u, v, lod, xi, wix, wiy, wiz, wox, woy, woz;
};
struct ChunkIn {
  int64_t start;
  int count, mat;
};

__device__ __forceinline__ ChunkIn chunk_at(const LaunchCommon& L, int64_t c) {
  ChunkIn ci;
  if (L.chunks) {
    const Chunk ch = L.chunks[c];
    ci.start = ch.start;
    ci.count = ch.count;
    ci.mat = ch.material;
  } else {
    ci.start = c * 128;
    ci.count = (int)((L.n - ci.start) < 128 ? (L.n - ci.start) : 128);
    ci.mat = 0;
  }
  return ci;
}

__device__ __forceinline__ QueryIn load_query(const QueryPtrs& q, int64_t i) {
  QueryIn x;
  x.u = __ldg(q.u + i);
  x.v = __ldg(q.v + i);
  x.lod = __ldg(q.lod + i);
  x.xi = q.xi ? __ldg(q.xi + i) : 0.0f;
  x.wix = __ldg(q.wix + i);
  x.wiy = __ldg(q.wiy + i);
  x.wiz = __ldg(q.wiz + i);
  x.wox = __ldg(q.wox + i);
  x.woy = __ldg(q.woy + i);
  x.woz = __ldg(q.woz + i);
  return x;
}

template <int H, bool FRAME, bool F16P>
__global__ void __launch_bounds__(128, 4) eval_tc_kernel(const LaunchCommon L) {
  using Lay = TcLayout<H, FRAME>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sW = smem;
  uint8_t* sA = smem + Lay::BLOB_ALIGNED;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + Lay::A_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);

  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t bar_w = ptx::smem_u32(&bars[0]);
  const uint32_t bar_m = ptx::smem_u32(&bars[1]);
  const uint32_t aW = ptx::smem_u32(sW);
  const uint32_t aA = ptx::smem_u32(sA);
  const uint32_t aConst = aA + Lay::KB * 2048;  // (1, 0, ...) | 0 blocks

  if (tid == 0) {
    ptx::mbar_init(bar_w, 1);
    ptx::mbar_init(bar_m, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), 64);
    ptx::tmem_relinquish();
  }
  ptx::st_shared_v4(aConst + tid * 16, 0x3C00u, 0u, 0u, 0u);
  ptx::st_shared_v4(aConst + 2048 + tid * 16, 0u, 0u, 0u, 0u);
  ptx::fence_proxy_async();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);

  const int64_t nchunks = L.chunks ? (int64_t)L.n_chunks : (L.n + 127) / 128;
  const int64_t per = (nchunks + gridDim.x - 1) / gridDim.x;
  const int64_t c_begin = (int64_t)blockIdx.x * per;
  const int64_t c_end = c_begin + per < nchunks ? c_begin + per : nchunks;

  uint32_t ph_w = 0, ph_m = 0;
  bool bad = false, mma_pending = false, w_pending = false;
  int cur_mat = -1;
  const void* pyr = L.pyr0;
  const bool cosine = (L.flags & NAM_OUT_COSINE) != 0;
  const int r = tid;

  constexpr uint32_t ID_16 = ptx::idesc_f16(128, 16);
  constexpr uint32_t ID_H = ptx::idesc_f16(128, H);

  // make this thread's A-operand writes visible to the tensor core, sync the
  // CTA, let one thread issue `issue`, wait for completion.  Returns false
  // (for every thread) if any thread's wait ran out.
  auto mma_stage = [&](auto issue) -> bool {
    ptx::fence_proxy_async();
    ptx::tc_fence_before();
    if (__syncthreads_or(bad)) return false;
    if (tid == 0) {
      ptx::tc_fence_after();
      issue();
      ptx::mma_commit(bar_m);
    }
    mma_pending = true;
    bad |= !ptx::mbar_wait(bar_m, ph_m, L.timeout_ns);
    ph_m ^= 1;
    if (!bad) mma_pending = false;
    ptx::tc_fence_after();
    return true;
  };

  ChunkIn ci{};
  QueryIn qc{};
  Taps8 tc{};  // texels of the current tile (FP16 pyramids), loaded a tile ahead
  if (c_begin < c_end) {
    ci = chunk_at(L, c_begin);
    qc = load_query(L.q, ci.start + (r < ci.count ? r : 0));
  }
  bool taps_ready = false;
  for (int64_t c = c_begin; c < c_end; ++c) {
    // prefetch the next tile's inputs; consumed one iteration later
    ChunkIn cn = ci;
    QueryIn qn = qc;
    if (c + 1 < c_end) {
      cn = chunk_at(L, c + 1);
      qn = load_query(L.q, cn.start + (r < cn.count ? r : 0));
    }
    if (ci.mat != cur_mat) {
      // (re)stage the material's weights; no MMA is in flight here
      if (__syncthreads_or(bad)) break;
      const void* wsrc = L.chunks ? L.mats.weights[ci.mat] : L.w0;
      pyr = L.chunks ? L.mats.pyramid[ci.mat] : L.pyr0;
      if (tid == 0) {
        ptx::fence_proxy_async();
        ptx::mbar_arrive_expect_tx(bar_w, Lay::BLOB);
        ptx::bulk_g2s(aW, wsrc, Lay::BLOB, bar_w);
      }
      w_pending = true;
      bad |= !ptx::mbar_wait(bar_w, ph_w, L.timeout_ns);
      ph_w ^= 1;
      if (!bad) w_pending = false;
      cur_mat = ci.mat;
    }
    const bool valid = r < ci.count;
    const int64_t i = ci.start + (valid ? r : 0);

    // ---- 1. latent fetch ------------------------------------------------
    float z[8];
    if (F16P) {
      if (!taps_ready) issue_taps(L.pyr, pyr, qc.u, qc.v, qc.lod, qc.xi, tc);
      finish_taps(tc, z);
    } else {
      fetch_latent<F16P>(L.pyr, pyr, qc.u, qc.v, qc.lod, qc.xi, z);
    }
    taps_ready = false;
    const uint32_t z01 = ptx::pack_h2(z[0], z[1]), z23 = ptx::pack_h2(z[2], z[3]);
    const uint32_t z45 = ptx::pack_h2(z[4], z[5]), z67 = ptx::pack_h2(z[6], z[7]);

    float xl[6];
    if (FRAME) {
      // ---- 2. frame MLP at FP32 accuracy (split FP16 operands) -----------
      {
        uint32_t lo0, lo1, lo2, lo3, h0, h1, h2, h3;
        split2(z[0], z[1], h0, lo0);
        split2(z[2], z[3], h1, lo1);
        split2(z[4], z[5], h2, lo2);
        split2(z[6], z[7], h3, lo3);
        ptx::st_shared_v4(aA + 0 * 2048 + r * 16, h0, h1, h2, h3);
        ptx::st_shared_v4(aA + 1 * 2048 + r * 16, lo0, lo1, lo2, lo3);
      }
      if (!mma_stage([&] {
            ptx::mma_f16(tmem, ptx::sdesc(aA, 2048, 128), ptx::sdesc(aW + Lay::B_F1, 256, 128), ID_16, 0);
            ptx::mma_f16(tmem, ptx::sdesc(aConst, 2048, 128), ptx::sdesc(aW + Lay::B_F1 + 512, 256, 128), ID_16, 1);
          }))
        break;
      {
        uint32_t acc[16];
        ptx::tmem_ld16(tlane, acc);
        ptx::tmem_ld_wait();
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          split2(fmaxf(u2f(acc[2 * j]), 0.0f), fmaxf(u2f(acc[2 * j + 1]), 0.0f), hi[j], lo[j]);
        ptx::st_shared_v4(aA + 0 * 2048 + r * 16, hi[0], hi[1], hi[2], hi[3]);
        ptx::st_shared_v4(aA + 1 * 2048 + r * 16, hi[4], hi[5], hi[6], hi[7]);
        ptx::st_shared_v4(aA + 2 * 2048 + r * 16, lo[0], lo[1], lo[2], lo[3]);
        ptx::st_shared_v4(aA + 3 * 2048 + r * 16, lo[4], lo[5], lo[6], lo[7]);
      }
      if (!mma_stage([&] {
            ptx::mma_f16(tmem, ptx::sdesc(aA, 2048, 128), ptx::sdesc(aW + Lay::B_F2, 256, 128), ID_16, 0);
            ptx::mma_f16(tmem, ptx::sdesc(aA + 2 * 2048, 2048, 128), ptx::sdesc(aW + Lay::B_F2 + 512, 256, 128),
                         ID_16, 1);
            ptx::mma_f16(tmem, ptx::sdesc(aConst, 2048, 128), ptx::sdesc(aW + Lay::B_F2 + 1024, 256, 128), ID_16, 1);
          }))
        break;
      {
        uint32_t acc[8];
        ptx::tmem_ld8(tlane, acc);
        ptx::tmem_ld_wait();
        float rr[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) rr[j] = u2f(acc[j]);
        // ---- 3. frame + transform ---------------------------------------
        Frame F = build_frame(rr);
        to_local(F, qc.wix, qc.wiy, qc.wiz, xl);
        to_local(F, qc.wox, qc.woy, qc.woz, xl + 3);
      }
    } else {
      xl[0] = qc.wix; xl[1] = qc.wiy; xl[2] = qc.wiz;
      xl[3] = qc.wox; xl[4] = qc.woy; xl[5] = qc.woz;
    }

    // ---- 4. decoder ---------------------------------------------------------
    // L1 operand: block 0 = z (fp16), block 1 = (wi', wo', 1, 0)
    ptx::st_shared_v4(aA + 0 * 2048 + r * 16, z01, z23, z45, z67);
    ptx::st_shared_v4(aA + 1 * 2048 + r * 16, ptx::pack_h2(xl[0], xl[1]), ptx::pack_h2(xl[2], xl[3]),
                      ptx::pack_h2(xl[4], xl[5]), 0x00003C00u);
    if (!mma_stage([&] {
          ptx::mma_f16(tmem, ptx::sdesc(aA, 2048, 128), ptx::sdesc(aW + Lay::B_L1, H * 16, 128), ID_H, 0);
        }))
      break;

    // texels of the next tile start loading now, under the hidden layers
    if (F16P && c + 1 < c_end && cn.mat == ci.mat) {
      issue_taps(L.pyr, pyr, qn.u, qn.v, qn.lod, qn.xi, tc);
      taps_ready = true;
    }

    // hidden -> hidden and hidden -> out share the epilogue: TMEM row ->
    // ReLU -> FP16 -> A blocks [0, H/8)
    bool ok = true;
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += (H < 32 ? H : 32)) {
        constexpr int NC = H < 32 ? H : 32;
        uint32_t pk[NC / 2];
        if (NC == 32) {
          uint32_t acc[32];
          ptx::tmem_ld32(tlane + c0, acc);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) pk[j] = ptx::pack_h2_relu(u2f(acc[2 * j]), u2f(acc[2 * j + 1]));
        } else {
          uint32_t acc[16];
          ptx::tmem_ld16(tlane + c0, acc);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 8; ++j) pk[j] = ptx::pack_h2_relu(u2f(acc[2 * j]), u2f(acc[2 * j + 1]));
        }
#pragma unroll
        for (int b = 0; b < NC / 8; ++b)
          ptx::st_shared_v4(aA + (c0 / 8 + b) * 2048 + r * 16, pk[4 * b], pk[4 * b + 1], pk[4 * b + 2],
                            pk[4 * b + 3]);
      }
      const int boff = layer == 0 ? Lay::B_L2 : Lay::B_LO;
      const int nrows = layer == 0 ? H : 16;
      const uint32_t id = layer == 0 ? ID_H : ID_16;
      if (!mma_stage([&] {
#pragma unroll
            for (int s2 = 0; s2 < H / 16; ++s2)
              ptx::mma_f16(tmem, ptx::sdesc(aA + s2 * 4096, 2048, 128),
                           ptx::sdesc(aW + boff + s2 * 2 * nrows * 16, nrows * 16, 128), id, s2 > 0 ? 1u : 0u);
            // bias step: A constant blocks x B blocks (H/8, H/8+1)
            ptx::mma_f16(tmem, ptx::sdesc(aConst, 2048, 128),
                         ptx::sdesc(aW + boff + (H / 8) * nrows * 16, nrows * 16, 128), id, 1u);
          })) {
        ok = false;
        break;
      }
    }
    if (!ok) break;

    // ---- 5. output ----------------------------------------------------------
    {
      uint32_t acc[4];
      ptx::tmem_ld4(tlane, acc);
      ptx::tmem_ld_wait();
      float y0 = u2f(acc[0]), y1 = u2f(acc[1]), y2 = u2f(acc[2]);
      if (cosine) {
        const float cz = fmaxf(qc.wiz, 0.0f);
        y0 *= cz; y1 *= cz; y2 *= cz;
      }
      if (valid) {
        L.rgb[3 * i + 0] = y0;
        L.rgb[3 * i + 1] = y1;
        L.rgb[3 * i + 2] = y2;
      }
    }
    ptx::tc_fence_before();
    ci = cn;
    qc = qn;
  }

  // ---- teardown: wait (bounded) for copies / MMAs still in flight ----------
  if (tid == 0) {
    if (mma_pending) ptx::mbar_wait(bar_m, ph_m ^ 1, L.timeout_ns);
    if (w_pending) ptx::mbar_wait(bar_w, ph_w ^ 1, L.timeout_ns);
    if (bad) record_error(L.err, DEVERR_WAIT_TIMEOUT);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 64);
  }
}

// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------
template <int H, bool FRAME, bool F16P>
static int launch_tc_one(const LaunchCommon& L, cudaStream_t s) {
  using Lay = TcLayout<H, FRAME>;
  auto k = eval_tc_kernel<H, FRAME, F16P>;
  static int occ = -1;
  if (occ < 0) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM);
    // TMEM: 512 columns per SM, 64 per CTA -> at most 8 resident CTAs
    occ = blocks_per_sm((const void*)k, 128, Lay::SMEM, 8, true);
  }
  const int64_t nchunks = L.chunks ? (int64_t)L.n_chunks : (L.n + 127) / 128;
  if (nchunks == 0) return 0;
  int64_t cap = (int64_t)occ * L.num_sms;
  int grid = (int)(nchunks < cap ? nchunks : cap);
  k<<<grid, 128, Lay::SMEM, s>>>(L);
  return (int)cudaGetLastError();
}

template <int H>
static int tc_dispatch(const LaunchCommon& L, cudaStream_t s) {
  if (L.shape.frame)
    return L.pyr.f16 ? launch_tc_one<H, true, true>(L, s) : launch_tc_one<H, true, false>(L, s);
  return L.pyr.f16 ? launch_tc_one<H, false, true>(L, s) : launch_tc_one<H, false, false>(L, s);
}

int launch_eval_tc(const LaunchCommon& L, int precision, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (precision != NAM_PREC_F16 || L.shape.NH != 2) return (int)cudaErrorInvalidValue;
  if (L.shape.H == 16) return tc_dispatch<16>(L, s);
  if (L.shape.H == 32) return tc_dispatch<32>(L, s);
  if (L.shape.H == 64) return tc_dispatch<64>(L, s);
  return (int)cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// single-MMA self test: D[128][N] = A[128][K] * B[N][K]^T with FP16 operands
// given in the canonical K-major layout (K = 32: two K steps), used by the
// tests to check descriptor and TMEM conventions in isolation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) mma_selftest_kernel(const uint8_t* A, const uint8_t* B, float* D,
                                                           uint64_t timeout_ns, int* err) {
  // A: 128 x 32 fp16 = 8 KB, B: 64 x 32 fp16 = 4 KB; the regions are sized
  // 32 KB and 16 KB so that every address a descriptor can form stays inside.
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + 32768;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 32768 + 16384);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < 8192 / 16; k += 128) reinterpret_cast<uint4*>(sA)[k] = reinterpret_cast<const uint4*>(A)[k];
  for (int k = tid; k < 4096 / 16; k += 128) reinterpret_cast<uint4*>(sB)[k] = reinterpret_cast<const uint4*>(B)[k];
  const uint32_t b = ptx::smem_u32(bar);
  if (tid == 0) {
    ptx::mbar_init(b, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), 64);
    ptx::tmem_relinquish();
  }
  ptx::fence_proxy_async();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t aA = ptx::smem_u32(sA), aB = ptx::smem_u32(sB);
  if (tid == 0) {
    constexpr uint32_t id = ptx::idesc_f16(128, 64);
    ptx::mma_f16(tmem, ptx::sdesc(aA, 2048, 128), ptx::sdesc(aB, 64 * 16, 128), id, 0);
    ptx::mma_f16(tmem, ptx::sdesc(aA + 4096, 2048, 128), ptx::sdesc(aB + 2 * 64 * 16, 64 * 16, 128), id, 1);
    ptx::mma_commit(b);
  }
  bool ok = ptx::mbar_wait(b, 0, timeout_ns);
  if (!ok && tid == 0) record_error(err, DEVERR_WAIT_TIMEOUT);
  ptx::tc_fence_after();
  if (ok) {
    uint32_t acc[32];
    for (int c0 = 0; c0 < 64; c0 += 32) {
      ptx::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, acc);
      ptx::tmem_ld_wait();
      for (int j = 0; j < 32; ++j) D[tid * 64 + c0 + j] = u2f(acc[j]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 64);
  }
}

// Same product with A taken from TMEM: thread r stores row r of A (two fp16
// per 32-bit column, element 2j in the low half of column j) with
// tcgen05.st, and two K=16 MMAs read it at columns +0 and +8.
__global__ void __launch_bounds__(128) mma_selftest_ts_kernel(const uint16_t* A, const uint8_t* B, float* D,
                                                              uint64_t timeout_ns, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 16384);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < 4096 / 16; k += 128) reinterpret_cast<uint4*>(sB)[k] = reinterpret_cast<const uint4*>(B)[k];
  const uint32_t b = ptx::smem_u32(bar);
  if (tid == 0) {
    ptx::mbar_init(b, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), 128);
    ptx::tmem_relinquish();
  }
  ptx::fence_proxy_async();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t lane = (uint32_t)(warp * 32) << 16;
  uint32_t row[16];
  for (int j = 0; j < 16; ++j) row[j] = (uint32_t)A[tid * 32 + 2 * j] | ((uint32_t)A[tid * 32 + 2 * j + 1] << 16);
  ptx::tmem_st16(tmem + lane + 64, row);
  ptx::tmem_st_wait();
  ptx::tc_fence_before();
  __syncthreads();
  const uint32_t aB = ptx::smem_u32(sB);
  if (tid == 0) {
    ptx::tc_fence_after();
    constexpr uint32_t id = ptx::idesc_f16(128, 64);
    ptx::mma_f16_ts(tmem, tmem + 64, ptx::sdesc(aB, 64 * 16, 128), id, 0);
    ptx::mma_f16_ts(tmem, tmem + 64 + 8, ptx::sdesc(aB + 2 * 64 * 16, 64 * 16, 128), id, 1);
    ptx::mma_commit(b);
  }
  bool ok = ptx::mbar_wait(b, 0, timeout_ns);
  if (!ok && tid == 0) record_error(err, DEVERR_WAIT_TIMEOUT);
  ptx::tc_fence_after();
  if (ok) {
    uint32_t acc[32];
    for (int c0 = 0; c0 < 64; c0 += 32) {
      ptx::tmem_ld32(tmem + lane + c0, acc);
      ptx::tmem_ld_wait();
      for (int j = 0; j < 32; ++j) D[tid * 64 + c0 + j] = u2f(acc[j]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 128);
  }
}

int launch_mma_selftest_ts(const uint16_t* A, const uint8_t* B, float* D, uint64_t timeout_ns, int* err,
                           void* stream) {
  const int smem = 16384 + 64;
  mma_selftest_ts_kernel<<<1, 128, smem, (cudaStream_t)stream>>>(A, B, D, timeout_ns, err);
  return (int)cudaGetLastError();
}

int launch_mma_selftest(const uint8_t* A, const uint8_t* B, float* D, uint64_t timeout_ns, int* err,
                        void* stream) {
  const int smem = 32768 + 16384 + 64;
  cudaFuncSetAttribute(mma_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  mma_selftest_kernel<<<1, 128, smem, (cudaStream_t)stream>>>(A, B, D, timeout_ns, err);
  return (int)cudaGetLastError();
}

}  // namespace nam
