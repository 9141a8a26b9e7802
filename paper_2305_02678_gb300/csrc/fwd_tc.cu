// Tensor-core evaluation of the neural BRDF on sm_103a (tcgen05 + TMEM).
//
// One CTA per SM with five warpgroups; each warpgroup owns a tile of up to
// 128 queries at a time (thread r = query r = TMEM lane r) and runs it
// through the whole path on its own TMEM columns, weight copy and mbarriers:
//   1. coalesced planar query loads, latent fetch (16-byte texel gathers,
//      FP32 filter) -> z                                     (Sec. 4.1)
//   2. frame MLP 8 -> 16 -> 6 on the tensor core with each FP16 operand
//      split into a high and a low half (z = z_hi + z_lo), so the frame has
//      FP32 accuracy; ReLU between the layers                 (Sec. 4.2)
//   3. frame build (Gram-Schmidt, b = n x t) and the direction transform in
//      FP32 registers: each thread holds its own query's TMEM row, so the
//      six frame outputs need no cross-lane exchange          (Eq. 4)
//   4. decoder layers 14 -> H -> H -> 3: FP16 operands (or E4M3 with
//      per-layer scales), FP32 accumulation in TMEM; FP16 biases ride in the
//      MMA as the weight of a constant-1 input
//   5. RGB store (x max(0, wi.z) if requested)
// The FP16 A operands are written to TMEM (tcgen05.st) and read by the MMA
// from there, so shared memory holds little more than the weights, and most
// of the SM's L1/shared storage caches the texel gathers.  MLP weights are
// staged per warpgroup, again when a multi-material launch switches
// material, with one bulk TMA copy of a blob that the host laid out in the
// MMA operand order at material creation.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
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

// Weight blob offsets (bytes) for hidden width H, frame form FK (0 none,
// 1 MLP 8-16-6, 2 the paper's linear 8 -> 12) and NH hidden layers.  Every
// FP16 bias rides in the MMA as the weight of a constant-1 input column.
struct TcOff {
  int b_f1, b_f2;  // FK 1: 16 x 32 [Wf1 | Wf1 | bf1 0..], 16 x 48 [Wf2 | Wf2 | bf2 0..]
                   // FK 2: b_f1 = 16 x 32 [Wf | Wf | bf 0..] (12 rows used)
  int b_l1, kl1;   // H x kl1: [W1 | b1 0..], kl1 = 16 (14 inputs) or 32 (20 inputs)
  int b_l2;        // (NH - 1) blocks of H x (H + 16): hidden -> hidden
  int b_lo;        // 16 x (H + 16): hidden -> RGB (3 rows used)
  int blob;
};
__host__ __device__ constexpr TcOff tc_off(int H, int FK, int NH) {
  TcOff o{};
  o.b_f1 = 0;
  o.b_f2 = 1024;
  o.b_l1 = FK == 1 ? 2560 : FK == 2 ? 1024 : 0;
  o.kl1 = FK == 2 ? 32 : 16;
  o.b_l2 = o.b_l1 + H * o.kl1 * 2;
  o.b_lo = o.b_l2 + (NH - 1) * H * (H + 16) * 2;
  o.blob = o.b_lo + 16 * (H + 16) * 2;
  return o;
}

// FP8 (E4M3) decoder (frame forms 0 and 1, two hidden layers): the frame
// blocks are those of the FP16 layout; the decoder's B operands hold E4M3
// codes in the canonical K-major layout for 8-bit types (8-row x 16-byte core
// matrices = 16 codes along K), K padded to the 32 of one kind::f8f6f4 MMA.
// The biases stay FP32 and are added in the epilogue together with the
// per-layer scales:
//   next-layer code = E4M3(relu(D * c_l + b'_l)),  c_l = s_l sw_l / s_{l+1},
//   b'_l = b_l / s_{l+1};  output = D * c_2 + b_2,  c_2 = s_2 sw_2,
// where D = sum of code products (FP32, in TMEM), s_l the static input scale
// of decoder layer l and sw_l its weight scale.
template <int H, int FK>
struct TcLayout8 {
  static constexpr int KP = H < 32 ? 32 : H;              // hidden K padded to one MMA step
  static constexpr int B_L1 = FK ? 2560 : 0;              // H x 32 codes
  static constexpr int B_L2 = B_L1 + H * 32;              // H x KP codes
  static constexpr int B_LO = B_L2 + H * KP;              // 16 x KP codes
  static constexpr int B_SC = (B_LO + 16 * KP + 15) / 16 * 16;  // FP32: inv_s0, c0, c1, c2
  static constexpr int B_B1 = B_SC + 16;                  // FP32 b'_0 [H]
  static constexpr int B_B2 = B_B1 + H * 4;               // FP32 b'_1 [H]
  static constexpr int B_B3 = B_B2 + H * 4;               // FP32 b_2 [8]: RGB, albedo head
  static constexpr int BLOB = B_B3 + 32;
};

template <int H, int FK>
static size_t blob8_bytes() {
  return (size_t)TcLayout8<H, FK>::BLOB;
}

// Shapes with a tensor-core kernel: two hidden layers of 16, 32 or 64, or
// three of 64; FP8 with frame forms 0 and 1 and two hidden layers.
static bool tc_supported(const Shape& s, int precision) {
  if (precision != NAM_PREC_F16 && precision != NAM_PREC_FP8) return false;
  const bool hidden_ok = (s.NH == 2 && (s.H == 16 || s.H == 32 || s.H == 64)) || (s.NH == 3 && s.H == 64);
  if (!hidden_ok || s.frame < 0 || s.frame > 2) return false;
  if (precision == NAM_PREC_FP8 && (s.NH != 2 || s.frame == 2)) return false;
  return true;
}

size_t tc_blob_bytes(const Shape& s, int precision) {
  if (precision == NAM_PREC_F16) return f16_blob_bytes(s);
  if (!tc_supported(s, precision)) return 0;
  const bool f = s.frame == 1;
  if (s.H == 16) return f ? blob8_bytes<16, 1>() : blob8_bytes<16, 0>();
  if (s.H == 32) return f ? blob8_bytes<32, 1>() : blob8_bytes<32, 0>();
  return f ? blob8_bytes<64, 1>() : blob8_bytes<64, 0>();
}

static void put_h(uint8_t* base, int R, int row, int k, float v) {
  __half h = __float2half_rn(v);
  std::memcpy(base + kmajor_off(R, row, k), &h, 2);
}

// E4M3 (OCP 8-bit float, "FN" variant: bias 7, no infinities, S.1111.111 the
// only NaN, largest finite 448) of an FP32 value, round to nearest even,
// saturating to +-448.  Written from the format's definition.
static uint8_t e4m3_of(float x) {
  if (std::isnan(x)) return 0x7F;
  const uint8_t sign = std::signbit(x) ? 0x80 : 0x00;
  const double a = std::fabs((double)x);
  if (a >= 448.0) return sign | 0x7E;
  if (a < 0.015625) {  // below 2^-6: subnormal codes, spacing 2^-9
    const int m = (int)std::nearbyint(a * 512.0);  // m = 8 is the smallest normal
    return sign | (uint8_t)m;
  }
  int e2;
  const double f = std::frexp(a, &e2);  // a = f 2^e2, f in [0.5, 1)
  int E = e2 - 1;
  int m = (int)std::nearbyint((f * 2.0 - 1.0) * 8.0);
  if (m == 8) {
    m = 0;
    ++E;
  }
  if (E > 8 || (E == 8 && m == 7)) return sign | 0x7E;
  return sign | (uint8_t)(((E + 7) << 3) | m);
}

// Canonical no-swizzle K-major 8-bit layout of an R x K operand: element
// (row, k) at byte (k / 16) * (R * 16) + row * 16 + (k % 16).
static inline int kmajor_off8(int R, int row, int k) { return (k / 16) * (R * 16) + row * 16 + (k % 16); }

// Per-layer E4M3 weights: sw = absmax(W) / 448 in FP32, code = E4M3(W / sw)
// with the division in FP32.
static float quantize_layer_e4m3(const float* W, int rows, int cols, uint8_t* base, int R, float* sw_out) {
  float amax = 0.0f;
  for (int i = 0; i < rows * cols; ++i) amax = std::fmax(amax, std::fabs(W[i]));
  const float sw = amax > 0.0f ? amax / 448.0f : 1.0f;
  for (int n = 0; n < rows; ++n)
    for (int k = 0; k < cols; ++k) base[kmajor_off8(R, n, k)] = e4m3_of(W[n * cols + k] / sw);
  *sw_out = sw;
  return sw;
}

// The value of an E4M3 code: sign bit, exponent field E (bias 7), mantissa
// m; E = 0 holds the subnormals m 2^-9.
static float e4m3_value(uint8_t c) {
  const int E = (c >> 3) & 15, m = c & 7;
  const float a = E == 0 ? std::ldexp((float)m, -9) : std::ldexp(1.0f + (float)m / 8.0f, E - 7);
  return (c & 0x80) ? -a : a;
}

float e4m3_dequant(float w, float sw) { return e4m3_value(e4m3_of(w / sw)) * sw; }

static void put_f(uint8_t* base, int idx, float v) { std::memcpy(base + 4 * idx, &v, 4); }

// Lay out the FP16-quantised weights as MMA B operands (N rows = outputs,
// K = inputs, K-major), each layer's bias in the extra input column that
// meets the constant-1 column of the A operand.  The frame layers take their
// FP16 operand in two halves (high part, residual), so their weights appear
// twice along K.  FP8: the frame part is the same; the decoder part is laid
// out as TcLayout8 describes.
int pack_tc_blob(const Shape& s, int precision, const float* frame, const float* dec, const float* act_scale,
                 uint8_t* out, float* weight_scales_out) {
  if (precision == NAM_PREC_F16) return pack_f16_blob(s, frame, dec, out);
  if (precision != NAM_PREC_FP8) return -1;
  const size_t bytes = tc_blob_bytes(s, precision);
  if (!bytes) return -1;
  std::memset(out, 0, bytes);
  const int H = s.H, IN = s.in;
  const TcOff o = tc_off(H, s.frame, s.NH);
  if (s.frame == 1) {
    const float* Wf1 = frame;            // [16][8]
    const float* bf1 = Wf1 + 128;        // [16]
    const float* Wf2 = bf1 + 16;         // [6][16]
    const float* bf2 = Wf2 + 96;         // [6]
    for (int n = 0; n < 16; ++n) {
      for (int k = 0; k < 16; ++k) put_h(out + o.b_f1, 16, n, k, Wf1[n * 8 + (k & 7)]);
      put_h(out + o.b_f1, 16, n, 16, bf1[n]);
    }
    for (int n = 0; n < 6; ++n) {
      for (int k = 0; k < 32; ++k) put_h(out + o.b_f2, 16, n, k, Wf2[n * 16 + (k & 15)]);
      put_h(out + o.b_f2, 16, n, 32, bf2[n]);
    }
  } else if (s.frame == 2) {
    const float* Wf = frame;             // [12][8]
    const float* bf = Wf + 96;           // [12]
    for (int n = 0; n < 12; ++n) {
      for (int k = 0; k < 16; ++k) put_h(out + o.b_f1, 16, n, k, Wf[n * 8 + (k & 7)]);
      put_h(out + o.b_f1, 16, n, 16, bf[n]);
    }
  }
  const float* W1 = dec;                 // [H][IN]
  const float* b1 = W1 + IN * H;
  const float* W2 = b1 + H;              // [H][H] (then the third layer's, NH = 3)
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;              // [out][H] (NH = 2): RGB rows, then the albedo head's
  const float* b3 = W3 + s.out * H;
  if (precision == NAM_PREC_FP8) {
    if (!act_scale) return -1;
    const int KP = H < 32 ? 32 : H;
    const int b_l1 = s.frame ? 2560 : 0, b_l2 = b_l1 + H * 32, b_lo = b_l2 + H * KP;
    const int b_sc = (b_lo + 16 * KP + 15) / 16 * 16, b_b1 = b_sc + 16, b_b2 = b_b1 + H * 4, b_b3 = b_b2 + H * 4;
    float sw[3];
    quantize_layer_e4m3(W1, H, 14, out + b_l1, H, &sw[0]);
    quantize_layer_e4m3(W2, H, H, out + b_l2, H, &sw[1]);
    quantize_layer_e4m3(W3, s.out, H, out + b_lo, 16, &sw[2]);
    const float inv0 = 1.0f / act_scale[0], inv1 = 1.0f / act_scale[1], inv2 = 1.0f / act_scale[2];
    put_f(out + b_sc, 0, inv0);
    put_f(out + b_sc, 1, (act_scale[0] * sw[0]) * inv1);
    put_f(out + b_sc, 2, (act_scale[1] * sw[1]) * inv2);
    put_f(out + b_sc, 3, act_scale[2] * sw[2]);
    for (int n = 0; n < H; ++n) {
      put_f(out + b_b1, n, b1[n] * inv1);
      put_f(out + b_b2, n, b2[n] * inv2);
    }
    for (int n = 0; n < s.out; ++n) put_f(out + b_b3, n, b3[n]);
    if (weight_scales_out)
      for (int l = 0; l < 3; ++l) weight_scales_out[l] = sw[l];
    return 0;
  }
  for (int n = 0; n < H; ++n) {
    for (int k = 0; k < IN; ++k) put_h(out + o.b_l1, H, n, k, W1[n * IN + k]);
    put_h(out + o.b_l1, H, n, IN, b1[n]);
  }
  const float* p = b1 + H;
  for (int l = 0; l < s.NH - 1; ++l) {
    const float* Wh = p;
    const float* bh = Wh + H * H;
    uint8_t* dst = out + o.b_l2 + l * H * (H + 16) * 2;
    for (int n = 0; n < H; ++n) {
      for (int k = 0; k < H; ++k) put_h(dst, H, n, k, Wh[n * H + k]);
      put_h(dst, H, n, H, bh[n]);
    }
    p = bh + H;
  }
  const float* Wo = p;
  const float* bo = Wo + s.out * H;
  for (int n = 0; n < s.out; ++n) {
    for (int k = 0; k < H; ++k) put_h(out + o.b_lo, 16, n, k, Wo[n * H + k]);
    put_h(out + o.b_lo, 16, n, H, bo[n]);
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

// Shared memory of one CTA: a constant block (1.0 in column 0 of every row)
// and a zero block, shared by the warpgroups; then one slot per warpgroup:
// its copy of the weight blob, for FP8 its A blocks (E4M3 codes, plus a zero
// block), and its two mbarriers.  The FP16 operands of every MMA that is not
// a bias step live in TMEM instead of shared memory, which leaves most of the
// SM's 256 KB of L1/shared storage to the L1 cache that serves the texel
// gathers.
template <int H, int FK, int NH, bool P8>
struct WgSlot {
  static constexpr int BLOB = P8 ? TcLayout8<H, (FK == 1 ? 1 : 0)>::BLOB : tc_off(H, FK, NH).blob;
  static constexpr int BLOB_AL = (BLOB + 127) / 128 * 128;
  static constexpr int A8_BLOCKS = P8 ? ((H / 16) > 1 ? (H / 16) : 1) : 0;  // E4M3 A blocks
  static constexpr int A8_BYTES = P8 ? (A8_BLOCKS + 1) * 2048 : 0;          // + zero block
  static constexpr int BYTES = BLOB_AL + A8_BYTES + 128;                     // + mbarriers
};
template <int H, int FK, int NH, bool P8, int NWG>
__host__ __device__ constexpr int smem_bytes() {
  return 4096 + NWG * WgSlot<H, FK, NH, P8>::BYTES + 16;
}

// TMEM columns of one warpgroup: FP32 accumulator [0, 64), FP16 A operand
// [64, 96) (two values per column, row = query).
constexpr int kTmemPerWg = 96;

// Warpgroups per CTA (one CTA per SM): 640 threads at <= 96 registers.  Five
// warpgroups without register prefetch of the next tile's texels measured
// faster than four with it (the gathers then hit a larger L1).
constexpr int kNwg = 5;

// One CTA per SM with NWG warpgroups; each warpgroup runs the whole path on
// its own tiles of 128 queries (thread r = query r = TMEM lane r), with its
// own TMEM columns, weight copy and mbarriers, so warpgroups never wait for
// each other.  P8: the decoder in E4M3 (kind::f8f6f4) instead of FP16.
template <int H, int FK, int NH, bool F16P, bool P8, int NWG>
__global__ void __launch_bounds__(NWG * 128, 1) eval_tc_kernel(const LaunchCommon L) {
  static_assert(!P8 || (NH == 2 && FK != 2), "FP8: frame forms 0 and 1, two hidden layers");
  constexpr TcOff O = tc_off(H, FK, NH);
  using Lay8 = TcLayout8<H, (FK == 1 ? 1 : 0)>;
  using S = WgSlot<H, FK, NH, P8>;
  constexpr int BLOB = S::BLOB;
  extern __shared__ __align__(1024) uint8_t smem[];

  const int tid = threadIdx.x, wg = tid >> 7, r = tid & 127, warp = tid >> 5;
  const uint32_t aConst = ptx::smem_u32(smem);
  const uint32_t aZero = aConst + 2048;
  uint8_t* sW = smem + 4096 + wg * S::BYTES;
  const uint32_t aW = ptx::smem_u32(sW);
  const uint32_t aA8 = aW + S::BLOB_AL;                 // P8: E4M3 A blocks
  const uint32_t aZ8 = aA8 + S::A8_BLOCKS * 2048;       // P8: this slot's zero block
  uint64_t* bars = reinterpret_cast<uint64_t*>(sW + S::BLOB_AL + S::A8_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 4096 + NWG * S::BYTES);
  const uint32_t bar_w = ptx::smem_u32(&bars[0]);
  const uint32_t bar_m = ptx::smem_u32(&bars[1]);
  const float* sc8 = reinterpret_cast<const float*>(sW + Lay8::B_SC);  // P8: inv_s0, c0, c1, c2
  const uint32_t bar_id = 1 + wg;                       // named barrier of this warpgroup

  if (r == 0) {
    ptx::mbar_init(bar_w, 1);
    ptx::mbar_init(bar_m, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), 512);
    ptx::tmem_relinquish();
  }
  if (tid < 128) {
    ptx::st_shared_v4(aConst + tid * 16, 0x3C00u, 0u, 0u, 0u);
    ptx::st_shared_v4(aZero + tid * 16, 0u, 0u, 0u, 0u);
  }
  if (P8) ptx::st_shared_v4(aZ8 + r * 16, 0u, 0u, 0u, 0u);
  ptx::fence_proxy_async();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t tD = tmem + wg * kTmemPerWg;           // accumulator (MMA address: lane 0)
  const uint32_t tA = tD + 64;                          // FP16 A operand
  const uint32_t tDl = tD + lane, tAl = tA + lane;      // this warp's rows

  int64_t nchunks = L.chunks ? (int64_t)L.n_chunks : (L.n + 127) / 128;
  if (L.n_chunks_dev) {
    const int64_t d = *L.n_chunks_dev;  // written by an earlier launch on this stream
    nchunks = d < 0 ? 0 : d < nchunks ? d : nchunks;
  }
  const int64_t per = (nchunks + gridDim.x - 1) / gridDim.x;
  const int64_t c_begin = (int64_t)blockIdx.x * per;
  const int64_t c_end = c_begin + per < nchunks ? c_begin + per : nchunks;

  uint32_t ph_w = 0, ph_m = 0;
  bool bad = false, mma_pending = false, w_pending = false;
  int cur_mat = -1;
  const void* pyr = L.pyr0;
  const bool cosine = (L.flags & NAM_OUT_COSINE) != 0;

  constexpr uint32_t ID_16 = ptx::idesc_f16(128, 16);
  constexpr uint32_t ID_H = ptx::idesc_f16(128, H);
  constexpr uint32_t ID8_16 = ptx::idesc_e4m3(128, 16);
  constexpr uint32_t ID8_H = ptx::idesc_e4m3(128, H);

  // make this thread's operand writes (shared memory and TMEM) visible to the
  // tensor core, sync the warpgroup, let one thread issue `issue`, wait for
  // completion.  Returns false (for every thread of the warpgroup) if any
  // thread's wait ran out.
  auto mma_stage = [&](auto issue) -> bool {
    if (P8) ptx::fence_proxy_async();
    ptx::tc_fence_before();
    if (ptx::bar_red_or(bar_id, 128, bad)) return false;
    if (r == 0) {
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
  int64_t c = c_begin + wg;
  if (c < c_end) {
    ci = chunk_at(L, c);
    qc = load_query(L.q, ci.start + (r < ci.count ? r : 0));
  }
  for (; c < c_end; c += NWG) {
    // prefetch the next tile's inputs; consumed one iteration later
    ChunkIn cn = ci;
    QueryIn qn = qc;
    const bool has_next = c + NWG < c_end;
    if (has_next) {
      cn = chunk_at(L, c + NWG);
      qn = load_query(L.q, cn.start + (r < cn.count ? r : 0));
    }
    if (ci.count <= 0) {
      // an empty slot of a chunk table (count is uniform over the warpgroup)
      ci = cn;
      qc = qn;
      continue;
    }
    if (ci.mat != cur_mat) {
      // (re)stage the material's weights; no MMA of this warpgroup is in flight
      if (ptx::bar_red_or(bar_id, 128, bad)) break;
      const void* wsrc = L.chunks ? L.mats.weights[ci.mat] : L.w0;
      pyr = L.chunks ? L.mats.pyramid[ci.mat] : L.pyr0;
      if (r == 0) {
        ptx::fence_proxy_async();
        ptx::mbar_arrive_expect_tx(bar_w, BLOB);
        ptx::bulk_g2s(aW, wsrc, BLOB, bar_w);
      }
      w_pending = true;
      bad |= !ptx::mbar_wait(bar_w, ph_w, L.timeout_ns);
      ph_w ^= 1;
      if (!bad) w_pending = false;
      cur_mat = ci.mat;
    }
    const bool valid = r < ci.count;
    const int64_t i = ci.start + (valid ? r : 0);
    // masked pass: this row's material, loaded now and compared at the store
    const int32_t row_mat = L.row_ids ? __ldg(L.row_ids + i) : ci.mat;

    // ---- 1. latent fetch ------------------------------------------------
    float z[8];
    if (F16P) {
      Taps8 tc;
      issue_taps(L.pyr, pyr, qc.u, qc.v, qc.lod, qc.xi, tc);
      finish_taps(tc, z);
    } else {
      fetch_latent<F16P>(L.pyr, pyr, qc.u, qc.v, qc.lod, qc.xi, z);
    }
    // the decoder's copy of z, packed now so that only 2 or 4 registers live
    // through the frame stages: FP16 pairs, or E4M3(z / s_0) quadruples
    uint32_t zp[4];
    if (P8) {
      const float inv0 = sc8[0];
      zp[0] = ptx::pack_e4m3x2(z[0] * inv0, z[1] * inv0) | (ptx::pack_e4m3x2(z[2] * inv0, z[3] * inv0) << 16);
      zp[1] = ptx::pack_e4m3x2(z[4] * inv0, z[5] * inv0) | (ptx::pack_e4m3x2(z[6] * inv0, z[7] * inv0) << 16);
      zp[2] = zp[3] = 0;
    } else {
      zp[0] = ptx::pack_h2(z[0], z[1]);
      zp[1] = ptx::pack_h2(z[2], z[3]);
      zp[2] = ptx::pack_h2(z[4], z[5]);
      zp[3] = ptx::pack_h2(z[6], z[7]);
    }

    float xl[12];
    if (FK == 2) {
      // ---- 2'. the paper's frame layer 8 -> 12 at FP32 accuracy -----------
      {
        uint32_t v[8];
        split2(z[0], z[1], v[0], v[4]);
        split2(z[2], z[3], v[1], v[5]);
        split2(z[4], z[5], v[2], v[6]);
        split2(z[6], z[7], v[3], v[7]);
        ptx::tmem_st8(tAl, v);  // A = (z_hi, z_lo)
        ptx::tmem_st_wait();
      }
      if (!mma_stage([&] {
            ptx::mma_f16_ts(tD, tA, ptx::sdesc(aW + O.b_f1, 256, 128), ID_16, 0);
            ptx::mma_f16(tD, ptx::sdesc(aConst, 2048, 128), ptx::sdesc(aW + O.b_f1 + 512, 256, 128), ID_16, 1);
          }))
        break;
      {
        uint32_t acc[16];
        ptx::tmem_ld16(tDl, acc);
        ptx::tmem_ld_wait();
        float rr[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) rr[j] = u2f(acc[j]);
        // ---- 3'. two frames (normalised n, t; b = n x t / |n x t|) --------
        const Frame F1 = paper_frame(rr), F2 = paper_frame(rr + 6);
        to_local(F1, qc.wix, qc.wiy, qc.wiz, xl);
        to_local(F2, qc.wix, qc.wiy, qc.wiz, xl + 3);
        to_local(F1, qc.wox, qc.woy, qc.woz, xl + 6);
        to_local(F2, qc.wox, qc.woy, qc.woz, xl + 9);
      }
    } else if (FK == 1) {
      // ---- 2. frame MLP at FP32 accuracy (split FP16 operands) -----------
      {
        uint32_t v[8];
        split2(z[0], z[1], v[0], v[4]);
        split2(z[2], z[3], v[1], v[5]);
        split2(z[4], z[5], v[2], v[6]);
        split2(z[6], z[7], v[3], v[7]);
        ptx::tmem_st8(tAl, v);  // A = (z_hi, z_lo)
        ptx::tmem_st_wait();
      }
      if (!mma_stage([&] {
            ptx::mma_f16_ts(tD, tA, ptx::sdesc(aW + O.b_f1, 256, 128), ID_16, 0);
            ptx::mma_f16(tD, ptx::sdesc(aConst, 2048, 128), ptx::sdesc(aW + O.b_f1 + 512, 256, 128), ID_16, 1);
          }))
        break;
      {
        uint32_t acc[16];
        ptx::tmem_ld16(tDl, acc);
        ptx::tmem_ld_wait();
        uint32_t v[16];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          split2(fmaxf(u2f(acc[2 * j]), 0.0f), fmaxf(u2f(acc[2 * j + 1]), 0.0f), v[j], v[8 + j]);
        ptx::tmem_st16(tAl, v);  // A = (h_hi, h_lo)
        ptx::tmem_st_wait();
      }
      if (!mma_stage([&] {
            ptx::mma_f16_ts(tD, tA, ptx::sdesc(aW + O.b_f2, 256, 128), ID_16, 0);
            ptx::mma_f16_ts(tD, tA + 8, ptx::sdesc(aW + O.b_f2 + 512, 256, 128), ID_16, 1);
            ptx::mma_f16(tD, ptx::sdesc(aConst, 2048, 128), ptx::sdesc(aW + O.b_f2 + 1024, 256, 128), ID_16, 1);
          }))
        break;
      {
        uint32_t acc[8];
        ptx::tmem_ld8(tDl, acc);
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
    if (P8) {
      // L1 operand: block 0 = E4M3(x / s_0) for x = (z, wi', wo'), two zero
      // codes; the second K block of the MMA is the slot's zero block
      const float inv0 = sc8[0];
      const uint32_t w2 =
          ptx::pack_e4m3x2(xl[0] * inv0, xl[1] * inv0) | (ptx::pack_e4m3x2(xl[2] * inv0, xl[3] * inv0) << 16);
      const uint32_t w3 = ptx::pack_e4m3x2(xl[4] * inv0, xl[5] * inv0);
      ptx::st_shared_v4(aA8 + r * 16, zp[0], zp[1], w2, w3);
      if (!mma_stage([&] {
            ptx::mma_f8(tD, ptx::sdesc(aA8, aZ8 - aA8, 128), ptx::sdesc(aW + Lay8::B_L1, H * 16, 128), ID8_H, 0);
          }))
        break;
    } else if (FK == 2) {
      // L1 operand: (z, T wi (6), T wo (6), 1, 0...), K = 32; the 1 meets
      // the bias column of W1
      uint32_t v[16] = {zp[0],
                        zp[1],
                        zp[2],
                        zp[3],
                        ptx::pack_h2(xl[0], xl[1]),
                        ptx::pack_h2(xl[2], xl[3]),
                        ptx::pack_h2(xl[4], xl[5]),
                        ptx::pack_h2(xl[6], xl[7]),
                        ptx::pack_h2(xl[8], xl[9]),
                        ptx::pack_h2(xl[10], xl[11]),
                        0x00003C00u,
                        0u,
                        0u,
                        0u,
                        0u,
                        0u};
      ptx::tmem_st16(tAl, v);
      ptx::tmem_st_wait();
      if (!mma_stage([&] {
            ptx::mma_f16_ts(tD, tA, ptx::sdesc(aW + O.b_l1, H * 16, 128), ID_H, 0);
            ptx::mma_f16_ts(tD, tA + 8, ptx::sdesc(aW + O.b_l1 + 2 * H * 16, H * 16, 128), ID_H, 1);
          }))
        break;
    } else {
      // L1 operand: (z, wi', wo', 1, 0); the 1 meets the bias column of W1
      uint32_t v[8] = {zp[0], zp[1], zp[2], zp[3], ptx::pack_h2(xl[0], xl[1]), ptx::pack_h2(xl[2], xl[3]),
                       ptx::pack_h2(xl[4], xl[5]), 0x00003C00u};
      ptx::tmem_st8(tAl, v);
      ptx::tmem_st_wait();
      if (!mma_stage([&] { ptx::mma_f16_ts(tD, tA, ptx::sdesc(aW + O.b_l1, H * 16, 128), ID_H, 0); }))
        break;
    }

    // hidden -> hidden and hidden -> out share the epilogue: TMEM row ->
    // ReLU -> FP16 (or scaled E4M3) -> A operand
    bool ok = true;
#pragma unroll
    for (int layer = 0; layer < NH; ++layer) {
      constexpr int NC = H < 32 ? H : 32;
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += NC) {
        uint32_t acc[NC];
        if constexpr (NC == 32) {
          ptx::tmem_ld32(tDl + c0, acc);
        } else {
          ptx::tmem_ld16(tDl + c0, acc);
        }
        ptx::tmem_ld_wait();
        if (P8) {
          // code = E4M3(relu(D c_l + b'_l)), four codes per 32-bit word
          const float cl = sc8[1 + layer];
          const float2 c2v = make_float2(cl, cl);
          const float4* bq = reinterpret_cast<const float4*>(sW + (layer == 0 ? Lay8::B_B1 : Lay8::B_B2)) + c0 / 4;
          uint32_t pk[NC / 4];
#pragma unroll
          for (int j = 0; j < NC / 4; ++j) {
            const float4 b = bq[j];
            const float2 q01 = ptx::fma2(make_float2(u2f(acc[4 * j]), u2f(acc[4 * j + 1])), c2v, make_float2(b.x, b.y));
            const float2 q23 =
                ptx::fma2(make_float2(u2f(acc[4 * j + 2]), u2f(acc[4 * j + 3])), c2v, make_float2(b.z, b.w));
            pk[j] = ptx::pack_e4m3x2_relu(q01.x, q01.y) | (ptx::pack_e4m3x2_relu(q23.x, q23.y) << 16);
          }
#pragma unroll
          for (int b = 0; b < NC / 16; ++b)
            ptx::st_shared_v4(aA8 + (c0 / 16 + b) * 2048 + r * 16, pk[4 * b], pk[4 * b + 1], pk[4 * b + 2],
                              pk[4 * b + 3]);
        } else {
          uint32_t pk[NC / 2];
#pragma unroll
          for (int j = 0; j < NC / 2; ++j) pk[j] = ptx::pack_h2_relu(u2f(acc[2 * j]), u2f(acc[2 * j + 1]));
          if constexpr (NC == 32) {
            ptx::tmem_st16(tAl + c0 / 2, pk);
          } else {
            ptx::tmem_st8(tAl + c0 / 2, pk);
          }
        }
      }
      if (!P8) ptx::tmem_st_wait();
      bool staged;
      if (P8) {
        const int boff = layer == 0 ? Lay8::B_L2 : Lay8::B_LO;
        const int nrows = layer == 0 ? H : 16;
        const uint32_t id = layer == 0 ? ID8_H : ID8_16;
        staged = mma_stage([&] {
          // K steps of 32 codes = two 16-code blocks; an odd last block pairs
          // with the zero block
#pragma unroll
          for (int s2 = 0; s2 < (H + 31) / 32; ++s2) {
            const uint32_t a0 = aA8 + s2 * 4096;
            const uint32_t lbo = (2 * s2 + 1 < H / 16) ? 2048u : (aZ8 - a0);
            ptx::mma_f8(tD, ptx::sdesc(a0, lbo, 128), ptx::sdesc(aW + boff + s2 * 2 * nrows * 16, nrows * 16, 128),
                        id, s2 > 0 ? 1u : 0u);
          }
        });
      } else {
        const bool last = layer == NH - 1;
        const int boff = last ? O.b_lo : O.b_l2 + layer * H * (H + 16) * 2;
        const int nrows = last ? 16 : H;
        const uint32_t id = last ? ID_16 : ID_H;
        staged = mma_stage([&] {
#pragma unroll
          for (int s2 = 0; s2 < H / 16; ++s2)
            ptx::mma_f16_ts(tD, tA + 8 * s2, ptx::sdesc(aW + boff + s2 * 2 * nrows * 16, nrows * 16, 128), id,
                            s2 > 0 ? 1u : 0u);
          // bias step: (constant block, zero block) x B blocks (H/8, H/8+1)
          ptx::mma_f16(tD, ptx::sdesc(aConst, 2048, 128),
                       ptx::sdesc(aW + boff + (H / 8) * nrows * 16, nrows * 16, 128), id, 1u);
        });
      }
      if (!staged) {
        ok = false;
        break;
      }
    }
    if (!ok) break;

    // ---- 5. output ----------------------------------------------------------
    {
      uint32_t acc[4];
      ptx::tmem_ld4(tDl, acc);
      ptx::tmem_ld_wait();
      float y0 = u2f(acc[0]), y1 = u2f(acc[1]), y2 = u2f(acc[2]);
      if (P8) {
        const float c2 = sc8[3];
        const float* b3 = reinterpret_cast<const float*>(sW + Lay8::B_B3);
        y0 = fmaf(y0, c2, b3[0]);
        y1 = fmaf(y1, c2, b3[1]);
        y2 = fmaf(y2, c2, b3[2]);
      }
      if (L.albedo) {
        // albedo head: output columns 3..5 (no cosine factor)
        uint32_t acc2[4];
        ptx::tmem_ld4(tDl + 4, acc2);
        ptx::tmem_ld_wait();
        float a0 = u2f(acc[3]), a1 = u2f(acc2[0]), a2 = u2f(acc2[1]);
        if (P8) {
          const float c2 = sc8[3];
          const float* b3 = reinterpret_cast<const float*>(sW + Lay8::B_B3);
          a0 = fmaf(a0, c2, b3[3]);
          a1 = fmaf(a1, c2, b3[4]);
          a2 = fmaf(a2, c2, b3[5]);
        }
        if (valid && row_mat == ci.mat) {
          L.albedo[3 * i + 0] = a0;
          L.albedo[3 * i + 1] = a1;
          L.albedo[3 * i + 2] = a2;
        }
      }
      if (cosine) {
        const float cz = fmaxf(qc.wiz, 0.0f);
        y0 *= cz; y1 *= cz; y2 *= cz;
      }
      if (valid && row_mat == ci.mat) {
        L.rgb[3 * i + 0] = y0;
        L.rgb[3 * i + 1] = y1;
        L.rgb[3 * i + 2] = y2;
      }
    }
    ptx::tc_fence_before();
    ci = cn;
    qc = qn;
  }

  // ---- teardown -------------------------------------------------------------
  // MMAs and bulk copies still in flight after a wait gave up are waited for
  // with the fixed drain limit (not the caller's), and TMEM is freed only if
  // they all completed.
  bool drained = true;
  if (r == 0) {
    if (mma_pending) drained &= ptx::mbar_wait(bar_m, ph_m ^ 1, ptx::kDrainTimeoutNs);
    if (w_pending) drained &= ptx::mbar_wait(bar_w, ph_w ^ 1, ptx::kDrainTimeoutNs);
    if (bad) record_error(L.err, DEVERR_WAIT_TIMEOUT);
    if (!drained) record_error(L.err, DEVERR_DRAIN_TIMEOUT);
  }
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
template <int H, int FK, int NH, bool F16P, bool P8>
static int launch_tc_one(const LaunchCommon& L, cudaStream_t s) {
  constexpr int SMEM = smem_bytes<H, FK, NH, P8, kNwg>();
  auto k = eval_tc_kernel<H, FK, NH, F16P, P8, kNwg>;
  static std::atomic<uint64_t> configured{0};
  once_per_device(configured, [&] {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    // ask for the smallest shared-memory carveout that holds the CTA: the
    // rest of the SM's L1/shared storage caches the texel gathers
    const int pct = (SMEM + 1024) * 100 / (228 * 1024) + 1;
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  });
  const int64_t nchunks = L.chunks ? (int64_t)L.n_chunks : (L.n + 127) / 128;
  if (nchunks == 0) return 0;
  // one CTA per SM (TMEM: kNwg x 96 of 512 columns)
  const int64_t want = (nchunks + kNwg - 1) / kNwg;
  const int grid = (int)(want < L.num_sms ? want : L.num_sms);
  k<<<grid, kNwg * 128, SMEM, s>>>(L);
  return (int)cudaGetLastError();
}

template <int H, int NH, bool P8>
static int tc_dispatch(const LaunchCommon& L, cudaStream_t s) {
  const bool f16 = L.pyr.f16;
  if (L.shape.frame == 1)
    return f16 ? launch_tc_one<H, 1, NH, true, P8>(L, s) : launch_tc_one<H, 1, NH, false, P8>(L, s);
  if constexpr (!P8) {
    if (L.shape.frame == 2)
      return f16 ? launch_tc_one<H, 2, NH, true, P8>(L, s) : launch_tc_one<H, 2, NH, false, P8>(L, s);
  }
  if (L.shape.frame != 0) return (int)cudaErrorInvalidValue;
  return f16 ? launch_tc_one<H, 0, NH, true, P8>(L, s) : launch_tc_one<H, 0, NH, false, P8>(L, s);
}

int launch_eval_tc(const LaunchCommon& L, int precision, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == NAM_PREC_F16) return launch_eval_f16(L, stream);
  if (!tc_supported(L.shape, precision)) return (int)cudaErrorInvalidValue;
  if (L.shape.H == 16) return tc_dispatch<16, 2, true>(L, s);
  if (L.shape.H == 32) return tc_dispatch<32, 2, true>(L, s);
  return tc_dispatch<64, 2, true>(L, s);
}

}  // namespace nam
