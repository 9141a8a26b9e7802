// Plain FP32 evaluation: one query per thread, MLP weights staged in shared
// memory, FP32 FMA on CUDA cores.  This is the "divergent" per-thread form
// of the decoder (Sec. 7.1: whole network per thread, unrolled FMAs) and the
// FP32 reference point the reduced-precision tensor-core path is compared to.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstring>

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

// One query's evaluation from a parameter image S (shared memory in the
// staged kernel, a material's global image in the divergent one): latent
// fetch, frame, direction transform, decoder; y = RGB.  With `calib` the
// maxima of |layer input| are folded into am0..am2.
template <int H, int NH, int FK, bool F16>
__device__ __forceinline__ void eval_query(const SmemF32<H, NH, FK, FK == 2 ? 20 : 16>& S, const PyrDesc& pd,
                                           const void* pyr, const QueryPtrs& q, int64_t i, bool cosine, bool calib,
                                           float& am0, float& am1, float& am2, float y[3]) {
  constexpr int INP = FK == 2 ? 20 : 16;
  float z[8];
  const float xi = q.xi ? q.xi[i] : 0.0f;
  fetch_latent<F16>(pd, pyr, q.u[i], q.v[i], q.lod[i], xi, z);
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
  y[0] = y0;
  y[1] = y1;
  y[2] = y2;
}

template <int H, int NH, int FK, bool F16>
__global__ void __launch_bounds__(128) eval_f32_kernel(LaunchCommon L) {
  constexpr int INP = FK == 2 ? 20 : 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemF32<H, NH, FK, INP>& S = *reinterpret_cast<SmemF32<H, NH, FK, INP>*>(smem_raw);
  load_params_f32<H, NH, FK, INP>(S, reinterpret_cast<const float*>(L.w0), FK == 2 ? 20 : 14);
  __syncthreads();
  const bool cosine = (L.flags & NAM_OUT_COSINE) != 0;
  const bool calib = L.amax != nullptr;
  float am0 = 0.0f, am1 = 0.0f, am2 = 0.0f;  // calibration: max |layer input|
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float y[3];
    eval_query<H, NH, FK, F16>(S, L.pyr, L.pyr0, L.q, i, cosine, calib, am0, am1, am2, y);
    if (L.rgb) {
      L.rgb[3 * i + 0] = y[0];
      L.rgb[3 * i + 1] = y[1];
      L.rgb[3 * i + 2] = y[2];
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

// ---------------------------------------------------------------------------
// divergent path of per-tile selection
// ---------------------------------------------------------------------------
// Tiles of many materials: one query per thread, each thread reading the
// weights of its own material from that material's global image (Sec. 7.1:
// the divergent code path evaluates the whole network per thread with FMAs
// and leaves divergence to the SIMT hardware).  A warp whose queries share a
// material issues each weight load once for all lanes; a warp over k
// materials issues it for k addresses.
template <int H, int NH, int FK, bool F16>
__global__ void __launch_bounds__(128) eval_divergent_kernel(const LaunchCommon L,
                                                             const float* const* __restrict__ images,
                                                             const int32_t* __restrict__ ids,
                                                             const int32_t* __restrict__ tiles,
                                                             const int32_t* __restrict__ n_tiles) {
  using Img = SmemF32<H, NH, FK, FK == 2 ? 20 : 16>;
  const bool cosine = (L.flags & NAM_OUT_COSINE) != 0;
  const int32_t count = *n_tiles;
  for (int32_t j = blockIdx.x; j < count; j += gridDim.x) {
    const int64_t i = (int64_t)__ldg(tiles + j) * 128 + threadIdx.x;
    if (i >= L.n) continue;
    const int m = __ldg(ids + i);
    if (m < 0 || m >= L.mats.nmat) continue;  // recorded by the selection pass
    const Img& S = *reinterpret_cast<const Img*>(images[m]);
    float am0 = 0.0f, am1 = 0.0f, am2 = 0.0f, y[3];
    eval_query<H, NH, FK, F16>(S, L.pyr, L.mats.pyramid[m], L.q, i, cosine, false, am0, am1, am2, y);
    L.rgb[3 * i + 0] = y[0];
    L.rgb[3 * i + 1] = y[1];
    L.rgb[3 * i + 2] = y[2];
  }
}

template <int H, int NH, int FK, bool F16>
static int launch_divergent_one(const LaunchCommon& L, const float* const* images, const int32_t* ids,
                                const int32_t* tiles, const int32_t* n_tiles, cudaStream_t s) {
  auto k = eval_divergent_kernel<H, NH, FK, F16>;
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> occ{0};
  once_per_device(configured, [&] { occ.store(blocks_per_sm((const void*)k, 128, 0, 16)); });
  const int64_t most = (L.n + 127) / 128;  // the divergent tiles are at most all of them
  const int64_t cap = (int64_t)occ.load() * L.num_sms;
  int grid = (int)(most < cap ? most : cap);
  if (grid < 1) grid = 1;
  k<<<grid, 128, 0, s>>>(L, images, ids, tiles, n_tiles);
  return (int)cudaGetLastError();
}

template <int H, int NH>
static int divergent_frame(const LaunchCommon& L, const float* const* images, const int32_t* ids,
                           const int32_t* tiles, const int32_t* n_tiles, cudaStream_t s) {
  const bool f16 = L.pyr.f16;
  switch (L.shape.frame) {
    case 1: return f16 ? launch_divergent_one<H, NH, 1, true>(L, images, ids, tiles, n_tiles, s)
                       : launch_divergent_one<H, NH, 1, false>(L, images, ids, tiles, n_tiles, s);
    case 2: return f16 ? launch_divergent_one<H, NH, 2, true>(L, images, ids, tiles, n_tiles, s)
                       : launch_divergent_one<H, NH, 2, false>(L, images, ids, tiles, n_tiles, s);
    default: return f16 ? launch_divergent_one<H, NH, 0, true>(L, images, ids, tiles, n_tiles, s)
                        : launch_divergent_one<H, NH, 0, false>(L, images, ids, tiles, n_tiles, s);
  }
}

int launch_eval_divergent(const LaunchCommon& L, const float* const* images, const int32_t* ids,
                          const int32_t* tiles, const int32_t* n_tiles, void* stream) {
  if (L.n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const Shape& sh = L.shape;
  if (sh.NH == 2) {
    if (sh.H == 16) return divergent_frame<16, 2>(L, images, ids, tiles, n_tiles, s);
    if (sh.H == 32) return divergent_frame<32, 2>(L, images, ids, tiles, n_tiles, s);
    if (sh.H == 64) return divergent_frame<64, 2>(L, images, ids, tiles, n_tiles, s);
  }
  if (sh.NH == 3 && sh.H == 64) return divergent_frame<64, 3>(L, images, ids, tiles, n_tiles, s);
  return (int)cudaErrorInvalidValue;
}

// Host: the image in the staged layout, each value as the tensor-core blob
// encodes it.
template <int H, int NH, int FK>
static void pack_image(const float* frame, const float* dec, int in, int precision, const float* sw, float* out) {
  using Img = SmemF32<H, NH, FK, FK == 2 ? 20 : 16>;
  constexpr int INP = FK == 2 ? 20 : 16;
  std::memset(out, 0, sizeof(Img));
  Img& S = *reinterpret_cast<Img*>(out);
  auto h = [](float v) { return __half2float(__float2half_rn(v)); };
  const bool p8 = precision == NAM_PREC_FP8;
  auto wq = [&](float v, int layer) { return p8 ? e4m3_dequant(v, sw[layer]) : h(v); };
  auto bq = [&](float v) { return p8 ? v : h(v); };
  if (FK == 1) {
    for (int i = 0; i < 128; ++i) S.fW1[i] = h(frame[i]);
    for (int i = 0; i < 16; ++i) S.fb1[i] = h(frame[128 + i]);
    for (int i = 0; i < 96; ++i) S.fW2[i] = h(frame[144 + i]);
    for (int i = 0; i < 6; ++i) S.fb2[i] = h(frame[240 + i]);
  } else if (FK == 2) {
    for (int i = 0; i < 96; ++i) S.fW1[i] = h(frame[i]);
    for (int i = 0; i < 12; ++i) S.fb1[i] = h(frame[96 + i]);
  }
  const float* p = dec;
  for (int j = 0; j < H; ++j)
    for (int k = 0; k < in; ++k) S.W1[j * INP + k] = wq(p[j * in + k], 0);
  p += in * H;
  for (int j = 0; j < H; ++j) S.b1[j] = bq(p[j]);
  p += H;
  for (int l = 0; l < NH - 1; ++l) {
    for (int i = 0; i < H * H; ++i) S.Wh[l][i] = wq(p[i], 1 + l);
    p += H * H;
    for (int j = 0; j < H; ++j) S.bh[l][j] = bq(p[j]);
    p += H;
  }
  for (int j = 0; j < H; ++j)
    for (int c = 0; c < 3; ++c) S.WoT[j * 4 + c] = wq(p[c * H + j], NH);
  p += 3 * H;
  for (int c = 0; c < 3; ++c) S.bo[c] = bq(p[c]);
}

template <int H, int NH>
static size_t image_floats_hn(int frame) {
  switch (frame) {
    case 1: return sizeof(SmemF32<H, NH, 1, 16>) / 4;
    case 2: return sizeof(SmemF32<H, NH, 2, 20>) / 4;
    default: return sizeof(SmemF32<H, NH, 0, 16>) / 4;
  }
}

size_t simt_image_floats(const Shape& s) {
  if (s.NH == 2 && s.H == 16) return image_floats_hn<16, 2>(s.frame);
  if (s.NH == 2 && s.H == 32) return image_floats_hn<32, 2>(s.frame);
  if (s.NH == 2 && s.H == 64) return image_floats_hn<64, 2>(s.frame);
  if (s.NH == 3 && s.H == 64) return image_floats_hn<64, 3>(s.frame);
  return 0;
}

template <int H, int NH>
static void pack_image_hn(const Shape& s, int precision, const float* frame, const float* dec, const float* sw,
                          float* out) {
  switch (s.frame) {
    case 1: return pack_image<H, NH, 1>(frame, dec, s.in, precision, sw, out);
    case 2: return pack_image<H, NH, 2>(frame, dec, s.in, precision, sw, out);
    default: return pack_image<H, NH, 0>(frame, dec, s.in, precision, sw, out);
  }
}

void pack_simt_image(const Shape& s, int precision, const float* frame, const float* dec, const float* sw,
                     float* out) {
  if (s.NH == 2 && s.H == 16) return pack_image_hn<16, 2>(s, precision, frame, dec, sw, out);
  if (s.NH == 2 && s.H == 32) return pack_image_hn<32, 2>(s, precision, frame, dec, sw, out);
  if (s.NH == 2 && s.H == 64) return pack_image_hn<64, 2>(s, precision, frame, dec, sw, out);
  if (s.NH == 3 && s.H == 64) return pack_image_hn<64, 3>(s, precision, frame, dec, sw, out);
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
