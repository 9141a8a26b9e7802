// Divergent path of per-tile selection (Sec. 7.1) and the per-material FP32
// images it reads.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "common.cuh"
#include "f32_body.cuh"

namespace nam {

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
static void pack_image(const float* frame, const float* dec, int in, int n_out, int precision, const float* sw,
                       float* out) {
  using Img = SmemF32<H, NH, FK, FK == 2 ? 20 : 16>;
  constexpr int INP = FK == 2 ? 20 : 16;
  std::memset(out, 0, sizeof(Img));
  Img& S = *reinterpret_cast<Img*>(out);
  auto h = [](float v) { return __half2float(__float2half_rn(v)); };
  // FP8: E4M3 weights (times their layer scale) on the hidden -> hidden
  // layers only; every other parameter binary16, as in the tensor-core blob
  const bool p8 = precision == NAM_PREC_FP8;
  auto wq = [&](float v, int layer) { return p8 && layer >= 1 && layer < NH ? e4m3_dequant(v, sw[layer]) : h(v); };
  auto bq = [&](float v) { return h(v); };
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
  p += n_out * H;  // the albedo head's rows (if any) are not read by this path
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
    case 1: return pack_image<H, NH, 1>(frame, dec, s.in, s.out, precision, sw, out);
    case 2: return pack_image<H, NH, 2>(frame, dec, s.in, s.out, precision, sw, out);
    default: return pack_image<H, NH, 0>(frame, dec, s.in, s.out, precision, sw, out);
  }
}

void pack_simt_image(const Shape& s, int precision, const float* frame, const float* dec, const float* sw,
                     float* out) {
  if (s.NH == 2 && s.H == 16) return pack_image_hn<16, 2>(s, precision, frame, dec, sw, out);
  if (s.NH == 2 && s.H == 32) return pack_image_hn<32, 2>(s, precision, frame, dec, sw, out);
  if (s.NH == 2 && s.H == 64) return pack_image_hn<64, 2>(s, precision, frame, dec, sw, out);
  if (s.NH == 3 && s.H == 64) return pack_image_hn<64, 3>(s, precision, frame, dec, sw, out);
}

}  // namespace nam
