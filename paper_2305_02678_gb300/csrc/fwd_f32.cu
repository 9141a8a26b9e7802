// Plain FP32 evaluation: one query per thread, MLP weights staged in shared
// memory, FP32 FMA on CUDA cores.  This is the "divergent" per-thread form
// of the decoder (Sec. 7.1: whole network per thread, unrolled FMAs) and the
// FP32 reference point the reduced-precision tensor-core path is compared to.
// With the albedo head the kernel also writes the albedo triplet.
#include <cuda_runtime.h>

#include "common.cuh"
#include "f32_body.cuh"

namespace nam {

int64_t n_params_of(const Shape& s) {
  int64_t n = frame_params_of(s.frame);
  n += (int64_t)s.in * s.H + s.H;
  for (int i = 1; i < s.NH; ++i) n += (int64_t)s.H * s.H + s.H;
  n += (int64_t)s.out * s.H + s.out;
  return n;
}

template <int H, int NH, int FK, bool F16>
__global__ void __launch_bounds__(128) eval_f32_kernel(LaunchCommon L) {
  constexpr int INP = FK == 2 ? 20 : 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemF32<H, NH, FK, INP>& S = *reinterpret_cast<SmemF32<H, NH, FK, INP>*>(smem_raw);
  load_params_f32<H, NH, FK, INP>(S, reinterpret_cast<const float*>(L.w0), FK == 2 ? 20 : 14, L.shape.out);
  __syncthreads();
  const bool cosine = (L.flags & NAM_OUT_COSINE) != 0;
  const bool calib = L.amax != nullptr;
  const bool alb = L.albedo != nullptr && L.shape.out == 6;
  float am0 = 0.0f, am1 = 0.0f, am2 = 0.0f;  // calibration: max |layer input|
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float y[3], a[3];
    eval_query<H, NH, FK, F16>(S, L.pyr, L.pyr0, L.q, i, cosine, calib, am0, am1, am2, y, alb, a);
    if (alb) {
      L.albedo[3 * i + 0] = a[0];
      L.albedo[3 * i + 1] = a[1];
      L.albedo[3 * i + 2] = a[2];
    }
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
