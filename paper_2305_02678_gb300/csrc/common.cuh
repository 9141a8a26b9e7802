// Device helpers shared by the libnam kernels: latent-pyramid fetch and
// shading-frame construction.  One thread evaluates one query.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "nam_internal.h"

namespace nam {

// Level index of a query (Sec. 4.1: the level may be fractional and lie
// between two levels).  l = clamp(lod, 0, L-1) (NaN -> 0), l0 = floor(l),
// l1 = min(l0+1, L-1), t = l - l0.
struct LevelPick {
  int l0, l1;
  float t;
};

__device__ __forceinline__ LevelPick pick_levels(const PyrDesc& P, float lod) {
  float l = fminf(fmaxf(lod, 0.0f), (float)(P.levels - 1));  // fmaxf(NaN, 0) = 0
  float f = floorf(l);
  LevelPick r;
  r.l0 = (int)f;
  r.l1 = min(r.l0 + 1, P.levels - 1);
  r.t = l - f;
  return r;
}

// Integer texel coordinate of the lower bilinear tap and its fraction, plus
// the upper tap, under the material's addressing.  Texel centres sit at
// (i + 1/2) / W, so the continuous coordinate is x = u W - 1/2.  X = u W is
// exact for power-of-two W; the 1/2 is then applied to X's fractional part
// (which cannot lose bits, unlike X - 1/2 itself when |X - 1/2| crosses a
// power of two), so tap index and fraction are exact while |X| < 2^23.
// Larger |X| (no fraction left in FP32) is reduced with the exact fmodf for
// wrap; non-finite coordinates read texel 0.
__device__ __forceinline__ void tap_axis(const PyrDesc& P, float u, int W, int& i0, int& i1, float& f) {
  float X = u * (float)W;
  if (!(fabsf(X) < 8388608.0f)) X = isfinite(X) ? (P.address == NAM_ADDRESS_CLAMP ? X : fmodf(X, (float)W)) : 0.0f;
  const float Xf = floorf(X);
  const float r = X - Xf;  // [0, 1]
  float x0;
  if (r >= 0.5f) {
    x0 = Xf;
    f = r - 0.5f;
  } else {
    x0 = Xf - 1.0f;
    f = r + 0.5f;
  }
  if (P.address == NAM_ADDRESS_CLAMP) {
    // clamp in float first so that huge |u| cannot overflow the int conversion
    i0 = (int)fminf(fmaxf(x0, 0.0f), (float)(W - 1));
    i1 = (int)fminf(fmaxf(x0 + 1.0f, 0.0f), (float)(W - 1));
  } else {
    int k = (int)x0;  // |k| <= 2^23
    if (P.pow2) {
      i0 = k & (W - 1);
      i1 = (k + 1) & (W - 1);
    } else {
      k %= W;
      if (k < 0) k += W;
      i0 = k;
      i1 = k + 1 == W ? 0 : k + 1;
    }
  }
}

// Accumulate wgt * bilinear(level l) into z[8].
template <bool F16>
__device__ __forceinline__ void bilinear_acc(const PyrDesc& P, const void* pyr, int l, float u, float v,
                                             float wgt, float z[8]) {
  const int W = P.w[l], H = P.h[l];
  int x0, x1, y0, y1;
  float fx, fy;
  tap_axis(P, u, W, x0, x1, fx);
  tap_axis(P, v, H, y0, y1, fy);
  // texel indices fit 32 bits (pyramids up to 2^32 texels, 64 GiB at FP16)
  const uint32_t base = (uint32_t)P.off[l];
  const uint32_t r0 = base + (uint32_t)y0 * (uint32_t)W, r1 = base + (uint32_t)y1 * (uint32_t)W;
  const uint32_t idx[4] = {r0 + x0, r0 + x1, r1 + x0, r1 + x1};
  const float gx = 1.0f - fx, gy = 1.0f - fy;
  const float w4[4] = {gx * gy * wgt, fx * gy * wgt, gx * fy * wgt, fx * fy * wgt};
  if (F16) {
    const uint4* p = reinterpret_cast<const uint4*>(pyr);
    uint4 t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] = __ldg(p + idx[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __half2* h = reinterpret_cast<const __half2*>(&t[k]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float2 f2 = __half22float2(h[c]);
        z[2 * c] = fmaf(w4[k], f2.x, z[2 * c]);
        z[2 * c + 1] = fmaf(w4[k], f2.y, z[2 * c + 1]);
      }
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(pyr);
    float4 a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = __ldg(p + 2 * (size_t)idx[k]);
      b[k] = __ldg(p + 2 * (size_t)idx[k] + 1);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      z[0] = fmaf(w4[k], a[k].x, z[0]);
      z[1] = fmaf(w4[k], a[k].y, z[1]);
      z[2] = fmaf(w4[k], a[k].z, z[2]);
      z[3] = fmaf(w4[k], a[k].w, z[3]);
      z[4] = fmaf(w4[k], b[k].x, z[4]);
      z[5] = fmaf(w4[k], b[k].y, z[5]);
      z[6] = fmaf(w4[k], b[k].z, z[6]);
      z[7] = fmaf(w4[k], b[k].w, z[7]);
    }
  }
}

// Filtered latent code z(x) (Sec. 4.1).  Trilinear blends the two levels
// with weights 1-t and t (the upper level is skipped when t == 0, where its
// weight is zero); stochastic takes l1 when xi < t and l0 otherwise.
template <bool F16>
__device__ __forceinline__ void fetch_latent(const PyrDesc& P, const void* pyr, float u, float v, float lod,
                                             float xi, float z[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) z[c] = 0.0f;
  LevelPick lp = pick_levels(P, lod);
  if (P.filter == NAM_FILTER_STOCHASTIC) {
    bilinear_acc<F16>(P, pyr, xi < lp.t ? lp.l1 : lp.l0, u, v, 1.0f, z);
  } else {
    bilinear_acc<F16>(P, pyr, lp.l0, u, v, 1.0f - lp.t, z);
    if (lp.t != 0.0f) bilinear_acc<F16>(P, pyr, lp.l1, u, v, lp.t, z);
  }
}

// The same fetch split in two so that the texel loads can be issued a tile
// ahead of their use (FP16 pyramids): issue_taps computes the (up to) eight
// tap indices and weights and starts the 16-byte loads; finish_taps filters.
// Taps of a level with zero weight are not loaded.
struct Taps8 {
  uint4 t[8];
  float w[8];
};

__device__ __forceinline__ void level_taps_f16(const PyrDesc& P, const uint4* __restrict__ p, int l, float u, float v,
                                               float wgt, uint4* t, float* w) {
  const int W = P.w[l], H = P.h[l];
  int x0, x1, y0, y1;
  float fx, fy;
  tap_axis(P, u, W, x0, x1, fx);
  tap_axis(P, v, H, y0, y1, fy);
  const uint32_t base = (uint32_t)P.off[l];
  const uint32_t r0 = base + (uint32_t)y0 * (uint32_t)W, r1 = base + (uint32_t)y1 * (uint32_t)W;
  const float gx = 1.0f - fx, gy = 1.0f - fy;
  w[0] = gx * gy * wgt;
  w[1] = fx * gy * wgt;
  w[2] = gx * fy * wgt;
  w[3] = fx * fy * wgt;
  t[0] = __ldg(p + r0 + x0);
  t[1] = __ldg(p + r0 + x1);
  t[2] = __ldg(p + r1 + x0);
  t[3] = __ldg(p + r1 + x1);
}

__device__ __forceinline__ void issue_taps(const PyrDesc& P, const void* pyr, float u, float v, float lod, float xi,
                                           Taps8& T) {
  const uint4* p = reinterpret_cast<const uint4*>(pyr);
  LevelPick lp = pick_levels(P, lod);
  if (P.filter == NAM_FILTER_STOCHASTIC) {
    level_taps_f16(P, p, xi < lp.t ? lp.l1 : lp.l0, u, v, 1.0f, T.t, T.w);
  } else {
    level_taps_f16(P, p, lp.l0, u, v, 1.0f - lp.t, T.t, T.w);
    if (lp.t != 0.0f) {
      level_taps_f16(P, p, lp.l1, u, v, lp.t, T.t + 4, T.w + 4);
      return;
    }
  }
#pragma unroll
  for (int k = 4; k < 8; ++k) {
    T.t[k] = make_uint4(0u, 0u, 0u, 0u);
    T.w[k] = 0.0f;
  }
}

// Packed FP32x2 FMA (sm_100 family); defined with the tensor-core helpers.
__device__ __forceinline__ float2 fma2_f32(float2 a, float2 b, float2 c) {
  unsigned long long ra = *reinterpret_cast<unsigned long long*>(&a);
  unsigned long long rb = *reinterpret_cast<unsigned long long*>(&b);
  unsigned long long rc = *reinterpret_cast<unsigned long long*>(&c);
  unsigned long long rd;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  return *reinterpret_cast<float2*>(&rd);
}

__device__ __forceinline__ void finish_taps(const Taps8& T, float z[8]) {
  float2 acc[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const __half2* h = reinterpret_cast<const __half2*>(&T.t[k]);
    const float2 wk = make_float2(T.w[k], T.w[k]);
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = fma2_f32(wk, __half22float2(h[c]), acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    z[2 * c] = acc[c].x;
    z[2 * c + 1] = acc[c].y;
  }
}

// Shading frame from r = (n_raw, t_raw) (Sec. 4.2, Eq. 4; b = n x t / |n x t|,
// Sec. 9): n = n_raw / |n_raw|, t = Gram-Schmidt of t_raw against n,
// normalised.  Degenerate inputs: |n_raw| < 1e-20 -> n = (0,0,1);
// |t'| <= 1e-6 |t_raw| -> t from n alone (branch-free orthonormal basis of
// Duff et al., JCGT 2017).  Writes T's rows t, b, n.
struct Frame {
  float t[3], b[3], n[3];
};

__device__ __forceinline__ Frame build_frame(const float r[6]) {
  Frame F;
  const float nl2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  if (!(nl2 >= 1e-40f)) {
    F.n[0] = 0.0f; F.n[1] = 0.0f; F.n[2] = 1.0f;
  } else {
    const float inv = rsqrtf(nl2);
    F.n[0] = r[0] * inv; F.n[1] = r[1] * inv; F.n[2] = r[2] * inv;
  }
  const float s = r[3] * F.n[0] + r[4] * F.n[1] + r[5] * F.n[2];
  const float tp0 = r[3] - s * F.n[0], tp1 = r[4] - s * F.n[1], tp2 = r[5] - s * F.n[2];
  const float tpl2 = tp0 * tp0 + tp1 * tp1 + tp2 * tp2;
  const float trl2 = r[3] * r[3] + r[4] * r[4] + r[5] * r[5];
  if (!(tpl2 > 1e-12f * trl2)) {
    const float sg = copysignf(1.0f, F.n[2]);
    const float a = -1.0f / (sg + F.n[2]);
    const float bb = F.n[0] * F.n[1] * a;
    F.t[0] = 1.0f + sg * F.n[0] * F.n[0] * a;
    F.t[1] = sg * bb;
    F.t[2] = -sg * F.n[0];
  } else {
    const float inv = rsqrtf(tpl2);
    F.t[0] = tp0 * inv; F.t[1] = tp1 * inv; F.t[2] = tp2 * inv;
  }
  const float c0 = F.n[1] * F.t[2] - F.n[2] * F.t[1];
  const float c1 = F.n[2] * F.t[0] - F.n[0] * F.t[2];
  const float c2 = F.n[0] * F.t[1] - F.n[1] * F.t[0];
  const float inv = rsqrtf(c0 * c0 + c1 * c1 + c2 * c2);
  F.b[0] = c0 * inv; F.b[1] = c1 * inv; F.b[2] = c2 * inv;
  return F;
}

// One frame of the paper's form (Sec. 4.2, Eq. 4; Sec. 9) from r = (n_raw,
// t_raw): n and t normalised but not orthogonalised, b = n x t / |n x t|.
// Degenerate outputs: |n_raw|^2 < 1e-40 -> n = (0,0,1); |t_raw|^2 < 1e-40, or
// |n x t|^2 <= 1e-12 (parallel), -> t from n by Duff et al.'s basis.
__device__ __forceinline__ Frame paper_frame(const float r[6]) {
  Frame F;
  const float nl2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  if (!(nl2 >= 1e-40f)) {
    F.n[0] = 0.0f; F.n[1] = 0.0f; F.n[2] = 1.0f;
  } else {
    const float inv = rsqrtf(nl2);
    F.n[0] = r[0] * inv; F.n[1] = r[1] * inv; F.n[2] = r[2] * inv;
  }
  const float tl2 = r[3] * r[3] + r[4] * r[4] + r[5] * r[5];
  bool basis = !(tl2 >= 1e-40f);
  if (!basis) {
    const float inv = rsqrtf(tl2);
    F.t[0] = r[3] * inv; F.t[1] = r[4] * inv; F.t[2] = r[5] * inv;
  }
  float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
  if (!basis) {
    c0 = F.n[1] * F.t[2] - F.n[2] * F.t[1];
    c1 = F.n[2] * F.t[0] - F.n[0] * F.t[2];
    c2 = F.n[0] * F.t[1] - F.n[1] * F.t[0];
    basis = !(c0 * c0 + c1 * c1 + c2 * c2 > 1e-12f);
  }
  if (basis) {
    const float sg = copysignf(1.0f, F.n[2]);
    const float a = -1.0f / (sg + F.n[2]);
    const float bb = F.n[0] * F.n[1] * a;
    F.t[0] = 1.0f + sg * F.n[0] * F.n[0] * a;
    F.t[1] = sg * bb;
    F.t[2] = -sg * F.n[0];
    c0 = F.n[1] * F.t[2] - F.n[2] * F.t[1];
    c1 = F.n[2] * F.t[0] - F.n[0] * F.t[2];
    c2 = F.n[0] * F.t[1] - F.n[1] * F.t[0];
  }
  const float inv = rsqrtf(c0 * c0 + c1 * c1 + c2 * c2);
  F.b[0] = c0 * inv; F.b[1] = c1 * inv; F.b[2] = c2 * inv;
  return F;
}

__device__ __forceinline__ void to_local(const Frame& F, float x, float y, float z, float out[3]) {
  out[0] = F.t[0] * x + F.t[1] * y + F.t[2] * z;
  out[1] = F.b[0] * x + F.b[1] * y + F.b[2] * z;
  out[2] = F.n[0] * x + F.n[1] * y + F.n[2] * z;
}

// Record a device-side error code (first one wins).
__device__ __forceinline__ void record_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

}  // namespace nam
