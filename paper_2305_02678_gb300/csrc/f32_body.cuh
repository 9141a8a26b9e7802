// The per-query body of the FP32 evaluation (weights staged in shared
// memory): the parameter image layout, its loader, and one query's
// evaluation.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace nam {

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
  float WaT[H * 4];         // albedo head: its output weights transposed [H][4]
  float ba[4];              // (zero without the head)
};

template <int H, int NH, int FK, int INP>
__device__ void load_params_f32(SmemF32<H, NH, FK, INP>& S, const float* __restrict__ p, int in, int out) {
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
  const bool alb = out == 6;
  for (int i = tid; i < H * 4; i += nt) {
    int j = i >> 2, c = i & 3;
    S.WoT[i] = c < 3 ? p[c * H + j] : 0.0f;
    S.WaT[i] = alb && c < 3 ? p[(3 + c) * H + j] : 0.0f;
  }
  p += out * H;
  for (int i = tid; i < 4; i += nt) {
    S.bo[i] = i < 3 ? p[i] : 0.0f;
    S.ba[i] = alb && i < 3 ? p[3 + i] : 0.0f;
  }
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

// One query's evaluation from the parameter image S in shared memory: latent
// fetch, frame, direction transform, decoder; y = RGB.  With `calib` the
// maxima of |layer input| are folded into am0..am2; with `alb` the albedo
// head's outputs (no cosine factor: the albedo depends on x and wo alone)
// go to alb_out.
template <int H, int NH, int FK, bool F16>
__device__ __forceinline__ void eval_query(const SmemF32<H, NH, FK, FK == 2 ? 20 : 16>& S, const PyrDesc& pd,
                                           const void* pyr, const QueryPtrs& q, int64_t i, bool cosine, bool calib,
                                           float& am0, float& am1, float& am2, float y[3], bool alb = false,
                                           float* alb_out = nullptr) {
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
  float a0 = S.ba[0], a1 = S.ba[1], a2 = S.ba[2];
  if (NH == 2) {
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
      float s = fmaxf(S.bh[0][j] + dot_row<H>(&S.Wh[0][j * H], h1), 0.0f);
      am2 = fmaxf(am2, s);
      float4 wo = reinterpret_cast<const float4*>(S.WoT)[j];
      y0 = fmaf(wo.x, s, y0);
      y1 = fmaf(wo.y, s, y1);
      y2 = fmaf(wo.z, s, y2);
      if (alb) {
        const float4 wa = reinterpret_cast<const float4*>(S.WaT)[j];
        a0 = fmaf(wa.x, s, a0);
        a1 = fmaf(wa.y, s, a1);
        a2 = fmaf(wa.z, s, a2);
      }
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
      if (alb) {
        const float4 wa = reinterpret_cast<const float4*>(S.WaT)[j];
        a0 = fmaf(wa.x, s, a0);
        a1 = fmaf(wa.y, s, a1);
        a2 = fmaf(wa.z, s, a2);
      }
    }
  }
  if (alb) {
    alb_out[0] = a0;
    alb_out[1] = a1;
    alb_out[2] = a2;
  }
  if (cosine) {
    float c = fmaxf(wiz, 0.0f);
    y0 *= c; y1 *= c; y2 *= c;
  }
  y[0] = y0;
  y[1] = y1;
  y[2] = y2;
}

}  // namespace nam
