// Reverse mode of the FP32 evaluation, the log-space L1 loss and Adam
// (training of the decoder and the latent texture, Sec. 5).
//
// Backward kernel: a CTA of 128 threads takes tiles of 128 queries.
//  Phase A (thread = query): recompute the forward, then back-propagate
//   dL/drgb through the decoder, the direction transform, the frame
//   construction and the frame MLP to dL/dz; scatter tap_weight * dL/dz into
//   the pyramid gradient with vector atomics.  The per-query vectors every
//   weight gradient needs (layer inputs and output deltas) go to shared
//   memory.
//  Phase B (thread = weight): each thread owns a fixed set of weight and
//   bias gradients and sums their per-query outer-product terms over the
//   tile into registers.
//  The registers are added to the global gradient with one atomic per
//   parameter per CTA after the CTA's last tile.
#include <cuda_runtime.h>

#include "common.cuh"

namespace nam {

template <int H>
struct BwdSmem {
  static constexpr int S = H + 4;  // padded row stride (16-byte rows, no bank conflicts)
  // parameters
  float fW1[16 * 8], fb1[16], fW2[6 * 16], fb2[8];
  float W1[H * 16], b1[H];
  float W2[H * H], b2[H];
  float Wo[3 * H], bo[4];
  // per-query vectors of the current tile
  float Z[128][12];    // frame MLP input (z)
  float HF[128][20];   // frame hidden activations
  float DHF[128][20];  // delta at the frame hidden pre-activations
  float DR[128][8];    // delta at r = (n_raw, t_raw)
  float X[128][20];    // decoder input x (14)
  float D1[128][S];    // delta at decoder layer-1 pre-activations
  float H1[128][S];    // decoder layer-1 activations
  float D2[128][S];    // delta at layer-2 pre-activations
  float H2[128][S];    // layer-2 activations
  float DY[128][4];    // delta at the output (after the cosine factor)
};

template <int H, bool FRAME, bool F16>
__global__ void __launch_bounds__(128, 1) backward_kernel(const BackwardArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem<H>& S = *reinterpret_cast<BwdSmem<H>*>(smem_raw);
  const int t = threadIdx.x;
  // ---- parameters -> shared (master layout, W1 rows padded to 16) ----------
  {
    const float* p = A.params;
    if (FRAME) {
      for (int i = t; i < 128; i += 128) S.fW1[i] = p[i];
      if (t < 16) S.fb1[t] = p[128 + t];
      for (int i = t; i < 96; i += 128) S.fW2[i] = p[144 + i];
      if (t < 8) S.fb2[t] = t < 6 ? p[240 + t] : 0.0f;
      p += 246;
    }
    for (int i = t; i < H * 16; i += 128) {
      int j = i >> 4, k = i & 15;
      S.W1[i] = k < 14 ? p[j * 14 + k] : 0.0f;
    }
    p += 14 * H;
    for (int i = t; i < H; i += 128) S.b1[i] = p[i];
    p += H;
    for (int i = t; i < H * H; i += 128) S.W2[i] = p[i];
    p += H * H;
    for (int i = t; i < H; i += 128) S.b2[i] = p[i];
    p += H;
    for (int i = t; i < 3 * H; i += 128) S.Wo[i] = p[i];
    p += 3 * H;
    if (t < 4) S.bo[t] = t < 3 ? p[t] : 0.0f;
  }
  __syncthreads();

  // ---- phase-B ownership -----------------------------------------------------
  constexpr int PER2 = H * H / 128;          // dW2 entries per thread, one row segment
  const int j2 = (t * PER2) / H, k2 = (t * PER2) % H;
  float acc2[PER2];
#pragma unroll
  for (int i = 0; i < PER2; ++i) acc2[i] = 0.0f;
  constexpr int N1 = (14 * H + 127) / 128;   // dW1 entries (strided by 128)
  float acc1[N1];
#pragma unroll
  for (int i = 0; i < N1; ++i) acc1[i] = 0.0f;
  constexpr int NO = (3 * H + 127) / 128;    // dWo entries
  float accO[NO];
#pragma unroll
  for (int i = 0; i < NO; ++i) accO[i] = 0.0f;
  // small: bias slots (db1 H, db2 H, dbo 3, dbf1 16, dbf2 6) and frame weights
  constexpr int NB = (2 * H + 25 + 127) / 128;
  float accB[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) accB[i] = 0.0f;
  float accF1 = 0.0f, accF2 = 0.0f;

  const bool cosine = (A.flags & NAM_OUT_COSINE) != 0;
  const int64_t ntiles = (A.n + 127) / 128;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t start = tile * 128;
    const int count = (int)((A.n - start) < 128 ? (A.n - start) : 128);
    const bool valid = t < count;
    const int64_t i = start + (valid ? t : 0);
    // =================== phase A ===========================================
    float z[8];
    const float xi = A.q.xi ? A.q.xi[i] : 0.0f;
    const float u = A.q.u[i], v = A.q.v[i], lod = A.q.lod[i];
    fetch_latent<F16>(A.pyr, A.pyramid, u, v, lod, xi, z);
    const float wi[3] = {A.q.wix[i], A.q.wiy[i], A.q.wiz[i]};
    const float wo[3] = {A.q.wox[i], A.q.woy[i], A.q.woz[i]};
    float x[16];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = z[c];
    x[14] = 0.0f;
    x[15] = 0.0f;
    float hfp[16], r[6];
    Frame F;
    float nl = 0.0f, tpl = 0.0f, cl = 0.0f, sdot = 0.0f;
    bool ndeg = false, tdeg = false;
    if (FRAME) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float s = S.fb1[j];
#pragma unroll
        for (int c = 0; c < 8; ++c) s = fmaf(S.fW1[j * 8 + c], z[c], s);
        hfp[j] = s;
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        float s = S.fb2[j];
#pragma unroll
        for (int k = 0; k < 16; ++k) s = fmaf(S.fW2[j * 16 + k], fmaxf(hfp[k], 0.0f), s);
        r[j] = s;
      }
      F = build_frame(r);
      // the quantities the frame backward needs
      nl = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
      ndeg = !(nl >= 1e-20f);
      sdot = r[3] * F.n[0] + r[4] * F.n[1] + r[5] * F.n[2];
      float tp0 = r[3] - sdot * F.n[0], tp1 = r[4] - sdot * F.n[1], tp2 = r[5] - sdot * F.n[2];
      tpl = sqrtf(tp0 * tp0 + tp1 * tp1 + tp2 * tp2);
      float trl = sqrtf(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
      tdeg = !(tpl > 1e-6f * trl);
      float c0 = F.n[1] * F.t[2] - F.n[2] * F.t[1];
      float c1 = F.n[2] * F.t[0] - F.n[0] * F.t[2];
      float c2 = F.n[0] * F.t[1] - F.n[1] * F.t[0];
      cl = sqrtf(c0 * c0 + c1 * c1 + c2 * c2);
      to_local(F, wi[0], wi[1], wi[2], x + 8);
      to_local(F, wo[0], wo[1], wo[2], x + 11);
    } else {
      x[8] = wi[0]; x[9] = wi[1]; x[10] = wi[2];
      x[11] = wo[0]; x[12] = wo[1]; x[13] = wo[2];
    }
    // decoder forward
    float h1[H];
    uint32_t mask1[(H + 31) / 32];
#pragma unroll
    for (int w = 0; w < (H + 31) / 32; ++w) mask1[w] = 0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const float4* row = reinterpret_cast<const float4*>(&S.W1[j * 16]);
      float s = S.b1[j];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float4 w = row[k];
        s = fmaf(w.x, x[4 * k], s);
        s = fmaf(w.y, x[4 * k + 1], s);
        s = fmaf(w.z, x[4 * k + 2], s);
        s = fmaf(w.w, x[4 * k + 3], s);
      }
      h1[j] = fmaxf(s, 0.0f);
      if (s > 0.0f) mask1[j >> 5] |= 1u << (j & 31);
    }
    // layer 2 and output: h2 -> shared row, y accumulated
    float y[3] = {S.bo[0], S.bo[1], S.bo[2]};
#pragma unroll 1
    for (int j = 0; j < H; ++j) {
      const float4* row = reinterpret_cast<const float4*>(&S.W2[j * H]);
      float s = S.b2[j];
#pragma unroll
      for (int k = 0; k < H / 4; ++k) {
        float4 w = row[k];
        s = fmaf(w.x, h1[4 * k], s);
        s = fmaf(w.y, h1[4 * k + 1], s);
        s = fmaf(w.z, h1[4 * k + 2], s);
        s = fmaf(w.w, h1[4 * k + 3], s);
      }
      const float h2 = fmaxf(s, 0.0f);
      S.H2[t][j] = h2;
#pragma unroll
      for (int c = 0; c < 3; ++c) y[c] = fmaf(S.Wo[c * H + j], h2, y[c]);
    }
    // store activations for phase B (rows padded, float4 stores)
#pragma unroll
    for (int k = 0; k < H / 4; ++k)
      reinterpret_cast<float4*>(&S.H1[t][0])[k] = make_float4(h1[4 * k], h1[4 * k + 1], h1[4 * k + 2], h1[4 * k + 3]);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      reinterpret_cast<float4*>(&S.X[t][0])[k] = make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
    // output delta
    const float cf = cosine ? fmaxf(wi[2], 0.0f) : 1.0f;
    float dy[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dy[c] = valid ? A.grad_rgb[3 * i + c] * cf : 0.0f;
    reinterpret_cast<float4*>(&S.DY[t][0])[0] = make_float4(dy[0], dy[1], dy[2], 0.0f);
    // layer-2 delta d2 = (Wo^T dy) masked, and d1 = W2^T d2 accumulated in
    // registers (reusing h1)
#pragma unroll
    for (int k = 0; k < H; ++k) h1[k] = 0.0f;
#pragma unroll 1
    for (int j = 0; j < H; ++j) {
      const float g = S.Wo[j] * dy[0] + S.Wo[H + j] * dy[1] + S.Wo[2 * H + j] * dy[2];
      const float dj = S.H2[t][j] > 0.0f ? g : 0.0f;
      S.D2[t][j] = dj;
      const float4* row = reinterpret_cast<const float4*>(&S.W2[j * H]);
#pragma unroll
      for (int k = 0; k < H / 4; ++k) {
        float4 w = row[k];
        h1[4 * k] = fmaf(w.x, dj, h1[4 * k]);
        h1[4 * k + 1] = fmaf(w.y, dj, h1[4 * k + 1]);
        h1[4 * k + 2] = fmaf(w.z, dj, h1[4 * k + 2]);
        h1[4 * k + 3] = fmaf(w.w, dj, h1[4 * k + 3]);
      }
    }
#pragma unroll
    for (int k = 0; k < H; ++k)
      if (!((mask1[k >> 5] >> (k & 31)) & 1u)) h1[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < H / 4; ++k)
      reinterpret_cast<float4*>(&S.D1[t][0])[k] = make_float4(h1[4 * k], h1[4 * k + 1], h1[4 * k + 2], h1[4 * k + 3]);
    // dx = W1^T d1
    float dx[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) dx[k] = 0.0f;
#pragma unroll 1
    for (int j = 0; j < H; ++j) {
      const float4* row = reinterpret_cast<const float4*>(&S.W1[j * 16]);
      const float dj = S.D1[t][j];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float4 w = row[k];
        dx[4 * k] = fmaf(w.x, dj, dx[4 * k]);
        dx[4 * k + 1] = fmaf(w.y, dj, dx[4 * k + 1]);
        dx[4 * k + 2] = fmaf(w.z, dj, dx[4 * k + 2]);
        dx[4 * k + 3] = fmaf(w.w, dj, dx[4 * k + 3]);
      }
    }
    float dz[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) dz[c] = dx[c];
    if (FRAME) {
      // x' = T w: dT row k += dx'_k w
      float dt[3], db[3], dn[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dt[k] = dx[8] * wi[k] + dx[11] * wo[k];
        db[k] = dx[9] * wi[k] + dx[12] * wo[k];
        dn[k] = dx[10] * wi[k] + dx[13] * wo[k];
      }
      // b = c / |c|, c = n x t
      float bdb = F.b[0] * db[0] + F.b[1] * db[1] + F.b[2] * db[2];
      float gc[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) gc[k] = (db[k] - F.b[k] * bdb) / cl;
      dn[0] += F.t[1] * gc[2] - F.t[2] * gc[1];
      dn[1] += F.t[2] * gc[0] - F.t[0] * gc[2];
      dn[2] += F.t[0] * gc[1] - F.t[1] * gc[0];
      dt[0] += gc[1] * F.n[2] - gc[2] * F.n[1];
      dt[1] += gc[2] * F.n[0] - gc[0] * F.n[2];
      dt[2] += gc[0] * F.n[1] - gc[1] * F.n[0];
      float dr[6] = {0, 0, 0, 0, 0, 0};
      if (!tdeg) {
        float tdt = F.t[0] * dt[0] + F.t[1] * dt[1] + F.t[2] * dt[2];
        float dtp[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) dtp[k] = (dt[k] - F.t[k] * tdt) / tpl;
        float ndtp = F.n[0] * dtp[0] + F.n[1] * dtp[1] + F.n[2] * dtp[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          dr[3 + k] += dtp[k] - F.n[k] * ndtp;
          dn[k] += -ndtp * r[3 + k] - sdot * dtp[k];
        }
      }
      if (!ndeg) {
        float ndn = F.n[0] * dn[0] + F.n[1] * dn[1] + F.n[2] * dn[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) dr[k] += (dn[k] - F.n[k] * ndn) / nl;
      }
      if (!valid) {
#pragma unroll
        for (int k = 0; k < 6; ++k) dr[k] = 0.0f;
      }
      reinterpret_cast<float4*>(&S.DR[t][0])[0] = make_float4(dr[0], dr[1], dr[2], dr[3]);
      reinterpret_cast<float4*>(&S.DR[t][0])[1] = make_float4(dr[4], dr[5], 0.0f, 0.0f);
      float dhf[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float g = 0.0f;
#pragma unroll
        for (int j = 0; j < 6; ++j) g = fmaf(S.fW2[j * 16 + k], dr[j], g);
        dhf[k] = hfp[k] > 0.0f ? g : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        reinterpret_cast<float4*>(&S.DHF[t][0])[k] = make_float4(dhf[4 * k], dhf[4 * k + 1], dhf[4 * k + 2], dhf[4 * k + 3]);
        reinterpret_cast<float4*>(&S.HF[t][0])[k] =
            make_float4(fmaxf(hfp[4 * k], 0.0f), fmaxf(hfp[4 * k + 1], 0.0f), fmaxf(hfp[4 * k + 2], 0.0f),
                        fmaxf(hfp[4 * k + 3], 0.0f));
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float g = 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k) g = fmaf(S.fW1[k * 8 + c], dhf[k], g);
        dz[c] += g;
      }
      reinterpret_cast<float4*>(&S.Z[t][0])[0] = make_float4(z[0], z[1], z[2], z[3]);
      reinterpret_cast<float4*>(&S.Z[t][0])[1] = make_float4(z[4], z[5], z[6], z[7]);
    }
    // pyramid scatter: z = sum_k w_k texel_k  =>  dtexel_k += w_k dz
    if (valid && A.grad_pyramid) {
      LevelPick lp = pick_levels(A.pyr, lod);
      int lv[2];
      float lw[2];
      int nl2;
      if (A.pyr.filter == NAM_FILTER_STOCHASTIC) {
        lv[0] = xi < lp.t ? lp.l1 : lp.l0;
        lw[0] = 1.0f;
        nl2 = 1;
      } else {
        lv[0] = lp.l0; lw[0] = 1.0f - lp.t;
        lv[1] = lp.l1; lw[1] = lp.t;
        nl2 = lp.t != 0.0f ? 2 : 1;
      }
      for (int e = 0; e < nl2; ++e) {
        const int l = lv[e];
        const int W = A.pyr.w[l], Hh = A.pyr.h[l];
        int x0, x1, y0, y1;
        float fx, fy;
        tap_axis(A.pyr, u, W, x0, x1, fx);
        tap_axis(A.pyr, v, Hh, y0, y1, fy);
        const int64_t base = A.pyr.off[l];
        const int64_t idx[4] = {base + (int64_t)y0 * W + x0, base + (int64_t)y0 * W + x1,
                                base + (int64_t)y1 * W + x0, base + (int64_t)y1 * W + x1};
        const float gx = 1.0f - fx, gy = 1.0f - fy;
        const float w4[4] = {gx * gy * lw[e], fx * gy * lw[e], gx * fy * lw[e], fx * fy * lw[e]};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float4* g = reinterpret_cast<float4*>(A.grad_pyramid + idx[k] * 8);
          atomicAdd(g, make_float4(w4[k] * dz[0], w4[k] * dz[1], w4[k] * dz[2], w4[k] * dz[3]));
          atomicAdd(g + 1, make_float4(w4[k] * dz[4], w4[k] * dz[5], w4[k] * dz[6], w4[k] * dz[7]));
        }
      }
    }
    if (!valid) {
      // zero the deltas of padding rows so that phase B can sum all 128
#pragma unroll
      for (int k = 0; k < H / 4; ++k) {
        reinterpret_cast<float4*>(&S.D1[t][0])[k] = make_float4(0, 0, 0, 0);
        reinterpret_cast<float4*>(&S.D2[t][0])[k] = make_float4(0, 0, 0, 0);
      }
      if (FRAME)
#pragma unroll
        for (int k = 0; k < 4; ++k) reinterpret_cast<float4*>(&S.DHF[t][0])[k] = make_float4(0, 0, 0, 0);
    }
    __syncthreads();
    // =================== phase B ===========================================
    for (int qq = 0; qq < count; ++qq) {
      // dW2[j2][k2 .. k2+PER2) += D2[q][j2] * H1[q][k2 ..]
      const float d = S.D2[qq][j2];
#pragma unroll
      for (int i2 = 0; i2 < PER2; i2 += 4) {
        float4 h = *reinterpret_cast<const float4*>(&S.H1[qq][k2 + i2]);
        acc2[i2] = fmaf(d, h.x, acc2[i2]);
        if (PER2 > 1) acc2[i2 + 1] = fmaf(d, h.y, acc2[i2 + 1]);
        if (PER2 > 2) acc2[i2 + 2] = fmaf(d, h.z, acc2[i2 + 2]);
        if (PER2 > 3) acc2[i2 + 3] = fmaf(d, h.w, acc2[i2 + 3]);
      }
#pragma unroll
      for (int e = 0; e < N1; ++e) {
        const int idx = t + 128 * e;
        if (idx < 14 * H) acc1[e] = fmaf(S.D1[qq][idx / 14], S.X[qq][idx % 14], acc1[e]);
      }
#pragma unroll
      for (int e = 0; e < NO; ++e) {
        const int idx = t + 128 * e;
        if (idx < 3 * H) accO[e] = fmaf(S.DY[qq][idx / H], S.H2[qq][idx % H], accO[e]);
      }
#pragma unroll
      for (int e = 0; e < NB; ++e) {
        const int slot = t + 128 * e;
        float d2 = 0.0f;
        if (slot < H) d2 = S.D1[qq][slot];
        else if (slot < 2 * H) d2 = S.D2[qq][slot - H];
        else if (slot < 2 * H + 3) d2 = S.DY[qq][slot - 2 * H];
        else if (FRAME && slot < 2 * H + 19) d2 = S.DHF[qq][slot - 2 * H - 3];
        else if (FRAME && slot < 2 * H + 25) d2 = S.DR[qq][slot - 2 * H - 19];
        accB[e] += d2;
      }
      if (FRAME) {
        accF1 = fmaf(S.DHF[qq][t >> 3], S.Z[qq][t & 7], accF1);            // dWf1 [16][8]
        if (t < 96) accF2 = fmaf(S.DR[qq][t >> 4], S.HF[qq][t & 15], accF2);  // dWf2 [6][16]
      }
    }
    __syncthreads();
  }
  // ---- flush: one atomic per parameter per CTA -------------------------------
  float* g = A.grad_params;
  int o = 0;
  if (FRAME) {
    atomicAdd(&g[t], accF1);                       // Wf1 (128)
    if (t < 96) atomicAdd(&g[144 + t], accF2);     // Wf2 (96)
    o = 246;
  }
  const int oW1 = o, ob1 = o + 14 * H, oW2 = ob1 + H, ob2 = oW2 + H * H, oWo = ob2 + H, obo = oWo + 3 * H;
#pragma unroll
  for (int i2 = 0; i2 < PER2; ++i2) atomicAdd(&g[oW2 + j2 * H + k2 + i2], acc2[i2]);
#pragma unroll
  for (int e = 0; e < N1; ++e) {
    const int idx = t + 128 * e;
    if (idx < 14 * H) atomicAdd(&g[oW1 + idx], acc1[e]);
  }
#pragma unroll
  for (int e = 0; e < NO; ++e) {
    const int idx = t + 128 * e;
    if (idx < 3 * H) atomicAdd(&g[oWo + idx], accO[e]);
  }
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    const int slot = t + 128 * e;
    if (slot < H) atomicAdd(&g[ob1 + slot], accB[e]);
    else if (slot < 2 * H) atomicAdd(&g[ob2 + slot - H], accB[e]);
    else if (slot < 2 * H + 3) atomicAdd(&g[obo + slot - 2 * H], accB[e]);
    else if (FRAME && slot < 2 * H + 19) atomicAdd(&g[128 + slot - 2 * H - 3], accB[e]);
    else if (FRAME && slot < 2 * H + 25) atomicAdd(&g[240 + slot - 2 * H - 19], accB[e]);
  }
}

template <int H, bool FRAME, bool F16>
static int launch_bwd_one(const BackwardArgs& a, cudaStream_t s) {
  auto k = backward_kernel<H, FRAME, F16>;
  const int smem = (int)sizeof(BwdSmem<H>);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int64_t tiles = (a.n + 127) / 128;
  int grid = (int)(tiles < a.num_sms ? tiles : a.num_sms);
  if (grid < 1) grid = 1;
  k<<<grid, 128, smem, s>>>(a);
  return (int)cudaGetLastError();
}

// Trainable materials keep FP32 latents (the pyramid is an Adam master).
template <int H>
static int bwd_dispatch(const BackwardArgs& a, cudaStream_t s) {
  if (a.pyr.f16) return (int)cudaErrorInvalidValue;
  return a.shape.frame ? launch_bwd_one<H, true, false>(a, s) : launch_bwd_one<H, false, false>(a, s);
}

int launch_backward(const BackwardArgs& a, void* stream) {
  if (a.n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (a.shape.NH != 2) return (int)cudaErrorInvalidValue;
  if (a.shape.H == 16) return bwd_dispatch<16>(a, s);
  if (a.shape.H == 32) return bwd_dispatch<32>(a, s);
  if (a.shape.H == 64) return bwd_dispatch<64>(a, s);
  return (int)cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// loss: L = mean |log(1+max(g,0)) - log(1+y)| + 0.01 mean max(-g,0)
// ---------------------------------------------------------------------------
__global__ void loss_kernel(const float* __restrict__ g, const float* __restrict__ y, int64_t m, float inv,
                            float* __restrict__ dg, float* __restrict__ acc) {
  float local = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float d = log1pf(fmaxf(gi, 0.0f)) - log1pf(y[i]);
    float l = fabsf(d);
    float grad = 0.0f;
    if (gi > 0.0f) grad = (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f)) / (1.0f + gi);
    if (gi < 0.0f) {
      l += 0.01f * (-gi);
      grad -= 0.01f;
    }
    dg[i] = grad * inv;
    local += l;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(acc, v * inv);
  }
}

int launch_loss(const float* rgb, const float* target, int64_t n, float* grad_rgb, float* loss_accum, void* stream) {
  const int64_t m = 3 * n;
  if (m == 0) return 0;
  int grid = (int)((m + 255) / 256);
  if (grid > 1024) grid = 1024;
  loss_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(rgb, target, m, 1.0f / (float)m, grad_rgb, loss_accum);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba): bias-corrected first and second moments; the gradient
// buffer is cleared after use so the next backward accumulates afresh.
// ---------------------------------------------------------------------------
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            int64_t count, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.0f;
  }
}

int launch_adam(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2, float eps,
                int step, void* stream) {
  if (count == 0) return 0;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  int grid = (int)((count + 255) / 256);
  if (grid > 4096) grid = 4096;
  adam_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(p, const_cast<float*>(g), m, v, count, lr, b1, b2, eps, c1, c2);
  return (int)cudaGetLastError();
}

}  // namespace nam
