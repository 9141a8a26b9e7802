// Reverse mode of the FP32 evaluation, the log-space L1 loss and Adam
// (training of the decoder and the latent texture, Sec. 5).
//
// Backward kernel: a CTA of 512 threads takes tiles of 128 queries.  Two
// lane mappings share the tile:
//  - a quad of four adjacent lanes per query, for the per-query work: the
//    latent fetch, the frame MLP (lane p owns frame hidden units p + 4e, the
//    six outputs are summed over the quad), the frame construction and its
//    backward (redundant in the quad, ALU only), dL/dx (lane p owns x
//    entries 4p..4p+3) and the pyramid scatter (lane p takes bilinear tap p;
//    taps that coincide, as at the coarsest levels, are merged so that each
//    distinct texel of a query takes one update);
//  - a half-warp per four queries for the decoder layers: lane l owns hidden
//    units l + 16 jj of all four queries, a 4 x (H/16) register block, so
//    that every shared-memory operand feeds four FMAs per query block.
//  Activations and deltas go to shared-memory rows; the lanes that read them
//  are in the writer's warp, so a __syncwarp orders them.
//  Training step variant (LOSS): the decoder blocks also finish the forward
//  (y = Wo h2 + bo, summed over the half-warp), evaluate the log-space L1
//  loss against the target and start the backward from its gradient, so a
//  training step needs no separate forward or loss pass.  With the albedo
//  head (ALB: six outputs, RGB then albedo) the fused loss adds the albedo's
//  L2 error against one-sample albedo estimates (the paper's albedo
//  inference), and the output layer's gradient blocks span eight rows.
//  Phase B (thread = 4x4 block of one weight matrix): each owner sums the
//  outer products delta[q][rows] * act[q][cols] over the tile in registers
//  (two 16-byte shared loads per 16 FMAs), the column-0 owners also sum the
//  bias deltas.  The registers are added to the global gradient with one
//  atomic per parameter per CTA after the CTA's last tile.
//  Same-address atomics serialise in L2, and every query whose lod reaches
//  the coarsest levels lands on a handful of texels there: the gradient of
//  the coarsest levels is summed in shared memory first (per warp for the
//  tiniest ones, per CTA for the next) and added to the global buffer once
//  per CTA.
#include <cuda_runtime.h>

#include "common.cuh"

namespace nam {

constexpr int kBwdQ = 128;             // queries per tile
constexpr int kBwdThreads = 4 * kBwdQ;  // a quad per query

template <int H, bool ALB = false>
struct BwdSmem {
  static constexpr int NO = ALB ? 6 : 3;  // decoder outputs
  static constexpr int DW = ALB ? 8 : 4;  // DY row length
  static constexpr int S = H + 4;  // padded row stride: rows l + 16 jj of a half-warp hit distinct banks
  // parameters
  float fW1[16 * 8], fb1[16], fW2[6 * 16], fb2[8];
  float W1[H][20];   // W1[j][0..13], zero padding
  float b1[H];
  float W2[H][S];    // W2[j][k]
  float b2[H];
  float Wo[NO * H], bo[8];
  float lred[16];  // per-warp loss partials
  // per-query vectors of the current tile (deltas at pre-activations)
  float Z[kBwdQ][8];     // frame MLP input (z)
  float HF[kBwdQ][16];   // frame hidden activations
  float DHF[kBwdQ][16];  // delta at the frame hidden pre-activations
  float R[kBwdQ][8];     // frame MLP output r = (n_raw, t_raw)
  float DR[kBwdQ][8];    // delta at r, zero padding
  float X[kBwdQ][16];    // decoder input x (14), zero padding
  float DX[kBwdQ][16];   // dL/dx
  float D1[kBwdQ][S];    // delta at decoder layer-1 pre-activations
  float H1[kBwdQ][S];    // decoder layer-1 activations
  float D2[kBwdQ][S];    // delta at layer-2 pre-activations
  float H2[kBwdQ][S];    // layer-2 activations
  float DY[kBwdQ][DW];   // delta at the outputs (after the cosine factor), zero padding;
                         // with the fused loss first the targets and the cosine
                         // factor: (t_r, t_g, t_b, cf), or with ALB (t_r, t_g, t_b,
                         // albedo t_r, t_g, t_b, 0, cf)
};

// Log-space L1 loss of one output element g against its target y (Sec. 5.2
// names an L1 loss in log space; read as |log(1 + max(g, 0)) - log(1 + y)|
// plus 0.01 max(-g, 0), which keeps a gradient on negative outputs); returns
// the loss, *grad = dloss/dg.
__device__ __forceinline__ float log_l1(float g, float y, float* grad) {
  const float d = log1pf(fmaxf(g, 0.0f)) - log1pf(y);
  float l = fabsf(d);
  float gr = 0.0f;
  if (g > 0.0f) gr = (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f)) / (1.0f + g);
  if (g < 0.0f) {
    l += 0.01f * (-g);
    gr -= 0.01f;
  }
  *grad = gr;
  return l;
}

__device__ __forceinline__ float quad_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b, float s) {
  s = fmaf(a.x, b.x, s);
  s = fmaf(a.y, b.y, s);
  s = fmaf(a.z, b.z, s);
  return fmaf(a.w, b.w, s);
}

template <int H, bool FRAME, bool F16, bool LOSS, bool ALB>
__global__ void __launch_bounds__(kBwdThreads, 1) backward_kernel(const BackwardArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Sm = BwdSmem<H, ALB>;
  Sm& S = *reinterpret_cast<Sm*>(smem_raw);
  constexpr int NO = Sm::NO, DW = Sm::DW;
  constexpr int JB = H / 16;  // hidden units per lane in the decoder blocks
  const int t = threadIdx.x;
  // ---- parameters -> shared ---------------------------------------------------
  {
    const float* p = A.params;
    if (FRAME) {
      for (int i = t; i < 128; i += kBwdThreads) S.fW1[i] = p[i];
      if (t < 16) S.fb1[t] = p[128 + t];
      for (int i = t; i < 96; i += kBwdThreads) S.fW2[i] = p[144 + i];
      if (t < 8) S.fb2[t] = t < 6 ? p[240 + t] : 0.0f;
      p += 246;
    }
    for (int i = t; i < H * 20; i += kBwdThreads) {
      const int j = i / 20, k = i % 20;
      S.W1[j][k] = k < 14 ? p[j * 14 + k] : 0.0f;
    }
    p += 14 * H;
    for (int i = t; i < H; i += kBwdThreads) S.b1[i] = p[i];
    p += H;
    for (int i = t; i < H * H; i += kBwdThreads) S.W2[i / H][i % H] = p[i];
    p += H * H;
    for (int i = t; i < H; i += kBwdThreads) S.b2[i] = p[i];
    p += H;
    for (int i = t; i < NO * H; i += kBwdThreads) S.Wo[i] = p[i];
    p += NO * H;
    if (t < 8) S.bo[t] = t < NO ? p[t] : 0.0f;
  }
  // coarse-level accumulators after the tile: [16 warps][tiny_n][8], [cta_n][8]
  float* wacc = reinterpret_cast<float*>(smem_raw + sizeof(Sm));
  float* cacc = wacc + 16 * 8 * A.tiny_n;
  for (int i = t; i < 8 * (16 * A.tiny_n + A.cta_n); i += kBwdThreads) wacc[i] = 0.0f;
  float* my_wacc = wacc + (t >> 5) * 8 * A.tiny_n;

  // ---- phase-B ownership: one 4x4 block of one gradient matrix ------------------
  // blocks: dW2 (H/4)^2, dW1 H/4 x 4 (14 columns padded to 16), dWo
  // DW/4 x H/4 (3 rows padded to 4, or 6 padded to 8), dWf1 4 x 2, dWf2 2 x 4
  // (6 rows padded to 8)
  constexpr int NB2 = (H / 4) * (H / 4), NB1 = H, NBO = (DW / 4) * (H / 4);
  int role = -1, r0 = 0, c0 = 0;
  const float* dp = nullptr;
  const float* ap = nullptr;
  int dstride = 0, astride = 0;
  {
    int b = t;
    if (b < NB2) {
      role = 0; r0 = 4 * (b / (H / 4)); c0 = 4 * (b % (H / 4));
      dp = &S.D2[0][r0]; dstride = Sm::S; ap = &S.H1[0][c0]; astride = Sm::S;
    } else if ((b -= NB2) < NB1) {
      role = 1; r0 = 4 * (b >> 2); c0 = 4 * (b & 3);
      dp = &S.D1[0][r0]; dstride = Sm::S; ap = &S.X[0][c0]; astride = 16;
    } else if ((b -= NB1) < NBO) {
      role = 2; r0 = 4 * (b / (H / 4)); c0 = 4 * (b % (H / 4));
      dp = &S.DY[0][r0]; dstride = DW; ap = &S.H2[0][c0]; astride = Sm::S;
    } else if (FRAME && (b -= NBO) < 8) {
      role = 3; r0 = 4 * (b >> 1); c0 = 4 * (b & 1);
      dp = &S.DHF[0][r0]; dstride = 16; ap = &S.Z[0][c0]; astride = 8;
    } else if (FRAME && (b -= 8) < 8) {
      role = 4; r0 = 4 * (b >> 2); c0 = 4 * (b & 3);
      dp = &S.DR[0][r0]; dstride = 8; ap = &S.HF[0][c0]; astride = 16;
    }
  }
  float acc[16], accb[4];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) accb[i] = 0.0f;
  __syncthreads();

  float lsum = 0.0f;  // fused loss: this lane's share of the sum
  const int ql = t >> 2, p = t & 3;         // quad: query ql, lane p
  const int hl = t & 15, qb = (t >> 4) * 4;  // half-warp: queries qb..qb+3, units hl + 16 jj
  const bool cosine = (A.flags & NAM_OUT_COSINE) != 0;
  const int64_t ntiles = (A.n + kBwdQ - 1) / kBwdQ;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t start = tile * kBwdQ;
    const int count = (int)((A.n - start) < kBwdQ ? (A.n - start) : kBwdQ);
    const bool valid = ql < count;
    const int64_t i = start + (valid ? ql : 0);
    // =================== phase A ===========================================
    // ---- quad: latent, frame MLP, frame, decoder input ----------------------
    {
      float z[8];
      if (A.z_in) {
        // encoder phase (Sec. 5.1): the latent is given, the texture bypassed
        const float4 a = reinterpret_cast<const float4*>(A.z_in + 8 * i)[0];
        const float4 b = reinterpret_cast<const float4*>(A.z_in + 8 * i)[1];
        z[0] = a.x; z[1] = a.y; z[2] = a.z; z[3] = a.w; z[4] = b.x; z[5] = b.y; z[6] = b.z; z[7] = b.w;
      } else {
        const float xi = A.q.xi ? A.q.xi[i] : 0.0f;
        fetch_latent<F16>(A.pyr, A.pyramid, A.q.u[i], A.q.v[i], A.q.lod[i], xi, z);
      }
      const float wi[3] = {A.q.wix[i], A.q.wiy[i], A.q.wiz[i]};
      const float wo[3] = {A.q.wox[i], A.q.woy[i], A.q.woz[i]};
      float x[14];
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = z[c];
      if (FRAME) {
        // lane p owns frame hidden units p + 4e (rows 8 floats apart in four
        // distinct bank groups)
        float hf[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4* row = reinterpret_cast<const float4*>(&S.fW1[(p + 4 * e) * 8]);
          const float4 a = row[0], b = row[1];
          float s = S.fb1[p + 4 * e];
          s = dot4(a, make_float4(z[0], z[1], z[2], z[3]), s);
          s = dot4(b, make_float4(z[4], z[5], z[6], z[7]), s);
          hf[e] = fmaxf(s, 0.0f);
          S.HF[ql][p + 4 * e] = hf[e];
        }
        float r[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          float t = 0.0f;
#pragma unroll
          for (int e = 0; e < 4; ++e) t = fmaf(S.fW2[j * 16 + p + 4 * e], hf[e], t);
          r[j] = quad_sum(t) + S.fb2[j];
        }
        const Frame F = build_frame(r);
        to_local(F, wi[0], wi[1], wi[2], x + 8);
        to_local(F, wo[0], wo[1], wo[2], x + 11);
        if (p == 0) {
          reinterpret_cast<float4*>(&S.R[ql][0])[0] = make_float4(r[0], r[1], r[2], r[3]);
          reinterpret_cast<float4*>(&S.R[ql][0])[1] = make_float4(r[4], r[5], 0.0f, 0.0f);
        }
      } else {
        x[8] = wi[0]; x[9] = wi[1]; x[10] = wi[2];
        x[11] = wo[0]; x[12] = wo[1]; x[13] = wo[2];
      }
      if (p == 0) {
        float4* X4 = reinterpret_cast<float4*>(&S.X[ql][0]);
        X4[0] = make_float4(x[0], x[1], x[2], x[3]);
        X4[1] = make_float4(x[4], x[5], x[6], x[7]);
        X4[2] = make_float4(x[8], x[9], x[10], x[11]);
        X4[3] = make_float4(x[12], x[13], 0.0f, 0.0f);
        reinterpret_cast<float4*>(&S.Z[ql][0])[0] = make_float4(z[0], z[1], z[2], z[3]);
        reinterpret_cast<float4*>(&S.Z[ql][0])[1] = make_float4(z[4], z[5], z[6], z[7]);
        const float cf = cosine ? fmaxf(wi[2], 0.0f) : 1.0f;
        float4* dy4 = reinterpret_cast<float4*>(&S.DY[ql][0]);
        if (LOSS) {
          const float* tg = A.target + 3 * i;
          if (ALB) {
            const float* ta = A.target_albedo + 3 * i;
            dy4[0] = valid ? make_float4(tg[0], tg[1], tg[2], ta[0]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            dy4[1] = valid ? make_float4(ta[1], ta[2], 0.0f, cf) : make_float4(0.0f, 0.0f, 0.0f, cf);
          } else {
            dy4[0] = valid ? make_float4(tg[0], tg[1], tg[2], cf) : make_float4(0.0f, 0.0f, 0.0f, cf);
          }
        } else if constexpr (ALB) {
          // dL/d(output) of the caller, [n][6]; the cosine factor scales the RGB only
          float dy[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) dy[c] = valid ? A.grad_rgb[6 * i + c] * (c < 3 ? cf : 1.0f) : 0.0f;
          dy4[0] = make_float4(dy[0], dy[1], dy[2], dy[3]);
          dy4[1] = make_float4(dy[4], dy[5], 0.0f, 0.0f);
        } else {
          float dy[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) dy[c] = valid ? A.grad_rgb[3 * i + c] * cf : 0.0f;
          dy4[0] = make_float4(dy[0], dy[1], dy[2], 0.0f);
        }
      }
    }
    __syncwarp();
    // ---- half-warp blocks: decoder forward and backward ---------------------
    uint32_t mask1 = 0;  // bit jj * 4 + qq: layer-1 unit hl + 16 jj of query qb + qq is active
    {
      float a[4][JB];
      // layer 1 (the forward value of y is not needed: dL/dy comes in)
#pragma unroll
      for (int jj = 0; jj < JB; ++jj)
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) a[qq][jj] = S.b1[hl + 16 * jj];
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        float4 xv[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) xv[qq] = reinterpret_cast<const float4*>(&S.X[qb + qq][0])[c4];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          const float4 w = reinterpret_cast<const float4*>(&S.W1[hl + 16 * jj][0])[c4];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) a[qq][jj] = dot4(w, xv[qq], a[qq][jj]);
        }
      }
#pragma unroll
      for (int jj = 0; jj < JB; ++jj)
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          S.H1[qb + qq][hl + 16 * jj] = fmaxf(a[qq][jj], 0.0f);
          if (a[qq][jj] > 0.0f) mask1 |= 1u << (jj * 4 + qq);
        }
      __syncwarp();
      // layer 2
#pragma unroll
      for (int jj = 0; jj < JB; ++jj)
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) a[qq][jj] = S.b2[hl + 16 * jj];
#pragma unroll 2
      for (int m = 0; m < H / 4; ++m) {
        float4 hv[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) hv[qq] = reinterpret_cast<const float4*>(&S.H1[qb + qq][0])[m];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          const float4 w = reinterpret_cast<const float4*>(&S.W2[hl + 16 * jj][0])[m];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) a[qq][jj] = dot4(w, hv[qq], a[qq][jj]);
        }
      }
      if (LOSS) {
        // output y = Wo relu(a) + bo of the four queries, summed over the
        // half-warp; lane (mq, mc) = (hl / 4, hl % 4) takes element mc of
        // query qb + mq: loss and dL/dy (times the cosine factor) into DY
        if constexpr (ALB) {
          float y[4][NO];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq)
#pragma unroll
            for (int c = 0; c < NO; ++c) y[qq][c] = 0.0f;
#pragma unroll
          for (int jj = 0; jj < JB; ++jj) {
            const int j = hl + 16 * jj;
            float o[NO];
#pragma unroll
            for (int c = 0; c < NO; ++c) o[c] = S.Wo[c * H + j];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const float h = fmaxf(a[qq][jj], 0.0f);
#pragma unroll
              for (int c = 0; c < NO; ++c) y[qq][c] = fmaf(o[c], h, y[qq][c]);
            }
          }
#pragma unroll
          for (int off = 1; off < 16; off <<= 1)
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
#pragma unroll
              for (int c = 0; c < NO; ++c) y[qq][c] += __shfl_xor_sync(0xffffffffu, y[qq][c], off);
          // lane (mq, mc) takes output elements mc and, with ALB, mc + 4 of query qb + mq
          const int mq = hl >> 2, mc = hl & 3;
          float ym[2] = {0.0f, 0.0f};
#pragma unroll
          for (int qq = 0; qq < 4; ++qq)
#pragma unroll
            for (int c = 0; c < NO; ++c) {
              if (qq == mq && c == mc) ym[0] = y[qq][c];
              if (qq == mq && c == mc + 4) ym[1] = y[qq][c];
            }
          float tv[DW];  // targets; the cosine factor last
#pragma unroll
          for (int c4 = 0; c4 < DW / 4; ++c4) {
            const float4 v = reinterpret_cast<const float4*>(&S.DY[qb + mq][0])[c4];
            tv[4 * c4] = v.x; tv[4 * c4 + 1] = v.y; tv[4 * c4 + 2] = v.z; tv[4 * c4 + 3] = v.w;
          }
          const float cf = tv[DW - 1];
          const bool vq = qb + mq < count;
          __syncwarp();
#pragma unroll
          for (int h2 = 0; h2 < DW / 4; ++h2) {
            const int e = mc + 4 * h2;  // output element of this lane
            float tgt = 0.0f;
#pragma unroll
            for (int c = 0; c < NO; ++c)
              if (c == e) tgt = tv[c];
            float d = 0.0f;
            if (e < 3) {
              // BRDF: log-space L1 of the cosine-weighted output
              const float g = (ym[h2] + S.bo[e]) * cf;
              float gr;
              const float l = log_l1(g, tgt, &gr);
              if (vq) lsum += l;
              d = gr * A.loss_inv * cf;
            } else if (e < NO) {
              // albedo head: L2 against the one-sample albedo estimate
              const float r = ym[h2] + S.bo[e] - tgt;
              if (vq) lsum += r * r;
              d = 2.0f * r * A.loss_inv;
            }
            S.DY[qb + mq][e] = vq ? d : 0.0f;
          }
          __syncwarp();
        } else {
          float y[4][3];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq)
#pragma unroll
            for (int c = 0; c < 3; ++c) y[qq][c] = 0.0f;
#pragma unroll
          for (int jj = 0; jj < JB; ++jj) {
            const int j = hl + 16 * jj;
            const float o[3] = {S.Wo[j], S.Wo[H + j], S.Wo[2 * H + j]};
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const float h = fmaxf(a[qq][jj], 0.0f);
#pragma unroll
              for (int c = 0; c < 3; ++c) y[qq][c] = fmaf(o[c], h, y[qq][c]);
            }
          }
#pragma unroll
          for (int off = 1; off < 16; off <<= 1)
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
#pragma unroll
              for (int c = 0; c < 3; ++c) y[qq][c] += __shfl_xor_sync(0xffffffffu, y[qq][c], off);
          const int mq = hl >> 2, mc = hl & 3;
          float ym = 0.0f;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              if (qq == mq && c == mc) ym = y[qq][c];
          const float4 tv = *reinterpret_cast<const float4*>(&S.DY[qb + mq][0]);
          __syncwarp();
          if (mc < 3) {
            const float g = (ym + S.bo[mc]) * tv.w;
            float gr;
            const float l = log_l1(g, mc == 0 ? tv.x : mc == 1 ? tv.y : tv.z, &gr);
            const bool vq = qb + mq < count;
            if (vq) lsum += l;
            S.DY[qb + mq][mc] = vq ? gr * A.loss_inv * tv.w : 0.0f;
          } else {
            S.DY[qb + mq][3] = 0.0f;
          }
          __syncwarp();
        }
      }
      // layer-2 delta d2 = (Wo^T dy) where the unit is active
      if constexpr (ALB) {
        float dyv[4][NO];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
#pragma unroll
          for (int c = 0; c < NO; ++c) dyv[qq][c] = S.DY[qb + qq][c];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          const int j = hl + 16 * jj;
          float o[NO];
#pragma unroll
          for (int c = 0; c < NO; ++c) o[c] = S.Wo[c * H + j];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float s = a[qq][jj];
            float d = o[NO - 1] * dyv[qq][NO - 1];
#pragma unroll
            for (int c = NO - 2; c >= 0; --c) d = fmaf(o[c], dyv[qq][c], d);
            S.H2[qb + qq][j] = fmaxf(s, 0.0f);
            S.D2[qb + qq][j] = s > 0.0f ? d : 0.0f;
          }
        }
      } else {
        float4 dyv[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) dyv[qq] = *reinterpret_cast<const float4*>(&S.DY[qb + qq][0]);
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          const int j = hl + 16 * jj;
          const float o0 = S.Wo[j], o1 = S.Wo[H + j], o2 = S.Wo[2 * H + j];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float s = a[qq][jj];
            S.H2[qb + qq][j] = fmaxf(s, 0.0f);
            S.D2[qb + qq][j] = s > 0.0f ? fmaf(o0, dyv[qq].x, fmaf(o1, dyv[qq].y, o2 * dyv[qq].z)) : 0.0f;
          }
        }
      }
      __syncwarp();
      // layer-1 delta d1 = (W2^T d2) where the unit is active; W2 is read by
      // column (unit k of lane hl is column hl + 16 kk)
#pragma unroll
      for (int kk = 0; kk < JB; ++kk)
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) a[qq][kk] = 0.0f;
#pragma unroll 2
      for (int m = 0; m < H / 4; ++m) {
        float4 dv[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) dv[qq] = reinterpret_cast<const float4*>(&S.D2[qb + qq][0])[m];
#pragma unroll
        for (int kk = 0; kk < JB; ++kk) {
          const float4 w = make_float4(S.W2[4 * m][hl + 16 * kk], S.W2[4 * m + 1][hl + 16 * kk],
                                       S.W2[4 * m + 2][hl + 16 * kk], S.W2[4 * m + 3][hl + 16 * kk]);
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) a[qq][kk] = dot4(w, dv[qq], a[qq][kk]);
        }
      }
#pragma unroll
      for (int kk = 0; kk < JB; ++kk)
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
          S.D1[qb + qq][hl + 16 * kk] = ((mask1 >> (kk * 4 + qq)) & 1u) ? a[qq][kk] : 0.0f;
    }
    __syncwarp();
    // ---- quad: dL/dx, frame backward, pyramid scatter ------------------------
    {
      // dx[4p .. 4p+3] = sum_k W1[k][4p ..] d1[k]
      float4 dxp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 4
      for (int k4 = 0; k4 < H / 4; ++k4) {
        const float4 d = reinterpret_cast<const float4*>(&S.D1[ql][0])[k4];
        const float dk[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4 w = reinterpret_cast<const float4*>(&S.W1[4 * k4 + e][0])[p];
          dxp.x = fmaf(w.x, dk[e], dxp.x);
          dxp.y = fmaf(w.y, dk[e], dxp.y);
          dxp.z = fmaf(w.z, dk[e], dxp.z);
          dxp.w = fmaf(w.w, dk[e], dxp.w);
        }
      }
      reinterpret_cast<float4*>(&S.DX[ql][0])[p] = dxp;
      __syncwarp();
      float dx[16];
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        const float4 d = reinterpret_cast<const float4*>(&S.DX[ql][0])[c4];
        dx[4 * c4] = d.x; dx[4 * c4 + 1] = d.y; dx[4 * c4 + 2] = d.z; dx[4 * c4 + 3] = d.w;
      }
      float dz[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) dz[c] = dx[c];
      if (FRAME) {
        float r[6];
        {
          const float4 r0 = reinterpret_cast<const float4*>(&S.R[ql][0])[0];
          const float4 r1 = reinterpret_cast<const float4*>(&S.R[ql][0])[1];
          r[0] = r0.x; r[1] = r0.y; r[2] = r0.z; r[3] = r0.w; r[4] = r1.x; r[5] = r1.y;
        }
        const Frame F = build_frame(r);
        // the quantities the frame backward needs
        const float nl = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        const bool ndeg = !(nl >= 1e-20f);
        const float sdot = r[3] * F.n[0] + r[4] * F.n[1] + r[5] * F.n[2];
        const float tp0 = r[3] - sdot * F.n[0], tp1 = r[4] - sdot * F.n[1], tp2 = r[5] - sdot * F.n[2];
        const float tpl = sqrtf(tp0 * tp0 + tp1 * tp1 + tp2 * tp2);
        const float trl = sqrtf(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
        const bool tdeg = !(tpl > 1e-6f * trl);
        const float c0_ = F.n[1] * F.t[2] - F.n[2] * F.t[1];
        const float c1_ = F.n[2] * F.t[0] - F.n[0] * F.t[2];
        const float c2_ = F.n[0] * F.t[1] - F.n[1] * F.t[0];
        const float cl = sqrtf(c0_ * c0_ + c1_ * c1_ + c2_ * c2_);
        const float wi[3] = {A.q.wix[i], A.q.wiy[i], A.q.wiz[i]};
        const float wo[3] = {A.q.wox[i], A.q.woy[i], A.q.woz[i]};
        // x' = T w: dT row k += dx'_k w
        float dt[3], db[3], dn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          dt[k] = dx[8] * wi[k] + dx[11] * wo[k];
          db[k] = dx[9] * wi[k] + dx[12] * wo[k];
          dn[k] = dx[10] * wi[k] + dx[13] * wo[k];
        }
        // b = c / |c|, c = n x t
        const float bdb = F.b[0] * db[0] + F.b[1] * db[1] + F.b[2] * db[2];
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
          const float tdt = F.t[0] * dt[0] + F.t[1] * dt[1] + F.t[2] * dt[2];
          float dtp[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) dtp[k] = (dt[k] - F.t[k] * tdt) / tpl;
          const float ndtp = F.n[0] * dtp[0] + F.n[1] * dtp[1] + F.n[2] * dtp[2];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            dr[3 + k] += dtp[k] - F.n[k] * ndtp;
            dn[k] += -ndtp * r[3 + k] - sdot * dtp[k];
          }
        }
        if (!ndeg) {
          const float ndn = F.n[0] * dn[0] + F.n[1] * dn[1] + F.n[2] * dn[2];
#pragma unroll
          for (int k = 0; k < 3; ++k) dr[k] += (dn[k] - F.n[k] * ndn) / nl;
        }
        if (!valid) {
#pragma unroll
          for (int k = 0; k < 6; ++k) dr[k] = 0.0f;
        }
        // frame hidden delta, own units p + 4e, and its share of dz
        float dhf[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float g = 0.0f;
#pragma unroll
          for (int j = 0; j < 6; ++j) g = fmaf(S.fW2[j * 16 + p + 4 * e], dr[j], g);
          dhf[e] = S.HF[ql][p + 4 * e] > 0.0f ? g : 0.0f;
          S.DHF[ql][p + 4 * e] = dhf[e];
        }
        if (p == 0) {
          reinterpret_cast<float4*>(&S.DR[ql][0])[0] = make_float4(dr[0], dr[1], dr[2], dr[3]);
          reinterpret_cast<float4*>(&S.DR[ql][0])[1] = make_float4(dr[4], dr[5], 0.0f, 0.0f);
        }
        float gz[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) gz[c] = 0.0f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4* row = reinterpret_cast<const float4*>(&S.fW1[(p + 4 * e) * 8]);
          const float4 a = row[0], b = row[1];
          gz[0] = fmaf(a.x, dhf[e], gz[0]); gz[1] = fmaf(a.y, dhf[e], gz[1]);
          gz[2] = fmaf(a.z, dhf[e], gz[2]); gz[3] = fmaf(a.w, dhf[e], gz[3]);
          gz[4] = fmaf(b.x, dhf[e], gz[4]); gz[5] = fmaf(b.y, dhf[e], gz[5]);
          gz[6] = fmaf(b.z, dhf[e], gz[6]); gz[7] = fmaf(b.w, dhf[e], gz[7]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) dz[c] += quad_sum(gz[c]);
      }
      if (A.dz_out) {
        // encoder phase: dL/dz goes to the encoder's backward
        if (valid && p == 0) {
          reinterpret_cast<float4*>(A.dz_out + 8 * i)[0] = make_float4(dz[0], dz[1], dz[2], dz[3]);
          reinterpret_cast<float4*>(A.dz_out + 8 * i)[1] = make_float4(dz[4], dz[5], dz[6], dz[7]);
        }
      } else if (valid && A.grad_pyramid) {
        // pyramid scatter: z = sum_k w_k texel_k  =>  dtexel_k += w_k dz
        const float u = A.q.u[i], v = A.q.v[i], lod = A.q.lod[i];
        const float xi = A.q.xi ? A.q.xi[i] : 0.0f;
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
          // lane p takes tap p = (y bit, x bit) and the weights of every later
          // tap on the same texel; a tap already taken by an earlier lane is skipped
          int tx[4];
          float tw[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            tx[k] = ((k & 2) ? y1 : y0) * W + ((k & 1) ? x1 : x0);
            tw[k] = ((k & 1) ? fx : 1.0f - fx) * ((k & 2) ? fy : 1.0f - fy);
          }
          const int mine = p == 0 ? tx[0] : p == 1 ? tx[1] : p == 2 ? tx[2] : tx[3];
          bool first = true;
          float w = 0.0f;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (tx[k] == mine) {
              if (k < p) first = false;
              else w += tw[k];
            }
          }
          if (!first) continue;
          w *= lw[e];
          const int64_t tex = A.pyr.off[l] + mine;
          if (tex >= A.cta_tex0) {
            float* c = tex >= A.tiny_tex0 ? my_wacc + 8 * (tex - A.tiny_tex0) : cacc + 8 * (tex - A.cta_tex0);
#pragma unroll
            for (int k = 0; k < 8; ++k) atomicAdd(c + k, w * dz[k]);
          } else {
            float4* g = reinterpret_cast<float4*>(A.grad_pyramid + tex * 8);
            atomicAdd(g, make_float4(w * dz[0], w * dz[1], w * dz[2], w * dz[3]));
            atomicAdd(g + 1, make_float4(w * dz[4], w * dz[5], w * dz[6], w * dz[7]));
          }
        }
      }
    }
    __syncthreads();
    // =================== phase B ===========================================
    if (role >= 0) {
#pragma unroll 2
      for (int qq = 0; qq < count; ++qq) {
        const float4 d = *reinterpret_cast<const float4*>(dp + qq * dstride);
        const float4 a = *reinterpret_cast<const float4*>(ap + qq * astride);
        const float dv[4] = {d.x, d.y, d.z, d.w};
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) acc[4 * rr + cc] = fmaf(dv[rr], av[cc], acc[4 * rr + cc]);
          accb[rr] += dv[rr];
        }
      }
    }
    __syncthreads();
  }
  // ---- flush: one atomic per parameter and coarse texel channel per CTA -------
  // (the last tile ended with a barrier)
  if (LOSS) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if ((t & 31) == 0) S.lred[t >> 5] = lsum;
    __syncthreads();
    if (t == 0) {
      float tot = 0.0f;
      for (int w = 0; w < 16; ++w) tot += S.lred[w];
      atomicAdd(A.loss_acc, tot * A.loss_inv);
    }
  }
  for (int k = t; k < 8 * A.tiny_n; k += kBwdThreads) {
    float c = 0.0f;
    for (int w = 0; w < 16; ++w) c += wacc[w * 8 * A.tiny_n + k];
    if (c != 0.0f) atomicAdd(A.grad_pyramid + A.tiny_tex0 * 8 + k, c);
  }
  for (int k = t; k < 8 * A.cta_n; k += kBwdThreads) {
    const float c = cacc[k];
    if (c != 0.0f) atomicAdd(A.grad_pyramid + A.cta_tex0 * 8 + k, c);
  }
  if (role < 0) return;
  float* g = A.grad_params;
  const int o = FRAME ? 246 : 0;
  const int oW1 = o, ob1 = o + 14 * H, oW2 = ob1 + H, ob2 = oW2 + H * H, oWo = ob2 + H, obo = oWo + NO * H;
  // (weight offset, row stride, valid rows, valid columns, bias offset)
  int wo_ = 0, ws = 0, nr = 0, nc = 0, bo_ = 0;
  switch (role) {
    case 0: wo_ = oW2; ws = H; nr = H; nc = H; bo_ = ob2; break;
    case 1: wo_ = oW1; ws = 14; nr = H; nc = 14; bo_ = ob1; break;
    case 2: wo_ = oWo; ws = H; nr = NO; nc = H; bo_ = obo; break;
    case 3: wo_ = 0; ws = 8; nr = 16; nc = 8; bo_ = 128; break;
    default: wo_ = 144; ws = 16; nr = 6; nc = 16; bo_ = 240; break;
  }
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int row = r0 + rr;
    if (row >= nr) continue;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
      if (c0 + cc < nc) atomicAdd(&g[wo_ + row * ws + c0 + cc], acc[4 * rr + cc]);
    if (c0 == 0) atomicAdd(&g[bo_ + row], accb[rr]);
  }
}

template <int H, bool FRAME, bool F16, bool LOSS, bool ALB>
static int launch_bwd_one(const BackwardArgs& a, cudaStream_t s) {
  auto k = backward_kernel<H, FRAME, F16, LOSS, ALB>;
  constexpr int kSmemMax = 227 * 1024;
  constexpr int kBase = (int)sizeof(BwdSmem<H, ALB>);
  static_assert(kBase <= kSmemMax, "backward tile does not fit in shared memory");
  // coarse-level accumulators in what the tile leaves: per-warp copies of the
  // coarsest levels up to kTiny texels, then one copy of the next levels
  constexpr int64_t kTiny = 24;
  BackwardArgs b = a;
  b.tiny_tex0 = b.cta_tex0 = a.pyr.texels;
  b.tiny_n = b.cta_n = 0;
  if (a.grad_pyramid) {
    int64_t room = (kSmemMax - kBase) / 32;  // texels of 8 floats
    int l = a.pyr.levels - 1;
    for (; l >= 0; --l) {
      const int64_t cum = a.pyr.texels - a.pyr.off[l];
      if (cum > kTiny || 16 * cum > room) break;
      b.tiny_tex0 = a.pyr.off[l];
    }
    b.tiny_n = (int32_t)(a.pyr.texels - b.tiny_tex0);
    room -= 16 * (int64_t)b.tiny_n;
    b.cta_tex0 = b.tiny_tex0;
    for (; l >= 0 && b.tiny_tex0 - a.pyr.off[l] <= room; --l) b.cta_tex0 = a.pyr.off[l];
    b.cta_n = (int32_t)(b.tiny_tex0 - b.cta_tex0);
  }
  const int smem = kBase + 32 * (16 * b.tiny_n + b.cta_n);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax); });
  const int64_t tiles = (a.n + kBwdQ - 1) / kBwdQ;
  int grid = (int)(tiles < a.num_sms ? tiles : a.num_sms);
  if (grid < 1) grid = 1;
  k<<<grid, kBwdThreads, smem, s>>>(b);
  return (int)cudaGetLastError();
}

// Trainable materials keep FP32 latents (the pyramid is an Adam master).
template <int H, bool ALB>
static int bwd_dispatch_alb(const BackwardArgs& a, cudaStream_t s) {
  if (a.target)
    return a.shape.frame ? launch_bwd_one<H, true, false, true, ALB>(a, s)
                         : launch_bwd_one<H, false, false, true, ALB>(a, s);
  return a.shape.frame ? launch_bwd_one<H, true, false, false, ALB>(a, s)
                       : launch_bwd_one<H, false, false, false, ALB>(a, s);
}

template <int H>
static int bwd_dispatch(const BackwardArgs& a, cudaStream_t s) {
  if (a.pyr.f16) return (int)cudaErrorInvalidValue;
  if (a.shape.out == 6) {
    if (a.target && !a.target_albedo) return (int)cudaErrorInvalidValue;
    return bwd_dispatch_alb<H, true>(a, s);
  }
  return bwd_dispatch_alb<H, false>(a, s);
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
    float grad;
    local += log_l1(g[i], y[i], &grad);
    dg[i] = grad * inv;
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
struct AdamStep {
  float lr, b1, b2, eps, c1, c2;
};

__device__ __forceinline__ void adam_one(float& p, float& g, float& m, float& v, const AdamStep& a) {
  const float gi = g;
  m = a.b1 * m + (1.0f - a.b1) * gi;
  v = a.b2 * v + (1.0f - a.b2) * gi * gi;
  p -= a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
  g = 0.0f;
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            int64_t count, const AdamStep a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    adam_one(p[i], g[i], m[i], v[i], a);
}

// 16-byte vector form of the same per-element update (the update is HBM
// bound: four streams read, four written)
__global__ void adam4_kernel(float4* __restrict__ p, float4* __restrict__ g, float4* __restrict__ m,
                             float4* __restrict__ v, int64_t count4, const AdamStep a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 P = p[i], G = g[i], M = m[i], V = v[i];
    adam_one(P.x, G.x, M.x, V.x, a);
    adam_one(P.y, G.y, M.y, V.y, a);
    adam_one(P.z, G.z, M.z, V.z, a);
    adam_one(P.w, G.w, M.w, V.w, a);
    p[i] = P;
    g[i] = G;
    m[i] = M;
    v[i] = V;
  }
}

int launch_adam(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2, float eps,
                int step, void* stream) {
  if (count == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const AdamStep a{lr, b1, b2, eps, 1.0f - powf(b1, (float)step), 1.0f - powf(b2, (float)step)};
  float* gm = const_cast<float*>(g);
  int64_t head = 0;
  // small arrays (the MLP masters) in one scalar launch
  if (count >= (1 << 16) && (((uintptr_t)p | (uintptr_t)g | (uintptr_t)m | (uintptr_t)v) & 15u) == 0) {
    const int64_t count4 = count / 4;
    if (count4 > 0) {
      int grid = (int)((count4 + 255) / 256);
      if (grid > 8192) grid = 8192;
      adam4_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<float4*>(p), reinterpret_cast<float4*>(gm),
                                        reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), count4, a);
    }
    head = 4 * count4;
  }
  const int64_t rest = count - head;
  if (rest > 0) {
    int grid = (int)((rest + 255) / 256);
    if (grid > 4096) grid = 4096;
    adam_kernel<<<grid, 256, 0, s>>>(p + head, gm + head, m + head, v + head, rest, a);
  }
  return (int)cudaGetLastError();
}

}  // namespace nam
