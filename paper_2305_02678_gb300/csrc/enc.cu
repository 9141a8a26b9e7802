// Encoder of the first training phase (Sec. 5.1): an MLP from the material
// parameters k(x) to the 8-channel latent, K -> 32 -> 32 -> 8 with ReLU
// hidden layers and a linear output.  It runs only in training: per query in
// the first phase (its output replaces the latent texture fetch) and once
// per texel to initialise the texture.
//
// Forward (encode_kernel): one thread per row, weights in shared memory.
// Backward (encoder_backward_kernel): a CTA of 128 threads takes tiles of 128
// rows; phase A (thread = row) recomputes the forward and back-propagates
// dL/dz to the hidden pre-activations, keeping the layer inputs and deltas of
// the tile in shared memory; phase B (thread = 4x4 block of one weight
// matrix) sums the outer products over the tile in registers; one atomic per
// parameter per CTA at the end.
#include <cuda_runtime.h>

#include "nam_internal.h"

namespace nam {
namespace {

constexpr int kE = 32;        // hidden width
constexpr int kKMax = 16;     // inputs, padded
constexpr int kTile = 128;    // rows per backward tile

// weights in shared memory, rows padded to 16-byte multiples
struct EncW {
  float W1[kE][kKMax];  // zero beyond K
  float b1[kE];
  float W2[kE][kE];
  float b2[kE];
  float W3[8][kE];
  float b3[8];
};

__device__ void load_encoder(EncW& S, const float* __restrict__ p, int K, int t, int nt) {
  for (int i = t; i < kE * kKMax; i += nt) {
    const int j = i / kKMax, c = i % kKMax;
    S.W1[j][c] = c < K ? p[j * K + c] : 0.0f;
  }
  p += kE * K;
  for (int i = t; i < kE; i += nt) S.b1[i] = p[i];
  p += kE;
  for (int i = t; i < kE * kE; i += nt) S.W2[i / kE][i % kE] = p[i];
  p += kE * kE;
  for (int i = t; i < kE; i += nt) S.b2[i] = p[i];
  p += kE;
  for (int i = t; i < 8 * kE; i += nt) S.W3[i / kE][i % kE] = p[i];
  p += 8 * kE;
  for (int i = t; i < 8; i += nt) S.b3[i] = p[i];
}

__device__ __forceinline__ void load_row(const float* __restrict__ attrs, int K, int64_t i, float k[kKMax]) {
#pragma unroll
  for (int c = 0; c < kKMax; ++c) k[c] = c < K ? attrs[i * K + c] : 0.0f;
}

// h1 = ReLU(W1 k + b1) into registers, h2 = ReLU(W2 h1 + b2) into the
// caller's shared-memory row; pre-activation signs in masks
__device__ __forceinline__ void hidden(const EncW& S, const float k[kKMax], float h1[kE], float* h2row,
                                       uint32_t& m1, uint32_t& m2) {
  m1 = m2 = 0;
#pragma unroll
  for (int j = 0; j < kE; ++j) {
    float s = S.b1[j];
#pragma unroll
    for (int c = 0; c < kKMax; ++c) s = fmaf(S.W1[j][c], k[c], s);
    h1[j] = fmaxf(s, 0.0f);
    if (s > 0.0f) m1 |= 1u << j;
  }
#pragma unroll 1
  for (int j = 0; j < kE; ++j) {
    float s = S.b2[j];
#pragma unroll
    for (int c = 0; c < kE; ++c) s = fmaf(S.W2[j][c], h1[c], s);
    h2row[j] = fmaxf(s, 0.0f);
    if (s > 0.0f) m2 |= 1u << j;
  }
}

constexpr int kFwdThreads = 256;

__global__ void __launch_bounds__(kFwdThreads) encode_kernel(const float* __restrict__ W, int K,
                                                             const float* __restrict__ attrs, int64_t n,
                                                             float* __restrict__ z_out) {
  __shared__ __align__(16) EncW S;
  __shared__ float H2[kFwdThreads][kE + 1];  // odd stride: a thread's row, conflict-free
  load_encoder(S, W, K, threadIdx.x, blockDim.x);
  __syncthreads();
  float* h2 = H2[threadIdx.x];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float k[kKMax], h1[kE];
    uint32_t m1, m2;
    load_row(attrs, K, i, k);
    hidden(S, k, h1, h2, m1, m2);
    float z[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) z[c] = S.b3[c];
#pragma unroll 4
    for (int j = 0; j < kE; ++j) {
      const float h = h2[j];
#pragma unroll
      for (int c = 0; c < 8; ++c) z[c] = fmaf(S.W3[c][j], h, z[c]);
    }
    float4* o = reinterpret_cast<float4*>(z_out + i * 8);
    o[0] = make_float4(z[0], z[1], z[2], z[3]);
    o[1] = make_float4(z[4], z[5], z[6], z[7]);
  }
}

struct EncBwdSmem {
  EncW w;
  static constexpr int S = kE + 4;  // padded row stride
  float X[kTile][kKMax];            // inputs k
  float H1[kTile][S], D1[kTile][S];
  float H2[kTile][S], D2[kTile][S];
  float DZ[kTile][8];
};

__global__ void __launch_bounds__(kTile) encoder_backward_kernel(const float* __restrict__ W, int K,
                                                                 const float* __restrict__ attrs,
                                                                 const float* __restrict__ dz, int64_t n,
                                                                 float* __restrict__ grad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EncBwdSmem& S = *reinterpret_cast<EncBwdSmem*>(smem_raw);
  const int t = threadIdx.x;
  load_encoder(S.w, W, K, t, kTile);
  // phase-B ownership: 4x4 blocks of dW3 [8][32] (16), dW2 [32][32] (64),
  // dW1 [32][16] (32, columns beyond K dropped at the flush)
  int role = -1, r0 = 0, c0 = 0;
  const float* dp = nullptr;
  const float* ap = nullptr;
  int dstride = 0, astride = 0;
  {
    int b = t;
    if (b < 16) {
      role = 0; r0 = 4 * (b >> 3); c0 = 4 * (b & 7);
      dp = &S.DZ[0][r0]; dstride = 8; ap = &S.H2[0][c0]; astride = EncBwdSmem::S;
    } else if ((b -= 16) < 64) {
      role = 1; r0 = 4 * (b >> 3); c0 = 4 * (b & 7);
      dp = &S.D2[0][r0]; dstride = EncBwdSmem::S; ap = &S.H1[0][c0]; astride = EncBwdSmem::S;
    } else if ((b -= 64) < 32) {
      role = 2; r0 = 4 * (b >> 2); c0 = 4 * (b & 3);
      dp = &S.D1[0][r0]; dstride = EncBwdSmem::S; ap = &S.X[0][c0]; astride = kKMax;
    }
  }
  float acc[16], accb[4];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = 0.0f;
#pragma unroll
  for (int e = 0; e < 4; ++e) accb[e] = 0.0f;
  __syncthreads();
  const int64_t ntiles = (n + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t start = tile * kTile;
    const int count = (int)((n - start) < kTile ? (n - start) : kTile);
    // ---- phase A: thread = row -----------------------------------------------
    if (t < count) {
      const int64_t i = start + t;
      float k[kKMax], h1[kE];
      uint32_t m1, m2;
      load_row(attrs, K, i, k);
      hidden(S.w, k, h1, S.H2[t], m1, m2);
      float g[8];
      {
        const float4 a = reinterpret_cast<const float4*>(dz + i * 8)[0];
        const float4 b = reinterpret_cast<const float4*>(dz + i * 8)[1];
        g[0] = a.x; g[1] = a.y; g[2] = a.z; g[3] = a.w; g[4] = b.x; g[5] = b.y; g[6] = b.z; g[7] = b.w;
      }
#pragma unroll
      for (int c4 = 0; c4 < kKMax / 4; ++c4)
        reinterpret_cast<float4*>(&S.X[t][0])[c4] = make_float4(k[4 * c4], k[4 * c4 + 1], k[4 * c4 + 2], k[4 * c4 + 3]);
#pragma unroll
      for (int j4 = 0; j4 < kE / 4; ++j4)
        reinterpret_cast<float4*>(&S.H1[t][0])[j4] = make_float4(h1[4 * j4], h1[4 * j4 + 1], h1[4 * j4 + 2], h1[4 * j4 + 3]);
      reinterpret_cast<float4*>(&S.DZ[t][0])[0] = make_float4(g[0], g[1], g[2], g[3]);
      reinterpret_cast<float4*>(&S.DZ[t][0])[1] = make_float4(g[4], g[5], g[6], g[7]);
      // d2 = (W3^T dz) where layer 2 is active
#pragma unroll 1
      for (int j = 0; j < kE; ++j) {
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) s = fmaf(S.w.W3[c][j], g[c], s);
        S.D2[t][j] = ((m2 >> j) & 1u) ? s : 0.0f;
      }
      // d1 = (W2^T d2) where layer 1 is active (accumulated in h1's registers)
#pragma unroll
      for (int c = 0; c < kE; ++c) h1[c] = 0.0f;
#pragma unroll 2
      for (int j = 0; j < kE; ++j) {
        const float d = S.D2[t][j];
#pragma unroll
        for (int c = 0; c < kE; ++c) h1[c] = fmaf(S.w.W2[j][c], d, h1[c]);
      }
#pragma unroll
      for (int j4 = 0; j4 < kE / 4; ++j4) {
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = ((m1 >> (4 * j4 + e)) & 1u) ? h1[4 * j4 + e] : 0.0f;
        reinterpret_cast<float4*>(&S.D1[t][0])[j4] = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
    __syncthreads();
    // ---- phase B: thread = 4x4 gradient block ---------------------------------
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
  if (role < 0) return;
  // (weight offset, row stride, valid rows, valid columns, bias offset)
  const int oW1 = 0, ob1 = kE * K, oW2 = ob1 + kE, ob2 = oW2 + kE * kE, oW3 = ob2 + kE, ob3 = oW3 + 8 * kE;
  int wo = 0, ws = 0, nc = 0, bo = 0;
  switch (role) {
    case 0: wo = oW3; ws = kE; nc = kE; bo = ob3; break;
    case 1: wo = oW2; ws = kE; nc = kE; bo = ob2; break;
    default: wo = oW1; ws = K; nc = K; bo = ob1; break;
  }
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int row = r0 + rr;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
      if (c0 + cc < nc) atomicAdd(&grad[wo + row * ws + c0 + cc], acc[4 * rr + cc]);
    if (c0 == 0) atomicAdd(&grad[bo + row], accb[rr]);
  }
}

}  // namespace

int launch_encode(const float* W, int K, const float* attrs, int64_t n, float* z_out, int num_sms, void* stream) {
  if (n == 0) return 0;
  if (K < 1 || K > kKMax) return (int)cudaErrorInvalidValue;
  int64_t blocks = (n + kFwdThreads - 1) / kFwdThreads;
  const int64_t cap = (int64_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
  encode_kernel<<<(int)blocks, kFwdThreads, 0, (cudaStream_t)stream>>>(W, K, attrs, n, z_out);
  return (int)cudaGetLastError();
}

int launch_encoder_backward(const float* W, int K, const float* attrs, const float* dz, int64_t n, float* grad,
                            int num_sms, void* stream) {
  if (n == 0) return 0;
  if (K < 1 || K > kKMax) return (int)cudaErrorInvalidValue;
  const int smem = (int)sizeof(EncBwdSmem);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(encoder_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  const int64_t tiles = (n + kTile - 1) / kTile;
  int64_t grid = (int64_t)num_sms * 2;
  if (grid > tiles) grid = tiles;
  encoder_backward_kernel<<<(int)grid, kTile, smem, (cudaStream_t)stream>>>(W, K, attrs, dz, n, grad);
  return (int)cudaGetLastError();
}

}  // namespace nam
