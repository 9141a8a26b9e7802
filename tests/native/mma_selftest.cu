// Test-only library (built by tests/test_g0_mma_selftest.py, not part of
// libnam): one tcgen05 MMA in isolation, to check the shared-memory and
// instruction descriptors and the TMEM read-back conventions that every
// tensor-core kernel of the library relies on.
//
//   D[128][64] = A[128][32] B[64][32]^T, binary16 operands, FP32 result.
//
// mma_selftest(A, B, D, a_in_tmem): A, B host arrays of binary16 bits; with
// a_in_tmem == 0 both in the canonical K-major layout (element (r, k) of an
// R-row operand at byte (k/8)*R*16 + r*16 + (k%8)*2), with a_in_tmem == 1 A
// row-major [128][32] (stored to TMEM two elements per 32-bit column by the
// kernel) and B as before; D host [128][64] row-major.  Returns 0, a CUDA
// error code, or -1 if the kernel's wait for the MMA ran out (it then waits
// for the MMA with a fixed drain limit and frees its TMEM only if it
// completed, -2 if it did not).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../paper_2305_02678_gb300/csrc/tc_ptx.cuh"

using namespace nam;

namespace {

__global__ void __launch_bounds__(128) selftest_kernel(const uint8_t* A, const uint8_t* B, float* D, int a_in_tmem,
                                                      int* status) {
  // A: 128 x 32 binary16 = 8 KB, B: 64 x 32 = 4 KB, at offsets sized so that
  // every address a descriptor can form stays inside the 48 KB region
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + 32768;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 32768 + 16384);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (!a_in_tmem)
    for (int k = tid; k < 8192 / 16; k += 128) reinterpret_cast<uint4*>(sA)[k] = reinterpret_cast<const uint4*>(A)[k];
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
  if (a_in_tmem) {
    const uint16_t* Ar = reinterpret_cast<const uint16_t*>(A);
    uint32_t row[16];
    for (int j = 0; j < 16; ++j) row[j] = (uint32_t)Ar[tid * 32 + 2 * j] | ((uint32_t)Ar[tid * 32 + 2 * j + 1] << 16);
    ptx::tmem_st16(tmem + lane + 64, row);
    ptx::tmem_st_wait();
    ptx::tc_fence_before();
    __syncthreads();
  }
  const uint32_t aA = ptx::smem_u32(sA), aB = ptx::smem_u32(sB);
  if (tid == 0) {
    ptx::tc_fence_after();
    constexpr uint32_t id = ptx::idesc_f16(128, 64);
    if (a_in_tmem) {
      ptx::mma_f16_ts(tmem, tmem + 64, ptx::sdesc(aB, 64 * 16, 128), id, 0);
      ptx::mma_f16_ts(tmem, tmem + 64 + 8, ptx::sdesc(aB + 2 * 64 * 16, 64 * 16, 128), id, 1);
    } else {
      ptx::mma_f16(tmem, ptx::sdesc(aA, 2048, 128), ptx::sdesc(aB, 64 * 16, 128), id, 0);
      ptx::mma_f16(tmem, ptx::sdesc(aA + 4096, 2048, 128), ptx::sdesc(aB + 2 * 64 * 16, 64 * 16, 128), id, 1);
    }
    ptx::mma_commit(b);
  }
  bool ok = ptx::mbar_wait(b, 0, 1000000000ull);
  bool drained = ok || ptx::mbar_wait(b, 0, ptx::kDrainTimeoutNs);
  ptx::tc_fence_after();
  if (ok) {
    uint32_t acc[32];
    for (int c0 = 0; c0 < 64; c0 += 32) {
      ptx::tmem_ld32(tmem + lane + c0, acc);
      ptx::tmem_ld_wait();
      for (int j = 0; j < 32; ++j) D[tid * 64 + c0 + j] = __uint_as_float(acc[j]);
    }
  } else if (tid == 0) {
    *status = drained ? -1 : -2;
  }
  ptx::tc_fence_before();
  const bool all = __syncthreads_and(drained ? 1 : 0) != 0;
  if (warp == 0 && all) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 128);
  }
}

}  // namespace

extern "C" int mma_selftest(const uint16_t* A_host, const uint16_t* B_host, float* D_host, int a_in_tmem) {
  void *A = nullptr, *B = nullptr, *D = nullptr, *S = nullptr;
  int status = 0;
  cudaError_t e = cudaMalloc(&A, 8192);
  if (e == cudaSuccess) e = cudaMalloc(&B, 4096);
  if (e == cudaSuccess) e = cudaMalloc(&D, 128 * 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&S, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(A, A_host, 8192, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B, B_host, 4096, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(D, 0, 128 * 64 * 4);
  if (e == cudaSuccess) e = cudaMemset(S, 0, sizeof(int));
  const int smem = 32768 + 16384 + 64;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) {
    // every operand was allocated and copied: only now does the kernel run
    selftest_kernel<<<1, 128, smem>>>((const uint8_t*)A, (const uint8_t*)B, (float*)D, a_in_tmem, (int*)S);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(D_host, D, 128 * 64 * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&status, S, sizeof(int), cudaMemcpyDeviceToHost);
  }
  cudaFree(A);
  cudaFree(B);
  cudaFree(D);
  cudaFree(S);
  return e != cudaSuccess ? (int)e : status;
}
