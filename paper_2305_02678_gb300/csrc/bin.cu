// Material binning for queries whose material varies per query (Sec. 7.3:
// the paper has the ray tracer reorder shading work so that threads that
// evaluate the same material run together).  Three passes on the device,
// then the evaluation:
//   count   per-material histogram (each block sums a segment of queries in
//           shared memory and adds one count per material to the global
//           histogram: same-address atomics serialise in L2);
//   plan    exclusive scan of the counts into per-material cursors, and the
//           chunk table of the tensor-core kernel (each material's range cut
//           into 128-query chunks; empty slots have count 0; the number of
//           chunks in use for the kernel to read on the device);
//   permute each block reserves, per material, one run of slots for its
//           segment (one global atomic per block and material) and writes
//           each query's index to a slot of its run;
//   launch  the chunked tensor-core kernel reads each slot's query through
//           the permutation (its fields from the caller's arrays) and writes
//           its RGB in the caller's order.
// Inside a material's range, runs follow the order in which blocks reserve
// them and slots inside a run the order in which warps claim them; neither
// changes any result, since each query is evaluated on its own, and a run
// keeps its segment's screen-space neighbours together.
#include <cuda_runtime.h>

#include <climits>

#include "common.cuh"

namespace nam {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

constexpr int kSeg = 1024;  // queries per block in count and scatter

// warp-aggregated add of 1 per lane to cnt[m] in shared memory; returns the
// value this lane's increment starts from
__device__ __forceinline__ uint32_t warp_bump(uint32_t* cnt, int m, uint32_t act) {
  const uint32_t same = __match_any_sync(act, m);
  const int leader = __ffs(same) - 1;
  uint32_t base = 0;
  if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(cnt + m, (uint32_t)__popc(same));
  return __shfl_sync(same, base, leader) + __popc(same & lanemask_lt());
}

// A query takes part in binning unless `tile_k` is given and its 128-query
// tile's entry there is non-negative (a tile the selection passes handle).
__device__ __forceinline__ bool binned_query(const int32_t* tile_k, int64_t i) {
  return tile_k == nullptr || __ldg(tile_k + (i >> 7)) < 0;
}

__global__ void __launch_bounds__(kThreads) bin_count_kernel(const int32_t* __restrict__ ids, int64_t n, int nmat,
                                                             const int32_t* __restrict__ tile_k,
                                                             uint32_t* __restrict__ counts, int* err) {
  extern __shared__ uint32_t cnt[];  // [nmat]
  for (int m = threadIdx.x; m < nmat; m += blockDim.x) cnt[m] = 0;
  __syncthreads();
  const int64_t seg = (int64_t)blockIdx.x * kSeg;
  const int64_t end = seg + kSeg < n ? seg + kSeg : n;
  for (int64_t base = seg; base < end; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int m = -1;
    if (i < end && binned_query(tile_k, i)) {
      m = __ldg(ids + i);
      if (m < 0 || m >= nmat) {
        record_error(err, DEVERR_BOUNDS);
        m = -1;
      }
    }
    const uint32_t act = __ballot_sync(0xffffffffu, m >= 0);
    if (m >= 0) warp_bump(cnt, m, act);
  }
  __syncthreads();
  for (int m = threadIdx.x; m < nmat; m += blockDim.x)
    if (cnt[m]) atomicAdd(counts + m, cnt[m]);
}

// One block: cursors[m] = sum of counts before m; chunks[c] for every slot
// c < max_chunks (a material with k queries owns ceil(k / 128) chunks);
// *n_used = the chunks in use (the tensor-core kernel's table length).
__global__ void __launch_bounds__(1024) bin_plan_kernel(const uint32_t* __restrict__ counts, int nmat,
                                                        uint32_t* __restrict__ cursors, Chunk* __restrict__ chunks,
                                                        int32_t max_chunks, int32_t* __restrict__ n_used) {
  extern __shared__ uint32_t sh[];
  uint32_t* qoff = sh;             // [nmat + 1] first query of each material
  uint32_t* coff = sh + nmat + 1;  // [nmat + 1] first chunk of each material
  if (threadIdx.x == 0) {
    uint32_t q = 0, c = 0;
    for (int m = 0; m < nmat; ++m) {
      qoff[m] = q;
      coff[m] = c;
      q += counts[m];
      c += (counts[m] + 127) / 128;
    }
    qoff[nmat] = q;
    coff[nmat] = c;
  }
  __syncthreads();
  for (int m = threadIdx.x; m < nmat; m += blockDim.x) cursors[m] = qoff[m];
  const uint32_t used = coff[nmat];
  if (threadIdx.x == 0) *n_used = (int32_t)used;
  for (int32_t c = threadIdx.x; c < max_chunks; c += blockDim.x) {
    Chunk ch;
    if ((uint32_t)c < used) {
      int lo = 0, hi = nmat - 1;  // the material whose chunk range holds c
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (coff[mid] <= (uint32_t)c) lo = mid;
        else hi = mid - 1;
      }
      const uint32_t k = (uint32_t)c - coff[lo];
      ch.start = (int64_t)qoff[lo] + 128ll * k;
      const uint32_t left = qoff[lo + 1] - (qoff[lo] + 128u * k);
      ch.count = (int32_t)(left < 128u ? left : 128u);
      ch.material = lo;
    } else {
      ch.start = 0;
      ch.count = 0;
      ch.material = 0;
    }
    chunks[c] = ch;
  }
}

// Permutation.  Each query's index goes to a slot of its material's range: a
// segment of at most kDirectMaterials materials writes each index at its
// warp's bump (a warp's lanes of one material take consecutive slots); a
// segment of more is ordered first (the indices of its valid queries placed
// in shared memory by material, a local counting sort), then each
// material's run is written to consecutive slots.  Either way a run keeps
// its segment's queries in their order, so that the chunked launch, which
// reads every slot's query through the permutation, gathers from few
// neighbourhoods of the caller's arrays.
// Shared memory: cnt, run, excl [nmat] each, then the query index and the
// material of each local position [kSeg] each.
constexpr int kStage = 1;
constexpr int kDirectMaterials = 4;  // segments of at most this many materials skip the ordering

__global__ void __launch_bounds__(kThreads) bin_scatter_kernel(const int32_t* __restrict__ ids, int64_t n, int nmat,
                                                               const int32_t* __restrict__ tile_k,
                                                               uint32_t* __restrict__ cursors,
                                                               int32_t* __restrict__ orig) {
  extern __shared__ uint32_t sh[];
  uint32_t* cnt = sh;               // [nmat] this segment's queries per material, then a bump counter
  uint32_t* run = sh + nmat;        // [nmat] first slot of the segment's run
  uint32_t* excl = sh + 2 * nmat;   // [nmat] first local position of each material
  uint32_t* stage = sh + 3 * nmat;  // [kSeg] query index of each local position
  int32_t* smat = reinterpret_cast<int32_t*>(stage + kStage * kSeg);  // [kSeg]
  __shared__ uint32_t wsum[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = (int64_t)blockIdx.x * kSeg;
  const int64_t end = seg + kSeg < n ? seg + kSeg : n;
  for (int m = threadIdx.x; m < nmat; m += blockDim.x) cnt[m] = 0;
  __syncthreads();
  for (int64_t base = seg; base < end; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int m = i < end && binned_query(tile_k, i) ? __ldg(ids + i) : -1;
    if (m >= nmat) m = -1;
    const uint32_t act = __ballot_sync(0xffffffffu, m >= 0);
    if (m >= 0) warp_bump(cnt, m, act);
  }
  __syncthreads();
  // exclusive scan of cnt over the materials: each thread sums a contiguous
  // block of entries, the block scans the thread sums
  const int per = (nmat + kThreads - 1) / kThreads;
  const int m0 = threadIdx.x * per, m1 = m0 + per < nmat ? m0 + per : nmat;
  uint32_t mine = 0;
  for (int m = m0; m < m1; ++m) mine += cnt[m];
  uint32_t x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t before = x - mine;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  for (int m = m0; m < m1; ++m) {
    excl[m] = before;
    before += cnt[m];
  }
  uint32_t total = 0;
  for (int w = 0; w < kThreads / 32; ++w) total += wsum[w];
  // a segment of a few materials is written directly below: each warp's
  // lanes of one material already take consecutive slots; staging pays off
  // only for many (threads whose materials are present, a lower bound on the
  // segment's materials when a thread covers several)
  bool present = false;
  for (int m = m0; m < m1; ++m) present |= cnt[m] != 0;
  const bool one = __syncthreads_count(present) <= kDirectMaterials;
  for (int m = threadIdx.x; m < nmat; m += blockDim.x) {
    run[m] = cnt[m] ? atomicAdd(cursors + m, cnt[m]) : 0u;
    cnt[m] = 0;
  }
  __syncthreads();
  if (one) {
    for (int64_t base = seg; base < end; base += blockDim.x) {
      const int64_t i = base + threadIdx.x;
      int m = i < end && binned_query(tile_k, i) ? __ldg(ids + i) : -1;
      if (m >= nmat) m = -1;
      const uint32_t act = __ballot_sync(0xffffffffu, m >= 0);
      if (m < 0) continue;
      const uint32_t slot = run[m] + warp_bump(cnt, m, act);
      orig[slot] = (int32_t)i;
    }
    return;
  }
  // stage: local position = the material's first position + its bump
  for (int64_t base = seg; base < end; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int m = i < end && binned_query(tile_k, i) ? __ldg(ids + i) : -1;
    if (m >= nmat) m = -1;
    const uint32_t act = __ballot_sync(0xffffffffu, m >= 0);
    if (m < 0) continue;
    const uint32_t lp = excl[m] + warp_bump(cnt, m, act);
    stage[lp] = (uint32_t)i;
    smat[lp] = m;
  }
  __syncthreads();
  // write: consecutive positions of one material go to consecutive slots
  for (uint32_t p = threadIdx.x; p < total; p += blockDim.x) {
    const int m = smat[p];
    const int64_t i = stage[p];
    const uint32_t slot = run[m] + (p - excl[m]);
    orig[slot] = (int32_t)i;
  }
}


// Per-tile selection (Sec. 7.1: the shader picks per warp between a code
// path for coherent and one for divergent execution).  A tcgen05 MMA covers
// the 128 rows of a CTA's tile, so the choice is made per 128-query tile, in
// place (no query moves):
//   k <= kSelectPasses   k tensor-core passes over the whole tile, one per
//                        material, each storing only its own material's
//                        rows (SIMT divergence serialises a warp over its
//                        branch targets the same way); k = 1 is the
//                        coherent path;
//   k > kSelectPasses    the tile's queries are binned by material with those
//                        of the other such tiles (the binning passes above,
//                        limited to them) and run in material-coherent
//                        chunks: the reordering the paper gets from SER
//                        (Sec. 7.3).
// With kSelectPasses = 1 every tile of two or more materials is binned:
// even two masked passes over a tile cost more tensor-core time than the
// binning of its queries.
// Three passes build the pass table grouped by material: per-tile material
// lists and per-material pass counts (one warp per tile), an exclusive scan
// of the counts (one block, which also writes the table's length for the
// tensor-core kernel), and the table itself; tile_k = -1 marks the tiles
// left to binning.
constexpr int kTilesPerBlock = kThreads / 32;  // one tile per warp in the list pass
constexpr int kWriteThreads = 256;             // one tile per thread in the write pass

// One warp per tile: the tile's distinct materials in increasing order (at
// most kSelectPasses; tile_k = -1 beyond), and one count per pass added to
// its material's total.
__global__ void __launch_bounds__(kThreads) select_tiles_kernel(const int32_t* __restrict__ ids, int64_t n,
                                                                int nmat, int32_t* __restrict__ tile_k,
                                                                int32_t* __restrict__ tile_mats,
                                                                int32_t* __restrict__ mat_passes, int* err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (n + 127) / 128;
  const int64_t t = (int64_t)blockIdx.x * kTilesPerBlock + warp;
  if (t >= ntiles) return;  // uniform over the warp
  const int64_t base = t * 128;
  const int cnt = (int)(n - base < 128 ? n - base : 128);
  int v[4];  // this lane's ids; INT_MAX once taken (or absent, or invalid)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = lane + 32 * q;
    v[q] = INT_MAX;
    if (r < cnt) {
      const int m = __ldg(ids + base + r);
      if (m < 0 || m >= nmat) record_error(err, DEVERR_BOUNDS);
      else v[q] = m;
    }
  }
  int k = 0, mine = 0;  // mine: the material of this lane's pass (lane < k)
  bool over = false;
  for (;;) {
    const int lm = min(min(v[0], v[1]), min(v[2], v[3]));
    const int m = __reduce_min_sync(0xffffffffu, lm);
    if (m == INT_MAX) break;
    if (k == kSelectPasses) {
      over = true;
      break;
    }
    if (lane == k) mine = m;
    if (lane == 0) tile_mats[t * kSelectPasses + k] = m;
    ++k;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (v[q] == m) v[q] = INT_MAX;
  }
  if (lane == 0) tile_k[t] = over ? -1 : k;
  // lane j counts the tile's pass j (same-address adds of one material
  // from many tiles serialise in L2, a few thousand per frame)
  if (!over && lane < k) atomicAdd(mat_passes + mine, 1);
}

// inclusive scan over a warp
__device__ __forceinline__ int32_t warp_scan(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// One block of 1024: the material counts become cursors (exclusive scan, in
// place) and *total their sum, the pass table's length.
__global__ void __launch_bounds__(1024) select_scan_kernel(int32_t* __restrict__ counts, int nmat,
                                                           int32_t* __restrict__ total) {
  __shared__ int32_t wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t carry = 0;
  for (int base = 0; base < nmat; base += 1024) {
    const int i = base + threadIdx.x;
    const int32_t v = i < nmat ? counts[i] : 0;
    const int32_t x = warp_scan(v);
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) wsum[lane] = warp_scan(wsum[lane]);
    __syncthreads();
    if (i < nmat) counts[i] = carry + (warp ? wsum[warp - 1] : 0) + x - v;
    carry += wsum[31];
    __syncthreads();  // wsum is rewritten by the next iteration
  }
  if (threadIdx.x == 0) *total = carry;
}

// One thread per tile: each of its passes goes to the next slot of its
// material's run, so that the pass table is grouped by material (a CTA's
// range of it then meets few materials, and warpgroups share their weight
// slots); the order inside a run does not change any result.  A tile left
// to binning has no pass.
__global__ void __launch_bounds__(kWriteThreads) select_write_kernel(const int32_t* __restrict__ tile_k,
                                                                     const int32_t* __restrict__ tile_mats,
                                                                     int64_t n, int32_t* __restrict__ cursors,
                                                                     Chunk* __restrict__ passes) {
  const int64_t ntiles = (n + 127) / 128;
  const int64_t t = (int64_t)blockIdx.x * kWriteThreads + threadIdx.x;
  if (t >= ntiles) return;
  const int32_t k = __ldg(tile_k + t);
  if (k <= 0) return;
  const int64_t base = t * 128;
  const int cnt = (int)(n - base < 128 ? n - base : 128);
  for (int j = 0; j < k; ++j) {
    Chunk ch;
    ch.start = base;
    ch.count = cnt;
    ch.material = __ldg(tile_mats + t * kSelectPasses + j);
    passes[atomicAdd(cursors + ch.material, 1)] = ch;
  }
}

}  // namespace

size_t bin_scratch_bytes(int64_t n, int nmat, bool xi) {
  (void)xi;
  const size_t f = ((size_t)n * 4 + 255) / 256 * 256;
  return f /* slot -> query */ + 2 * (((size_t)nmat * 4 + 255) / 256 * 256) + 256 /* chunks in use */ +
         ((size_t)max_bin_chunks(n, nmat) * sizeof(Chunk) + 255) / 256 * 256;
}

int32_t max_bin_chunks(int64_t n, int nmat) { return (int32_t)((n + 127) / 128 + nmat); }

// The binning passes over the queries of `a` (with `tile_k`, only those of
// the tiles whose entry is negative), the tensor-core launch over the
// binned ranges (as many chunks as the plan fills) and the write-back.
static int bin_eval(const BinArgs& a, const int32_t* tile_k, cudaStream_t s) {
  const int64_t n = a.n;
  const size_t f = ((size_t)n * 4 + 255) / 256 * 256;
  uint8_t* p = (uint8_t*)a.scratch;
  int32_t* orig = (int32_t*)p; p += f;
  const size_t mb = ((size_t)a.nmat * 4 + 255) / 256 * 256;
  uint32_t* counts = (uint32_t*)p; p += mb;
  uint32_t* cursors = (uint32_t*)p; p += mb;
  int32_t* n_used = (int32_t*)p; p += 256;
  Chunk* chunks = (Chunk*)p;
  const int32_t maxc = max_bin_chunks(n, a.nmat);

  int e = (int)cudaMemsetAsync(counts, 0, (size_t)a.nmat * 4, s);
  if (e) return e;
  const int gseg = (int)((n + kSeg - 1) / kSeg);
  bin_count_kernel<<<gseg, kThreads, a.nmat * sizeof(uint32_t), s>>>(a.ids, n, a.nmat, tile_k, counts, a.L.err);
  bin_plan_kernel<<<1, 1024, 2 * (a.nmat + 1) * sizeof(uint32_t), s>>>(counts, a.nmat, cursors, chunks, maxc, n_used);
  const int scatter_smem = (3 * a.nmat + (kStage + 1) * kSeg) * (int)sizeof(uint32_t);
  static std::atomic<uint64_t> scatter_attr{0};
  once_per_device(scatter_attr, [] {
    cudaFuncSetAttribute(bin_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (3 * NAM_MAX_BIN_MATERIALS + (kStage + 1) * kSeg) * (int)sizeof(uint32_t));
  });
  bin_scatter_kernel<<<gseg, kThreads, scatter_smem, s>>>(a.ids, n, a.nmat, tile_k, cursors, orig);
  e = (int)cudaGetLastError();
  if (e) return e;
  // the chunked launch reads each slot's query through the permutation and
  // writes its RGB in the caller's order
  LaunchCommon L = a.L;
  L.rgb = a.rgb_out;
  L.chunks = chunks;
  L.n_chunks = maxc;
  L.n_chunks_dev = n_used;
  L.row_ids = nullptr;
  L.gather = orig;
  return launch_material(L, a.precision, s);
}

int launch_bin_eval(const BinArgs& a, void* stream) { return bin_eval(a, nullptr, (cudaStream_t)stream); }

// Scratch of a selection launch: tile_k [ntiles], tile_mats [ntiles][kSelectPasses],
// per material its pass count, then cursor [nmat], the pass count, the pass
// table (at most one pass per query and kSelectPasses per tile), then the
// binning scratch of the tiles left to binning (bin_scratch_bytes).
namespace {
struct SelectLayout {
  size_t tile_k, tile_mats, counts, total, passes, bin, bytes;
  int64_t ntiles, nb, cap;
};
SelectLayout select_layout(int64_t n, int nmat, bool xi) {
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  SelectLayout l;
  l.ntiles = (n + 127) / 128;
  l.nb = (l.ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
  l.cap = l.ntiles * kSelectPasses < n ? l.ntiles * kSelectPasses : n;
  l.tile_k = 0;
  l.tile_mats = l.tile_k + r((size_t)l.ntiles * 4);
  l.counts = l.tile_mats + r((size_t)l.ntiles * kSelectPasses * 4);
  l.total = l.counts + r((size_t)nmat * 4);
  l.passes = l.total + 256;
  l.bin = l.passes + r((size_t)l.cap * sizeof(Chunk));
  l.bytes = l.bin + bin_scratch_bytes(n, nmat, xi);
  return l;
}
}  // namespace

size_t select_scratch_bytes(int64_t n, int nmat, bool xi) { return select_layout(n, nmat, xi).bytes; }

int launch_select_eval(const SelectArgs& a, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = a.L.n;
  if (n == 0) return 0;
  const int nmat = a.L.mats.nmat;
  const SelectLayout l = select_layout(n, nmat, a.L.q.xi != nullptr);
  uint8_t* p = (uint8_t*)a.scratch;
  int32_t* tile_k = (int32_t*)(p + l.tile_k);
  int32_t* tile_mats = (int32_t*)(p + l.tile_mats);
  int32_t* counts = (int32_t*)(p + l.counts);
  int32_t* total = (int32_t*)(p + l.total);
  Chunk* passes = (Chunk*)(p + l.passes);
  int e = (int)cudaMemsetAsync(counts, 0, (size_t)nmat * 4, s);
  if (e) return e;
  select_tiles_kernel<<<(int)l.nb, kThreads, 0, s>>>(a.ids, n, nmat, tile_k, tile_mats, counts, a.L.err);
  select_scan_kernel<<<1, 1024, 0, s>>>(counts, nmat, total);
  select_write_kernel<<<(int)((l.ntiles + kWriteThreads - 1) / kWriteThreads), kWriteThreads, 0, s>>>(
      tile_k, tile_mats, n, counts, passes);
  e = (int)cudaGetLastError();
  if (e) return e;
  LaunchCommon L = a.L;
  L.chunks = passes;
  L.n_chunks = (int32_t)l.cap;
  L.n_chunks_dev = total;
  // a pass stores only the rows of its material: the other materials of
  // its tile, and ids out of range, are left alone
  L.row_ids = a.ids;
  e = launch_material(L, a.precision, stream);
  if (e) return e;
  BinArgs b;
  b.L = a.L;
  b.ids = a.ids;
  b.nmat = nmat;
  b.n = n;
  b.rgb_out = a.L.rgb;
  b.precision = a.precision;
  b.num_sms = a.L.num_sms;
  b.scratch = p + l.bin;
  return bin_eval(b, tile_k, s);
}

}  // namespace nam
