// Internal types shared by the libnam translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/nam.h"

namespace nam {

// Device error codes recorded by kernels in the context's error word.
enum DevError : int {
  DEVERR_NONE = 0,
  DEVERR_WAIT_TIMEOUT = 1,  // a bounded mbarrier wait ran out
  DEVERR_BOUNDS = 2,        // an index failed a device-side check
  DEVERR_DRAIN_TIMEOUT = 3, // after a wait gave up, the kernel's own MMAs or
                            // copies did not complete within the drain limit;
                            // its TMEM was left allocated
};

// Latent pyramid geometry, passed by value to kernels.
struct PyrDesc {
  int32_t levels;
  int32_t f16;      // 1: binary16 texels (16 B per texel), 0: float32 (32 B)
  int32_t filter;   // NAM_FILTER_*
  int32_t address;  // NAM_ADDRESS_*
  int32_t pow2;     // every level width and height is a power of two
  int32_t w[NAM_MAX_LEVELS], h[NAM_MAX_LEVELS];
  int64_t off[NAM_MAX_LEVELS];  // first texel of each level
  int64_t texels;
};

// Planar query arrays (device) with an optional base offset.
struct QueryPtrs {
  const float *u, *v, *lod, *wix, *wiy, *wiz, *wox, *woy, *woz, *xi;
};

// Decoder shape supported by the kernels: 14 -> H (x NH hidden layers) -> 3,
// optional frame MLP 8 -> 16 -> 6.
struct Shape {
  int32_t H;        // hidden width: 16, 32, 64
  int32_t NH;       // hidden layers: 2 or 3 (3 only with H = 64)
  int32_t frame;    // 0: none, 1: frame MLP 8 -> 16 -> 6 + Gram-Schmidt,
                    // 2: the paper's linear 8 -> 12, two frames
  int32_t in;       // decoder inputs: 14, or 20 with frame == 2
  int32_t out;      // decoder outputs: 3 (RGB), or 6 with the albedo head
                    // (RGB, then the directional albedo's RGB)
};

// Frame parameters per form: MLP 16*8 + 16 + 6*16 + 6, paper 12*8 + 12.
inline int64_t frame_params_of(int frame) { return frame == 1 ? 246 : frame == 2 ? 108 : 0; }

// A chunk of at most 128 consecutive queries that all use one material.
struct Chunk {
  int64_t start;
  int32_t count;
  int32_t material;
};

// Per-launch description of the materials a kernel may use.
struct MatTable {
  const void* const* pyramid;  // device array [nmat] of pyramid pointers
  const void* const* weights;  // device array [nmat] of weight blobs
  int32_t nmat;
};

// ---------------------------------------------------------------------------
// launchers (return cudaError_t as int)
// ---------------------------------------------------------------------------
struct LaunchCommon {
  PyrDesc pyr;
  Shape shape;
  QueryPtrs q;
  float* rgb;
  int64_t n;             // queries (single-material launches)
  const Chunk* chunks;   // device chunk list (multi-material) or nullptr
  int32_t n_chunks;      // chunks when `chunks` is set (an upper bound when
                         // n_chunks_dev is set)
  const int32_t* n_chunks_dev;  // tensor-core kernel: if set, the number of
                                // chunks, written on the device by an earlier
                                // launch (at most n_chunks)
  const int32_t* row_ids;       // tensor-core kernel: if set, a chunk's row i
                                // is stored only where row_ids[i] equals the
                                // chunk's material (masked passes)
  const int32_t* gather;        // tensor-core kernel, chunked launches: if set,
                                // a chunk's row i is query gather[i] (its
                                // fields read and its outputs written there)
  MatTable mats;         // single material: nmat = 1
  const void* pyr0;      // single material pyramid
  const void* w0;        // single material weight blob
  uint32_t flags;
  int* err;
  uint64_t timeout_ns;
  int num_sms;
  float* amax;           // FP32 kernel only: if set, max |input| of each decoder
                         // layer over the batch (atomic max, starts at 0);
                         // rgb may then be null
  float* albedo;         // albedo head (shape.out == 6): if set, [n][3]
                         // directional albedo of each query
};

// Resident blocks per SM of a kernel: the occupancy API, or (resources_only,
// and as a fallback) the limit computed from the kernel's registers, shared
// memory and threads.  The API answers 1 for kernels that use TMEM, whose
// true limit (columns allocated per CTA) the caller passes as `cap`.
int blocks_per_sm(const void* func, int threads, int dyn_smem, int cap, bool resources_only = false);

// Kernel attributes (dynamic shared memory, carveout) belong to a device's
// context: `fn` runs once per device for each call site's `done` mask.
template <class F>
inline void once_per_device(std::atomic<uint64_t>& done, F fn) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    fn();
    return;
  }
  const uint64_t bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return;
  fn();
  done.fetch_or(bit, std::memory_order_acq_rel);
}

int launch_eval_f32(const LaunchCommon& L, void* stream);
// tensor-core evaluation (every shape with a tensor-core kernel): FP16, and
// FP8 (E4M3 hidden -> hidden layers)
int launch_eval_f16(const LaunchCommon& L, void* stream);
int launch_eval_fp8(const LaunchCommon& L, void* stream);
size_t f16_blob_bytes(const Shape& s);
int pack_f16_blob(const Shape& s, int precision, const float* frame, const float* dec, const float* act_scale,
                  uint8_t* out, float* weight_scales_out);
int launch_eval_tc(const LaunchCommon& L, int precision, void* stream);

// Weight blob sizes and packing (host side).
size_t f32_blob_floats(const Shape& s);
void pack_f32_blob(const Shape& s, const float* frame, const float* dec, float* out);
size_t tc_blob_bytes(const Shape& s, int precision);
int pack_tc_blob(const Shape& s, int precision, const float* frame, const float* dec,
                 const float* act_scale, uint8_t* out, float* weight_scales_out);


// Importance sampler (11 -> 32 -> 32 -> 32 -> 9 FP32 MLP + proxy density).
constexpr int kSamplerFloats = (11 * 32 + 32) + 2 * (32 * 32 + 32) + (32 * 9 + 9);
// The sampler's weights packed as tensor-core operands (binary16 hi/lo
// splits of the FP32 masters); -1 if a weight is beyond the split's range.
size_t sampler_blob_bytes();
int pack_sampler_blob(const float* weights, uint8_t* out);
// mode 0: density of each query's wo; mode 1: sample from u [n][3].
int launch_sampler(const LaunchCommon& L, const void* sampler_blob, int mode, const float* u, float* wo_out,
                   float* pdf_out, void* stream);

// Backward / training.
struct BackwardArgs {
  PyrDesc pyr;
  Shape shape;
  QueryPtrs q;
  int64_t n;
  const void* pyramid;     // FP32 master pyramid
  const float* params;     // FP32 master params (frame then decoder)
  const float* grad_rgb;   // [n][3] dL/drgb, or null when target is set
  // fused log-space L1 loss (training step): when target is set the kernel
  // takes dL/drgb from the loss of its own forward values against target
  // [n][3] and adds loss_inv * sum of the per-element losses to *loss_acc
  const float* target;
  float* loss_acc;
  float loss_inv;
  // albedo head (shape.out == 6): with target set, target_albedo [n][3]
  // holds one-sample estimates of the directional albedo and the loss adds
  // loss_inv * sum of the squared albedo errors (L2); without target,
  // grad_rgb is [n][6] (RGB, then albedo)
  const float* target_albedo;
  // encoder phase (Sec. 5.1): when z_in is set the latent of query i is
  // z_in[8 i ..] (the texture is not read) and, when dz_out is set, dL/dz of
  // query i goes to dz_out[8 i ..] instead of the pyramid gradient
  const float* z_in;
  float* dz_out;
  float* grad_params;
  float* grad_pyramid;     // may be null
  uint32_t flags;
  int num_sms;
  // set by the launcher: the gradient of texels [tiny_tex0, texels) is summed
  // in per-warp shared copies, that of [cta_tex0, tiny_tex0) in one shared
  // copy per CTA, before it reaches the global buffer
  int64_t tiny_tex0, cta_tex0;
  int32_t tiny_n, cta_n;
};
int launch_backward(const BackwardArgs& a, void* stream);

// the evaluation launch for a material's precision (tensor-core or FP32 path)
int launch_material(const LaunchCommon& L, int precision, void* stream);

// Material binning (per-query material ids): count, plan, a permutation of
// the query indices by material, one chunked launch that reads each query
// through the permutation and writes its output in place.
struct BinArgs {
  LaunchCommon L;          // caller's query pointers, flags, error word, materials table
  const int32_t* ids;      // [n] material of each query
  int32_t nmat;
  int64_t n;
  float* rgb_out;          // [n][3], the caller's order
  int precision;
  int num_sms;
  void* scratch;           // bin_scratch_bytes(n, nmat, xi) bytes, 256-byte aligned
};
int32_t max_bin_chunks(int64_t n, int nmat);
size_t bin_scratch_bytes(int64_t n, int nmat, bool xi);
int launch_bin_eval(const BinArgs& a, void* stream);

// Per-tile selection (per-query material ids), in place: a tile of 128
// queries with k <= kSelectPasses distinct materials runs as k tensor-core
// passes (one per material, each storing its own material's rows); the
// queries of tiles with more are binned by material and run in
// material-coherent chunks.  One pass per tile at most: tiles of two or
// more materials are binned (cheaper than two or more masked passes).
constexpr int kSelectPasses = NAM_SELECT_MAX_PASSES;
struct SelectArgs {
  LaunchCommon L;              // caller's queries, rgb, n, flags, materials table
  const int32_t* ids;          // [n] material of each query
  int precision;
  void* scratch;               // select_scratch_bytes(n, nmat, xi), 256-byte aligned
};
size_t select_scratch_bytes(int64_t n, int nmat, bool xi);
int launch_select_eval(const SelectArgs& a, void* stream);

// encoder (Sec. 5.1): K -> 32 -> 32 -> 8, ReLU hidden layers, linear output;
// W = per layer W[out][in] then b[out]
inline int64_t encoder_params_of(int K) { return 32 * (int64_t)K + 32 + 32 * 32 + 32 + 8 * 32 + 8; }
int launch_encode(const float* W, int K, const float* attrs, int64_t n, float* z_out, int num_sms, void* stream);
// accumulates the gradient of sum <dz, encoder(attrs)> into grad (layout of W)
int launch_encoder_backward(const float* W, int K, const float* attrs, const float* dz, int64_t n, float* grad,
                            int num_sms, void* stream);
int launch_loss(const float* rgb, const float* target, int64_t n, float* grad_rgb, float* loss_accum,
                void* stream);
int launch_adam(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2,
                float eps, int step, void* stream);
int64_t n_params_of(const Shape& s);

}  // namespace nam
