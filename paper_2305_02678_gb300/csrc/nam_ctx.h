// Host-side state behind the opaque handles (internal).
#pragma once
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "nam_internal.h"

struct nam_material_s {
  nam_material_desc desc;     // pointers in it are not kept
  nam::Shape shape;
  nam::PyrDesc pyr;
  int64_t n_params = 0;
  void* pyramid = nullptr;    // device pyramid (FP16 or FP32 texels)
  void* blob = nullptr;       // tensor-core weight blob (F16 / FP8)
  float* params = nullptr;    // FP32 masters (frame then decoder)
  void* sampler = nullptr;    // importance-sampler weights as tensor-core operands, or null
  int64_t pyr_off = 0;        // trainable: offset of the pyramid block in
                              // adam_m / adam_v / grad (n_params rounded up
                              // to 16 bytes, for the 16-byte vector atomics)
  float* adam_m = nullptr;    // trainable: [pyr_off + texels*8]
  float* adam_v = nullptr;
  float* grad = nullptr;      // trainable: gradient buffer, same layout
  void* train_scratch = nullptr;  // trainable: the training step's loss accumulator
  size_t train_scratch_bytes = 0;
  // encoder (Sec. 5.1), trainable materials created with encoder_inputs > 0:
  // one allocation of 4 x enc_n floats: masters, gradient, Adam m, Adam v
  int32_t enc_in = 0;
  int64_t enc_n = 0;
  float* enc = nullptr;
  void* enc_scratch = nullptr;    // a batch's latents and their gradients
  size_t enc_scratch_bytes = 0;
  nam_material_info info{};
};

namespace nam {
struct ServeState;
}

struct nam_ctx {
  int device = 0;
  int num_sms = 0;
  bool host_direct = false;             // kernels may read host memory (page tables)
  uint64_t budget = 0;
  uint64_t timeout_ns = 0;
  int serve_streams = 4;
  int serve_queue_depth = 256;
  std::atomic<uint64_t> resident{0};
  int* err_word = nullptr;
  std::mutex mu;                        // guards `materials`
  std::set<nam_material> materials;
  // staging for nam_eval_host
  std::mutex stage_mu;
  void* stage_dev = nullptr;
  size_t stage_bytes = 0;
  void* stage_stream = nullptr;
  void* h2d_stream = nullptr;           // nam_eval_host: copies in / out, overlapping
  void* d2h_stream = nullptr;           // the kernels on the caller's stream
  std::vector<void*> stage_events;
  // fault injection
  std::atomic<bool> fault_alloc{false};
  std::atomic<bool> fault_launch{false};
  std::atomic<bool> fault_stall{false};
  // stream-ordered allocations (serving frame buffers, work tables): a pool
  // of the context's own that keeps freed memory instead of returning it to
  // the driver, so that steady-state frames do not pay for remapping
  cudaMemPool_t pool = nullptr;
  // serving
  nam::ServeState* serve = nullptr;
  std::mutex serve_mu;                  // guards `serve` creation
};

namespace nam {

struct DeviceGuard {
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
  int prev_ = 0, dev_ = 0;
};

nam_status fail(nam_status s, const char* fmt, ...);
nam_status cuda_fail(int e, const char* what);
int dev_alloc(nam_ctx* ctx, void** p, size_t bytes);
bool budget_reserve(nam_ctx* ctx, uint64_t bytes);
void budget_release(nam_ctx* ctx, uint64_t bytes);
nam_status validate_desc(const nam_material_desc* d, Shape* shape, PyrDesc* pyr);
nam_status check_queries(const nam_material_s* m, const nam_queries* q);
void fill_launch(nam_ctx* ctx, const nam_material_s* m, const nam_queries* q, int64_t n, float* rgb, uint32_t flags,
                 LaunchCommon* L);
int launch_material(const LaunchCommon& L, int precision, void* stream);
void build_chunks(const nam_work_item* items, int32_t n_items, std::vector<Chunk>* out);
nam_status check_multi(nam_ctx* ctx, const nam_material* mats, int32_t nmat);
void serve_stop(nam_ctx* ctx);

}  // namespace nam
