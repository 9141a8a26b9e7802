// A training step for callers that cannot allocate device memory.
//
// nam_train_step keeps its loss accumulator in device memory it allocates on
// its first call.  Callers that must not allocate once they are running -- a
// renderer or trainer with a fixed memory plan, a host that forbids
// cudaMalloc outside its own allocator, code that must not synchronise the
// device (cudaMalloc/cudaFree may) -- use nam_train_step_noalloc instead,
// which runs the forward, the loss and the backward as separate passes and
// keeps their per-batch buffers (the forward's RGB, dL/dRGB and the loss
// accumulator) in the file-scope device array below.  The array is part of the library image:
// every GPU that loads libnam holds it (NAM_NOALLOC_TRAIN_MAX_QUERIES * 24 +
// 256 bytes, 1.5 MiB) until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "nam_ctx.h"

using namespace nam;

namespace {

constexpr int64_t kMaxQueries = NAM_NOALLOC_TRAIN_MAX_QUERIES;
constexpr int64_t kHeaderFloats = 64;  // loss accumulator, padded to 256 bytes

// [0, 64): loss accumulator; then rgb [max][3]; then dL/drgb [max][3]
__device__ __align__(256) float g_train_scratch[kHeaderFloats + 6 * kMaxQueries];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the array on the current device.  The host-side name
// g_train_scratch is only a stand-in and must never reach a kernel.
nam_status scratch_on_device(int dev, float** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(NAM_ERR_UNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_train_scratch);
    if (e != cudaSuccess) return cuda_fail((int)e, "nam_train_step_noalloc: cudaGetSymbolAddress");
    g_scratch_dev[dev] = (float*)p;
  }
  *out = g_scratch_dev[dev];
  return NAM_OK;
}

}  // namespace

extern "C" nam_status nam_train_step_noalloc(nam_ctx* ctx, nam_material m, const nam_queries* q,
                                             const float* target_rgb, int64_t n, const nam_adam* opt, float* loss_out,
                                             void* stream, uint32_t flags) {
  if (!ctx || !m) return fail(NAM_ERR_INVALID_ARG, "nam_train_step_noalloc: NULL context or material");
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->materials.count(m)) return fail(NAM_ERR_NOT_FOUND, "nam_train_step_noalloc: unknown material");
  }
  if (!m->desc.trainable) return fail(NAM_ERR_UNSUPPORTED, "nam_train_step_noalloc: material is not trainable");
  if (m->shape.NH != 2 || m->shape.frame == 2)
    return fail(NAM_ERR_UNSUPPORTED, "nam_train_step_noalloc: reverse mode supports the frame MLP form with two hidden layers");
  if (m->shape.out != 3)
    return fail(NAM_ERR_UNSUPPORTED, "nam_train_step_noalloc: the material has the albedo head (nam_train_step_albedo)");
  if (n <= 0) return fail(NAM_ERR_INVALID_ARG, "nam_train_step_noalloc: n must be > 0");
  if (n > kMaxQueries)
    return fail(NAM_ERR_INVALID_ARG, "nam_train_step_noalloc: batch of %lld queries exceeds the %lld the static buffer holds",
                (long long)n, (long long)kMaxQueries);
  if (!target_rgb || !opt) return fail(NAM_ERR_INVALID_ARG, "nam_train_step_noalloc: NULL target or optimiser settings");
  if (opt->step < 1) return fail(NAM_ERR_INVALID_ARG, "nam_train_step_noalloc: Adam step is 1-based");
  nam_status st = check_queries(m, q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  float* scratch = nullptr;
  st = scratch_on_device(ctx->device, &scratch);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  float* loss_acc = scratch;
  float* rgb = scratch + kHeaderFloats;
  float* grad_rgb = rgb + 3 * n;
  // the accumulator keeps the previous call's value: clear it
  cudaError_t ce = cudaMemsetAsync(loss_acc, 0, sizeof(float), s);
  if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_train_step_noalloc: clear");
  LaunchCommon L;
  fill_launch(ctx, m, q, n, rgb, flags, &L);
  int e = launch_eval_f32(L, s);
  if (!e) e = launch_loss(rgb, target_rgb, n, grad_rgb, loss_acc, s);
  BackwardArgs a;
  std::memset(&a, 0, sizeof a);
  a.pyr = m->pyr;
  a.shape = m->shape;
  a.q = QueryPtrs{q->u, q->v, q->lod, q->wix, q->wiy, q->wiz, q->wox, q->woy, q->woz, q->xi};
  a.n = n;
  a.pyramid = m->pyramid;
  a.params = m->params;
  a.grad_rgb = grad_rgb;
  a.grad_params = m->grad;
  a.grad_pyramid = m->grad + m->pyr_off;
  a.flags = flags;
  a.num_sms = ctx->num_sms;
  if (!e) e = launch_backward(a, s);
  const int64_t np = m->n_params, po = m->pyr_off, nt = m->pyr.texels * 8;
  if (!e)
    e = launch_adam(m->params, m->grad, m->adam_m, m->adam_v, np, opt->lr_params, opt->beta1, opt->beta2, opt->eps,
                    opt->step, s);
  if (!e)
    e = launch_adam((float*)m->pyramid, m->grad + po, m->adam_m + po, m->adam_v + po, nt, opt->lr_pyramid,
                    opt->beta1, opt->beta2, opt->eps, opt->step, s);
  if (e) return cuda_fail(e, "nam_train_step_noalloc: launch");
  if (loss_out) {
    ce = cudaMemcpyAsync(loss_out, loss_acc, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_train_step_noalloc: loss readback");
  }
  return NAM_OK;
}
