// C ABI: reverse mode and the training step (Sec. 5.2).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "nam_ctx.h"

using namespace nam;

static nam_status check_trainable(nam_ctx* ctx, nam_material m) {
  if (!ctx || !m) return fail(NAM_ERR_INVALID_ARG, "NULL context or material");
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->materials.count(m)) return fail(NAM_ERR_NOT_FOUND, "unknown material");
  }
  if (!m->desc.trainable) return fail(NAM_ERR_UNSUPPORTED, "material is not trainable");
  if (m->shape.NH != 2 || m->shape.frame == 2)
    return fail(NAM_ERR_UNSUPPORTED, "reverse mode supports the frame MLP form with two hidden layers");
  return NAM_OK;
}

static void fill_bwd(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n, const float* grad_rgb,
                     float* grad_params, float* grad_pyramid, uint32_t flags, BackwardArgs* a) {
  std::memset(a, 0, sizeof *a);
  a->pyr = m->pyr;
  a->shape = m->shape;
  a->q = QueryPtrs{q->u, q->v, q->lod, q->wix, q->wiy, q->wiz, q->wox, q->woy, q->woz, q->xi};
  a->n = n;
  a->pyramid = m->pyramid;
  a->params = m->params;
  a->grad_rgb = grad_rgb;
  a->grad_params = grad_params;
  a->grad_pyramid = grad_pyramid;
  a->flags = flags;
  a->num_sms = ctx->num_sms;
}

extern "C" nam_status nam_backward(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n,
                                   const float* grad_rgb, float* grad_params, float* grad_pyramid, void* stream,
                                   uint32_t flags) {
  nam_status st = check_trainable(ctx, m);
  if (st) return st;
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NAM_OK;
  if (!grad_rgb || !grad_params) return fail(NAM_ERR_INVALID_ARG, "NULL gradient buffer");
  if (((uintptr_t)grad_pyramid & 15u) != 0)
    return fail(NAM_ERR_INVALID_ARG, "grad_pyramid must be 16-byte aligned (it takes 16-byte vector atomics)");
  st = check_queries(m, q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  BackwardArgs a;
  fill_bwd(ctx, m, q, n, grad_rgb, grad_params, grad_pyramid, flags, &a);
  int e = launch_backward(a, stream);
  if (e) return cuda_fail(e, "nam_backward: launch");
  return NAM_OK;
}

extern "C" nam_status nam_train_step(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* target_rgb,
                                     int64_t n, const nam_adam* opt, float* loss_out, void* stream, uint32_t flags) {
  nam_status st = check_trainable(ctx, m);
  if (st) return st;
  if (n <= 0) return fail(NAM_ERR_INVALID_ARG, "n must be > 0");
  if (!target_rgb || !opt) return fail(NAM_ERR_INVALID_ARG, "NULL target or optimiser settings");
  if (opt->step < 1) return fail(NAM_ERR_INVALID_ARG, "Adam step is 1-based");
  st = check_queries(m, q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  // per-material scratch: the loss accumulator (the backward kernel runs the
  // forward and the loss itself)
  const size_t need = 256;
  if (need > m->train_scratch_bytes) {
    if (m->train_scratch) {
      cudaStreamSynchronize(s);
      cudaFree(m->train_scratch);
      budget_release(ctx, m->train_scratch_bytes);
      m->info.resident_bytes -= m->train_scratch_bytes;
      m->train_scratch = nullptr;
      m->train_scratch_bytes = 0;
    }
    if (!budget_reserve(ctx, need)) return fail(NAM_ERR_BUDGET, "training scratch needs %zu bytes", need);
    int e = dev_alloc(ctx, &m->train_scratch, need);
    if (e) {
      budget_release(ctx, need);
      return cuda_fail(e, "nam_train_step: scratch");
    }
    m->train_scratch_bytes = need;
    m->info.resident_bytes += need;
  }
  float* loss_acc = (float*)m->train_scratch;
  int e = (int)cudaMemsetAsync(loss_acc, 0, sizeof(float), s);
  BackwardArgs a;
  const int64_t np = m->n_params, po = m->pyr_off, nt = m->pyr.texels * 8;
  fill_bwd(ctx, m, q, n, nullptr, m->grad, m->grad + po, flags, &a);
  a.target = target_rgb;
  a.loss_acc = loss_acc;
  a.loss_inv = 1.0f / (float)(3 * n);
  if (!e) e = launch_backward(a, s);
  if (!e)
    e = launch_adam(m->params, m->grad, m->adam_m, m->adam_v, np, opt->lr_params, opt->beta1, opt->beta2, opt->eps,
                    opt->step, s);
  if (!e)
    e = launch_adam((float*)m->pyramid, m->grad + po, m->adam_m + po, m->adam_v + po, nt, opt->lr_pyramid,
                    opt->beta1, opt->beta2, opt->eps, opt->step, s);
  if (e) return cuda_fail(e, "nam_train_step: launch");
  if (loss_out) {
    cudaError_t ce = cudaMemcpyAsync(loss_out, loss_acc, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_train_step: loss readback");
  }
  return NAM_OK;
}
