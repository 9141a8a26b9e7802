// C ABI: reverse mode and the training step (Sec. 5.2).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
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

// A per-material device buffer of at least `need` bytes (re-allocated when a
// batch outgrows it; the stream is synchronised before the old one is freed).
static nam_status grow_scratch(nam_ctx* ctx, nam_material m, void** buf, size_t* bytes, size_t need, cudaStream_t s,
                               const char* who) {
  if (need <= *bytes) return NAM_OK;
  if (*buf) {
    cudaStreamSynchronize(s);
    cudaFree(*buf);
    budget_release(ctx, *bytes);
    m->info.resident_bytes -= *bytes;
    *buf = nullptr;
    *bytes = 0;
  }
  if (!budget_reserve(ctx, need)) return fail(NAM_ERR_BUDGET, "%s: scratch needs %zu bytes", who, need);
  int e = dev_alloc(ctx, buf, need);
  if (e) {
    budget_release(ctx, need);
    char what[96];
    std::snprintf(what, sizeof what, "%s: scratch", who);
    return cuda_fail(e, what);
  }
  *bytes = need;
  m->info.resident_bytes += need;
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

// The fused training step; target_albedo (albedo head only) [n][3].
static nam_status train_step(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* target_rgb,
                             const float* target_albedo, int64_t n, const nam_adam* opt, float* loss_out,
                             void* stream, uint32_t flags) {
  nam_status st = check_trainable(ctx, m);
  if (st) return st;
  if (n <= 0) return fail(NAM_ERR_INVALID_ARG, "n must be > 0");
  if (!target_rgb || !opt) return fail(NAM_ERR_INVALID_ARG, "NULL target or optimiser settings");
  if (m->shape.out == 6 && !target_albedo)
    return fail(NAM_ERR_UNSUPPORTED, "the material has the albedo head: nam_train_step_albedo trains it");
  if (m->shape.out == 3 && target_albedo) return fail(NAM_ERR_UNSUPPORTED, "the material has no albedo head");
  if (opt->step < 1) return fail(NAM_ERR_INVALID_ARG, "Adam step is 1-based");
  st = check_queries(m, q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  // per-material scratch: the loss accumulator (the backward kernel runs the
  // forward and the loss itself)
  st = grow_scratch(ctx, m, &m->train_scratch, &m->train_scratch_bytes, 256, s, "nam_train_step");
  if (st) return st;
  float* loss_acc = (float*)m->train_scratch;
  int e = (int)cudaMemsetAsync(loss_acc, 0, sizeof(float), s);
  BackwardArgs a;
  const int64_t np = m->n_params, po = m->pyr_off, nt = m->pyr.texels * 8;
  fill_bwd(ctx, m, q, n, nullptr, m->grad, m->grad + po, flags, &a);
  a.target = target_rgb;
  a.target_albedo = target_albedo;
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

extern "C" nam_status nam_train_step(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* target_rgb,
                                     int64_t n, const nam_adam* opt, float* loss_out, void* stream, uint32_t flags) {
  return train_step(ctx, m, q, target_rgb, nullptr, n, opt, loss_out, stream, flags);
}

extern "C" nam_status nam_train_step_albedo(nam_ctx* ctx, nam_material m, const nam_queries* q,
                                            const float* target_rgb, const float* target_albedo, int64_t n,
                                            const nam_adam* opt, float* loss_out, void* stream, uint32_t flags) {
  if (!target_albedo) return fail(NAM_ERR_INVALID_ARG, "nam_train_step_albedo: NULL albedo targets");
  return train_step(ctx, m, q, target_rgb, target_albedo, n, opt, loss_out, stream, flags);
}

// ---------------------------------------------------------------------------
// encoder phase of training (Sec. 5.1)
// ---------------------------------------------------------------------------
static nam_status check_encoder(nam_ctx* ctx, nam_material m, const char* who) {
  nam_status st = check_trainable(ctx, m);
  if (st) return st;
  if (!m->enc) return fail(NAM_ERR_UNSUPPORTED, "%s: the material has no encoder", who);
  return NAM_OK;
}

// wi and wo are read; u, v, lod and xi are not (the latent comes from the encoder)
static nam_status check_directions(const nam_queries* q) {
  if (!q || !q->wix || !q->wiy || !q->wiz || !q->wox || !q->woy || !q->woz)
    return fail(NAM_ERR_INVALID_ARG, "queries need wi and wo");
  return NAM_OK;
}

// latents [n][8] then their gradients [n][8], 256-byte aligned
static nam_status encoder_scratch(nam_ctx* ctx, nam_material m, int64_t n, cudaStream_t s, float** z, float** dz,
                                  const char* who) {
  const size_t half = ((size_t)n * 32 + 255) / 256 * 256;
  nam_status st = grow_scratch(ctx, m, &m->enc_scratch, &m->enc_scratch_bytes, 2 * half, s, who);
  if (st) return st;
  *z = (float*)m->enc_scratch;
  *dz = (float*)((char*)m->enc_scratch + half);
  return NAM_OK;
}

extern "C" nam_status nam_encode(nam_ctx* ctx, nam_material m, const float* attrs, int64_t n, float* z_out,
                                 void* stream) {
  nam_status st = check_encoder(ctx, m, "nam_encode");
  if (st) return st;
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NAM_OK;
  if (!attrs || !z_out) return fail(NAM_ERR_INVALID_ARG, "NULL attributes or output");
  if (((uintptr_t)z_out & 15u) != 0) return fail(NAM_ERR_INVALID_ARG, "z_out must be 16-byte aligned");
  DeviceGuard g(ctx->device);
  int e = launch_encode(m->enc, m->enc_in, attrs, n, z_out, ctx->num_sms, stream);
  if (e) return cuda_fail(e, "nam_encode: launch");
  return NAM_OK;
}

extern "C" nam_status nam_encoder_bake(nam_ctx* ctx, nam_material m, const float* texel_attrs, void* stream) {
  nam_status st = check_encoder(ctx, m, "nam_encoder_bake");
  if (st) return st;
  if (!texel_attrs) return fail(NAM_ERR_INVALID_ARG, "NULL texel attributes");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t texels = m->pyr.texels, po = m->pyr_off;
  int e = launch_encode(m->enc, m->enc_in, texel_attrs, texels, (float*)m->pyramid, ctx->num_sms, s);
  // finetuning starts afresh: the pyramid's Adam moments and gradient
  if (!e) e = (int)cudaMemsetAsync(m->adam_m + po, 0, (size_t)texels * 32, s);
  if (!e) e = (int)cudaMemsetAsync(m->adam_v + po, 0, (size_t)texels * 32, s);
  if (!e) e = (int)cudaMemsetAsync(m->grad + po, 0, (size_t)texels * 32, s);
  if (e) return cuda_fail(e, "nam_encoder_bake: launch");
  return NAM_OK;
}

extern "C" nam_status nam_backward_encoded(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* attrs,
                                           int64_t n, const float* grad_rgb, float* grad_params, float* grad_encoder,
                                           void* stream, uint32_t flags) {
  nam_status st = check_encoder(ctx, m, "nam_backward_encoded");
  if (st) return st;
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NAM_OK;
  if (!attrs || !grad_rgb || !grad_params || !grad_encoder)
    return fail(NAM_ERR_INVALID_ARG, "NULL attributes or gradient buffer");
  st = check_directions(q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  float *z, *dz;
  st = encoder_scratch(ctx, m, n, s, &z, &dz, "nam_backward_encoded");
  if (st) return st;
  int e = launch_encode(m->enc, m->enc_in, attrs, n, z, ctx->num_sms, s);
  BackwardArgs a;
  fill_bwd(ctx, m, q, n, grad_rgb, grad_params, nullptr, flags, &a);
  a.z_in = z;
  a.dz_out = dz;
  if (!e) e = launch_backward(a, s);
  if (!e) e = launch_encoder_backward(m->enc, m->enc_in, attrs, dz, n, grad_encoder, ctx->num_sms, s);
  if (e) return cuda_fail(e, "nam_backward_encoded: launch");
  return NAM_OK;
}

extern "C" nam_status nam_train_step_encoded(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* attrs,
                                             const float* target_rgb, int64_t n, const nam_adam* opt,
                                             float* loss_out, void* stream, uint32_t flags) {
  nam_status st = check_encoder(ctx, m, "nam_train_step_encoded");
  if (st) return st;
  if (n <= 0) return fail(NAM_ERR_INVALID_ARG, "n must be > 0");
  if (!attrs || !target_rgb || !opt) return fail(NAM_ERR_INVALID_ARG, "NULL attributes, target or optimiser settings");
  if (opt->step < 1) return fail(NAM_ERR_INVALID_ARG, "Adam step is 1-based");
  st = check_directions(q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  st = grow_scratch(ctx, m, &m->train_scratch, &m->train_scratch_bytes, 256, s, "nam_train_step_encoded");
  if (st) return st;
  float *z, *dz;
  st = encoder_scratch(ctx, m, n, s, &z, &dz, "nam_train_step_encoded");
  if (st) return st;
  float* loss_acc = (float*)m->train_scratch;
  const int64_t en = m->enc_n;
  float* enc_grad = m->enc + en;
  int e = (int)cudaMemsetAsync(loss_acc, 0, sizeof(float), s);
  if (!e) e = launch_encode(m->enc, m->enc_in, attrs, n, z, ctx->num_sms, s);
  BackwardArgs a;
  fill_bwd(ctx, m, q, n, nullptr, m->grad, nullptr, flags, &a);
  a.target = target_rgb;
  a.loss_acc = loss_acc;
  a.loss_inv = 1.0f / (float)(3 * n);
  a.z_in = z;
  a.dz_out = dz;
  if (!e) e = launch_backward(a, s);
  if (!e) e = launch_encoder_backward(m->enc, m->enc_in, attrs, dz, n, enc_grad, ctx->num_sms, s);
  if (!e)
    e = launch_adam(m->params, m->grad, m->adam_m, m->adam_v, m->n_params, opt->lr_params, opt->beta1, opt->beta2,
                    opt->eps, opt->step, s);
  if (!e)
    e = launch_adam(m->enc, enc_grad, m->enc + 2 * en, m->enc + 3 * en, en, opt->lr_params, opt->beta1, opt->beta2,
                    opt->eps, opt->step, s);
  if (e) return cuda_fail(e, "nam_train_step_encoded: launch");
  if (loss_out) {
    cudaError_t ce = cudaMemcpyAsync(loss_out, loss_acc, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_train_step_encoded: loss readback");
  }
  return NAM_OK;
}

extern "C" nam_status nam_material_encoder(nam_ctx* ctx, nam_material m, float** encoder_dev) {
  nam_status st = check_encoder(ctx, m, "nam_material_encoder");
  if (st) return st;
  if (encoder_dev) *encoder_dev = m->enc;
  return NAM_OK;
}
