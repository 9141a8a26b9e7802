// C ABI of libnam: contexts, materials, evaluation entry points.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "nam_internal.h"
#include "nam_ctx.h"

namespace nam {
}

using namespace nam;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

nam_status nam::fail(nam_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

nam_status nam::cuda_fail(int e, const char* what) {
  return fail(e == (int)cudaErrorMemoryAllocation ? NAM_ERR_OOM : NAM_ERR_CUDA, "%s: %s (%d)", what,
              cudaGetErrorString((cudaError_t)e), e);
}

extern "C" const char* nam_status_string(nam_status s) {
  switch (s) {
    case NAM_OK: return "ok";
    case NAM_ERR_INVALID_ARG: return "invalid argument";
    case NAM_ERR_OOM: return "out of memory";
    case NAM_ERR_BUDGET: return "HBM budget exceeded";
    case NAM_ERR_NOT_FOUND: return "not found";
    case NAM_ERR_BUSY: return "busy";
    case NAM_ERR_TIMEOUT: return "timeout";
    case NAM_ERR_CUDA: return "CUDA error";
    case NAM_ERR_DEVICE_ASSERT: return "device-side check failed";
    case NAM_ERR_UNSUPPORTED: return "unsupported";
    case NAM_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

extern "C" const char* nam_last_error_message(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// device guard
// ---------------------------------------------------------------------------
nam::DeviceGuard::DeviceGuard(int dev) {
  cudaGetDevice(&prev_);
  if (prev_ != dev) cudaSetDevice(dev);
  dev_ = dev;
}
nam::DeviceGuard::~DeviceGuard() {
  if (prev_ != dev_) cudaSetDevice(prev_);
}

// Device allocation that honours the fault-injection hook.
int nam::dev_alloc(nam_ctx* ctx, void** p, size_t bytes) {
  if (ctx->fault_alloc.exchange(false)) {
    *p = nullptr;
    return (int)cudaErrorMemoryAllocation;
  }
  return (int)cudaMalloc(p, bytes ? bytes : 16);
}

bool nam::budget_reserve(nam_ctx* ctx, uint64_t bytes) {
  uint64_t cur = ctx->resident.load();
  for (;;) {
    if (ctx->budget && cur + bytes > ctx->budget) return false;
    if (ctx->resident.compare_exchange_weak(cur, cur + bytes)) return true;
  }
}
void nam::budget_release(nam_ctx* ctx, uint64_t bytes) { ctx->resident.fetch_sub(bytes); }

int nam::blocks_per_sm(const void* func, int threads, int dyn_smem, int cap, bool resources_only) {
  int o = 0;
  cudaError_t e = cudaSuccess;
  if (!resources_only) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, func, threads, dyn_smem);
  cudaFuncAttributes a{};
  cudaError_t ea = cudaFuncGetAttributes(&a, func);
  if (resources_only || e != cudaSuccess || o < 1) {
    cudaGetLastError();
    int regs = ea == cudaSuccess ? a.numRegs : 64;
    int smem = dyn_smem + (ea == cudaSuccess ? (int)a.sharedSizeBytes : 0) + 1024;
    int by_smem = (227 * 1024) / (smem > 0 ? smem : 1);
    int by_regs = 65536 / (((regs + 7) / 8 * 8) * threads);
    int by_thr = 2048 / threads;
    o = std::min(std::min(by_smem, by_regs), std::min(by_thr, 32));
  }
  if (o > cap) o = cap;
  if (o < 1) o = 1;
  if (getenv("NAM_VERBOSE"))
    fprintf(stderr, "[nam] occupancy: api=%d (%s) regs=%d static_smem=%zu dyn_smem=%d -> %d blocks/SM\n", o,
            cudaGetErrorString(e), ea == cudaSuccess ? a.numRegs : -1, ea == cudaSuccess ? a.sharedSizeBytes : 0,
            dyn_smem, o);
  return o;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" nam_status nam_init(nam_ctx** out, const nam_config* cfg) {
  if (!out) return fail(NAM_ERR_INVALID_ARG, "nam_init: out is NULL");
  *out = nullptr;
  nam_config c{};
  if (cfg) c = *cfg;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail((int)e, "nam_init: cudaGetDeviceCount");
  if (c.device < 0 || c.device >= ndev) return fail(NAM_ERR_INVALID_ARG, "nam_init: device %d of %d", c.device, ndev);
  DeviceGuard g(c.device);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, c.device);
  if (e != cudaSuccess) return cuda_fail((int)e, "nam_init: cudaGetDeviceProperties");
  if (prop.major < 10) return fail(NAM_ERR_UNSUPPORTED, "nam_init: device %s is sm_%d%d, libnam needs sm_103a", prop.name, prop.major, prop.minor);
  nam_ctx* ctx = new nam_ctx();
  ctx->device = c.device;
  ctx->num_sms = prop.multiProcessorCount;
  int pageable = 0;
  if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, c.device) != cudaSuccess) pageable = 0;
  ctx->host_direct = pageable == 1;
  ctx->budget = c.hbm_budget_bytes;
  ctx->timeout_ns = c.wait_timeout_ns ? c.wait_timeout_ns : 2000000000ull;
  ctx->serve_streams = c.serve_streams > 0 ? c.serve_streams : 4;
  ctx->serve_queue_depth = c.serve_queue_depth > 0 ? c.serve_queue_depth : 256;
  e = cudaMalloc(&ctx->err_word, sizeof(int));
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail((int)e, "nam_init: error word");
  }
  cudaMemset(ctx->err_word, 0, sizeof(int));
  cudaMemPoolProps pp{};
  pp.allocType = cudaMemAllocationTypePinned;
  pp.location.type = cudaMemLocationTypeDevice;
  pp.location.id = c.device;
  e = cudaMemPoolCreate(&ctx->pool, &pp);
  if (e != cudaSuccess) {
    cudaFree(ctx->err_word);
    delete ctx;
    return cuda_fail((int)e, "nam_init: memory pool");
  }
  uint64_t keep = UINT64_MAX;
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  cudaDeviceSynchronize();
  *out = ctx;
  return NAM_OK;
}

static void free_material(nam_ctx* ctx, nam_material m) {
  DeviceGuard g(ctx->device);
  cudaFree(m->pyramid);
  cudaFree(m->blob);
  cudaFree(m->params);
  cudaFree(m->sampler);
  cudaFree(m->adam_m);
  cudaFree(m->adam_v);
  cudaFree(m->grad);
  cudaFree(m->train_scratch);
  cudaFree(m->enc);
  cudaFree(m->enc_scratch);
  budget_release(ctx, m->info.resident_bytes);
  delete m;
}

extern "C" nam_status nam_shutdown(nam_ctx* ctx) {
  if (!ctx) return fail(NAM_ERR_INVALID_ARG, "nam_shutdown: NULL context");
  serve_stop(ctx);
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (nam_material m : ctx->materials) free_material(ctx, m);
  ctx->materials.clear();
  cudaFree(ctx->err_word);
  cudaFree(ctx->stage_dev);
  if (ctx->stage_stream) cudaStreamDestroy((cudaStream_t)ctx->stage_stream);
  if (ctx->h2d_stream) cudaStreamDestroy((cudaStream_t)ctx->h2d_stream);
  if (ctx->d2h_stream) cudaStreamDestroy((cudaStream_t)ctx->d2h_stream);
  for (void* ev : ctx->stage_events) cudaEventDestroy((cudaEvent_t)ev);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
  return NAM_OK;
}

extern "C" nam_status nam_check_device_error(nam_ctx* ctx) {
  if (!ctx) return fail(NAM_ERR_INVALID_ARG, "NULL context");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail((int)e, "nam_check_device_error");
  int code = 0;
  cudaMemcpy(&code, ctx->err_word, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemset(ctx->err_word, 0, sizeof(int));
  if (code == DEVERR_WAIT_TIMEOUT) return fail(NAM_ERR_TIMEOUT, "a device-side wait ran past its limit");
  if (code == DEVERR_DRAIN_TIMEOUT)
    return fail(NAM_ERR_TIMEOUT, "a kernel's own MMAs or copies did not complete within the drain limit");
  if (code) return fail(NAM_ERR_DEVICE_ASSERT, "device-side check failed (code %d)", code);
  return NAM_OK;
}

// ---------------------------------------------------------------------------
// materials
// ---------------------------------------------------------------------------
static bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

nam_status nam::validate_desc(const nam_material_desc* d, Shape* shape, PyrDesc* pyr) {
  if (!d) return fail(NAM_ERR_INVALID_ARG, "descriptor is NULL");
  if (d->channels != 8) return fail(NAM_ERR_INVALID_ARG, "channels must be 8 (got %d)", d->channels);
  if (d->base_w < 1 || d->base_h < 1 || d->base_w > (1 << 20) || d->base_h > (1 << 20))
    return fail(NAM_ERR_INVALID_ARG, "bad base size %dx%d", d->base_w, d->base_h);
  int maxl = 1;
  while ((std::max(d->base_w, d->base_h) >> maxl) > 0) ++maxl;
  if (d->levels < 1 || d->levels > NAM_MAX_LEVELS || d->levels > maxl)
    return fail(NAM_ERR_INVALID_ARG, "levels %d not in [1, %d]", d->levels, std::min(maxl, NAM_MAX_LEVELS));
  if (d->latent_dtype != NAM_LATENT_F32 && d->latent_dtype != NAM_LATENT_F16)
    return fail(NAM_ERR_INVALID_ARG, "bad latent dtype %d", d->latent_dtype);
  if (!d->pyramid) return fail(NAM_ERR_INVALID_ARG, "pyramid is NULL");
  if (d->frame_form != NAM_FRAME_MLP && d->frame_form != NAM_FRAME_PAPER)
    return fail(NAM_ERR_INVALID_ARG, "bad frame_form %d", d->frame_form);
  const bool paper = d->frame_form == NAM_FRAME_PAPER;
  if (d->frame_hidden != 0 && (d->frame_hidden != 16 || paper))
    return fail(NAM_ERR_UNSUPPORTED, "frame_hidden must be 0 or 16 (0 with the paper's frame form), got %d",
                d->frame_hidden);
  if ((d->frame_hidden || paper) && !d->frame_weights) return fail(NAM_ERR_INVALID_ARG, "frame weights are NULL");
  if (!d->decoder_weights) return fail(NAM_ERR_INVALID_ARG, "decoder weights are NULL");
  if (d->n_layers != 3 && d->n_layers != 4)
    return fail(NAM_ERR_UNSUPPORTED, "n_layers must be 3 or 4: two or three hidden layers (got %d)", d->n_layers);
  const int H = d->widths[1];
  const int in = paper ? 20 : 14;
  const int n_out = d->widths[d->n_layers];
  if (d->widths[0] != in || (n_out != 3 && n_out != 6))
    return fail(NAM_ERR_UNSUPPORTED, "decoder must map %d inputs to 3 outputs (6 with the albedo head)", in);
  for (int l = 1; l < d->n_layers; ++l)
    if (d->widths[l] != H) return fail(NAM_ERR_UNSUPPORTED, "hidden widths must be equal");
  if (H != 16 && H != 32 && H != 64) return fail(NAM_ERR_UNSUPPORTED, "hidden width %d not in {16, 32, 64}", H);
  if (d->n_layers == 4 && H != 64) return fail(NAM_ERR_UNSUPPORTED, "three hidden layers need H = 64");
  if (d->trainable && (paper || d->n_layers != 3))
    return fail(NAM_ERR_UNSUPPORTED, "training needs the frame MLP form and two hidden layers");
  if (d->precision < NAM_PREC_F32 || d->precision > NAM_PREC_FP8)
    return fail(NAM_ERR_INVALID_ARG, "bad precision %d", d->precision);
  if (d->filter != NAM_FILTER_TRILINEAR && d->filter != NAM_FILTER_STOCHASTIC)
    return fail(NAM_ERR_INVALID_ARG, "bad filter %d", d->filter);
  if (d->address != NAM_ADDRESS_WRAP && d->address != NAM_ADDRESS_CLAMP)
    return fail(NAM_ERR_INVALID_ARG, "bad address mode %d", d->address);
  if (d->trainable && (d->precision != NAM_PREC_F32 || d->latent_dtype != NAM_LATENT_F32))
    return fail(NAM_ERR_UNSUPPORTED, "trainable materials need F32 precision and F32 latents");
  if (d->precision == NAM_PREC_FP8) {
    if (!d->fp8_act_scale) return fail(NAM_ERR_INVALID_ARG, "FP8 needs fp8_act_scale");
    for (int l = 0; l < d->n_layers; ++l)
      if (!(d->fp8_act_scale[l] > 0.0f) || !std::isfinite(d->fp8_act_scale[l]))
        return fail(NAM_ERR_INVALID_ARG, "fp8_act_scale[%d] must be finite and > 0", l);
  }
  if (d->sampler_hidden != 0 && d->sampler_hidden != 32)
    return fail(NAM_ERR_UNSUPPORTED, "sampler_hidden must be 0 or 32");
  if (d->sampler_hidden && !d->sampler_weights) return fail(NAM_ERR_INVALID_ARG, "sampler_weights is NULL");
  if (d->encoder_inputs < 0 || d->encoder_inputs > NAM_ENCODER_MAX_INPUTS)
    return fail(NAM_ERR_INVALID_ARG, "encoder_inputs %d not in [0, %d]", d->encoder_inputs, NAM_ENCODER_MAX_INPUTS);
  if (d->encoder_inputs && !d->trainable)
    return fail(NAM_ERR_UNSUPPORTED, "an encoder needs a trainable material (it exists only for training)");
  if (d->encoder_inputs && !d->encoder_weights) return fail(NAM_ERR_INVALID_ARG, "encoder_weights is NULL");
  if (d->encoder_inputs && n_out != 3)
    return fail(NAM_ERR_UNSUPPORTED, "the encoder phase trains the RGB decoder only (no albedo head)");
  shape->H = H;
  shape->NH = d->n_layers - 1;
  shape->frame = paper ? 2 : (d->frame_hidden ? 1 : 0);
  shape->in = in;
  shape->out = n_out;
  std::memset(pyr, 0, sizeof *pyr);
  pyr->levels = d->levels;
  pyr->f16 = d->latent_dtype == NAM_LATENT_F16;
  pyr->filter = d->filter;
  pyr->address = d->address;
  pyr->pow2 = 1;
  int64_t off = 0;
  for (int l = 0; l < d->levels; ++l) {
    int w = std::max(1, d->base_w >> l), h = std::max(1, d->base_h >> l);
    pyr->w[l] = w;
    pyr->h[l] = h;
    pyr->off[l] = off;
    if (!is_pow2(w) || !is_pow2(h)) pyr->pow2 = 0;
    off += (int64_t)w * h;
  }
  pyr->texels = off;
  return NAM_OK;
}

extern "C" nam_status nam_create_material(nam_ctx* ctx, const nam_material_desc* d, nam_material* out) {
  if (!ctx || !out) return fail(NAM_ERR_INVALID_ARG, "nam_create_material: NULL argument");
  *out = nullptr;
  Shape sh;
  PyrDesc pd;
  nam_status st = validate_desc(d, &sh, &pd);
  if (st) return st;
  DeviceGuard g(ctx->device);
  const size_t texel_bytes = pd.f16 ? 16 : 32;
  const size_t pyr_bytes = (size_t)pd.texels * texel_bytes;
  const int64_t np = n_params_of(sh);
  // host copies of the FP32 masters (the descriptor may point to device memory)
  const int64_t nframe = frame_params_of(sh.frame);
  std::vector<float> master((size_t)np);
  cudaMemcpyKind kind = d->params_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  if (nframe) cudaMemcpy(master.data(), d->frame_weights, nframe * 4, kind);
  cudaMemcpy(master.data() + nframe, d->decoder_weights, (np - nframe) * 4, kind);
  for (float v : master)
    if (!std::isfinite(v)) return fail(NAM_ERR_INVALID_ARG, "non-finite weight");
  std::vector<float> encw;
  if (d->encoder_inputs) {
    encw.resize((size_t)encoder_params_of(d->encoder_inputs));
    cudaMemcpy(encw.data(), d->encoder_weights, encw.size() * 4, kind);
    for (float v : encw)
      if (!std::isfinite(v)) return fail(NAM_ERR_INVALID_ARG, "non-finite encoder weight");
  }
  std::vector<uint8_t> smp;
  if (d->sampler_hidden) {
    std::vector<float> w(kSamplerFloats);
    cudaMemcpy(w.data(), d->sampler_weights, kSamplerFloats * 4, kind);
    for (float v : w)
      if (!std::isfinite(v)) return fail(NAM_ERR_INVALID_ARG, "non-finite sampler weight");
    smp.resize(sampler_blob_bytes());
    if (pack_sampler_blob(w.data(), smp.data()) != 0)
      return fail(NAM_ERR_UNSUPPORTED, "sampler weight of magnitude >= 32768");
  }

  nam_material m = new nam_material_s();
  m->desc = *d;
  m->shape = sh;
  m->pyr = pd;
  m->n_params = np;
  size_t blob_bytes = 0;
  if (d->precision == NAM_PREC_F32) {
    blob_bytes = 0;  // the FP32 kernels read the master layout directly
  } else {
    blob_bytes = tc_blob_bytes(sh, d->precision);
    if (!blob_bytes) {
      delete m;
      return fail(NAM_ERR_UNSUPPORTED, "no tensor-core kernel for this shape/precision");
    }
  }
  uint64_t resident = pyr_bytes + blob_bytes + (uint64_t)np * 4 + (uint64_t)smp.size() +
                      4ull * encw.size() * 4;
  m->enc_in = d->encoder_inputs;
  m->enc_n = (int64_t)encw.size();
  m->pyr_off = (np + 3) / 4 * 4;
  if (d->trainable) {
    // FP32 pyramid masters are the pyramid itself; Adam moments and gradients
    // for params and pyramid
    resident += 3ull * (m->pyr_off + pd.texels * 8) * 4;
  }
  if (!budget_reserve(ctx, resident)) {
    delete m;
    return fail(NAM_ERR_BUDGET, "material needs %llu bytes; %llu of %llu in use", (unsigned long long)resident,
                (unsigned long long)ctx->resident.load(), (unsigned long long)ctx->budget);
  }
  m->info.resident_bytes = resident;
  int e = dev_alloc(ctx, &m->pyramid, pyr_bytes);
  if (!e) e = dev_alloc(ctx, (void**)&m->params, np * 4);
  if (!e && blob_bytes) e = dev_alloc(ctx, &m->blob, blob_bytes);
  if (!e && !smp.empty()) e = dev_alloc(ctx, &m->sampler, smp.size());
  if (!e && !encw.empty()) e = dev_alloc(ctx, (void**)&m->enc, 4 * encw.size() * 4);
  if (!e && d->trainable) {
    const size_t nb = (m->pyr_off + pd.texels * 8) * 4;
    e = dev_alloc(ctx, (void**)&m->adam_m, nb);
    if (!e) e = dev_alloc(ctx, (void**)&m->adam_v, nb);
    if (!e) e = dev_alloc(ctx, (void**)&m->grad, nb);
  }
  if (e) {
    free_material(ctx, m);
    return cuda_fail(e, "nam_create_material: allocation");
  }
  e = (int)cudaMemcpy(m->pyramid, d->pyramid, pyr_bytes,
                      d->params_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  if (!e) e = (int)cudaMemcpy(m->params, master.data(), np * 4, cudaMemcpyHostToDevice);
  if (!e && !smp.empty()) e = (int)cudaMemcpy(m->sampler, smp.data(), smp.size(), cudaMemcpyHostToDevice);
  if (!e && !encw.empty()) {
    e = (int)cudaMemcpy(m->enc, encw.data(), encw.size() * 4, cudaMemcpyHostToDevice);
    if (!e) e = (int)cudaMemset(m->enc + encw.size(), 0, 3 * encw.size() * 4);  // gradient, Adam m, v
  }
  if (!e && blob_bytes) {
    std::vector<uint8_t> blob(blob_bytes);
    if (pack_tc_blob(sh, d->precision, nframe ? master.data() : nullptr, master.data() + nframe,
                     d->fp8_act_scale, blob.data(), m->info.fp8_weight_scale) != 0) {
      free_material(ctx, m);
      return fail(NAM_ERR_UNSUPPORTED, "weight packing failed");
    }
    e = (int)cudaMemcpy(m->blob, blob.data(), blob_bytes, cudaMemcpyHostToDevice);
  }
  if (!e && d->trainable) {
    size_t nb = (m->pyr_off + pd.texels * 8) * 4;
    cudaMemset(m->adam_m, 0, nb);
    cudaMemset(m->adam_v, 0, nb);
    e = (int)cudaMemset(m->grad, 0, nb);
  }
  if (e) {
    free_material(ctx, m);
    return cuda_fail(e, "nam_create_material: upload");
  }
  m->info.texels = pd.texels;
  m->info.n_params = np;
  m->info.precision = d->precision;
  m->info.filter = d->filter;
  m->info.address = d->address;
  m->info.levels = d->levels;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->materials.insert(m);
  }
  *out = m;
  return NAM_OK;
}

static bool owns(nam_ctx* ctx, nam_material m) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  return ctx->materials.count(m) != 0;
}

extern "C" nam_status nam_destroy_material(nam_ctx* ctx, nam_material m) {
  if (!ctx || !m) return fail(NAM_ERR_INVALID_ARG, "NULL argument");
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->materials.count(m)) return fail(NAM_ERR_NOT_FOUND, "unknown material");
    ctx->materials.erase(m);
  }
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  free_material(ctx, m);
  return NAM_OK;
}

extern "C" nam_status nam_material_get_info(nam_ctx* ctx, nam_material m, nam_material_info* out) {
  if (!ctx || !m || !out) return fail(NAM_ERR_INVALID_ARG, "NULL argument");
  if (!owns(ctx, m)) return fail(NAM_ERR_NOT_FOUND, "unknown material");
  *out = m->info;
  return NAM_OK;
}

extern "C" nam_status nam_material_params(nam_ctx* ctx, nam_material m, float** params_dev, float** pyramid_dev) {
  if (!ctx || !m) return fail(NAM_ERR_INVALID_ARG, "NULL argument");
  if (!owns(ctx, m)) return fail(NAM_ERR_NOT_FOUND, "unknown material");
  if (!m->desc.trainable) return fail(NAM_ERR_UNSUPPORTED, "material is not trainable");
  if (params_dev) *params_dev = m->params;
  if (pyramid_dev) *pyramid_dev = (float*)m->pyramid;
  return NAM_OK;
}

// ---------------------------------------------------------------------------
// evaluation
// ---------------------------------------------------------------------------
nam_status nam::check_queries(const nam_material_s* m, const nam_queries* q) {
  if (!q || !q->u || !q->v || !q->lod || !q->wix || !q->wiy || !q->wiz || !q->wox || !q->woy || !q->woz)
    return fail(NAM_ERR_INVALID_ARG, "query arrays must not be NULL");
  if (m->desc.filter == NAM_FILTER_STOCHASTIC && !q->xi)
    return fail(NAM_ERR_INVALID_ARG, "stochastic filtering needs xi");
  return NAM_OK;
}

void nam::fill_launch(nam_ctx* ctx, const nam_material_s* m, const nam_queries* q, int64_t n, float* rgb,
                      uint32_t flags, LaunchCommon* L) {
  std::memset(L, 0, sizeof *L);
  L->pyr = m->pyr;
  L->shape = m->shape;
  L->q = QueryPtrs{q->u, q->v, q->lod, q->wix, q->wiy, q->wiz, q->wox, q->woy, q->woz, q->xi};
  L->rgb = rgb;
  L->n = n;
  L->pyr0 = m->pyramid;
  L->w0 = m->desc.precision == NAM_PREC_F32 ? (const void*)m->params : m->blob;
  L->mats.nmat = 1;
  L->flags = flags;
  L->err = ctx->err_word;
  L->timeout_ns = ctx->timeout_ns;
  L->num_sms = ctx->num_sms;
}

int nam::launch_material(const LaunchCommon& L, int precision, void* stream) {
  if (precision == NAM_PREC_F32) return launch_eval_f32(L, stream);
  return launch_eval_tc(L, precision, stream);
}

extern "C" nam_status nam_eval(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n, float* rgb_out,
                               void* stream, uint32_t flags) {
  if (!ctx || !m) return fail(NAM_ERR_INVALID_ARG, "nam_eval: NULL context or material");
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "nam_eval: n < 0");
  if (n == 0) return NAM_OK;
  if (!rgb_out) return fail(NAM_ERR_INVALID_ARG, "nam_eval: rgb_out is NULL");
  if (!owns(ctx, m)) return fail(NAM_ERR_NOT_FOUND, "nam_eval: unknown material");
  nam_status st = check_queries(m, q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  LaunchCommon L;
  fill_launch(ctx, m, q, n, rgb_out, flags, &L);
  int e = launch_material(L, m->desc.precision, stream);
  if (e) return cuda_fail(e, "nam_eval: launch");
  return NAM_OK;
}

extern "C" nam_status nam_eval_albedo(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n,
                                      float* rgb_out, float* albedo_out, void* stream, uint32_t flags) {
  if (!ctx || !m) return fail(NAM_ERR_INVALID_ARG, "nam_eval_albedo: NULL context or material");
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "nam_eval_albedo: n < 0");
  if (!owns(ctx, m)) return fail(NAM_ERR_NOT_FOUND, "nam_eval_albedo: unknown material");
  if (m->shape.out != 6) return fail(NAM_ERR_UNSUPPORTED, "nam_eval_albedo: the material has no albedo head");
  if (n == 0) return NAM_OK;
  if (!rgb_out || !albedo_out) return fail(NAM_ERR_INVALID_ARG, "nam_eval_albedo: NULL output");
  nam_status st = check_queries(m, q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  LaunchCommon L;
  fill_launch(ctx, m, q, n, rgb_out, flags, &L);
  L.albedo = albedo_out;
  int e = launch_material(L, m->desc.precision, stream);
  if (e) return cuda_fail(e, "nam_eval_albedo: launch");
  return NAM_OK;
}

extern "C" nam_status nam_fp8_calibrate(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n,
                                        float* act_scale_out, void* stream) {
  if (!ctx || !m || !act_scale_out) return fail(NAM_ERR_INVALID_ARG, "nam_fp8_calibrate: NULL argument");
  if (n <= 0) return fail(NAM_ERR_INVALID_ARG, "nam_fp8_calibrate: n must be > 0");
  if (!owns(ctx, m)) return fail(NAM_ERR_NOT_FOUND, "nam_fp8_calibrate: unknown material");
  nam_status st = check_queries(m, q);
  if (st) return st;
  const int nl = m->desc.n_layers;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  float* amax = nullptr;
  cudaError_t ce = cudaMallocFromPoolAsync((void**)&amax, 4 * sizeof(float), ctx->pool, s);
  if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_fp8_calibrate: allocation");
  ce = cudaMemsetAsync(amax, 0, 4 * sizeof(float), s);
  LaunchCommon L;
  fill_launch(ctx, m, q, n, nullptr, 0, &L);
  L.w0 = m->params;  // FP32 masters, whatever the material's precision
  L.amax = amax;
  int e = ce == cudaSuccess ? launch_eval_f32(L, stream) : (int)ce;
  float h[4] = {0, 0, 0, 0};
  if (!e) e = (int)cudaMemcpyAsync(h, amax, sizeof h, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(amax, s);
  if (!e) e = (int)cudaStreamSynchronize(s);
  if (e) return cuda_fail(e, "nam_fp8_calibrate");
  for (int l = 0; l < nl; ++l) act_scale_out[l] = h[l] > 0.0f ? h[l] / 448.0f : 1.0f;
  return NAM_OK;
}

static nam_status sampler_call(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n, int mode,
                               const float* u, float* wo_out, float* pdf_out, void* stream, const char* who) {
  if (!ctx || !m || !q) return fail(NAM_ERR_INVALID_ARG, "%s: NULL argument", who);
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "%s: n < 0", who);
  if (!owns(ctx, m)) return fail(NAM_ERR_NOT_FOUND, "%s: unknown material", who);
  if (!m->sampler) return fail(NAM_ERR_UNSUPPORTED, "%s: the material has no importance sampler", who);
  if (n == 0) return NAM_OK;
  if (!q->u || !q->v || !q->lod || !q->wix || !q->wiy || !q->wiz)
    return fail(NAM_ERR_INVALID_ARG, "%s: NULL query array", who);
  if (m->desc.filter == NAM_FILTER_STOCHASTIC && !q->xi) return fail(NAM_ERR_INVALID_ARG, "%s: xi is NULL", who);
  if (mode == 0 && (!q->wox || !q->woy || !q->woz || !pdf_out))
    return fail(NAM_ERR_INVALID_ARG, "%s: NULL wo or output", who);
  if (mode == 1 && (!u || !wo_out)) return fail(NAM_ERR_INVALID_ARG, "%s: NULL variates or output", who);
  DeviceGuard g(ctx->device);
  LaunchCommon L;
  fill_launch(ctx, m, q, n, nullptr, 0, &L);
  int e = launch_sampler(L, m->sampler, mode, u, wo_out, pdf_out, stream);
  if (e) return cuda_fail(e, who);
  return NAM_OK;
}

extern "C" nam_status nam_sample(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n, const float* u,
                                 float* wo_out, float* pdf_out, void* stream) {
  return sampler_call(ctx, m, q, n, 1, u, wo_out, pdf_out, stream, "nam_sample");
}

extern "C" nam_status nam_sample_pdf(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n, float* pdf_out,
                                     void* stream) {
  return sampler_call(ctx, m, q, n, 0, nullptr, nullptr, pdf_out, stream, "nam_sample_pdf");
}

extern "C" nam_status nam_eval_host(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n, float* rgb_out,
                                    void* stream, uint32_t flags) {
  if (!ctx || !m) return fail(NAM_ERR_INVALID_ARG, "nam_eval_host: NULL context or material");
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "nam_eval_host: n < 0");
  if (n == 0) return NAM_OK;
  if (!rgb_out) return fail(NAM_ERR_INVALID_ARG, "nam_eval_host: rgb_out is NULL");
  if (!owns(ctx, m)) return fail(NAM_ERR_NOT_FOUND, "nam_eval_host: unknown material");
  nam_status st = check_queries(m, q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  if (ctx->host_direct && !(flags & NAM_HOST_STAGED)) {
    // the kernel reads the host queries and writes the host RGB itself
    LaunchCommon L;
    fill_launch(ctx, m, q, n, rgb_out, flags, &L);
    int e = launch_material(L, m->desc.precision, stream);
    if (e) return cuda_fail(e, "nam_eval_host: launch");
    cudaError_t ce = cudaStreamSynchronize((cudaStream_t)stream);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_eval_host: sync");
    return NAM_OK;
  }
  std::lock_guard<std::mutex> lk(ctx->stage_mu);
  const bool has_xi = m->desc.filter == NAM_FILTER_STOCHASTIC;
  const int nf = has_xi ? 10 : 9;
  const size_t need = (size_t)n * 4 * (nf + 3);
  if (need > ctx->stage_bytes) {
    if (ctx->stage_dev) {
      cudaFree(ctx->stage_dev);
      budget_release(ctx, ctx->stage_bytes);
      ctx->stage_dev = nullptr;
      ctx->stage_bytes = 0;
    }
    if (!budget_reserve(ctx, need)) return fail(NAM_ERR_BUDGET, "nam_eval_host: staging needs %zu bytes", need);
    int e = dev_alloc(ctx, &ctx->stage_dev, need);
    if (e) {
      budget_release(ctx, need);
      return cuda_fail(e, "nam_eval_host: staging allocation");
    }
    ctx->stage_bytes = need;
  }
  // Pipelined over (at most four) chunks: host->device copies on one stream,
  // kernels on the caller's stream, device->host copies on another, ordered
  // by events, so that chunk k+1 arrives while chunk k runs and chunk k-1
  // returns.  Chunks hold at least 2^19 queries (2 MB per field copy: smaller
  // copies lose bandwidth to per-copy overhead).  Every chunk has its own
  // region of the staging area, so nothing is overwritten while in use.
  const int64_t kHostChunk = std::max<int64_t>(1 << 19, ((n + 3) / 4 + 127) / 128 * 128);
  const int64_t nchunk = (n + kHostChunk - 1) / kHostChunk;
  cudaError_t ce = cudaSuccess;
  if (!ctx->h2d_stream) ce = cudaStreamCreateWithFlags((cudaStream_t*)&ctx->h2d_stream, cudaStreamNonBlocking);
  if (ce == cudaSuccess && !ctx->d2h_stream)
    ce = cudaStreamCreateWithFlags((cudaStream_t*)&ctx->d2h_stream, cudaStreamNonBlocking);
  while (ce == cudaSuccess && (int64_t)ctx->stage_events.size() < 2 * nchunk) {
    cudaEvent_t ev;
    ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (ce == cudaSuccess) ctx->stage_events.push_back((void*)ev);
  }
  if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_eval_host: streams");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStream_t sin = (cudaStream_t)ctx->h2d_stream, sout = (cudaStream_t)ctx->d2h_stream;
  float* base = (float*)ctx->stage_dev;
  const float* src[10] = {q->u, q->v, q->lod, q->wix, q->wiy, q->wiz, q->wox, q->woy, q->woz, q->xi};
  float* dst[10];
  for (int f = 0; f < nf; ++f) dst[f] = base + (size_t)f * n;
  float* rgb_dev = base + (size_t)nf * n;
  for (int64_t k = 0; k < nchunk; ++k) {
    const int64_t off = k * kHostChunk, cnt = std::min<int64_t>(kHostChunk, n - off);
    cudaEvent_t ev_in = (cudaEvent_t)ctx->stage_events[2 * k], ev_done = (cudaEvent_t)ctx->stage_events[2 * k + 1];
    for (int f = 0; f < nf && ce == cudaSuccess; ++f)
      ce = cudaMemcpyAsync(dst[f] + off, src[f] + off, (size_t)cnt * 4, cudaMemcpyHostToDevice, sin);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev_in, sin);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, ev_in, 0);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_eval_host: H2D");
    nam_queries dq{dst[0] + off, dst[1] + off, dst[2] + off, dst[3] + off, dst[4] + off, dst[5] + off,
                   dst[6] + off, dst[7] + off, dst[8] + off, has_xi ? dst[9] + off : nullptr};
    LaunchCommon L;
    fill_launch(ctx, m, &dq, cnt, rgb_dev + 3 * off, flags, &L);
    int e = launch_material(L, m->desc.precision, stream);
    if (e) return cuda_fail(e, "nam_eval_host: launch");
    ce = cudaEventRecord(ev_done, s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(sout, ev_done, 0);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(rgb_out + 3 * off, rgb_dev + 3 * off, (size_t)cnt * 12, cudaMemcpyDeviceToHost, sout);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_eval_host: D2H");
  }
  ce = cudaStreamSynchronize(sout);
  if (ce != cudaSuccess) return cuda_fail((int)ce, "nam_eval_host: sync");
  return NAM_OK;
}

// Chunk table of a multi-material launch: every item split into runs of at
// most 128 queries so that no tensor-core tile mixes materials.
void nam::build_chunks(const nam_work_item* items, int32_t n_items, std::vector<Chunk>* out) {
  out->clear();
  for (int32_t i = 0; i < n_items; ++i) {
    for (int32_t o = 0; o < items[i].count; o += 128) {
      Chunk c;
      c.start = items[i].start + o;
      c.count = std::min(128, items[i].count - o);
      c.material = items[i].material;
      out->push_back(c);
    }
  }
}

nam_status nam::check_multi(nam_ctx* ctx, const nam_material* mats, int32_t nmat) {
  if (!mats || nmat < 1) return fail(NAM_ERR_INVALID_ARG, "no materials");
  const nam_material m0 = mats[0];
  for (int32_t k = 0; k < nmat; ++k) {
    if (!mats[k] || !owns(ctx, mats[k])) return fail(NAM_ERR_NOT_FOUND, "unknown material %d", k);
    const nam_material m = mats[k];
    if (m->desc.precision == NAM_PREC_F32) return fail(NAM_ERR_UNSUPPORTED, "multi-material launches use the tensor-core path");
    if (m->desc.precision != m0->desc.precision || m->shape.H != m0->shape.H || m->shape.NH != m0->shape.NH ||
        m->shape.frame != m0->shape.frame || m->shape.in != m0->shape.in || m->shape.out != m0->shape.out)
      return fail(NAM_ERR_INVALID_ARG, "materials must share precision and MLP shape");
    if (std::memcmp(&m->pyr, &m0->pyr, sizeof(PyrDesc)) != 0)
      return fail(NAM_ERR_INVALID_ARG, "materials must share pyramid geometry, dtype, filter and addressing");
  }
  return NAM_OK;
}

extern "C" nam_status nam_eval_multi(nam_ctx* ctx, const nam_material* mats, int32_t nmat, const nam_queries* q,
                                     const nam_work_item* items, int32_t n_items, float* rgb_out, void* stream,
                                     uint32_t flags) {
  if (!ctx) return fail(NAM_ERR_INVALID_ARG, "nam_eval_multi: NULL context");
  if (n_items < 0) return fail(NAM_ERR_INVALID_ARG, "n_items < 0");
  if (n_items == 0) return NAM_OK;
  if (!items || !rgb_out) return fail(NAM_ERR_INVALID_ARG, "NULL items or output");
  nam_status st = check_multi(ctx, mats, nmat);
  if (st) return st;
  st = check_queries(mats[0], q);
  if (st) return st;
  for (int32_t i = 0; i < n_items; ++i)
    if (items[i].material < 0 || items[i].material >= nmat || items[i].count < 0 || items[i].start < 0)
      return fail(NAM_ERR_INVALID_ARG, "bad work item %d", i);
  std::vector<Chunk> chunks;
  build_chunks(items, n_items, &chunks);
  if (chunks.empty()) return NAM_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  // one stream-ordered allocation: chunk table, pyramid pointers, weight pointers
  const size_t cb = chunks.size() * sizeof(Chunk);
  const size_t pb = (size_t)nmat * sizeof(void*);
  std::vector<uint8_t> host(cb + 2 * pb);
  std::memcpy(host.data(), chunks.data(), cb);
  for (int32_t k = 0; k < nmat; ++k) {
    const void* p = mats[k]->pyramid;
    const void* w = mats[k]->blob;
    std::memcpy(host.data() + cb + k * sizeof(void*), &p, sizeof p);
    std::memcpy(host.data() + cb + pb + k * sizeof(void*), &w, sizeof w);
  }
  void* dev = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&dev, host.size(), ctx->pool, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "nam_eval_multi: table allocation");
  e = cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(dev, s);
    return cuda_fail((int)e, "nam_eval_multi: table upload");
  }
  LaunchCommon L;
  fill_launch(ctx, mats[0], q, 0, rgb_out, flags, &L);
  L.chunks = (const Chunk*)dev;
  L.n_chunks = (int32_t)chunks.size();
  L.mats.pyramid = (const void* const*)((uint8_t*)dev + cb);
  L.mats.weights = (const void* const*)((uint8_t*)dev + cb + pb);
  L.mats.nmat = nmat;
  int le = launch_material(L, mats[0]->desc.precision, stream);
  cudaFreeAsync(dev, s);
  if (le) return cuda_fail(le, "nam_eval_multi: launch");
  return NAM_OK;
}

extern "C" nam_status nam_eval_binned(nam_ctx* ctx, const nam_material* mats, int32_t nmat, const nam_queries* q,
                                      const int32_t* material_ids, int64_t n, float* rgb_out, void* stream,
                                      uint32_t flags) {
  if (!ctx) return fail(NAM_ERR_INVALID_ARG, "nam_eval_binned: NULL context");
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "n < 0");
  if (n > INT32_MAX) return fail(NAM_ERR_INVALID_ARG, "n beyond 2^31 - 1");
  if (nmat > NAM_MAX_BIN_MATERIALS) return fail(NAM_ERR_INVALID_ARG, "more than %d materials", NAM_MAX_BIN_MATERIALS);
  nam_status st = check_multi(ctx, mats, nmat);
  if (st) return st;
  if (n == 0) return NAM_OK;
  if (!material_ids || !rgb_out) return fail(NAM_ERR_INVALID_ARG, "NULL material ids or output");
  st = check_queries(mats[0], q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  // one stream-ordered allocation: binning scratch, pyramid and weight pointers
  const size_t sb = bin_scratch_bytes(n, nmat, q->xi != nullptr);
  const size_t pb = (size_t)nmat * sizeof(void*);
  std::vector<uint8_t> host(2 * pb);
  for (int32_t k = 0; k < nmat; ++k) {
    const void* p = mats[k]->pyramid;
    const void* w = mats[k]->blob;
    std::memcpy(host.data() + k * sizeof(void*), &p, sizeof p);
    std::memcpy(host.data() + pb + k * sizeof(void*), &w, sizeof w);
  }
  void* dev = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&dev, sb + host.size(), ctx->pool, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "nam_eval_binned: scratch allocation");
  uint8_t* tab = (uint8_t*)dev + sb;
  e = cudaMemcpyAsync(tab, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(dev, s);
    return cuda_fail((int)e, "nam_eval_binned: table upload");
  }
  BinArgs a;
  fill_launch(ctx, mats[0], q, 0, nullptr, flags, &a.L);
  a.L.mats.pyramid = (const void* const*)tab;
  a.L.mats.weights = (const void* const*)(tab + pb);
  a.L.mats.nmat = nmat;
  a.ids = material_ids;
  a.nmat = nmat;
  a.n = n;
  a.rgb_out = rgb_out;
  a.precision = mats[0]->desc.precision;
  a.num_sms = ctx->num_sms;
  a.scratch = dev;
  int le = launch_bin_eval(a, s);
  cudaFreeAsync(dev, s);
  if (le) return cuda_fail(le, "nam_eval_binned: launch");
  return NAM_OK;
}

extern "C" nam_status nam_eval_select(nam_ctx* ctx, const nam_material* mats, int32_t nmat, const nam_queries* q,
                                      const int32_t* material_ids, int64_t n, float* rgb_out, void* stream,
                                      uint32_t flags) {
  if (!ctx) return fail(NAM_ERR_INVALID_ARG, "nam_eval_select: NULL context");
  if (n < 0) return fail(NAM_ERR_INVALID_ARG, "n < 0");
  if (n > INT32_MAX) return fail(NAM_ERR_INVALID_ARG, "n beyond 2^31 - 1");
  if (nmat > NAM_MAX_BIN_MATERIALS) return fail(NAM_ERR_INVALID_ARG, "more than %d materials", NAM_MAX_BIN_MATERIALS);
  nam_status st = check_multi(ctx, mats, nmat);
  if (st) return st;
  if (n == 0) return NAM_OK;
  if (!material_ids || !rgb_out) return fail(NAM_ERR_INVALID_ARG, "NULL material ids or output");
  st = check_queries(mats[0], q);
  if (st) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  // one stream-ordered allocation: tile tables and binning scratch, then
  // pyramid and weight pointers
  const size_t tb = (select_scratch_bytes(n, nmat, q->xi != nullptr) + 255) / 256 * 256;
  const size_t pb = (size_t)nmat * sizeof(void*);
  std::vector<uint8_t> host(2 * pb);
  for (int32_t k = 0; k < nmat; ++k) {
    const void* ptrs[2] = {mats[k]->pyramid, mats[k]->blob};
    for (int j = 0; j < 2; ++j) std::memcpy(host.data() + j * pb + k * sizeof(void*), &ptrs[j], sizeof(void*));
  }
  void* dev = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&dev, tb + host.size(), ctx->pool, s);
  if (e != cudaSuccess) return cuda_fail((int)e, "nam_eval_select: scratch allocation");
  uint8_t* tab = (uint8_t*)dev + tb;
  e = cudaMemcpyAsync(tab, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(dev, s);
    return cuda_fail((int)e, "nam_eval_select: table upload");
  }
  SelectArgs a;
  fill_launch(ctx, mats[0], q, n, rgb_out, flags, &a.L);
  a.L.mats.pyramid = (const void* const*)tab;
  a.L.mats.weights = (const void* const*)(tab + pb);
  a.L.mats.nmat = nmat;
  a.ids = material_ids;
  a.precision = mats[0]->desc.precision;
  a.scratch = dev;
  int le = launch_select_eval(a, s);
  cudaFreeAsync(dev, s);
  if (le) return cuda_fail(le, "nam_eval_select: launch");
  return NAM_OK;
}


