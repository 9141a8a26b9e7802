/*
 * nam.h -- C ABI of libnam, batched neural-BRDF evaluation on one GPU.
 *
 * The operation behind every entry point is the neural BRDF of Zeltner et
 * al., "Real-Time Neural Appearance Models" (ACM TOG 2024):
 *
 *     f(x, wi, wo) ~ g( z(x), T wi, T wo ; theta )                (Eq. 3)
 *
 * z(x)  8-channel latent code read from a per-material hierarchical latent
 *       texture (Sec. 4.1): level from the pixel footprint (the caller passes
 *       it as `lod`), bilinear inside a level, the two neighbouring levels
 *       either blended (trilinear) or picked by Russian roulette (stochastic).
 * T     rows (t, b, n) of a shading frame decoded from z (Sec. 4.2, Eq. 4),
 *       b = n x t / |n x t| (Sec. 9).  Here one frame from a frame MLP
 *       8 -> H -> 6 (n_raw, t_raw) with Gram-Schmidt, or the identity.
 * g     decoder MLP, ReLU hidden layers, linear RGB output (Sec. 7, Sec. 8),
 *       input order (z0..z7, (T wi)xyz, (T wo)xyz).
 *
 * Conventions (hold for every call):
 *  - Every function returns nam_status: NAM_OK (0) or a negative error code.
 *    No C++ exception crosses the ABI.  nam_last_error_message() gives a
 *    thread-local description of the last failure on the calling thread.
 *  - Handles are opaque.  A context owns its materials; destroying the
 *    context destroys them.
 *  - Queries are planar float32 arrays (one per field), in the memory space
 *    the call names (device for nam_eval, host for nam_eval_host and the
 *    serving frames).  Outputs are float32 RGB, [n][3] row-major.
 *  - Directions are unit vectors in the geometric frame (z = normal).
 *  - Asynchronous calls enqueue on the caller's CUDA stream (a cudaStream_t
 *    passed as void*, NULL = legacy default stream); outputs are valid after
 *    that stream is synchronised.  A call that returns an error enqueues
 *    nothing.
 *  - Device-side errors (a bounded wait that ran out, a bounds check) are
 *    recorded in the context and returned by the next synchronous call or by
 *    nam_check_device_error().
 */
#ifndef NAM_H
#define NAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* status                                                                   */
/* ------------------------------------------------------------------------ */
typedef int32_t nam_status;
enum {
  NAM_OK = 0,
  NAM_ERR_INVALID_ARG = -1,   /* a pointer, size or enum is out of range */
  NAM_ERR_OOM = -2,           /* device or pinned allocation failed */
  NAM_ERR_BUDGET = -3,        /* resident bytes would exceed the HBM budget */
  NAM_ERR_NOT_FOUND = -4,     /* unknown handle or ticket */
  NAM_ERR_BUSY = -5,          /* the serving admission queue is full */
  NAM_ERR_TIMEOUT = -6,       /* a host or device wait ran past its limit */
  NAM_ERR_CUDA = -7,          /* a CUDA runtime call failed */
  NAM_ERR_DEVICE_ASSERT = -8, /* a device-side check failed */
  NAM_ERR_UNSUPPORTED = -9,   /* a valid but unimplemented combination */
  NAM_ERR_CANCELLED = -10     /* the ticket was cancelled before it ran */
};

const char* nam_status_string(nam_status s);
/* Thread-local description of the last error on this thread ("" if none).
 * The pointer stays valid until the next nam_* call on this thread. */
const char* nam_last_error_message(void);

/* ------------------------------------------------------------------------ */
/* context                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct nam_ctx nam_ctx;

typedef struct {
  int32_t device;             /* CUDA device ordinal */
  int32_t serve_streams;      /* streams of the serving loop (0 -> 4) */
  int32_t serve_queue_depth;  /* frames the admission queue holds (0 -> 256) */
  int32_t reserved0;
  uint64_t hbm_budget_bytes;  /* cap on resident bytes: materials + serving
                                 buffers (0 -> no cap) */
  uint64_t wait_timeout_ns;   /* limit of every device-side wait and of
                                 nam_wait (0 -> 2 s) */
} nam_config;

/* Create a context on cfg->device (cfg NULL -> device 0, defaults).  The
 * calling thread's current device is left unchanged.  Starts no thread until
 * the first nam_submit. */
nam_status nam_init(nam_ctx** out, const nam_config* cfg);
/* Cancel queued serving frames, wait (bounded) for frames on the GPU, stop
 * the serving thread, free every material and buffer, free the context. */
nam_status nam_shutdown(nam_ctx* ctx);
/* Device-side error word of the context: NAM_OK or the first error a kernel
 * recorded since the last call; clears it.  Synchronises the device. */
nam_status nam_check_device_error(nam_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* materials                                                                */
/* ------------------------------------------------------------------------ */
typedef struct nam_material_s* nam_material;

enum { NAM_LATENT_F32 = 0, NAM_LATENT_F16 = 1 };
/* Arithmetic of the MLPs.
 * F32: plain FP32 FMA on CUDA cores, one query per thread.
 * F16: parameters quantised to binary16 at creation (post-training
 * quantisation, Sec. 5.2), MLP layers on tensor cores with FP16 operands and
 * FP32 accumulation.  The operands the result is most sensitive to (the
 * latent, the transformed directions, the frame MLP's hidden layer, the last
 * hidden layer; every hidden layer for hidden width < 64) enter as two FP16
 * halves, so the error against FP16 weights with exact activations stays
 * within 2e-3.
 * FP8 (beyond the paper): as F16, except that the hidden -> hidden decoder
 * layers have E4M3 weights with a power-of-two per-layer scale (the smallest
 * s_w with max |W| / s_w <= 448) and take their input as two E4M3 code sets
 * of x / s_a (s_a: the smallest power of two >= fp8_act_scale[l]), FP32
 * accumulation and FP32 bias; needs a decoder with at least two hidden
 * layers. */
enum { NAM_PREC_F32 = 0, NAM_PREC_F16 = 1, NAM_PREC_FP8 = 2 };
enum { NAM_FILTER_TRILINEAR = 0, NAM_FILTER_STOCHASTIC = 1 };
enum { NAM_ADDRESS_WRAP = 0, NAM_ADDRESS_CLAMP = 1 };
enum { NAM_FRAME_MLP = 0, NAM_FRAME_PAPER = 1 };

#define NAM_MAX_LEVELS 16
#define NAM_MAX_LAYERS 8

typedef struct {
  /* latent pyramid (Sec. 4.1): level l is max(1, base_w >> l) x
   * max(1, base_h >> l) texels, levels stored finest first, texel-major,
   * 8 channels per texel: pyramid[(offset_l + y * W_l + x) * 8 + c]. */
  int32_t base_w, base_h;
  int32_t levels;             /* 1 .. min(NAM_MAX_LEVELS, 1 + log2(max(w,h))) */
  int32_t channels;           /* must be 8 */
  int32_t latent_dtype;       /* NAM_LATENT_F32 or NAM_LATENT_F16 */
  int32_t params_on_device;   /* 1: pyramid and weight pointers are device memory */
  const void* pyramid;        /* copied at creation */

  /* shading frames (Sec. 4.2).  frame_form NAM_FRAME_MLP: frame MLP 8 ->
   * frame_hidden -> 6, ReLU hidden, linear out r = (n_raw, t_raw), one frame
   * by Gram-Schmidt, b = n x t / |n x t|; weights FP32 [Wf1 (h x 8), bf1 (h),
   * Wf2 (6 x h), bf2 (6)]; frame_hidden = 0: no frame, T = I (directions
   * are already local).  frame_form NAM_FRAME_PAPER: the paper's single
   * linear layer 8 -> 12 giving two (normal, tangent) pairs, each
   * normalised but not orthogonalised, b = n x t / |n x t| (Sec. 4.2, Eq. 4,
   * Sec. 9); weights [Wf (12 x 8), bf (12)]; frame_hidden must be 0; the
   * decoder then reads 20 inputs (z, T wi (6), T wo (6)).  Matrices are
   * [out][in] row-major. */
  int32_t frame_hidden;       /* 0 or 16 (NAM_FRAME_MLP) */
  int32_t n_layers;           /* decoder linear layers: 3 (two hidden layers) or
                                 4 (three hidden layers, H = 64) */
  const float* frame_weights;
  /* decoder widths[0] = 14 (20 with NAM_FRAME_PAPER), widths[1..n_layers-1]
   * = H (16, 32 or 64, all equal), widths[n_layers] = 3, or 6 with the
   * albedo head (the paper's albedo inference: outputs 3..5 approximate the
   * directional albedo of Eq. 2, read with nam_eval_albedo; the cosine
   * factor never applies to them; no encoder with the head).  Weights FP32
   * master values, per layer W (out x in) then b (out), layers in order. */
  int32_t widths[NAM_MAX_LAYERS + 1];
  const float* decoder_weights;

  int32_t precision;          /* NAM_PREC_* */
  int32_t filter;             /* NAM_FILTER_* */
  int32_t address;            /* NAM_ADDRESS_* */
  int32_t trainable;          /* 1: keep FP32 masters on the device for
                                 nam_backward / nam_train_step (F32 only;
                                 NAM_FRAME_MLP, two hidden layers) */
  const float* fp8_act_scale; /* NAM_PREC_FP8: host array, n_layers values
                                 > 0: max |input| / 448 of each decoder layer
                                 (nam_fp8_calibrate); the hidden -> hidden
                                 layers' entries set their input scales */
  /* importance sampler (Sec. 4.3, Appendix A): an MLP from (z, wi) to the
   * nine parameters of the analytic proxy density.  sampler_hidden = 0: no
   * sampler; 32: widths 11 -> 32 -> 32 -> 32 -> 9 with ReLU hidden layers,
   * FP32 weights per layer W (out x in) then b (out), layers in order (host
   * or device memory as params_on_device says), copied at creation
   * (NAM_ERR_UNSUPPORTED for a weight of magnitude >= 32768: the network
   * runs on the tensor cores with each weight split into two binary16
   * values). */
  int32_t sampler_hidden;
  const float* sampler_weights;
  int32_t frame_form;         /* NAM_FRAME_MLP (0) or NAM_FRAME_PAPER (1) */
  /* Encoder of the first training phase (Sec. 5.1): an MLP from the material
   * parameters k(x) (encoder_inputs of them, 1..16; 0: no encoder) to the
   * 8-channel latent, widths K -> 32 -> 32 -> 8, ReLU hidden layers, linear
   * output; FP32 weights per layer W (out x in) then b (out), host or device
   * memory as params_on_device says, copied at creation.  Trainable
   * materials only: the encoder exists for training and for initialising
   * the latent texture (nam_encoder_bake), never for evaluation. */
  int32_t encoder_inputs;
  const float* encoder_weights;
} nam_material_desc;

#define NAM_ENCODER_HIDDEN 32
#define NAM_ENCODER_MAX_INPUTS 16

typedef struct {
  uint64_t resident_bytes;    /* device bytes this material holds */
  int64_t texels;             /* texels over all levels */
  int64_t n_params;           /* FP32 master parameters (frame + decoder) */
  int32_t precision, filter, address, levels;
  float fp8_weight_scale[NAM_MAX_LAYERS]; /* NAM_PREC_FP8: weight scale s_w of
                                             each hidden -> hidden decoder
                                             layer, 0 for the others */
} nam_material_info;

/* Copy the pyramid and weights to the device in the layout the kernels read
 * (FP16/FP8 weights quantised here).  NAM_ERR_BUDGET if the context's
 * resident bytes would pass its budget; NAM_ERR_UNSUPPORTED for widths or a
 * precision/filter combination without a kernel. */
nam_status nam_create_material(nam_ctx* ctx, const nam_material_desc* d, nam_material* out);
nam_status nam_destroy_material(nam_ctx* ctx, nam_material m);
nam_status nam_material_get_info(nam_ctx* ctx, nam_material m, nam_material_info* out);
/* Trainable materials: device pointers to the FP32 masters the kernels read,
 * params [n_params] (frame then decoder, layouts as in the descriptor) and
 * pyramid [texels][8].  Owned by the material; valid until it is destroyed.
 * Writing them between launches (on the launch stream) changes the model. */
nam_status nam_material_params(nam_ctx* ctx, nam_material m, float** params_dev, float** pyramid_dev);

/* ------------------------------------------------------------------------ */
/* evaluation                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  const float *u, *v;         /* texture coordinates (wrap or clamp per material) */
  const float *lod;           /* fractional level; clamped to [0, levels-1], NaN -> 0 */
  const float *wix, *wiy, *wiz;
  const float *wox, *woy, *woz;
  const float *xi;            /* U[0,1) variate for the stochastic level pick:
                                 the coarser level iff xi < frac(lod).
                                 Required for NAM_FILTER_STOCHASTIC, else ignored. */
} nam_queries;

enum {
  NAM_OUT_COSINE = 1u << 0,  /* multiply the RGB by max(0, wi.z) (Eq. 1) */
  NAM_HOST_STAGED = 1u << 8,  /* nam_eval_host: always take the staged-copy path */
  NAM_FRAME_DEVICE = 1u << 9  /* nam_submit: the frame's query arrays and rgb_out are
                                 device memory (e.g. a renderer's G-buffer): no copies */
};

/* Evaluate n queries whose arrays are device memory; writes rgb_out (device,
 * [n][3]).  n = 0 is a no-op.  Asynchronous on `stream`.  A material with
 * the albedo head gives its RGB here (its albedo: nam_eval_albedo). */
nam_status nam_eval(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n,
                    float* rgb_out, void* stream, uint32_t flags);

/* The albedo head (a material created with widths[n_layers] = 6): one pass
 * writes the RGB of nam_eval to rgb_out and the directional albedo
 * alpha(x, wo) the decoder infers (the paper's albedo inference; its extra
 * RGB triplet, no cosine factor) to albedo_out, both device [n][3].  Every
 * precision; NAM_ERR_UNSUPPORTED for a material without the head. */
nam_status nam_eval_albedo(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n,
                           float* rgb_out, float* albedo_out, void* stream, uint32_t flags);

/* Same with HOST query and output arrays; synchronises the stream before it
 * returns.  Where the device reads host memory through the host's page
 * tables (cudaDevAttrPageableMemoryAccess, e.g. a GB300 sharing page tables
 * with its Grace CPU), the kernel reads the host queries and writes the host
 * RGB directly, with no staging copies; otherwise, or with NAM_HOST_STAGED in
 * flags, the inputs go to a device staging area owned by the context in up
 * to four chunks whose copies overlap the kernels (pinned host memory gives
 * full copy bandwidth).  Both paths give identical results. */
nam_status nam_eval_host(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n,
                         float* rgb_out, void* stream, uint32_t flags);

/* Static activation scales for NAM_PREC_FP8 from a calibration batch (FP8
 * inference is beyond the paper, which stops at FP16 parameters, Sec. 5.2):
 * evaluates material m's FP32 master parameters with the FP32 kernel on n
 * device queries and writes act_scale_out[l] = (max over the batch of
 * |input of decoder layer l|) / 448 for each of the n_layers decoder layers
 * (1 where that maximum is 0), so that the largest input seen maps to the
 * largest E4M3 magnitude.  Layer 0's input is (z, wi', wo'); later layers'
 * inputs are the previous layer's ReLU outputs.  act_scale_out: host array
 * of n_layers floats, ready for nam_material_desc.fp8_act_scale.  m may have
 * any precision.  Synchronises `stream`. */
nam_status nam_fp8_calibrate(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n,
                             float* act_scale_out, void* stream);

/* Importance sampling with the material's proxy density (Sec. 4.3,
 * Appendix A).  The sampler network maps (z(x), wi) to (w_d, mu_d, w_s,
 * alpha_x, alpha_y, rho, mu_s): w_d, w_s = softmax of two outputs; mu =
 * qsinh(o) = o (1 + |o|/2); alpha = 1e-3 + (1 - 1e-3) (qtanh(o) + 1) / 2 and
 * rho = 0.99 qtanh(o), qtanh(o) = o (1 - |o|/4) for |o| < 2 else sign(o).
 * Density: p(wo) = w_d max(0, wo . n_d) / pi + w_s p_s(wo), n_d =
 * normalize(-mu_dx, -mu_dy, 1); p_s(wo) = D_std(v/|v|) det(M^-1) / |v|^3 /
 * (4 |wo . h|), h = normalize(wi + wo), v = M^-1 h, D_std(w) = max(0, w_z) /
 * pi, M = [[alpha_x, 0, -mu_sx], [alpha_y rho, alpha_y sqrt(1 - rho^2),
 * -mu_sy], [0, 0, 1]].  Directions are in the query's geometric frame (z up).
 * All arrays are device memory; FP32 arithmetic (the network on the tensor
 * cores with binary16 hi/lo splits of weights and activations, relative
 * error ~2^-22 per product); asynchronous on `stream`; NAM_ERR_UNSUPPORTED
 * if the material has no sampler.
 *
 * nam_sample: one direction per query from the variates u ([n][3] in
 * [0, 1)): u[2] < w_d picks the diffuse lobe, (u[0], u[1]) drive the cosine
 * mapping (sqrt(u0) cos 2 pi u1, sqrt(u0) sin 2 pi u1, sqrt(1 - u0)), which is
 * rotated to n_d (diffuse) or mapped to the half vector normalize(M d) and
 * reflected about it (specular).  Writes wo_out [n][3] and, if pdf_out is not
 * NULL, the mixture density of each sampled direction [n].  The queries' wo
 * arrays are not read.
 * nam_sample_pdf: the mixture density of each query's wo given its wi. */
nam_status nam_sample(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n, const float* u,
                      float* wo_out, float* pdf_out, void* stream);
nam_status nam_sample_pdf(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n, float* pdf_out,
                          void* stream);

/* A contiguous run of queries [start, start+count) evaluated with
 * materials[material]. */
typedef struct {
  int64_t start;
  int32_t count;
  int32_t material;
} nam_work_item;

/* Evaluate work items (HOST array `items`, n_items entries, read before the
 * call returns) that each use one of nmat materials (device queries and
 * output, as nam_eval).  All materials must share precision and decoder
 * widths.  Each item's queries run on the path a single-material launch
 * would use, so a query's result does not depend on the other items. */
nam_status nam_eval_multi(nam_ctx* ctx, const nam_material* materials, int32_t nmat,
                          const nam_queries* q, const nam_work_item* items, int32_t n_items,
                          float* rgb_out, void* stream, uint32_t flags);

/* Evaluation of queries whose material varies per query, with no tile
 * coherence (Sec. 7.3: the paper has the ray tracer reorder shading work so
 * that threads evaluating the same material run together).  Bins the queries
 * by material on the device -- per-material histogram, exclusive scan, a
 * permutation that puts each query's index in its material's contiguous
 * range -- evaluates the ranges in one chunked launch of the materials'
 * kernel, which reads each query through the permutation, and writes
 * rgb_out [n][3] (device) in the caller's order.  Each query's result is bitwise
 * that of nam_eval on its material: no query's value depends on which others
 * share its range.  material_ids: device int32 [n], each in [0, nmat); a query
 * with an id outside that range is not evaluated (its rgb_out entries are
 * left as they were) and nam_check_device_error then reports
 * NAM_ERR_DEVICE_ASSERT.  Materials as for nam_eval_multi (tensor-core
 * precisions, one MLP shape and pyramid geometry); nmat <=
 * NAM_MAX_BIN_MATERIALS; n < 2^31.  Temporary device memory (≈ 4 bytes
 * per query, 16 per 128-query chunk and 8 per material) comes from the
 * context's stream-ordered pool. */
#define NAM_MAX_BIN_MATERIALS 4096
nam_status nam_eval_binned(nam_ctx* ctx, const nam_material* mats, int32_t n_materials, const nam_queries* q,
                           const int32_t* material_ids, int64_t n, float* rgb_out, void* stream, uint32_t flags);

/* Evaluation of queries whose material varies per query, in place, choosing
 * a code path per tile (Sec. 7.1: the shader picks per warp between a path
 * for coherent and one for divergent execution; a tcgen05 MMA spans a CTA's
 * 128-row tile, so here the unit is a tile of 128 consecutive queries in the
 * caller's order).  A pass over material_ids lists each tile's distinct
 * materials:
 *   1 to NAM_SELECT_MAX_PASSES  one tensor-core pass over the tile per
 *       material, each storing only the rows of its own material; every
 *       such query's result is bitwise that of nam_eval on its material;
 *   more  the queries of all such tiles are binned by material (the
 *       passes of nam_eval_binned, limited to those tiles: the reordering
 *       the paper's renderer gets from SER, Sec. 7.3) and run in
 *       material-coherent 128-query chunks, their results written in
 *       place; every such query's result is likewise bitwise that of
 *       nam_eval on its material.
 * NAM_SELECT_MAX_PASSES is 1: a tile whose queries share one material is
 * one pass (the coherent path), every other tile is binned, which costs
 * less than running even two masked passes over it.
 * So every result equals nam_eval's on the query's material; only the cost
 * differs: coherent ids (screen tiles of a few surfaces) move no query,
 * incoherent ones cost about what nam_eval_binned does.  Arguments, id
 * checks (an id outside [0, n_materials) leaves that query's rgb_out
 * untouched and makes nam_check_device_error report NAM_ERR_DEVICE_ASSERT)
 * and material requirements as nam_eval_binned.  Temporary device memory
 * (24 bytes per tile: its material list and its entry of the pass table;
 * the binning scratch of nam_eval_binned, and 20 bytes per material) comes
 * from the context's stream-ordered pool. */
#define NAM_SELECT_MAX_PASSES 1
nam_status nam_eval_select(nam_ctx* ctx, const nam_material* mats, int32_t n_materials, const nam_queries* q,
                           const int32_t* material_ids, int64_t n, float* rgb_out, void* stream, uint32_t flags);

/* ------------------------------------------------------------------------ */
/* synthetic-scene harness                                                  */
/* ------------------------------------------------------------------------ */
/* A small analytic scene that exercises evaluation, sampling and densities
 * the way a renderer does (the paper evaluates its materials inside a path
 * tracer, Sec. 7): primary rays of a pinhole camera against a ground plane
 * and spheres give a G-buffer; direct lighting from a constant sky is
 * estimated with one BSDF sample (nam_sample) and one cosine-weighted light
 * sample, combined with the power heuristic (Veach 1995), with analytic
 * shadow rays; the shading queries of each material run on their own
 * contiguous range (pixels binned by material on the device).
 *
 * Geometry: ground plane y = ground_y (normal +y, uv = (x, z) /
 * ground_uv_scale, tangent +x) when ground_material >= 0; spheres with uv =
 * (atan2(n_z, n_x) / 2 pi + 1/2, acos(n_y) / pi) and tangent along +phi.
 * Shading frame (t, b, n) with b = n x t; the query directions are in it.
 * Level of detail from a ray cone (Akenine-Moller et al. 2021): spread
 * 2 tan(fov_y / 2) / height per unit distance, footprint = spread * t /
 * max(|cos|, 0.05), converted to level-0 texels of a pyramid of width
 * lod_base_width through the primitive's world-to-uv scale (ground: 1 /
 * ground_uv_scale; sphere: 1 / (pi sqrt(2) r)); lod = log2(footprint). */
typedef struct {
  float center[3];
  float radius;
  int32_t material;
} nam_sphere;

typedef struct {
  int32_t width, height;
  float eye[3], target[3], up[3];
  float fov_y;                /* radians */
  float ground_y;
  int32_t ground_material;    /* < 0: no ground plane */
  float ground_uv_scale;
  const nam_sphere* spheres;  /* host array */
  int32_t n_spheres;
  float sky_radiance;
} nam_scene;

/* Per-pixel G-buffer, device arrays of width * height entries (row-major
 * from the top-left pixel): material (-1 where the ray leaves the scene), t,
 * u, v, lod, frame [9] (t, b, n rows, world space), view [3] (the direction
 * to the eye in the shading frame). */
typedef struct {
  int32_t* material;
  float *t, *u, *v, *lod;
  float* frame;
  float* view;
} nam_gbuffer;

#define NAM_SCENE_MAX_SPHERES 64
nam_status nam_scene_gbuffer(nam_ctx* ctx, const nam_scene* scene, int32_t lod_base_width, nam_gbuffer* out,
                             void* stream);

/* Direct lighting of every pixel (one sample per strategy) into image
 * [pixels][3] (device); pixels that see the sky get sky_radiance.  Material
 * k of the scene is mats[k]; all share pyramid geometry and MLP shape (as
 * for nam_eval_multi) and need an importance sampler.  variates: device
 * [pixels][5] in [0, 1): three for nam_sample, two for the light sample.
 * Estimator per pixel with BSDF sample d_b (density p_b, the sampler's, with
 * the view direction as its wi) and light sample d_l (density p_l = cos/pi):
 * sum over s of V(d_s) L f(d_s, view) cos(d_s) / p_s(d_s) * p_s^2 / (p_b^2 +
 * p_l^2), f the material's evaluation with wi = d_s, wo = view.  Synchronises
 * the stream (per-material ranges are sized on the host); temporary device
 * memory from the context's pool. */
nam_status nam_scene_render_direct(nam_ctx* ctx, const nam_scene* scene, const nam_material* mats, int32_t n_materials,
                                   const float* variates, float* image, void* stream);

/* Paths of up to `bounces` vertices: at every vertex the direct-lighting
 * estimate above, weighted by the path's throughput, then the path goes on
 * along the BSDF sample (throughput *= f cos / p_b; a sample below the
 * surface or of zero density ends it; a ray that leaves the scene ends it,
 * its sky light already counted by the MIS estimate at its vertex).  Cone
 * of a secondary vertex: spread times the distance travelled along the
 * path.  variates: device [bounces][pixels][5], one set per vertex.
 * bounces = 1 is nam_scene_render_direct. */
#define NAM_SCENE_MAX_BOUNCES 16
nam_status nam_scene_render_paths(nam_ctx* ctx, const nam_scene* scene, const nam_material* mats, int32_t n_materials,
                                  int32_t bounces, const float* variates, float* image, void* stream);

/* ------------------------------------------------------------------------ */
/* differentiation and training (Sec. 5.2)                                  */
/* ------------------------------------------------------------------------ */
/* Reverse mode of nam_eval for a trainable (F32) material: given grad_rgb
 * (device [n][3]; [n][6] for a material with the albedo head: dL/d(RGB),
 * then dL/d(albedo)) accumulates (adds, does not zero) the gradient of
 * sum <grad_rgb, rgb> into grad_params (device [n_params], layout of the
 * masters) and grad_pyramid (device [texels][8], 16-byte aligned; may be
 * NULL; a misaligned pointer is refused with NAM_ERR_INVALID_ARG).  Weight
 * gradients are reduced per CTA then added with one atomic per parameter and
 * CTA; pyramid gradients are scattered with atomics (tap weight x dL/dz).
 * ReLU'(0) = 0.  No gradient flows through the degenerate-frame fallbacks. */
nam_status nam_backward(nam_ctx* ctx, nam_material m, const nam_queries* q, int64_t n,
                        const float* grad_rgb, float* grad_params, float* grad_pyramid,
                        void* stream, uint32_t flags);

typedef struct {
  float lr_params, lr_pyramid;  /* learning rates of the MLP weights and of the latents */
  float beta1, beta2, eps;
  int32_t step;                 /* 1-based step used for bias correction */
} nam_adam;

/* One training step on a trainable material: forward, loss
 * L = mean |log(1+max(g,0)) - log(1+y)| + 0.01 mean max(-g,0) over the n x 3
 * outputs (L1 in log space, Sec. 5.2), backward, Adam on the MLP masters
 * and the pyramid.  One kernel runs the forward, the loss and the backward;
 * two more apply Adam.  target_rgb is device [n][3]; *loss_out (host)
 * receives L of this step's forward (the call synchronises the stream to
 * read it).  Optimiser moments live in the material; the first call
 * allocates the material's 256-byte loss accumulator. */
nam_status nam_train_step(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* target_rgb,
                          int64_t n, const nam_adam* opt, float* loss_out, void* stream, uint32_t flags);

/* nam_train_step for a material with the albedo head (the paper's albedo
 * inference): the loss adds mean (a - t)^2 over the n x 3 albedo outputs,
 * t the device [n][3] target_albedo, one-sample Monte Carlo estimates of the
 * directional albedo (Eq. 2: e.g. pi f(x, wi, wo) for wi drawn
 * cosine-weighted), so that the head converges to their mean.  *loss_out
 * receives the sum of both terms.  nam_train_step (and its no-allocation
 * form) refuses a material with the head, this call one without it. */
nam_status nam_train_step_albedo(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* target_rgb,
                                 const float* target_albedo, int64_t n, const nam_adam* opt, float* loss_out,
                                 void* stream, uint32_t flags);

/* A training step that allocates no device memory.  The paper has no
 * counterpart: this is a library facility.  nam_train_step allocates a
 * per-material buffer on its first call; callers that may not call
 * cudaMalloc while they run -- a fixed memory plan, an embedding host that
 * owns all allocation, a loop that must not synchronise the device the way
 * cudaMalloc/cudaFree can -- call this instead.  It computes what
 * nam_train_step computes (loss, gradients, Adam update) as separate passes:
 * the forward, the loss, the backward, Adam, with the per-batch buffers
 * (forward RGB, dL/dRGB, loss accumulator) in one static device array of the
 * library (NAM_NOALLOC_TRAIN_MAX_QUERIES * 24 + 256 bytes, held by every GPU
 * that loads libnam until the process exits).  Its results agree with
 * nam_train_step's to FP32 rounding: the fused step takes the forward values
 * from its backward kernel, which sums in another order.
 *  - n must be at most NAM_NOALLOC_TRAIN_MAX_QUERIES; larger batches are
 *    refused with NAM_ERR_INVALID_ARG before anything is enqueued.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) for that device; make that first call before any
 *    stream capture.
 *  - All calls share the array, which keeps the last call's contents (the
 *    loss accumulator is cleared by each call).  Calls whose work overlaps on
 *    the GPU (different streams, no ordering between them) race on it: order
 *    them on one stream.
 *  - Arguments, results and errors as nam_train_step. */
#define NAM_NOALLOC_TRAIN_MAX_QUERIES 65536
nam_status nam_train_step_noalloc(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* target_rgb,
                                  int64_t n, const nam_adam* opt, float* loss_out, void* stream, uint32_t flags);

/* ------------------------------------------------------------------------ */
/* encoder phase of training (Sec. 5.1)                                     */
/* ------------------------------------------------------------------------ */
/* The paper trains in two phases.  First the latent of a query is the
 * encoder's output for the material parameters at the query, fed to the
 * decoder directly (the latent texture is bypassed); then the texture is
 * initialised by evaluating the encoder for every texel, the encoder is
 * dropped and the texels are trained directly (nam_train_step).  All calls
 * below need a trainable material created with encoder_inputs = K > 0.
 * attrs are device arrays [n][K] (row-major, FP32): the K material
 * parameters of each query, or of each texel for the bake.  Queries need
 * wi and wo (and xi is ignored); u, v and lod are not read. */

/* z_out [n][8] (device, 16-byte aligned) = encoder(attrs). */
nam_status nam_encode(nam_ctx* ctx, nam_material m, const float* attrs, int64_t n, float* z_out, void* stream);

/* Initialise the latent texture: texel t of the FP32 pyramid master =
 * encoder(texel_attrs[t]) for all texels (levels packed finest first; the
 * caller prefilters the parameters of the coarse levels).  Clears the
 * pyramid's Adam moments and gradient, so that finetuning starts afresh. */
nam_status nam_encoder_bake(nam_ctx* ctx, nam_material m, const float* texel_attrs, void* stream);

/* Reverse mode with latents from the encoder: accumulates the gradient of
 * sum <grad_rgb, rgb> into grad_params (frame then decoder, as nam_backward)
 * and grad_encoder (device [encoder parameters], the layout of
 * encoder_weights).  Keeps a per-material buffer for the batch's latents and
 * their gradients (allocated on first use, grown with the batch). */
nam_status nam_backward_encoded(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* attrs,
                                int64_t n, const float* grad_rgb, float* grad_params, float* grad_encoder,
                                void* stream, uint32_t flags);

/* One step of the first training phase: forward with latents from the
 * encoder, the loss of nam_train_step, backward through decoder, frame and
 * encoder, Adam (lr_params) on the frame, decoder and encoder masters.  The
 * latent texture is untouched.  *loss_out as in nam_train_step. */
nam_status nam_train_step_encoded(nam_ctx* ctx, nam_material m, const nam_queries* q, const float* attrs,
                                  const float* target_rgb, int64_t n, const nam_adam* opt, float* loss_out,
                                  void* stream, uint32_t flags);

/* Device pointer to the encoder's FP32 masters (layout of encoder_weights);
 * owned by the material. */
nam_status nam_material_encoder(nam_ctx* ctx, nam_material m, float** encoder_dev);

/* ------------------------------------------------------------------------ */
/* serving: continuous batching of frames (Sec. 7.3 coherency analogue)      */
/* ------------------------------------------------------------------------ */
typedef uint64_t nam_ticket;

typedef struct {
  int64_t n_queries;          /* queries of the frame */
  nam_queries q;              /* HOST arrays (device with NAM_FRAME_DEVICE), n_queries each,
                                 valid until the ticket completes */
  const nam_work_item* items; /* HOST array: the frame's tiles, each one material */
  int32_t n_items;
  int32_t n_materials;
  const nam_material* materials; /* HOST array of n_materials handles, resident in this context */
  float* rgb_out;             /* HOST [n_queries][3] (device with NAM_FRAME_DEVICE), written
                                 before the ticket completes */
  uint32_t flags;             /* NAM_OUT_*, NAM_FRAME_DEVICE */
  int32_t reserved0;
  double arrival_s;           /* arrival time on the nam_now() clock; <= 0 -> now.  A frame
                                 whose arrival lies in the future is held in the queue
                                 until then (a paced stream), so a caller may submit ahead
                                 of the arrival times without its own timing mattering. */
} nam_frame;

/* Times of one frame, all in seconds on the nam_now() clock.  The gpu_* times
 * are device timestamps (CUDA events on the frame's stream) mapped onto that
 * clock through an anchor event the serving thread takes while the GPU is
 * idle (error: a few microseconds); 0 where the frame never reached the GPU. */
typedef struct {
  double arrival_s;           /* the frame's arrival (nam_frame.arrival_s) */
  double admit_s;             /* the serving thread took it off the queue */
  double start_s;             /* it began enqueuing the frame's work */
  double finish_s;            /* the serving thread observed its completion */
  int64_t n_queries;
  nam_status status;          /* NAM_OK once done; an error if it failed */
  int32_t slot;               /* stream slot that ran it (-1: none) */
  double submit_s;            /* nam_submit was called */
  double enqueued_s;          /* all of the frame's work was on its stream */
  double gpu_begin_s;         /* its first copy began on the device */
  double gpu_kernel_begin_s;  /* its kernel began (inputs resident) */
  double gpu_kernel_end_s;    /* its kernel ended */
  double gpu_end_s;           /* its RGB was back in host memory */
  int32_t in_flight_at_admit; /* frames already on the GPU when it was admitted */
  int32_t reserved1;
} nam_frame_stats;

typedef struct {
  uint64_t resident_bytes;    /* materials + serving buffers in use */
  uint64_t budget_bytes;
  int64_t queued, in_flight, completed, failed;
  int64_t queries_completed;
  double p50_latency_ms, p99_latency_ms;  /* over the last <= 4096 completed frames */
  double evals_per_s;         /* completed queries / (last finish - first arrival) */
} nam_stats;

/* Seconds on a monotonic host clock shared by the serving calls. */
double nam_now(void);
/* Queue a frame (non-blocking).  A serving thread admits queued frames in
 * submission order, each once its arrival time has come, its device buffers
 * fit in the budget and a stream slot is free, so frames that arrive while
 * others run start at once and overlap with them on the GPU.  NAM_ERR_BUSY
 * if the queue is full; NAM_ERR_BUDGET if the frame alone can never fit. */
nam_status nam_submit(nam_ctx* ctx, const nam_frame* f, nam_ticket* out);
/* Non-blocking: *done = 1 once the frame's output is in rgb_out (or it
 * failed); fills *st if not NULL. */
nam_status nam_poll(nam_ctx* ctx, nam_ticket t, int32_t* done, nam_frame_stats* st);
/* Block until the ticket completes or timeout_ns passes (NAM_ERR_TIMEOUT). */
nam_status nam_wait(nam_ctx* ctx, nam_ticket t, uint64_t timeout_ns, nam_frame_stats* st);
/* Cancel a queued (not yet admitted) frame: it completes with
 * NAM_ERR_CANCELLED.  NAM_ERR_BUSY if it is already on the GPU. */
nam_status nam_cancel(nam_ctx* ctx, nam_ticket t);
nam_status nam_get_stats(nam_ctx* ctx, nam_stats* out);

/* ------------------------------------------------------------------------ */
/* test hooks (host-side fault injection; no GPU fault is ever made)         */
/* ------------------------------------------------------------------------ */
enum {
  NAM_FAULT_NONE = 0,
  NAM_FAULT_ALLOC = 1,        /* the next device allocation fails (NAM_ERR_OOM) */
  NAM_FAULT_LAUNCH = 2,       /* the next serving launch fails (NAM_ERR_CUDA) */
  NAM_FAULT_STALL = 3         /* the serving thread stops admitting frames */
};
nam_status nam_inject_fault(nam_ctx* ctx, int32_t fault);

#ifdef __cplusplus
}
#endif
#endif /* NAM_H */
