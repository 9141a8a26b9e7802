// Synthetic-scene harness: an analytic scene (ground plane, spheres) ray-cast
// to a G-buffer, and a small wavefront path tracer lit by a constant sky: at
// every vertex one BSDF sample and one cosine-weighted light sample under the
// power heuristic (Veach 1995), with analytic shadow rays, and the path goes
// on along the BSDF sample.  The materials' own entry points
// (nam_sample, nam_sample_pdf, nam_eval) run on material-contiguous ranges:
// the hit pixels are binned by material on the device first, the way a
// renderer reorders shading work so that threads evaluating one material run
// together (Sec. 7.3).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "nam_ctx.h"

using namespace nam;

namespace {

constexpr int kThreads = 256;
constexpr float kPi = 3.14159265358979323846f;
constexpr float kEps = 1e-4f;

struct SceneDev {
  int W, H;
  float eye[3], fwd[3], right[3], up[3];
  float tan_half, aspect, spread;
  float ground_y, ground_inv_scale;
  int ground_mat;
  int ns;
  float sph[NAM_SCENE_MAX_SPHERES][4];
  int sph_mat[NAM_SCENE_MAX_SPHERES];
  float sky;
  float lod_w0;  // level-0 texels per unit of uv
};

struct Hit {
  float t;
  int mat;
  int prim;  // -1 ground, else sphere index
};

__device__ __forceinline__ float dot3(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

__device__ void primary_dir(const SceneDev& S, int px, int py, float d[3]) {
  const float x = (2.0f * (px + 0.5f) / S.W - 1.0f) * S.tan_half * S.aspect;
  const float y = (1.0f - 2.0f * (py + 0.5f) / S.H) * S.tan_half;
  float v[3];
  for (int k = 0; k < 3; ++k) v[k] = S.fwd[k] + x * S.right[k] + y * S.up[k];
  const float inv = rsqrtf(dot3(v, v));
  for (int k = 0; k < 3; ++k) d[k] = v[k] * inv;
}

// closest hit with t > tmin (t = INF, mat = -1 on a miss)
__device__ Hit intersect(const SceneDev& S, const float o[3], const float d[3], float tmin) {
  Hit h{INFINITY, -1, -2};
  if (S.ground_mat >= 0 && fabsf(d[1]) > 1e-12f) {
    const float t = (S.ground_y - o[1]) / d[1];
    if (t > tmin && t < h.t) h = Hit{t, S.ground_mat, -1};
  }
  for (int s = 0; s < S.ns; ++s) {
    const float oc[3] = {o[0] - S.sph[s][0], o[1] - S.sph[s][1], o[2] - S.sph[s][2]};
    const float b = dot3(oc, d);
    const float c = dot3(oc, oc) - S.sph[s][3] * S.sph[s][3];
    const float disc = b * b - c;
    if (disc < 0.0f) continue;
    const float q = sqrtf(disc);
    float t = -b - q;
    if (!(t > tmin)) t = -b + q;
    if (t > tmin && t < h.t) h = Hit{t, S.sph_mat[s], s};
  }
  return h;
}

// shading frame rows (t, b, n), uv and the world-to-uv scale of a hit
__device__ void surface(const SceneDev& S, const Hit& h, const float p[3], float T[9], float& u, float& v,
                        float& uv_scale) {
  float n[3], t[3];
  if (h.prim < 0) {
    n[0] = 0.0f; n[1] = 1.0f; n[2] = 0.0f;
    t[0] = 1.0f; t[1] = 0.0f; t[2] = 0.0f;
    u = p[0] * S.ground_inv_scale;
    v = p[2] * S.ground_inv_scale;
    uv_scale = S.ground_inv_scale;
  } else {
    const float* c = S.sph[h.prim];
    const float inv_r = 1.0f / c[3];
    for (int k = 0; k < 3; ++k) n[k] = (p[k] - c[k]) * inv_r;
    const float inv_n = rsqrtf(dot3(n, n));
    for (int k = 0; k < 3; ++k) n[k] *= inv_n;
    const float h2 = n[0] * n[0] + n[2] * n[2];
    if (h2 > 1e-12f) {
      const float ih = rsqrtf(h2);
      t[0] = -n[2] * ih; t[1] = 0.0f; t[2] = n[0] * ih;
    } else {
      t[0] = 1.0f; t[1] = 0.0f; t[2] = 0.0f;
    }
    u = atan2f(n[2], n[0]) * (0.5f / kPi) + 0.5f;
    v = acosf(fminf(fmaxf(n[1], -1.0f), 1.0f)) * (1.0f / kPi);
    uv_scale = inv_r / (kPi * 1.41421356237f);
  }
  // b = n x t
  const float b[3] = {n[1] * t[2] - n[2] * t[1], n[2] * t[0] - n[0] * t[2], n[0] * t[1] - n[1] * t[0]};
  for (int k = 0; k < 3; ++k) {
    T[k] = t[k];
    T[3 + k] = b[k];
    T[6 + k] = n[k];
  }
}

// A path's current vertex; pos, dir and cone are kept for the path tracer
// (null in the public G-buffer call)
struct GBuf {
  int32_t* material;
  float *t, *u, *v, *lod, *frame, *view;
  float *pos, *dir, *cone;
};

// surface data of hit h on ray (o, d) whose cone has width `cone` at the hit
__device__ void write_vertex(const SceneDev& S, GBuf& g, int64_t i, const Hit& h, const float o[3], const float d[3],
                             float cone) {
  g.material[i] = h.mat;
  if (h.mat < 0) {
    g.t[i] = INFINITY;
    g.u[i] = g.v[i] = g.lod[i] = 0.0f;
    for (int k = 0; k < 9; ++k) g.frame[9 * i + k] = 0.0f;
    for (int k = 0; k < 3; ++k) g.view[3 * i + k] = 0.0f;
    return;
  }
  const float p[3] = {o[0] + h.t * d[0], o[1] + h.t * d[1], o[2] + h.t * d[2]};
  float T[9], u, v, uv_scale;
  surface(S, h, p, T, u, v, uv_scale);
  const float cosv = fabsf(dot3(T + 6, d));
  const float footprint = cone / fmaxf(cosv, 0.05f) * uv_scale * S.lod_w0;
  g.t[i] = h.t;
  g.u[i] = u;
  g.v[i] = v;
  g.lod[i] = log2f(fmaxf(footprint, 1e-6f));
  for (int k = 0; k < 9; ++k) g.frame[9 * i + k] = T[k];
  // direction back along the ray in the shading frame
  const float w[3] = {-d[0], -d[1], -d[2]};
  for (int k = 0; k < 3; ++k) g.view[3 * i + k] = dot3(T + 3 * k, w);
  if (g.pos) {
    for (int k = 0; k < 3; ++k) {
      g.pos[3 * i + k] = p[k];
      g.dir[3 * i + k] = d[k];
    }
    g.cone[i] = cone;
  }
}

__global__ void __launch_bounds__(kThreads) gbuffer_kernel(const SceneDev S, GBuf g) {
  const int64_t n = (int64_t)S.W * S.H;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int px = (int)(i % S.W), py = (int)(i / S.W);
    float d[3];
    primary_dir(S, px, py, d);
    const Hit h = intersect(S, S.eye, d, kEps);
    write_vertex(S, g, i, h, S.eye, d, S.spread * h.t);
  }
}

// the next vertex of every live path (ray ro, rd; live = rd[3i] is finite);
// the cone keeps widening with the distance travelled
__global__ void __launch_bounds__(kThreads) trace_kernel(const SceneDev S, int64_t n, const float* __restrict__ ro,
                                                         const float* __restrict__ rd, GBuf g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d[3] = {rd[3 * i], rd[3 * i + 1], rd[3 * i + 2]};
    if (!isfinite(d[0])) {
      g.material[i] = -1;
      continue;
    }
    const float o[3] = {ro[3 * i], ro[3 * i + 1], ro[3 * i + 2]};
    const Hit h = intersect(S, o, d, kEps);
    const float cone = g.cone[i] + S.spread * (h.mat >= 0 ? h.t : 0.0f);
    write_vertex(S, g, i, h, o, d, cone);
  }
}

__global__ void __launch_bounds__(kThreads) count_kernel(const int32_t* __restrict__ mat, int64_t n,
                                                         uint32_t* __restrict__ counts) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int m = mat[i];
    if (m >= 0) atomicAdd(counts + m, 1u);
  }
}

// perm[slot] = pixel, slots of material m from cursor[m] on
__global__ void __launch_bounds__(kThreads) scatter_kernel(const int32_t* __restrict__ mat, int64_t n,
                                                           uint32_t* __restrict__ cursor, int32_t* __restrict__ perm) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int m = mat[i];
    if (m >= 0) perm[atomicAdd(cursor + m, 1u)] = (int32_t)i;
  }
}

struct Slots {
  // sampler queries (wi = view), light-sample density queries (wo = d_l)
  float *u, *v, *lod, *xi, *vx, *vy, *vz, *lx, *ly, *lz;
  float* var;  // [n_hit][3] variates for nam_sample
};

__global__ void __launch_bounds__(kThreads) prep_kernel(const int32_t* __restrict__ perm, int64_t nh, GBuf g,
                                                        const float* __restrict__ variates, Slots s) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nh; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[p];
    s.u[p] = g.u[i];
    s.v[p] = g.v[i];
    s.lod[p] = g.lod[i];
    s.xi[p] = 0.5f;
    s.vx[p] = g.view[3 * i];
    s.vy[p] = g.view[3 * i + 1];
    s.vz[p] = g.view[3 * i + 2];
    const float* r = variates + 5 * i;
    for (int k = 0; k < 3; ++k) s.var[3 * p + k] = r[k];
    // cosine-weighted light sample about the shading normal
    float sp, cp;
    sincospif(2.0f * r[4], &sp, &cp);
    const float sr = sqrtf(r[3]);
    s.lx[p] = sr * cp;
    s.ly[p] = sr * sp;
    s.lz[p] = sqrtf(fmaxf(1.0f - r[3], 0.0f));
  }
}

struct EvalQ {
  float *u, *v, *lod, *xi, *wix, *wiy, *wiz, *wox, *woy, *woz;
};

// two shading queries per slot: 2p with wi = d_b, 2p + 1 with wi = d_l
__global__ void __launch_bounds__(kThreads) build_eval_kernel(int64_t nh, Slots s, const float* __restrict__ d_b,
                                                              EvalQ e) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nh; p += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < 2; ++k) {
      const int64_t q = 2 * p + k;
      e.u[q] = s.u[p];
      e.v[q] = s.v[p];
      e.lod[q] = s.lod[p];
      e.xi[q] = 0.5f;
      e.wix[q] = k ? s.lx[p] : d_b[3 * p];
      e.wiy[q] = k ? s.ly[p] : d_b[3 * p + 1];
      e.wiz[q] = k ? s.lz[p] : d_b[3 * p + 2];
      e.wox[q] = s.vx[p];
      e.woy[q] = s.vy[p];
      e.woz[q] = s.vz[p];
    }
  }
}

struct PathState {
  float* thr;  // [n][3] throughput
  float* rad;  // [n][3] radiance gathered so far
  float* ro;   // [n][3] next ray origin
  float* rd;   // [n][3] next ray direction (NaN: the path ends)
};

__global__ void __launch_bounds__(kThreads) shade_kernel(const SceneDev S, const int32_t* __restrict__ perm, int64_t nh,
                                                         GBuf g, Slots s, const float* __restrict__ d_b,
                                                         const float* __restrict__ pdf_b, const float* __restrict__ pdf_bl,
                                                         const float* __restrict__ rgb, PathState ps, bool more) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nh; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[p];
    const float* T = g.frame + 9 * i;
    const float t = g.t[i];
    // secondary rays leave from just above the surface
    const float off = 1e-3f * fmaxf(1.0f, t);
    const float o[3] = {g.pos[3 * i] + off * T[6], g.pos[3 * i + 1] + off * T[7], g.pos[3 * i + 2] + off * T[8]};
    float c[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < 2; ++k) {
      const float l[3] = {k ? s.lx[p] : d_b[3 * p], k ? s.ly[p] : d_b[3 * p + 1], k ? s.lz[p] : d_b[3 * p + 2]};
      if (!(l[2] > 0.0f)) continue;
      const float pl = l[2] * (1.0f / kPi);
      const float pb = k ? pdf_bl[p] : pdf_b[p];
      const float pd = k ? pl : pb;
      if (!(pd > 0.0f)) continue;
      const float w = pd * pd / (pb * pb + pl * pl);
      const float dw[3] = {T[0] * l[0] + T[3] * l[1] + T[6] * l[2], T[1] * l[0] + T[4] * l[1] + T[7] * l[2],
                           T[2] * l[0] + T[5] * l[1] + T[8] * l[2]};
      if (intersect(S, o, dw, kEps).mat >= 0) continue;  // the sky is blocked
      const float a = S.sky * w / pd;
      for (int ch = 0; ch < 3; ++ch) c[ch] += a * rgb[3 * (2 * p + k) + ch];
    }
    for (int ch = 0; ch < 3; ++ch) ps.rad[3 * i + ch] += ps.thr[3 * i + ch] * c[ch];
    if (!more) continue;
    // the path goes on along the BSDF sample
    const float l[3] = {d_b[3 * p], d_b[3 * p + 1], d_b[3 * p + 2]};
    const float pb = pdf_b[p];
    if (l[2] > 0.0f && pb > 0.0f) {
      for (int ch = 0; ch < 3; ++ch) ps.thr[3 * i + ch] *= rgb[3 * (2 * p) + ch] / pb;
      for (int k = 0; k < 3; ++k) {
        ps.ro[3 * i + k] = o[k];
        ps.rd[3 * i + k] = T[k] * l[0] + T[3 + k] * l[1] + T[6 + k] * l[2];
      }
    }
  }
}

// throughput 1, radiance 0 (the sky where the primary ray leaves the scene)
__global__ void __launch_bounds__(kThreads) init_paths_kernel(const int32_t* __restrict__ mat, int64_t n, float sky,
                                                              PathState ps) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int ch = 0; ch < 3; ++ch) {
      ps.thr[3 * i + ch] = 1.0f;
      ps.rad[3 * i + ch] = mat[i] < 0 ? sky : 0.0f;
    }
}

__global__ void __launch_bounds__(kThreads) end_paths_kernel(int64_t n, float* __restrict__ rd) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rd[3 * i] = NAN;
}

int grid_of(int64_t n, int sms) {
  int64_t g = (n + kThreads - 1) / kThreads;
  return (int)(g < (int64_t)sms * 8 ? (g > 0 ? g : 1) : (int64_t)sms * 8);
}

void normalize3(float v[3]) {
  const float l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int k = 0; k < 3; ++k) v[k] /= l;
}

void cross3(const float a[3], const float b[3], float c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

nam_status make_scene(const nam_scene* sc, int32_t lod_base_width, SceneDev* S) {
  if (!sc) return fail(NAM_ERR_INVALID_ARG, "NULL scene");
  if (sc->width < 1 || sc->height < 1 || (int64_t)sc->width * sc->height > INT32_MAX)
    return fail(NAM_ERR_INVALID_ARG, "bad image size %dx%d", sc->width, sc->height);
  if (sc->n_spheres < 0 || sc->n_spheres > NAM_SCENE_MAX_SPHERES || (sc->n_spheres && !sc->spheres))
    return fail(NAM_ERR_INVALID_ARG, "bad sphere list");
  if (!(sc->fov_y > 0.0f && sc->fov_y < 3.1f)) return fail(NAM_ERR_INVALID_ARG, "fov_y out of (0, 3.1)");
  if (sc->ground_material >= 0 && !(sc->ground_uv_scale > 0.0f))
    return fail(NAM_ERR_INVALID_ARG, "ground_uv_scale must be > 0");
  if (lod_base_width < 1) return fail(NAM_ERR_INVALID_ARG, "lod_base_width must be >= 1");
  std::memset(S, 0, sizeof *S);
  S->W = sc->width;
  S->H = sc->height;
  for (int k = 0; k < 3; ++k) {
    S->eye[k] = sc->eye[k];
    S->fwd[k] = sc->target[k] - sc->eye[k];
  }
  normalize3(S->fwd);
  cross3(S->fwd, sc->up, S->right);
  const float rl = std::sqrt(S->right[0] * S->right[0] + S->right[1] * S->right[1] + S->right[2] * S->right[2]);
  if (!(rl > 1e-6f)) return fail(NAM_ERR_INVALID_ARG, "camera up is parallel to the view direction");
  normalize3(S->right);
  cross3(S->right, S->fwd, S->up);
  S->tan_half = std::tan(0.5f * sc->fov_y);
  S->aspect = (float)sc->width / (float)sc->height;
  S->spread = 2.0f * S->tan_half / (float)sc->height;
  S->ground_y = sc->ground_y;
  S->ground_mat = sc->ground_material;
  S->ground_inv_scale = sc->ground_material >= 0 ? 1.0f / sc->ground_uv_scale : 0.0f;
  S->ns = sc->n_spheres;
  for (int s = 0; s < sc->n_spheres; ++s) {
    const nam_sphere& sp = sc->spheres[s];
    if (!(sp.radius > 0.0f)) return fail(NAM_ERR_INVALID_ARG, "sphere %d: radius must be > 0", s);
    for (int k = 0; k < 3; ++k) S->sph[s][k] = sp.center[k];
    S->sph[s][3] = sp.radius;
    S->sph_mat[s] = sp.material;
  }
  S->sky = sc->sky_radiance;
  S->lod_w0 = (float)lod_base_width;
  return NAM_OK;
}

int max_material(const nam_scene* sc) {
  int m = sc->ground_material;
  for (int s = 0; s < sc->n_spheres; ++s) m = sc->spheres[s].material > m ? sc->spheres[s].material : m;
  return m;
}

}  // namespace

extern "C" nam_status nam_scene_gbuffer(nam_ctx* ctx, const nam_scene* scene, int32_t lod_base_width, nam_gbuffer* out,
                                        void* stream) {
  if (!ctx || !out) return fail(NAM_ERR_INVALID_ARG, "nam_scene_gbuffer: NULL argument");
  SceneDev S;
  nam_status st = make_scene(scene, lod_base_width, &S);
  if (st) return st;
  for (int s = 0; s < scene->n_spheres; ++s)
    if (scene->spheres[s].material < 0) return fail(NAM_ERR_INVALID_ARG, "sphere %d: material < 0", s);
  if (!out->material || !out->t || !out->u || !out->v || !out->lod || !out->frame || !out->view)
    return fail(NAM_ERR_INVALID_ARG, "nam_scene_gbuffer: NULL output array");
  DeviceGuard g(ctx->device);
  GBuf gb{out->material, out->t, out->u, out->v, out->lod, out->frame, out->view, nullptr, nullptr, nullptr};
  const int64_t n = (int64_t)S.W * S.H;
  gbuffer_kernel<<<grid_of(n, ctx->num_sms), kThreads, 0, (cudaStream_t)stream>>>(S, gb);
  const int e = (int)cudaGetLastError();
  if (e) return cuda_fail(e, "nam_scene_gbuffer: launch");
  return NAM_OK;
}

static nam_status render_paths(nam_ctx* ctx, const nam_scene* scene, const nam_material* mats, int32_t nmat,
                               int32_t bounces, const float* variates, float* image, void* stream, const char* who) {
  if (!ctx || !variates || !image) return fail(NAM_ERR_INVALID_ARG, "%s: NULL argument", who);
  if (bounces < 1 || bounces > NAM_SCENE_MAX_BOUNCES)
    return fail(NAM_ERR_INVALID_ARG, "%s: bounces %d not in [1, %d]", who, bounces, NAM_SCENE_MAX_BOUNCES);
  nam_status st = check_multi(ctx, mats, nmat);
  if (st) return st;
  SceneDev S;
  st = make_scene(scene, mats[0]->pyr.w[0], &S);
  if (st) return st;
  if (max_material(scene) >= nmat) return fail(NAM_ERR_INVALID_ARG, "the scene names material %d of %d",
                                               max_material(scene), nmat);
  for (int s = 0; s < scene->n_spheres; ++s)
    if (scene->spheres[s].material < 0) return fail(NAM_ERR_INVALID_ARG, "sphere %d: material < 0", s);
  for (int k = 0; k < nmat; ++k)
    if (!mats[k]->sampler) return fail(NAM_ERR_UNSUPPORTED, "material %d has no importance sampler", k);
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = (int64_t)S.W * S.H;
  const int grid = grid_of(n, ctx->num_sms);
  // scratch, in units of one 4-byte value per pixel: the path vertex 24, slot
  // permutation 1, per-slot queries and variates 13, BSDF sample and the two
  // densities 5, shading queries (2 per slot) 20 and their RGB 6, throughput
  // and next ray 9 (the radiance accumulates in the image)
  const size_t F = ((size_t)n * 4 + 255) / 256 * 256;
  const size_t counts_b = ((size_t)nmat * 4 + 255) / 256 * 256;
  const size_t total = F * 78 + 2 * counts_b;
  uint8_t* base = nullptr;
  cudaError_t ce = cudaMallocFromPoolAsync((void**)&base, total, ctx->pool, s);
  if (ce != cudaSuccess) return cuda_fail((int)ce, "scene harness: scratch");
  uint8_t* p = base;
  auto take = [&](size_t k) {
    uint8_t* r = p;
    p += k * F;
    return (float*)r;
  };
  GBuf gb;
  gb.material = (int32_t*)take(1);
  gb.t = take(1); gb.u = take(1); gb.v = take(1); gb.lod = take(1);
  gb.frame = take(9); gb.view = take(3);
  gb.pos = take(3); gb.dir = take(3); gb.cone = take(1);
  int32_t* perm = (int32_t*)take(1);
  Slots sl;
  sl.u = take(1); sl.v = take(1); sl.lod = take(1); sl.xi = take(1);
  sl.vx = take(1); sl.vy = take(1); sl.vz = take(1); sl.lx = take(1); sl.ly = take(1); sl.lz = take(1);
  sl.var = take(3);
  float* d_b = take(3);
  float* pdf_b = take(1);
  float* pdf_bl = take(1);
  EvalQ eq;
  eq.u = take(2); eq.v = take(2); eq.lod = take(2); eq.xi = take(2);
  eq.wix = take(2); eq.wiy = take(2); eq.wiz = take(2); eq.wox = take(2); eq.woy = take(2); eq.woz = take(2);
  float* rgb = take(6);
  PathState ps;
  ps.thr = take(3);
  ps.ro = take(3);
  ps.rd = take(3);
  ps.rad = image;
  uint32_t* counts = (uint32_t*)p;
  uint32_t* cursor = (uint32_t*)(p + counts_b);

  int e = 0;
  gbuffer_kernel<<<grid, kThreads, 0, s>>>(S, gb);
  init_paths_kernel<<<grid, kThreads, 0, s>>>(gb.material, n, S.sky, ps);
  std::vector<uint32_t> hc((size_t)nmat), off((size_t)nmat + 1, 0);
  for (int32_t b = 0; b < bounces && !e && !st; ++b) {
    const bool more = b + 1 < bounces;
    if (more) end_paths_kernel<<<grid, kThreads, 0, s>>>(n, ps.rd);
    cudaMemsetAsync(counts, 0, (size_t)nmat * 4, s);
    count_kernel<<<grid, kThreads, 0, s>>>(gb.material, n, counts);
    ce = cudaMemcpyAsync(hc.data(), counts, (size_t)nmat * 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
      e = (int)ce;
      break;
    }
    for (int k = 0; k < nmat; ++k) off[k + 1] = off[k] + hc[k];
    const int64_t nh = off[nmat];
    if (nh == 0) break;  // every path has left the scene
    ce = cudaMemcpyAsync(cursor, off.data(), (size_t)nmat * 4, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) {
      e = (int)ce;
      break;
    }
    const int gh = grid_of(nh, ctx->num_sms);
    scatter_kernel<<<grid, kThreads, 0, s>>>(gb.material, n, cursor, perm);
    prep_kernel<<<gh, kThreads, 0, s>>>(perm, nh, gb, variates + (size_t)b * n * 5, sl);
    e = (int)cudaGetLastError();
    // per material: one BSDF sample, and the sampler's density of the light sample
    for (int k = 0; k < nmat && !e; ++k) {
      const int64_t o = off[k], c = hc[k];
      if (!c) continue;
      nam_queries qa{sl.u + o, sl.v + o, sl.lod + o, sl.vx + o, sl.vy + o, sl.vz + o, sl.lx + o, sl.ly + o, sl.lz + o,
                     sl.xi + o};
      st = nam_sample(ctx, mats[k], &qa, c, sl.var + 3 * o, d_b + 3 * o, pdf_b + o, s);
      if (!st) st = nam_sample_pdf(ctx, mats[k], &qa, c, pdf_bl + o, s);
      if (st) break;
    }
    if (!st && !e) {
      build_eval_kernel<<<gh, kThreads, 0, s>>>(nh, sl, d_b, eq);
      e = (int)cudaGetLastError();
    }
    for (int k = 0; k < nmat && !st && !e; ++k) {
      const int64_t o = 2 * (int64_t)off[k], c = 2 * (int64_t)hc[k];
      if (!c) continue;
      nam_queries qe{eq.u + o, eq.v + o, eq.lod + o, eq.wix + o, eq.wiy + o, eq.wiz + o, eq.wox + o, eq.woy + o,
                     eq.woz + o, eq.xi + o};
      st = nam_eval(ctx, mats[k], &qe, c, rgb + 3 * o, s, NAM_OUT_COSINE);
    }
    if (!st && !e) {
      shade_kernel<<<gh, kThreads, 0, s>>>(S, perm, nh, gb, sl, d_b, pdf_b, pdf_bl, rgb, ps, more);
      e = (int)cudaGetLastError();
    }
    if (more && !st && !e) {
      trace_kernel<<<grid, kThreads, 0, s>>>(S, n, ps.ro, ps.rd, gb);
      e = (int)cudaGetLastError();
    }
  }
  cudaFreeAsync(base, s);
  if (st) return st;
  if (e) return cuda_fail(e, who);
  return NAM_OK;
}

extern "C" nam_status nam_scene_render_direct(nam_ctx* ctx, const nam_scene* scene, const nam_material* mats,
                                              int32_t nmat, const float* variates, float* image, void* stream) {
  return render_paths(ctx, scene, mats, nmat, 1, variates, image, stream, "nam_scene_render_direct");
}

extern "C" nam_status nam_scene_render_paths(nam_ctx* ctx, const nam_scene* scene, const nam_material* mats,
                                             int32_t nmat, int32_t bounces, const float* variates, float* image,
                                             void* stream) {
  return render_paths(ctx, scene, mats, nmat, bounces, variates, image, stream, "nam_scene_render_paths");
}
