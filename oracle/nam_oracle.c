/*
 * FP64 CPU oracle for the neural-BRDF evaluation of "Real-Time Neural
 * Appearance Models" (Zeltner et al., ACM TOG 2024).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  It shares no code with the CUDA path:
 * everything below is written out plainly, one query at a time, in double
 * precision, following the paper's description:
 *
 *   f(x, wi, wo) ~ g(z(x), T wi, T wo; theta)                  (Eq. 3)
 *   z(x): hierarchical latent texture, level from the footprint area,
 *         one of the two neighbouring levels picked by Russian roulette
 *         (stochastic) or both blended (trilinear), bilinear inside a level
 *                                                              (Sec. 4.1)
 *   T: rows (t, b, n) of a shading frame decoded from z        (Eq. 4, Sec. 4.2)
 *      with b = n x t / |n x t|                                (Sec. 9)
 *   g: MLP with ReLU hidden layers and a linear RGB output     (Sec. 7, Sec. 8)
 *   FP16 parameters by post-training quantisation              (Sec. 5.2)
 *   training loss: L1 in log space                             (Sec. 5.2)
 *
 * Readings where the paper is silent (texel centres, level sizes, addressing,
 * lod clamp and tie-break, frame MLP form and degenerate frames, decoder input
 * order, activations, loss form, FP8 quantisation) are listed in the design
 * notes and restated at each function below.
 *
 * Pins: tests/test_oracle_pins*.py check every function here against closed
 * forms, invariants, library routines and brute force on tiny inputs.  The
 * composed evaluation is parity unpinned end to end: the paper prints no
 * worked example with values to compare against.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_C 8          /* latent channels (Sec. 4: eight-dimensional code) */
#define ORC_MAXW 256     /* widest layer the oracle accepts */
#define ORC_MAXL 8       /* most decoder layers */
#define ORC_MAXOUT 6     /* decoder outputs: RGB, or RGB then an albedo RGB (the
                            optional albedo head of the paper's albedo inference) */

/* ------------------------------------------------------------------------- */
/* number formats                                                             */
/* ------------------------------------------------------------------------- */

/* IEEE 754 binary16 -> double: sign, 5-bit exponent (bias 15), 10-bit
 * fraction; exponent 0 is subnormal (no implicit one), 31 is inf/NaN. */
double orc_f16_to_f64(uint16_t h) {
  int s = (h >> 15) & 1, e = (h >> 10) & 31, f = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)f, -24);
  else if (e == 31) v = f ? NAN : INFINITY;
  else v = ldexp((double)(1024 + f), e - 25);
  return s ? -v : v;
}

/* Round a double to the nearest binary16 value, ties to even; overflow past
 * the largest finite value (65504) rounds to infinity as IEEE prescribes. */
uint16_t orc_f64_to_f16(double x) {
  if (isnan(x)) return 0x7e00;
  uint16_t sign = signbit(x) ? 0x8000 : 0;
  double a = fabs(x);
  if (a >= 65520.0) return sign | 0x7c00; /* halfway to 2^16 and beyond */
  int e;
  frexp(a, &e);           /* a = m 2^e, m in [0.5, 1) */
  int ex = e - 1;         /* a in [2^ex, 2^(ex+1)) */
  if (ex < -14) ex = -14; /* subnormal spacing 2^-24 */
  double q = ldexp(a, 10 - ex); /* units of the spacing 2^(ex-10) */
  double r = nearbyint(q);      /* current rounding mode: ties to even */
  double v = ldexp(r, ex - 10);
  if (v == 0.0) return sign;
  /* re-encode the exact value v */
  int e2;
  frexp(v, &e2);
  int E = e2 - 1;
  if (E < -14) return sign | (uint16_t)ldexp(v, 24); /* subnormal */
  if (E > 15) return sign | 0x7c00;
  uint16_t frac = (uint16_t)(ldexp(v, 10 - E) - 1024.0);
  return sign | (uint16_t)((E + 15) << 10) | frac;
}

double orc_round_f16(double x) { return orc_f16_to_f64(orc_f64_to_f16(x)); }

/* OCP 8-bit floating point, E4M3FN variant: bias 7, no infinities, only
 * S.1111.111 is NaN, largest finite magnitude 448 = 1.75 * 2^8. */
double orc_e4m3_to_f64(uint8_t b) {
  int s = (b >> 7) & 1, e = (b >> 3) & 15, f = b & 7;
  double v;
  if (e == 15 && f == 7) v = NAN;
  else if (e == 0) v = ldexp((double)f, -9);
  else v = ldexp((double)(8 + f), e - 10);
  return s ? -v : v;
}

/* Round to nearest E4M3FN, ties to even, saturating at +-448 (the
 * "satfinite" conversion).  NaN maps to the NaN code 0x7f. */
uint8_t orc_f64_to_e4m3(double x) {
  if (isnan(x)) return 0x7f;
  uint8_t sign = signbit(x) ? 0x80 : 0;
  double a = fabs(x);
  if (a >= 448.0) return sign | 0x7e;
  int e;
  frexp(a, &e);
  int ex = e - 1;
  if (ex < -6) ex = -6; /* subnormal spacing 2^-9 */
  double r = nearbyint(ldexp(a, 3 - ex));
  double v = ldexp(r, ex - 3);
  if (v >= 448.0) return sign | 0x7e;
  if (v == 0.0) return sign;
  int e2;
  frexp(v, &e2);
  int E = e2 - 1;
  if (E < -6) return sign | (uint8_t)ldexp(v, 9);
  uint8_t frac = (uint8_t)(ldexp(v, 3 - E) - 8.0);
  return sign | (uint8_t)((E + 7) << 3) | frac;
}

double orc_round_e4m3(double x) { return orc_e4m3_to_f64(orc_f64_to_e4m3(x)); }

/* Per-layer FP8 weight quantisation (beyond the paper, which names lower
 * precision as future work in Sec. 5.2).  Reading: the scale is the power of
 * two s = 2^ceil(log2(absmax(W) / 448)) (1 for an all-zero layer), so that
 * |W| / s <= 448 and dividing by s is exact; each code = E4M3(W / s), round to
 * nearest even, saturating.  Writes s and the dequantised weights code * s. */
void orc_quantize_e4m3_layer(const float* W, int64_t n, float* scale_out, double* deq_out) {
  double amax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double a = fabs((double)W[i]);
    if (a > amax) amax = a;
  }
  /* the smallest power of two s with amax / s <= 448, found by doubling and
   * halving (exact in FP64) rather than through log2 */
  double s = 1.0;
  if (amax > 0.0) {
    while (amax / s > 448.0) s *= 2.0;
    while (amax / (s * 0.5) <= 448.0) s *= 0.5;
  }
  *scale_out = (float)s;
  for (int64_t i = 0; i < n; ++i) deq_out[i] = orc_round_e4m3((double)W[i] / s) * s;
}

/* ------------------------------------------------------------------------- */
/* model description                                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t W0, H0, L, C;     /* finest level size, level count, channels (8) */
  int32_t latent_f16;       /* 1: pyramid holds binary16 bit patterns, 0: float32 */
  int32_t address;          /* 0: wrap (repeat), 1: clamp to edge */
  int32_t filter;           /* 0: trilinear, 1: stochastic (Russian roulette) */
  int32_t out_cosine;       /* 1: multiply the output by max(0, wi.z) */
  int32_t frame_hidden;     /* hidden width of the frame MLP, 0: T = I */
  int32_t n_layers;         /* decoder linear layers */
  int32_t widths[ORC_MAXL + 1]; /* decoder widths, widths[0] = 14, widths[n_layers] = 3, or 6 with
                                   the albedo head (outputs 3..5: directional albedo) */
  const void* pyramid;      /* levels packed finest first, [texel][C] */
  const double* frame_params; /* Wf1[h][8], bf1[h], Wf2[6][h], bf2[6] */
  const double* dec_params;   /* per layer W[out][in] then b[out] */
  int32_t frame_form;         /* 0: frame MLP 8 -> h -> 6 with Gram-Schmidt (frame_hidden > 0);
                                 1: the paper's form, one linear layer 8 -> 12 giving two frames
                                 (frame_params = Wf[12][8], bf[12]; decoder widths[0] = 20) */
} orc_model;

typedef struct {
  const float *u, *v, *lod, *wix, *wiy, *wiz, *wox, *woy, *woz, *xi;
  /* encoder phase of training (Sec. 5.1): when set, the latent of query i is
   * z[8 i .. 8 i + 7] as given (the encoder's output), bypassing the latent
   * texture; u, v, lod and xi are then not read */
  const double* z;
} orc_queries;

/* Level sizes: level l is max(1, W0 >> l) by max(1, H0 >> l) texels, levels
 * stored one after the other starting with the finest. */
static int64_t level_offset(const orc_model* m, int l, int* Wl, int* Hl) {
  int64_t off = 0;
  for (int k = 0; k < l; ++k) {
    int w = m->W0 >> k, h = m->H0 >> k;
    off += (int64_t)(w > 0 ? w : 1) * (h > 0 ? h : 1);
  }
  int w = m->W0 >> l, h = m->H0 >> l;
  *Wl = w > 0 ? w : 1;
  *Hl = h > 0 ? h : 1;
  return off;
}

static double texel(const orc_model* m, int64_t idx, int c) {
  if (m->latent_f16) return orc_f16_to_f64(((const uint16_t*)m->pyramid)[idx * m->C + c]);
  return (double)((const float*)m->pyramid)[idx * m->C + c];
}

/* Integer texel coordinate under the addressing mode: wrap repeats the level
 * with period n, clamp holds the edge texel. */
static int64_t address(const orc_model* m, double i, int n) {
  if (m->address == 1) {
    if (i < 0) return 0;
    if (i > n - 1) return n - 1;
    return (int64_t)i;
  }
  double r = i - (double)n * floor(i / (double)n);
  int64_t k = (int64_t)r;
  if (k >= n) k -= n; /* guards r == n after rounding */
  return k;
}

/* One bilinear tap set at level l: texel centres sit at (i + 1/2) / W_l, so
 * the continuous texel coordinate is x = u W_l - 1/2; the four texels around
 * it get the usual bilinear weights.  Returns the taps' indices and weights. */
static void bilinear_taps(const orc_model* m, int l, double u, double v,
                          int64_t idx[4], double w[4]) {
  int Wl, Hl;
  int64_t off = level_offset(m, l, &Wl, &Hl);
  double x = u * Wl - 0.5, y = v * Hl - 0.5;
  double x0 = floor(x), y0 = floor(y);
  double fx = x - x0, fy = y - y0;
  int64_t ix0 = address(m, x0, Wl), ix1 = address(m, x0 + 1.0, Wl);
  int64_t iy0 = address(m, y0, Hl), iy1 = address(m, y0 + 1.0, Hl);
  idx[0] = off + iy0 * Wl + ix0; w[0] = (1.0 - fx) * (1.0 - fy);
  idx[1] = off + iy0 * Wl + ix1; w[1] = fx * (1.0 - fy);
  idx[2] = off + iy1 * Wl + ix0; w[2] = (1.0 - fx) * fy;
  idx[3] = off + iy1 * Wl + ix1; w[3] = fx * fy;
}

/* Level selection (Sec. 4.1): the level index may be fractional.  Reading:
 * l = clamp(lod, 0, L-1) (NaN -> 0), l0 = floor(l), l1 = min(l0+1, L-1),
 * t = l - l0.  Trilinear blends the two bilinear fetches with weights 1-t, t;
 * the stochastic variant takes l1 when xi < t and l0 otherwise, so that its
 * expectation over xi ~ U[0,1) is the trilinear result.
 * Fills up to 8 taps; returns the tap count. */
static int latent_taps(const orc_model* m, double u, double v, double lod, double xi,
                       int64_t idx[8], double w[8]) {
  double l = lod;
  if (!(l > 0.0)) l = 0.0; /* also maps NaN to 0 */
  if (l > m->L - 1) l = m->L - 1;
  double l0 = floor(l);
  double t = l - l0;
  int il0 = (int)l0;
  int il1 = il0 + 1 < m->L ? il0 + 1 : m->L - 1;
  if (m->filter == 1) {
    int lv = (xi < t) ? il1 : il0;
    bilinear_taps(m, lv, u, v, idx, w);
    return 4;
  }
  bilinear_taps(m, il0, u, v, idx, w);
  bilinear_taps(m, il1, u, v, idx + 4, w + 4);
  for (int k = 0; k < 4; ++k) {
    w[k] *= (1.0 - t);
    w[k + 4] *= t;
  }
  return 8;
}

static void latent(const orc_model* m, double u, double v, double lod, double xi, double z[ORC_C]) {
  int64_t idx[8];
  double w[8];
  int nt = latent_taps(m, u, v, lod, xi, idx, w);
  for (int c = 0; c < ORC_C; ++c) z[c] = 0.0;
  for (int k = 0; k < nt; ++k)
    for (int c = 0; c < ORC_C; ++c) z[c] += w[k] * texel(m, idx[k], c);
}

/* ------------------------------------------------------------------------- */
/* shading frame (Sec. 4.2, Eq. 4; bitangent from Sec. 9)                     */
/* ------------------------------------------------------------------------- */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Tangent orthogonal to a unit n when the decoded tangent is unusable:
 * the branch-free orthonormal basis of Duff et al. (JCGT 6(1), 2017). */
static void basis_tangent(const double n[3], double t[3]) {
  double s = copysign(1.0, n[2]);
  double a = -1.0 / (s + n[2]);
  double b = n[0] * n[1] * a;
  t[0] = 1.0 + s * n[0] * n[0] * a;
  t[1] = s * b;
  t[2] = -s * n[0];
}

typedef struct {
  double n[3], t[3], b[3];
  double nraw_len, tp_len, c_len, s; /* |n_raw|, |t'|, |n x t|, t_raw.n */
  int n_degenerate, t_degenerate;
} frame_state;

/* r = (n_raw, t_raw).  Reading of the frame step: normalise n; Gram-Schmidt
 * the tangent against n and normalise; b = n x t / |n x t|.  Degenerate
 * cases: |n_raw| < 1e-20 gives n = (0,0,1); |t'| <= 1e-6 |t_raw| takes the
 * tangent from n alone (Duff et al.).  T's rows are (t, b, n). */
static void build_frame(const double r[6], frame_state* f) {
  const double* nr = r;
  const double* tr = r + 3;
  double nl = sqrt(dot3(nr, nr));
  f->nraw_len = nl;
  f->n_degenerate = !(nl >= 1e-20);
  if (f->n_degenerate) {
    f->n[0] = 0; f->n[1] = 0; f->n[2] = 1;
  } else {
    for (int k = 0; k < 3; ++k) f->n[k] = nr[k] / nl;
  }
  double s = dot3(tr, f->n);
  f->s = s;
  double tp[3];
  for (int k = 0; k < 3; ++k) tp[k] = tr[k] - s * f->n[k];
  double tpl = sqrt(dot3(tp, tp));
  double trl = sqrt(dot3(tr, tr));
  f->tp_len = tpl;
  f->t_degenerate = !(tpl > 1e-6 * trl);
  if (f->t_degenerate) basis_tangent(f->n, f->t);
  else for (int k = 0; k < 3; ++k) f->t[k] = tp[k] / tpl;
  double c[3];
  cross3(f->n, f->t, c);
  double cl = sqrt(dot3(c, c));
  f->c_len = cl;
  for (int k = 0; k < 3; ++k) f->b[k] = c[k] / cl;
}

/* ------------------------------------------------------------------------- */
/* one query, forward, keeping what the backward pass needs                   */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t idx[8];
  double w[8];
  int ntaps;
  double z[ORC_C];        /* filtered latent */
  double hf_pre[ORC_MAXW];
  double hf[ORC_MAXW];
  double r[12];
  frame_state fr;
  double pf_n[2][3], pf_t[2][3], pf_b[2][3]; /* paper form: the two frames */
  double pf_nl[2], pf_tl[2], pf_sin[2];
  double wi[3], wo[3];
  double pre[ORC_MAXL][ORC_MAXW]; /* decoder pre-activations */
  double act[ORC_MAXL + 1][ORC_MAXW]; /* decoder layer inputs, act[0] = x */
  double y[ORC_MAXOUT];
  double cosf;            /* BRDF output factor: 1 or max(0, wi.z) (not applied to the albedo) */
} trace;

/* ------------------------------------------------------------------------- */
/* valid alternative roundings                                                */
/* ------------------------------------------------------------------------- */
/* The paper's frame form (Sec. 4.2, Eq. 4; Sec. 9): one linear layer maps z
 * to N = 2 (normal, tangent) pairs; each is normalised, not orthogonalised,
 * and b = n x t / |n x t|.  Readings for degenerate outputs: |n_raw| < 1e-20
 * gives n = (0,0,1); |t_raw| < 1e-20, or n and t parallel (|n x t| <= 1e-6),
 * takes t from n by Duff et al.'s basis. */
static void paper_frames(const orc_model* m, trace* tr) {
  const double* Wf = m->frame_params;
  const double* bf = Wf + 12 * ORC_C;
  for (int j = 0; j < 12; ++j) {
    double s = bf[j];
    for (int c = 0; c < ORC_C; ++c) s += Wf[j * ORC_C + c] * tr->z[c];
    tr->r[j] = s;
  }
  for (int k = 0; k < 2; ++k) {
    const double* nr = tr->r + 6 * k;
    const double* trw = tr->r + 6 * k + 3;
    double* n = tr->pf_n[k];
    double* t = tr->pf_t[k];
    double* b = tr->pf_b[k];
    double nl = sqrt(dot3(nr, nr)), tl = sqrt(dot3(trw, trw));
    tr->pf_nl[k] = nl;
    tr->pf_tl[k] = tl;
    if (nl >= 1e-20) for (int a = 0; a < 3; ++a) n[a] = nr[a] / nl;
    else { n[0] = 0; n[1] = 0; n[2] = 1; }
    if (tl >= 1e-20) for (int a = 0; a < 3; ++a) t[a] = trw[a] / tl;
    else basis_tangent(n, t);
    double c[3];
    cross3(n, t, c);
    double cl = sqrt(dot3(c, c));
    tr->pf_sin[k] = cl;
    if (!(cl > 1e-6)) {
      basis_tangent(n, t);
      cross3(n, t, c);
      cl = sqrt(dot3(c, c));
    }
    for (int a = 0; a < 3; ++a) b[a] = c[a] / cl;
  }
}

static void forward(const orc_model* m, const orc_queries* q, int64_t i, trace* tr) {
  if (q->z) {
    /* the latent comes from the encoder, not from the texture */
    tr->ntaps = 0;
    for (int c = 0; c < ORC_C; ++c) tr->z[c] = q->z[i * ORC_C + c];
  } else {
    double u = q->u[i], v = q->v[i], lod = q->lod[i];
    double xi = q->xi ? q->xi[i] : 0.0;
    tr->ntaps = latent_taps(m, u, v, lod, xi, tr->idx, tr->w);
    for (int c = 0; c < ORC_C; ++c) tr->z[c] = 0.0;
    for (int k = 0; k < tr->ntaps; ++k)
      for (int c = 0; c < ORC_C; ++c) tr->z[c] += tr->w[k] * texel(m, tr->idx[k], c);
  }
  tr->wi[0] = q->wix[i]; tr->wi[1] = q->wiy[i]; tr->wi[2] = q->wiz[i];
  tr->wo[0] = q->wox[i]; tr->wo[1] = q->woy[i]; tr->wo[2] = q->woz[i];

  double wi_l[6], wo_l[6];
  int nd = 3;  /* transformed components per direction */
  if (m->frame_form == 1) {
    paper_frames(m, tr);
    nd = 6;
    for (int k = 0; k < 2; ++k) {
      wi_l[3 * k + 0] = dot3(tr->pf_t[k], tr->wi);
      wi_l[3 * k + 1] = dot3(tr->pf_b[k], tr->wi);
      wi_l[3 * k + 2] = dot3(tr->pf_n[k], tr->wi);
      wo_l[3 * k + 0] = dot3(tr->pf_t[k], tr->wo);
      wo_l[3 * k + 1] = dot3(tr->pf_b[k], tr->wo);
      wo_l[3 * k + 2] = dot3(tr->pf_n[k], tr->wo);
    }
  } else if (m->frame_hidden > 0) {
    int H = m->frame_hidden;
    const double* Wf1 = m->frame_params;
    const double* bf1 = Wf1 + H * ORC_C;
    const double* Wf2 = bf1 + H;
    const double* bf2 = Wf2 + 6 * H;
    for (int j = 0; j < H; ++j) {
      double s = bf1[j];
      for (int c = 0; c < ORC_C; ++c) s += Wf1[j * ORC_C + c] * tr->z[c];
      tr->hf_pre[j] = s;
      tr->hf[j] = s > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < 6; ++j) {
      double s = bf2[j];
      for (int k = 0; k < H; ++k) s += Wf2[j * H + k] * tr->hf[k];
      tr->r[j] = s;
    }
    build_frame(tr->r, &tr->fr);
    wi_l[0] = dot3(tr->fr.t, tr->wi); wi_l[1] = dot3(tr->fr.b, tr->wi); wi_l[2] = dot3(tr->fr.n, tr->wi);
    wo_l[0] = dot3(tr->fr.t, tr->wo); wo_l[1] = dot3(tr->fr.b, tr->wo); wo_l[2] = dot3(tr->fr.n, tr->wo);
  } else {
    for (int k = 0; k < 3; ++k) { wi_l[k] = tr->wi[k]; wo_l[k] = tr->wo[k]; }
  }
  /* decoder input order: z0..z7, wi', wo' (paper form: T wi = (t1, b1, n1,
   * t2, b2, n2) . wi, then T wo) */
  double* x = tr->act[0];
  for (int c = 0; c < ORC_C; ++c) x[c] = tr->z[c];
  for (int k = 0; k < nd; ++k) {
    x[ORC_C + k] = wi_l[k];
    x[ORC_C + nd + k] = wo_l[k];
  }

  const double* p = m->dec_params;
  for (int l = 0; l < m->n_layers; ++l) {
    int in = m->widths[l], out = m->widths[l + 1];
    const double* W = p;
    const double* b = p + (int64_t)in * out;
    p = b + out;
    int last = (l == m->n_layers - 1);
    for (int j = 0; j < out; ++j) {
      double s = b[j];
      for (int k = 0; k < in; ++k) s += W[j * in + k] * tr->act[l][k];
      tr->pre[l][j] = s;
      if (!last) tr->act[l + 1][j] = s > 0.0 ? s : 0.0;
    }
  }
  int lastl = m->n_layers - 1;
  tr->cosf = 1.0;
  if (m->out_cosine) tr->cosf = tr->wi[2] > 0.0 ? tr->wi[2] : 0.0;
  for (int c = 0; c < m->widths[m->n_layers]; ++c) tr->y[c] = tr->pre[lastl][c] * (c < 3 ? tr->cosf : 1.0);
}


/* ------------------------------------------------------------------------- */
/* exported batch entry points                                                */
/* ------------------------------------------------------------------------- */
void orc_latent_batch(const orc_model* m, const orc_queries* q, int64_t n, double* z_out) {
  for (int64_t i = 0; i < n; ++i) {
    double xi = q->xi ? q->xi[i] : 0.0;
    latent(m, q->u[i], q->v[i], q->lod[i], xi, z_out + i * ORC_C);
  }
}

/* T rows (t, b, n) for each r = (n_raw, t_raw); out [n][9]. */
void orc_frame_batch(const double* r, int64_t n, double* T_out) {
  for (int64_t i = 0; i < n; ++i) {
    frame_state f;
    build_frame(r + i * 6, &f);
    double* T = T_out + i * 9;
    for (int k = 0; k < 3; ++k) { T[k] = f.t[k]; T[3 + k] = f.b[k]; T[6 + k] = f.n[k]; }
  }
}

/* The decoder MLP alone on given inputs x [n][widths[0]] -> y [n][widths[L]]. */
void orc_mlp_batch(const orc_model* m, const double* x, int64_t n, double* y_out) {
  int outw = m->widths[m->n_layers];
  double a[ORC_MAXW], h[ORC_MAXW];
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < m->widths[0]; ++k) a[k] = x[i * m->widths[0] + k];
    const double* p = m->dec_params;
    for (int l = 0; l < m->n_layers; ++l) {
      int in = m->widths[l], out = m->widths[l + 1];
      const double* W = p;
      const double* b = p + (int64_t)in * out;
      p = b + out;
      for (int j = 0; j < out; ++j) {
        double s = b[j];
        for (int k = 0; k < in; ++k) s += W[j * in + k] * a[k];
        h[j] = (l < m->n_layers - 1) ? (s > 0.0 ? s : 0.0) : s;
      }
      for (int j = 0; j < out; ++j) a[j] = h[j];
    }
    for (int c = 0; c < outw; ++c) y_out[i * outw + c] = a[c];
  }
}

typedef struct {
  const orc_model* m;
  const orc_queries* q;
  int64_t begin, end;
  double* out;
} eval_job;

static void* eval_worker(void* arg) {
  eval_job* j = (eval_job*)arg;
  trace* tr = (trace*)malloc(sizeof(trace));
  for (int64_t i = j->begin; i < j->end; ++i) {
    forward(j->m, j->q, i, tr);
    const int ow = j->m->widths[j->m->n_layers];
    for (int c = 0; c < ow; ++c) j->out[i * ow + c] = tr->y[c];
  }
  free(tr);
  return NULL;
}

/* Full evaluation of n queries -> out [n][widths[n_layers]] (RGB, then the
 * albedo RGB with the albedo head), split over nthreads. */
void orc_eval(const orc_model* m, const orc_queries* q, int64_t n, double* rgb_out, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < 4096) nthreads = 1;
  pthread_t th[256];
  eval_job jobs[256];
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].m = m; jobs[t].q = q; jobs[t].out = rgb_out;
    jobs[t].begin = (int64_t)t * chunk;
    jobs[t].end = jobs[t].begin + chunk < n ? jobs[t].begin + chunk : n;
    if (jobs[t].begin > n) jobs[t].begin = n;
  }
  if (nthreads == 1) { eval_worker(&jobs[0]); return; }
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, eval_worker, &jobs[t]);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* Largest |input| of each decoder layer over a batch (FP64 forward without
 * rounding): the static per-layer activation ranges for FP8 scales. */
void orc_decoder_input_absmax(const orc_model* m, const orc_queries* q, int64_t n, double* amax_out) {
  trace* tr = (trace*)malloc(sizeof(trace));
  for (int l = 0; l < m->n_layers; ++l) amax_out[l] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    forward(m, q, i, tr);
    for (int l = 0; l < m->n_layers; ++l)
      for (int k = 0; k < m->widths[l]; ++k) {
        double a = fabs(tr->act[l][k]);
        if (a > amax_out[l]) amax_out[l] = a;
      }
  }
  free(tr);
}

/* ------------------------------------------------------------------------- */
/* training loss (Sec. 5.2: L1 in log space)                                  */
/* ------------------------------------------------------------------------- */
/* Reading: L = mean |log(1 + max(g,0)) - log(1 + y)| + 0.01 mean max(-g, 0)
 * over the n x 3 outputs; the second term keeps a gradient on negative g.
 * Subgradients: sign(0) = 0, d max(g,0)/dg = 0 at g = 0. */
double orc_loss(const double* g, const float* y, int64_t n, double* dldg_out) {
  double acc = 0.0;
  double inv = 1.0 / (3.0 * (double)n);
  for (int64_t i = 0; i < 3 * n; ++i) {
    double gp = g[i] > 0.0 ? g[i] : 0.0;
    double d = log1p(gp) - log1p((double)y[i]);
    acc += fabs(d);
    double grad = 0.0;
    if (g[i] > 0.0) grad = (d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0)) / (1.0 + g[i]);
    if (g[i] < 0.0) {
      acc += 0.01 * (-g[i]);
      grad += -0.01;
    }
    if (dldg_out) dldg_out[i] = grad * inv;
  }
  return acc * inv;
}

/* Albedo loss (the paper's albedo inference: the extra RGB output is fitted
 * with an L2 loss to one-sample Monte Carlo estimates of the directional
 * albedo of Eq. 2).  Reading: L = mean (a - t)^2 over the n x 3 elements,
 * added to the BRDF loss with weight 1; dL/da = 2 (a - t) / (3 n). */
double orc_albedo_loss(const double* a, const float* t, int64_t n, double* dlda_out) {
  double acc = 0.0;
  double inv = 1.0 / (3.0 * (double)n);
  for (int64_t i = 0; i < 3 * n; ++i) {
    double d = a[i] - (double)t[i];
    acc += d * d;
    if (dlda_out) dlda_out[i] = 2.0 * d * inv;
  }
  return acc * inv;
}

/* ------------------------------------------------------------------------- */
/* reverse mode                                                               */
/* ------------------------------------------------------------------------- */
/* Gradient of sum_i <dl_dy[i], y_i> with respect to the frame MLP parameters,
 * the decoder parameters (same layouts as the model's arrays) and the
 * pyramid ([texel][C]).  Accumulates into the outputs.  Exact derivative of
 * the forward above (no activation rounding), with two readings: ReLU'(0) = 0,
 * and no gradient flows through the degenerate-frame fallbacks (a
 * degenerate n is a constant; the fallback tangent depends on n only).
 * g_z (may be NULL) receives dL/dz per query [n][8] (overwritten, not
 * accumulated): the gradient the encoder of Sec. 5.1 back-propagates. */
void orc_grad(const orc_model* m, const orc_queries* q, int64_t n, const double* dl_dy,
              double* g_frame, double* g_dec, double* g_pyr, double* g_z) {
  if (m->frame_form == 1) return; /* reverse mode of the paper's frame form is not built */
  trace* tr = (trace*)malloc(sizeof(trace));
  double da[ORC_MAXW], dpre[ORC_MAXW];
  for (int64_t i = 0; i < n; ++i) {
    forward(m, q, i, tr);
    int L = m->n_layers;
    /* output */
    const int ow = m->widths[L];
    for (int j = 0; j < ow; ++j) dpre[j] = dl_dy[i * ow + j] * (j < 3 ? tr->cosf : 1.0);
    /* decoder layers, last to first; parameter offsets */
    int64_t offs[ORC_MAXL];
    int64_t o = 0;
    for (int l = 0; l < L; ++l) {
      offs[l] = o;
      o += (int64_t)m->widths[l] * m->widths[l + 1] + m->widths[l + 1];
    }
    for (int l = L - 1; l >= 0; --l) {
      int in = m->widths[l], out = m->widths[l + 1];
      const double* W = m->dec_params + offs[l];
      double* gW = g_dec + offs[l];
      double* gb = gW + (int64_t)in * out;
      for (int j = 0; j < out; ++j) {
        gb[j] += dpre[j];
        for (int k = 0; k < in; ++k) gW[j * in + k] += dpre[j] * tr->act[l][k];
      }
      for (int k = 0; k < in; ++k) {
        double s = 0.0;
        for (int j = 0; j < out; ++j) s += W[j * in + k] * dpre[j];
        da[k] = s;
      }
      if (l > 0)
        for (int k = 0; k < in; ++k) dpre[k] = tr->pre[l - 1][k] > 0.0 ? da[k] : 0.0;
    }
    /* da = dL/dx, x = (z, T wi, T wo) */
    double dz[ORC_C];
    for (int c = 0; c < ORC_C; ++c) dz[c] = da[c];
    if (m->frame_hidden > 0) {
      const double* dwi = da + ORC_C;
      const double* dwo = da + ORC_C + 3;
      frame_state* f = &tr->fr;
      /* rows of T: t, b, n;  x' = T w  =>  dT_row_k += dx'_k * w */
      double dt[3], db[3], dn[3];
      for (int k = 0; k < 3; ++k) {
        dt[k] = dwi[0] * tr->wi[k] + dwo[0] * tr->wo[k];
        db[k] = dwi[1] * tr->wi[k] + dwo[1] * tr->wo[k];
        dn[k] = dwi[2] * tr->wi[k] + dwo[2] * tr->wo[k];
      }
      /* b = c / |c|, c = n x t */
      double bdb = dot3(f->b, db), gc[3], tmp[3];
      for (int k = 0; k < 3; ++k) gc[k] = (db[k] - f->b[k] * bdb) / f->c_len;
      cross3(f->t, gc, tmp);
      for (int k = 0; k < 3; ++k) dn[k] += tmp[k];
      cross3(gc, f->n, tmp);
      for (int k = 0; k < 3; ++k) dt[k] += tmp[k];
      double dr[6] = {0, 0, 0, 0, 0, 0};
      const double* traw = tr->r + 3;
      if (!f->t_degenerate) {
        /* t = t' / |t'|, t' = t_raw - (t_raw.n) n */
        double tdt = dot3(f->t, dt), dtp[3];
        for (int k = 0; k < 3; ++k) dtp[k] = (dt[k] - f->t[k] * tdt) / f->tp_len;
        double ndtp = dot3(f->n, dtp);
        for (int k = 0; k < 3; ++k) {
          dr[3 + k] += dtp[k] - f->n[k] * ndtp;
          dn[k] += -ndtp * traw[k] - f->s * dtp[k];
        }
      }
      if (!f->n_degenerate) {
        double ndn = dot3(f->n, dn);
        for (int k = 0; k < 3; ++k) dr[k] += (dn[k] - f->n[k] * ndn) / f->nraw_len;
      }
      /* frame MLP */
      int H = m->frame_hidden;
      const double* Wf1 = m->frame_params;
      const double* Wf2 = Wf1 + H * ORC_C + H;
      double* gWf1 = g_frame;
      double* gbf1 = gWf1 + H * ORC_C;
      double* gWf2 = gbf1 + H;
      double* gbf2 = gWf2 + 6 * H;
      double dh[ORC_MAXW];
      for (int j = 0; j < 6; ++j) {
        gbf2[j] += dr[j];
        for (int k = 0; k < H; ++k) gWf2[j * H + k] += dr[j] * tr->hf[k];
      }
      for (int k = 0; k < H; ++k) {
        double s = 0.0;
        for (int j = 0; j < 6; ++j) s += Wf2[j * H + k] * dr[j];
        dh[k] = tr->hf_pre[k] > 0.0 ? s : 0.0;
      }
      for (int k = 0; k < H; ++k) {
        gbf1[k] += dh[k];
        for (int c = 0; c < ORC_C; ++c) gWf1[k * ORC_C + c] += dh[k] * tr->z[c];
      }
      for (int c = 0; c < ORC_C; ++c) {
        double s = 0.0;
        for (int k = 0; k < H; ++k) s += Wf1[k * ORC_C + c] * dh[k];
        dz[c] += s;
      }
    }
    /* dL/dz of the query (the encoder's output gradient, Sec. 5.1) */
    if (g_z)
      for (int c = 0; c < ORC_C; ++c) g_z[i * ORC_C + c] = dz[c];
    /* z = sum_k w_k texel_k */
    if (g_pyr)
      for (int k = 0; k < tr->ntaps; ++k)
        for (int c = 0; c < ORC_C; ++c) g_pyr[tr->idx[k] * ORC_C + c] += tr->w[k] * dz[c];
  }
  free(tr);
}

/* Hash (FNV-1a) of the on/off pattern of every ReLU a query passes through
 * (frame hidden layer and decoder hidden layers), one per query.  Finite
 * difference checks use it to skip parameters whose step crosses a kink. */
void orc_relu_pattern(const orc_model* m, const orc_queries* q, int64_t n, uint64_t* out) {
  trace* tr = (trace*)malloc(sizeof(trace));
  for (int64_t i = 0; i < n; ++i) {
    forward(m, q, i, tr);
    uint64_t h = 1469598103934665603ull;
    for (int j = 0; j < m->frame_hidden; ++j) h = (h ^ (uint64_t)(tr->hf_pre[j] > 0.0)) * 1099511628211ull;
    for (int l = 0; l + 1 < m->n_layers; ++l)
      for (int j = 0; j < m->widths[l + 1]; ++j) h = (h ^ (uint64_t)(tr->pre[l][j] > 0.0)) * 1099511628211ull;
    out[i] = h;
  }
  free(tr);
}

/* Condition number of the frame step at each query: how much relative
 * rounding in r = (n_raw, t_raw) is amplified in T.  Each raw vector's
 * relative rounding is bounded by (sum of the magnitudes of the terms that
 * form it) / (its norm); Gram-Schmidt multiplies the tangent's by
 * 1 / sin(angle(n_raw, t_raw)).  kappa = max of the two ratios / sin.  1 when
 * there is no frame MLP.  Used by the parity tests to separate
 * ill-conditioned queries (where any finite-precision evaluation of the
 * method departs from the exact result) from the rest. */
static double frame_kappa(const orc_model* m, const trace* tr) {
  if (m->frame_form == 1) {
    /* each frame: relative rounding of n_raw, t_raw over 1 / sin(n, t) */
    const double* Wf = m->frame_params;
    const double* bf = Wf + 12 * ORC_C;
    double kmax = 1.0;
    for (int k = 0; k < 2; ++k) {
      double a[6];
      for (int j = 0; j < 6; ++j) {
        double s = fabs(bf[6 * k + j]);
        for (int c = 0; c < ORC_C; ++c) s += fabs(Wf[(6 * k + j) * ORC_C + c] * tr->z[c]);
        a[j] = s;
      }
      double An = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      double At = sqrt(a[3] * a[3] + a[4] * a[4] + a[5] * a[5]);
      double rn = An / tr->pf_nl[k], rt = At / tr->pf_tl[k];
      double kk = (rn > rt ? rn : rt) / tr->pf_sin[k];
      if (!isfinite(kk)) kk = 1e300;
      if (kk > kmax) kmax = kk;
    }
    return kmax;
  }
  if (m->frame_hidden <= 0) return 1.0;
  int H = m->frame_hidden;
  const double* Wf1 = m->frame_params;
  const double* Wf2 = Wf1 + H * ORC_C + H;
  const double* bf2 = Wf2 + 6 * H;
  double a[6];
  for (int j = 0; j < 6; ++j) {
    double s = fabs(bf2[j]);
    for (int k = 0; k < H; ++k) s += fabs(Wf2[j * H + k] * tr->hf[k]);
    a[j] = s;
  }
  double An = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double At = sqrt(a[3] * a[3] + a[4] * a[4] + a[5] * a[5]);
  const double* nr = tr->r;
  const double* trr = tr->r + 3;
  double nl = sqrt(dot3(nr, nr)), tl = sqrt(dot3(trr, trr)), c[3];
  cross3(nr, trr, c);
  double sn = sqrt(dot3(c, c)) / (nl * tl);
  double rn = An / nl, rt = At / tl;
  double k = (rn > rt ? rn : rt) / sn;
  return isfinite(k) ? k : 1e300;
}

/* Sensitivity of the decoder's RGB to its direction inputs (the transformed
 * wi', wo': 6 values, 12 in the paper's frame form): for each query and RGB
 * channel c, sum over those inputs k of |d y_c / d x_k|, the Jacobian taken
 * through the query's own ReLU pattern (ReLU'(0) = 0, reading 10) and the
 * cosine factor.  A perturbation of every direction input by at most d moves
 * y_c by at most d times this value (to first order).  Out [n][3]. */
void orc_direction_gain(const orc_model* m, const orc_queries* q, int64_t n, double* gain_out) {
  trace* tr = (trace*)malloc(sizeof(trace));
  const int nd = m->frame_form == 1 ? 6 : 3;
  const int ndir = 2 * nd;
  double J[ORC_MAXW][12], Jn[ORC_MAXW][12];
  for (int64_t i = 0; i < n; ++i) {
    forward(m, q, i, tr);
    const double* p = m->dec_params;
    for (int l = 0; l < m->n_layers; ++l) {
      const int in = m->widths[l], out = m->widths[l + 1];
      const double* W = p;
      p = W + (int64_t)in * out + out;
      for (int j = 0; j < out; ++j)
        for (int k = 0; k < ndir; ++k) {
          double s = 0.0;
          if (l == 0) {
            s = W[j * in + ORC_C + k];
          } else {
            for (int t = 0; t < in; ++t)
              if (tr->pre[l - 1][t] > 0.0) s += W[j * in + t] * J[t][k];
          }
          Jn[j][k] = s;
        }
      for (int j = 0; j < out; ++j)
        for (int k = 0; k < ndir; ++k) J[j][k] = Jn[j][k];
    }
    for (int c = 0; c < 3; ++c) {
      double g = 0.0;
      for (int k = 0; k < ndir; ++k) g += fabs(J[c][k]);
      gain_out[3 * i + c] = g * tr->cosf;
    }
  }
  free(tr);
}

void orc_frame_condition(const orc_model* m, const orc_queries* q, int64_t n, double* kappa_out) {
  trace* tr = (trace*)malloc(sizeof(trace));
  for (int64_t i = 0; i < n; ++i) {
    if (m->frame_hidden <= 0 && m->frame_form != 1) { kappa_out[i] = 1.0; continue; }
    forward(m, q, i, tr);
    kappa_out[i] = frame_kappa(m, tr);
  }
  free(tr);
}

/* ------------------------------------------------------------------------- */
/* importance sampling (Sec. 4.3, Appendix A)                                 */
/* ------------------------------------------------------------------------- */
/* A second MLP maps (z(x), wi) to the nine parameters of an analytic proxy
 * density: a blend of a tilted cosine lobe and a GGX half-vector density with
 * elliptical anisotropy and non-centred mean slopes (Appendix A).
 *
 * Readings where the paper leaves the form open:
 *  - network: input (z0..z7, wi_x, wi_y, wi_z), three ReLU hidden layers of
 *    32, nine linear outputs in the paper's order
 *    (w_d, mu_dx, mu_dy, w_s, alpha_x, alpha_y, rho, mu_sx, mu_sy);
 *  - "quadratic approximations of tanh and sinh": qtanh(x) = x (1 - |x|/4)
 *    for |x| < 2 and sign(x) beyond (odd, C1, onto [-1, 1]); qsinh(x) =
 *    x (1 + |x|/2) (odd, monotonic, unbounded);
 *  - alpha = 1e-3 + (1 - 1e-3) (qtanh + 1) / 2 in [1e-3, 1]; rho = 0.99 qtanh
 *    (so that sqrt(1 - rho^2) > 0); mu = qsinh; (w_d, w_s) = softmax;
 *  - D_std, the unit-roughness GGX density of the standard half-vector
 *    sampling technique, is cos(theta) / pi on the upper hemisphere (at
 *    alpha = 1 the GGX NDF is 1/pi, and the technique draws normals with
 *    density D cos(theta));
 *  - the half vector of the specular pdf is normalize(wi + wo) (zero density
 *    when wi + wo = 0 or when it points below the surface);
 *  - sampling takes three variates: u3 < w_d picks the diffuse lobe; (u1, u2)
 *    drive Malley's cosine mapping (which is also the alpha = 1 GGX normal
 *    sampling); the diffuse lobe is rotated to n_d with the Duff et al. basis;
 *    the returned density is the full mixture density of the sampled wo. */
#define ORC_SAMPLER_IN 11
#define ORC_SAMPLER_H 32
#define ORC_SAMPLER_OUT 9
#define ORC_ALPHA_MIN 1e-3
#define ORC_RHO_MAX 0.99
#define ORC_PI 3.14159265358979323846

double orc_qtanh(double x) {
  double a = fabs(x);
  if (a >= 2.0) return x > 0 ? 1.0 : -1.0;
  return x * (1.0 - a / 4.0);
}
double orc_qsinh(double x) { return x * (1.0 + fabs(x) / 2.0); }

/* Raw network outputs -> the nine proxy parameters. */
void orc_proxy_activate(const double o[9], double p[9]) {
  double mx = o[0] > o[3] ? o[0] : o[3];
  double ed = exp(o[0] - mx), es = exp(o[3] - mx);
  p[0] = ed / (ed + es);
  p[3] = es / (ed + es);
  p[1] = orc_qsinh(o[1]);
  p[2] = orc_qsinh(o[2]);
  p[4] = ORC_ALPHA_MIN + (1.0 - ORC_ALPHA_MIN) * 0.5 * (orc_qtanh(o[4]) + 1.0);
  p[5] = ORC_ALPHA_MIN + (1.0 - ORC_ALPHA_MIN) * 0.5 * (orc_qtanh(o[5]) + 1.0);
  p[6] = ORC_RHO_MAX * orc_qtanh(o[6]);
  p[7] = orc_qsinh(o[7]);
  p[8] = orc_qsinh(o[8]);
}

/* Sampler MLP: weights per layer W[out][in] then b[out], widths 11, 32, 32,
 * 32, 9. */
static void sampler_mlp(const double* sp, const double z[ORC_C], const double wi[3], double o[9]) {
  double x[ORC_SAMPLER_H], y[ORC_SAMPLER_H];
  double in[ORC_SAMPLER_IN];
  for (int c = 0; c < ORC_C; ++c) in[c] = z[c];
  for (int k = 0; k < 3; ++k) in[ORC_C + k] = wi[k];
  const int widths[5] = {ORC_SAMPLER_IN, ORC_SAMPLER_H, ORC_SAMPLER_H, ORC_SAMPLER_H, ORC_SAMPLER_OUT};
  const double* p = sp;
  const double* cur = in;
  for (int l = 0; l < 4; ++l) {
    int ni = widths[l], no = widths[l + 1];
    const double* W = p;
    const double* b = p + ni * no;
    p = b + no;
    double* out = (l == 3) ? o : (l % 2 == 0 ? x : y);
    for (int j = 0; j < no; ++j) {
      double s = b[j];
      for (int k = 0; k < ni; ++k) s += W[j * ni + k] * cur[k];
      out[j] = (l == 3) ? s : (s > 0.0 ? s : 0.0);
    }
    cur = out;
  }
}

static void normalize3(double v[3]) {
  double l = sqrt(dot3(v, v));
  for (int k = 0; k < 3; ++k) v[k] /= l;
}

/* Density of half vectors of the specular lobe (the LTC-style transform of
 * D_std by M, with its Jacobian det(M^-1) / |M^-1 h|^3). */
double orc_proxy_pdf_h(const double p[9], const double h[3]) {
  double ax = p[4], ay = p[5], rho = p[6], msx = p[7], msy = p[8];
  double s = sqrt(1.0 - rho * rho);
  /* v = M^-1 h, M = [[ax, 0, -msx], [ay rho, ay s, -msy], [0, 0, 1]] */
  double v[3];
  v[2] = h[2];
  v[0] = (h[0] + msx * h[2]) / ax;
  v[1] = (h[1] + msy * h[2] - ay * rho * v[0]) / (ay * s);
  double vl = sqrt(dot3(v, v));
  double cz = v[2] / vl;
  if (!(cz > 0.0)) return 0.0;
  double dstd = cz / ORC_PI;
  double detinv = 1.0 / (ax * ay * s);
  return dstd * detinv / (vl * vl * vl);
}

/* Full proxy density of wo given wi (Appendix A, pdf_full / pdf_spec). */
double orc_proxy_pdf(const double p[9], const double wi[3], const double wo[3]) {
  double nd[3] = {-p[1], -p[2], 1.0};
  normalize3(nd);
  double c = dot3(wo, nd);
  double pd = c > 0.0 ? c / ORC_PI : 0.0;
  double h[3] = {wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2]};
  double hl = sqrt(dot3(h, h));
  double ps = 0.0;
  if (hl > 0.0) {
    for (int k = 0; k < 3; ++k) h[k] /= hl;
    double oh = fabs(dot3(wo, h));
    if (oh > 0.0) ps = orc_proxy_pdf_h(p, h) / (4.0 * oh);
  }
  return p[0] * pd + p[3] * ps;
}

static void cosine_dir(double u1, double u2, double d[3]) {
  double r = sqrt(u1), phi = 2.0 * ORC_PI * u2;
  d[0] = r * cos(phi);
  d[1] = r * sin(phi);
  d[2] = sqrt(1.0 - u1 > 0.0 ? 1.0 - u1 : 0.0);
}

/* Sample transform W(u; wi) of the proxy (Appendix A, Sampling). */
void orc_proxy_sample(const double p[9], const double wi[3], const double u[3], double wo[3], double* pdf) {
  double l[3];
  cosine_dir(u[0], u[1], l);
  if (u[2] < p[0]) {
    double nd[3] = {-p[1], -p[2], 1.0}, t[3], b[3];
    normalize3(nd);
    basis_tangent(nd, t);
    cross3(nd, t, b);
    for (int k = 0; k < 3; ++k) wo[k] = t[k] * l[0] + b[k] * l[1] + nd[k] * l[2];
  } else {
    double ax = p[4], ay = p[5], rho = p[6], msx = p[7], msy = p[8];
    double s = sqrt(1.0 - rho * rho);
    double h[3] = {ax * l[0] - msx * l[2], ay * rho * l[0] + ay * s * l[1] - msy * l[2], l[2]};
    normalize3(h);
    double d = dot3(wi, h);
    for (int k = 0; k < 3; ++k) wo[k] = 2.0 * d * h[k] - wi[k];
  }
  *pdf = orc_proxy_pdf(p, wi, wo);
}

/* Per query: z from the latent pyramid as for the decoder, then the sampler
 * network and its activations.  params_out [n][9]. */
void orc_sampler_params(const orc_model* m, const double* sp, const orc_queries* q, int64_t n, double* params_out) {
  for (int64_t i = 0; i < n; ++i) {
    double z[ORC_C], o[9];
    double xi = q->xi ? q->xi[i] : 0.0;
    latent(m, q->u[i], q->v[i], q->lod[i], xi, z);
    double wi[3] = {q->wix[i], q->wiy[i], q->wiz[i]};
    sampler_mlp(sp, z, wi, o);
    orc_proxy_activate(o, params_out + i * 9);
  }
}

/* Proxy density of each query's wo given its wi; pdf_out [n]. */
void orc_sampler_pdf(const orc_model* m, const double* sp, const orc_queries* q, int64_t n, double* pdf_out) {
  for (int64_t i = 0; i < n; ++i) {
    double p[9], z[ORC_C], o[9];
    double xi = q->xi ? q->xi[i] : 0.0;
    latent(m, q->u[i], q->v[i], q->lod[i], xi, z);
    double wi[3] = {q->wix[i], q->wiy[i], q->wiz[i]};
    double wo[3] = {q->wox[i], q->woy[i], q->woz[i]};
    sampler_mlp(sp, z, wi, o);
    orc_proxy_activate(o, p);
    pdf_out[i] = orc_proxy_pdf(p, wi, wo);
  }
}

/* One sample per query from variates u [n][3]: wo_out [n][3], pdf_out [n]. */
void orc_sampler_sample(const orc_model* m, const double* sp, const orc_queries* q, int64_t n, const double* u,
                        double* wo_out, double* pdf_out) {
  for (int64_t i = 0; i < n; ++i) {
    double p[9], z[ORC_C], o[9];
    double xi = q->xi ? q->xi[i] : 0.0;
    latent(m, q->u[i], q->v[i], q->lod[i], xi, z);
    double wi[3] = {q->wix[i], q->wiy[i], q->wiz[i]};
    sampler_mlp(sp, z, wi, o);
    orc_proxy_activate(o, p);
    orc_proxy_sample(p, wi, u + i * 3, wo_out + i * 3, pdf_out + i);
  }
}

/* Batch forms for quadrature: out[k] = pdf of wo[k] given wi, and the
 * half-vector density at h[k]. */
void orc_proxy_pdf_batch(const double p[9], const double wi[3], const double* wo, int64_t n, double* out) {
  for (int64_t k = 0; k < n; ++k) out[k] = orc_proxy_pdf(p, wi, wo + 3 * k);
}
void orc_proxy_pdf_h_batch(const double p[9], const double* h, int64_t n, double* out) {
  for (int64_t k = 0; k < n; ++k) out[k] = orc_proxy_pdf_h(p, h + 3 * k);
}
