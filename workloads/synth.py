"""Seeded synthetic inputs with the shapes of the paper's workloads.

The paper's assets (layered MaterialX materials, trained latents and weights)
are not available, so every input here is synthetic.  The recipe:

* latent pyramids: every texel of every level an independent N(0, 0.5) draw
  (levels of a learned pyramid are optimised independently, Sec. 4.1), packed
  level after level, 8 channels per texel;
* MLP weights: Glorot-uniform U(+-sqrt(6/(fan_in+fan_out))), biases U(+-0.1),
  stored [out][in] row-major, FP32 masters;
* queries: either uniform (uv ~ U[0,1)^2, lod ~ U[0, lod_max]) or one query per
  pixel of a frame whose uv come from a smooth random warp, with lod taken from
  the area of the warp's pixel footprint (Sec. 4.1, footprint-area LOD);
* directions: cosine-weighted hemisphere (Malley's method) in the geometric
  frame, z up; xi ~ U[0,1) for the stochastic level choice;
* training targets: a procedural GGX-over-Lambert BRDF whose albedo and
  roughness vary over uv with gradient noise.

Query arrays are float32 and planar: one array per field.  Nothing in this
module evaluates the neural BRDF.
"""
from __future__ import annotations

import math

import numpy as np

CHANNELS = 8

#: one seed per workload: 1 = FP32 small, 2 = FP16 1080p, 3 = 4K sweep,
#: 4 = training, 5 = serving
SEEDS = {1: 2305026781, 2: 2305026782, 3: 2305026783, 4: 2305026784, 5: 2305026785}

QUERY_FIELDS = ("u", "v", "lod", "wix", "wiy", "wiz", "wox", "woy", "woz", "xi")


def rng_streams(seed: int, n: int):
    """n independent PCG64 generators derived from one seed."""
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(seed).spawn(n)]


# ----------------------------------------------------------------------------
# latent pyramid
# ----------------------------------------------------------------------------
def pyramid_texel_count(W0: int, H0: int, L: int) -> int:
    """Texels in a packed pyramid whose level l is max(1, W0>>l) x max(1, H0>>l)."""
    return sum(max(1, W0 >> l) * max(1, H0 >> l) for l in range(L))


def make_pyramid(rng, W0: int, H0: int, L: int, dtype=np.float16, std: float = 0.5):
    """[texels, 8] array of independent N(0, std) latents, levels packed in order."""
    n = pyramid_texel_count(W0, H0, L)
    x = rng.standard_normal((n, CHANNELS), dtype=np.float32)
    x *= np.float32(std)
    return x.astype(dtype, copy=False)


# ----------------------------------------------------------------------------
# weights
# ----------------------------------------------------------------------------
def glorot_layer(rng, fan_in: int, fan_out: int, bias_range: float = 0.1):
    lim = math.sqrt(6.0 / (fan_in + fan_out))
    W = rng.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32)
    b = rng.uniform(-bias_range, bias_range, size=fan_out).astype(np.float32)
    return W, b


def make_mlp(rng, widths):
    """List of (W [out][in], b [out]) float32 pairs for consecutive widths."""
    return [glorot_layer(rng, widths[i], widths[i + 1]) for i in range(len(widths) - 1)]


def make_model(rng, decoder_widths=(14, 64, 64, 3), frame_widths=(8, 16, 6)):
    """A random neural material: optional frame MLP and the decoder MLP."""
    frame = make_mlp(rng, frame_widths) if frame_widths is not None else None
    return {"frame": frame, "decoder": make_mlp(rng, decoder_widths)}


# ----------------------------------------------------------------------------
# queries
# ----------------------------------------------------------------------------
def cosine_hemisphere(rng, n: int) -> np.ndarray:
    """[3, n] float64 directions, pdf cos(theta)/pi (Malley's method)."""
    r1 = rng.random(n)
    r2 = rng.random(n)
    s = np.sqrt(r1)
    phi = 2.0 * np.pi * r2
    return np.stack([s * np.cos(phi), s * np.sin(phi), np.sqrt(1.0 - r1)])


def _pack(u, v, lod, wi, wo, xi):
    f = np.float32
    q = {"u": u.astype(f), "v": v.astype(f), "lod": lod.astype(f),
         "wix": wi[0].astype(f), "wiy": wi[1].astype(f), "wiz": wi[2].astype(f),
         "wox": wo[0].astype(f), "woy": wo[1].astype(f), "woz": wo[2].astype(f),
         "xi": xi.astype(f)}
    return {k: np.ascontiguousarray(a) for k, a in q.items()}


def uniform_queries(rng, n: int, lod_max: float):
    """uv ~ U[0,1)^2, lod ~ U[0, lod_max], cosine-hemisphere wi/wo, xi ~ U[0,1)."""
    u = rng.random(n)
    v = rng.random(n)
    lod = rng.uniform(0.0, lod_max, n)
    wi = cosine_hemisphere(rng, n)
    wo = cosine_hemisphere(rng, n)
    xi = rng.random(n)
    return _pack(u, v, lod, wi, wo, xi)


class SmoothWarp:
    """A random smooth map from pixel coordinates to uv.

    p = pixel / width (aspect kept).  A slowly varying zoom
    m(p) = (width / W0) * 2**(6 s(p)), s = 1/2 + 1/2 sin(2 pi <k0, p> + phi0),
    spans one texel per pixel (s = 0) to 64 texels per pixel (s = 1), and four
    small sinusoidal displacements bend the grid:
    uv = 1/2 + (p - 1/2) m(p) + sum_k a_k sin(2 pi <k_k, p> + phi_k) e_k.
    """

    def __init__(self, rng, width: int, W0: int):
        self.width = float(width)
        self.zoom0 = float(width) / float(W0)
        sgn = lambda: rng.choice([-1, 1], size=2)
        self.k0 = rng.integers(1, 4, size=2) * sgn()
        self.phi0 = rng.uniform(0.0, 2.0 * np.pi)
        self.k = [rng.integers(1, 4, size=2) * sgn() for _ in range(4)]
        self.a = rng.uniform(0.0, 0.02, size=4)
        self.phi = rng.uniform(0.0, 2.0 * np.pi, size=4)
        ang = rng.uniform(0.0, 2.0 * np.pi, size=4)
        self.e = np.stack([np.cos(ang), np.sin(ang)], axis=1)

    def __call__(self, px, py):
        p0 = px / self.width
        p1 = py / self.width
        s = 0.5 + 0.5 * np.sin(2 * np.pi * (self.k0[0] * p0 + self.k0[1] * p1) + self.phi0)
        m = self.zoom0 * np.exp2(6.0 * s)
        u = 0.5 + (p0 - 0.5) * m
        v = 0.5 + (p1 - 0.5) * m
        for k, a, ph, e in zip(self.k, self.a, self.phi, self.e):
            w = a * np.sin(2 * np.pi * (k[0] * p0 + k[1] * p1) + ph)
            u = u + w * e[0]
            v = v + w * e[1]
        return u, v


def footprint_lod(warp, px, py, W0: int, H0: int):
    """lod = 1/2 log2(|det J| W0 H0), J = d(uv)/d(pixel) by central differences
    at +-1 pixel: the level whose texel area matches the pixel footprint area."""
    ux1, vx1 = warp(px + 1.0, py)
    ux0, vx0 = warp(px - 1.0, py)
    uy1, vy1 = warp(px, py + 1.0)
    uy0, vy0 = warp(px, py - 1.0)
    jxx = 0.5 * (ux1 - ux0)
    jyx = 0.5 * (vx1 - vx0)
    jxy = 0.5 * (uy1 - uy0)
    jyy = 0.5 * (vy1 - vy0)
    det = np.abs(jxx * jyy - jxy * jyx)
    return 0.5 * np.log2(np.maximum(det * float(W0) * float(H0), 1e-30))


def frame_pixels(width: int, height: int, order: str = "row", tile: int = 64):
    """Pixel-centre coordinates of a frame, row-major or 64x64-tile-major."""
    if order == "row":
        yy, xx = np.divmod(np.arange(width * height, dtype=np.int64), width)
    elif order == "tile":
        xx, yy = tile_major_pixels(width, height, tile)
    else:
        raise ValueError(order)
    return xx.astype(np.float64) + 0.5, yy.astype(np.float64) + 0.5


def tile_major_pixels(width: int, height: int, tile: int = 64):
    """(x, y) of every pixel, tile by tile (tiles row-major, pixels row-major
    inside a tile; edge tiles are ragged)."""
    xs, ys = [], []
    for ty in range(0, height, tile):
        for tx in range(0, width, tile):
            h = min(tile, height - ty)
            w = min(tile, width - tx)
            yy, xx = np.divmod(np.arange(w * h, dtype=np.int64), w)
            xs.append(xx + tx)
            ys.append(yy + ty)
    return np.concatenate(xs), np.concatenate(ys)


def tile_ranges(width: int, height: int, tile: int = 64):
    """(start, count) of each tile's queries in tile-major order."""
    out, start = [], 0
    for ty in range(0, height, tile):
        for tx in range(0, width, tile):
            c = min(tile, width - tx) * min(tile, height - ty)
            out.append((start, c))
            start += c
    return out


def warp_queries(rng, width: int, height: int, W0: int, H0: int, order: str = "row"):
    """One query per pixel: uv from a random smooth warp, lod from its footprint,
    cosine-hemisphere wi/wo, xi ~ U[0,1)."""
    warp = SmoothWarp(rng, width, W0)
    px, py = frame_pixels(width, height, order)
    u, v = warp(px, py)
    lod = footprint_lod(warp, px, py, W0, H0)
    n = px.size
    wi = cosine_hemisphere(rng, n)
    wo = cosine_hemisphere(rng, n)
    xi = rng.random(n)
    return _pack(u, v, lod, wi, wo, xi)


def slice_queries(q, start: int, count: int):
    return {k: np.ascontiguousarray(a[start:start + count]) for k, a in q.items()}


# ----------------------------------------------------------------------------
# procedural training target (GGX specular over Lambertian, noise-textured)
# ----------------------------------------------------------------------------
class GradientNoise2D:
    """Periodic 2D gradient noise (Perlin's construction: random unit gradients
    on an integer lattice, quintic fade 6t^5 - 15t^4 + 10t^3, bilinear blend of
    the corner ramps), summed over octaves.  Period 1 in uv."""

    def __init__(self, rng, base_freq: int = 4, octaves: int = 3):
        self.freqs = [base_freq << o for o in range(octaves)]
        self.grads = []
        for f in self.freqs:
            ang = rng.uniform(0.0, 2.0 * np.pi, size=(f, f))
            self.grads.append(np.stack([np.cos(ang), np.sin(ang)], axis=-1))

    @staticmethod
    def _fade(t):
        return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)

    def __call__(self, u, v):
        total = np.zeros_like(u, dtype=np.float64)
        amp = 1.0
        for f, g in zip(self.freqs, self.grads):
            x = np.mod(u, 1.0) * f
            y = np.mod(v, 1.0) * f
            i0 = np.floor(x).astype(np.int64)
            j0 = np.floor(y).astype(np.int64)
            dx = x - i0
            dy = y - j0
            acc = 0.0
            for oi in (0, 1):
                for oj in (0, 1):
                    gi = g[(j0 + oj) % f, (i0 + oi) % f]
                    ramp = gi[..., 0] * (dx - oi) + gi[..., 1] * (dy - oj)
                    wx = self._fade(dx) if oi else 1.0 - self._fade(dx)
                    wy = self._fade(dy) if oj else 1.0 - self._fade(dy)
                    acc = acc + wx * wy * ramp
            total += amp * acc
            amp *= 0.5
        return total


class ProceduralBRDF:
    """f = a(x)/pi + D G2 F / (4 cos_i cos_o): isotropic GGX (alpha = r^2),
    height-correlated Smith G2, Schlick Fresnel with F0 = 0.04, zero below the
    horizon.  a (RGB) in [0.05, 0.95] and r in [0.05, 1] come from four seeded
    gradient-noise fields over uv."""

    def __init__(self, rng):
        self.albedo_fields = [GradientNoise2D(rng) for _ in range(3)]
        self.rough_field = GradientNoise2D(rng)

    @staticmethod
    def _to_range(n, lo, hi):
        return lo + (hi - lo) * 0.5 * (1.0 + np.tanh(2.0 * n))

    def params(self, u, v):
        a = np.stack([self._to_range(f(u, v), 0.05, 0.95) for f in self.albedo_fields], axis=-1)
        r = self._to_range(self.rough_field(u, v), 0.05, 1.0)
        return a, r

    def __call__(self, u, v, wi, wo):
        """wi, wo: [3, n] float64.  Returns [n, 3] float64."""
        return self.from_params(*self.params(u, v), wi, wo)

    @staticmethod
    def ggx_ndf(alpha, cos_h):
        """Isotropic GGX (Trowbridge-Reitz) normal distribution D(h) for the
        cosine of the half vector with the normal."""
        a2 = alpha * alpha
        return a2 / (np.pi * (cos_h * cos_h * (a2 - 1.0) + 1.0) ** 2)

    @staticmethod
    def smith_lambda(alpha, cos_t):
        """Smith's Lambda of the GGX distribution for a direction at cos_t
        from the normal: (-1 + sqrt(1 + alpha^2 tan^2)) / 2."""
        c = np.clip(cos_t, 1e-12, 1.0)
        tan2 = (1.0 - c * c) / (c * c)
        return 0.5 * (-1.0 + np.sqrt(1.0 + alpha * alpha * tan2))

    @staticmethod
    def schlick(f0, cos_d):
        """Schlick's Fresnel approximation."""
        return f0 + (1.0 - f0) * (1.0 - cos_d) ** 5

    @staticmethod
    def from_params(a, r, wi, wo):
        """The BRDF for albedo a [n, 3] and roughness r [n]."""
        P = ProceduralBRDF
        alpha = r * r
        ci, co = wi[2], wo[2]
        h = wi + wo
        h = h / np.maximum(np.linalg.norm(h, axis=0), 1e-300)
        D = P.ggx_ndf(alpha, h[2])
        G2 = 1.0 / (1.0 + P.smith_lambda(alpha, ci) + P.smith_lambda(alpha, co))  # height-correlated
        F = P.schlick(0.04, np.clip(np.sum(wi * h, axis=0), 0.0, 1.0))
        denom = np.maximum(4.0 * ci * co, 1e-12)
        spec = D * G2 * F / denom
        f = a / np.pi + spec[:, None]
        ok = (ci > 0.0) & (co > 0.0)
        return np.where(ok[:, None], f, 0.0)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------
def workload(i: int, scale: float = 1.0):
    """Inputs of workload i (see module docstring).  `scale` < 1 shrinks the
    query count (not the pyramid) for quick tests."""
    seed = SEEDS[i]
    r_pyr, r_w, r_q, r_t = rng_streams(seed, 4)
    if i == 1:
        W0 = H0 = 256
        L = 9
        pyr = make_pyramid(r_pyr, W0, H0, L, dtype=np.float32)
        model = make_model(r_w, (14, 32, 32, 3), None)
        n = max(1, int(65536 * scale))
        q = uniform_queries(r_q, n, 8.0)
        return dict(W0=W0, H0=H0, L=L, pyramid=pyr, model=model, queries=q, name="fp32-256sq-65536q")
    if i in (2, 3):
        W0 = H0 = 2048
        L = 12
        pyr = make_pyramid(r_pyr, W0, H0, L, dtype=np.float16)
        model = make_model(r_w, (14, 64, 64, 3), (8, 16, 6))
        width, height = (1920, 1080) if i == 2 else (3840, 2160)
        if scale != 1.0:
            height = max(1, int(round(height * scale)))
        q = warp_queries(r_q, width, height, W0, H0)
        return dict(W0=W0, H0=H0, L=L, pyramid=pyr, model=model, queries=q,
                    width=width, height=height,
                    name=f"fp16-2048sq-{width}x{height}")
    if i == 4:
        W0 = H0 = 1024
        L = 11
        pyr = make_pyramid(r_pyr, W0, H0, L, dtype=np.float32)
        model = make_model(r_w, (14, 64, 64, 3), (8, 16, 6))
        n = max(1, int(262144 * scale))
        q = uniform_queries(r_q, n, 10.0)
        target = ProceduralBRDF(r_t)
        return dict(W0=W0, H0=H0, L=L, pyramid=pyr, model=model, queries=q,
                    target=target, name="train-1024sq-262144")
    raise ValueError(f"workload {i}")


def calibration_queries(i: int, n_side: int = 256):
    """A calibration batch for static FP8 activation scales: n_side^2 (65,536)
    queries of workload i's kind (warp frame for 2 and 3, uniform otherwise)
    drawn from seed + 1000, so that it is disjoint from the evaluated batch."""
    r = rng_streams(SEEDS[i] + 1000, 1)[0]
    if i in (2, 3):
        return warp_queries(r, n_side, n_side, 2048, 2048)
    return uniform_queries(r, n_side * n_side, {1: 8.0, 4: 10.0}[i])


def target_rgb(target: ProceduralBRDF, q) -> np.ndarray:
    """[n, 3] float32 procedural BRDF values at the queries' uv and directions."""
    wi = np.stack([q["wix"], q["wiy"], q["wiz"]]).astype(np.float64)
    wo = np.stack([q["wox"], q["woy"], q["woz"]]).astype(np.float64)
    return target(q["u"].astype(np.float64), q["v"].astype(np.float64), wi, wo).astype(np.float32)


def albedo_targets(rng, target: ProceduralBRDF, q) -> np.ndarray:
    """[n, 3] float32 one-sample Monte Carlo estimates of the procedural
    material's directional albedo (Eq. 2: the integral over the upper
    hemisphere of f(x, wi, wo) cos(theta_i)) at each query's uv and wo: wi
    drawn cosine-weighted (pdf cos(theta_i) / pi), so the estimate is
    pi f(x, wi, wo).  The training data of the albedo head."""
    n = q["u"].shape[0]
    wi = cosine_hemisphere(rng, n)
    wo = np.stack([q["wox"], q["woy"], q["woz"]]).astype(np.float64)
    f = target(q["u"].astype(np.float64), q["v"].astype(np.float64), wi, wo)
    return (np.pi * f).astype(np.float32)


def material_attributes(target: ProceduralBRDF, q) -> np.ndarray:
    """[n, 4] float32 material parameters k(x) = (albedo RGB, roughness) of the
    procedural material at the queries' uv: the encoder's inputs."""
    a, r = target.params(q["u"].astype(np.float64), q["v"].astype(np.float64))
    return np.concatenate([a, r[:, None]], axis=1).astype(np.float32)


def texel_attributes(target: ProceduralBRDF, W0: int, H0: int, L: int) -> np.ndarray:
    """[texels, 4] float32 material parameters for every texel of an L-level
    pyramid, levels packed finest first: level 0 at the texel centres,
    each coarser level the mean of its 2x2 (or 2x1) finer texels (the
    prefiltered parameters the encoder maps to the coarse latents)."""
    xs, ys = np.meshgrid(np.arange(W0), np.arange(H0))
    u = (xs.ravel() + 0.5) / W0
    v = (ys.ravel() + 0.5) / H0
    a, r = target.params(u, v)
    lvl = np.concatenate([a, r[:, None]], axis=1).reshape(H0, W0, 4)
    out = [lvl.reshape(-1, 4)]
    w, h = W0, H0
    for _ in range(1, L):
        w2, h2 = max(1, w // 2), max(1, h // 2)
        fx, fy = w // w2, h // h2
        lvl = lvl.reshape(h2, fy, w2, fx, 4).mean(axis=(1, 3))
        out.append(lvl.reshape(-1, 4))
        w, h = w2, h2
    return np.concatenate(out).astype(np.float32)


def filtered_targets(rng, target: ProceduralBRDF, q, W0: int, max_samples: int = 8):
    """Footprint-filtered training data for queries q (the data generation of
    the paper's training, as this module reads it): a query at lod l stands
    for a Gaussian footprint of standard deviation 2^l / (2 W0) in uv; its
    target is the mean of the procedural BRDF, and its material parameters
    the mean of (albedo RGB, roughness), over m = min(max_samples, ceil(4^l))
    points drawn from that Gaussian (one point, the query itself, at lod 0),
    uv wrapped.  Returns (target [n, 3] float32, attributes [n, 4] float32)."""
    n = q["u"].shape[0]
    lod = q["lod"].astype(np.float64)
    m = np.minimum(max_samples, np.ceil(4.0 ** lod)).astype(np.int64)
    sigma = np.exp2(lod) / (2.0 * W0)
    S = max_samples
    off = rng.normal(size=(2, S, n)) * sigma[None, None, :]
    off[:, 0, m == 1] = 0.0
    us = np.mod(q["u"].astype(np.float64)[None, :] + off[0], 1.0)
    vs = np.mod(q["v"].astype(np.float64)[None, :] + off[1], 1.0)
    take = np.arange(S)[:, None] < m[None, :]            # [S, n]
    wi = np.stack([q["wix"], q["wiy"], q["wiz"]]).astype(np.float64)
    wo = np.stack([q["wox"], q["woy"], q["woz"]]).astype(np.float64)
    a, r = target.params(us.ravel(), vs.ravel())
    f = target.from_params(a, r, np.tile(wi, S), np.tile(wo, S)).reshape(S, n, 3)
    k = np.concatenate([a, r[:, None]], axis=1).reshape(S, n, 4)
    w = take / m[None, :]
    y = np.einsum("sn,snc->nc", w, f)
    attrs = np.einsum("sn,snc->nc", w, k)
    return y.astype(np.float32), attrs.astype(np.float32)
