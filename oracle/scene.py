"""FP64 numpy version of the synthetic-scene harness (ground plane and
spheres seen by a pinhole camera; a path tracer lit by a constant sky: at
every vertex one BSDF sample and one cosine-weighted light sample combined by
the power heuristic, Veach 1995, with analytic shadow rays, the path going on
along the BSDF sample).  The neural material's
evaluation, sampling and densities come from the FP64 oracle (oracle.py).

TEST INFRASTRUCTURE: only the tests import this module.  It shares nothing
with the CUDA path.

Geometry (the harness's definition): ground plane y = ground_y with normal
+y, tangent +x, uv = (x, z) / ground_uv_scale; spheres with n = (p - c) / r,
uv = (atan2(n_z, n_x) / 2 pi + 1/2, acos(n_y) / pi), tangent along +phi
((-n_z, 0, n_x) normalised; +x at the poles); b = n x t.  Ray-cone level of
detail: lod = log2(w / max(|cos|, 0.05) * s * W0), w the cone width (2
tan(fov/2) / height times the distance travelled along the path), s = 1 /
ground_uv_scale on the ground, 1 / (pi sqrt(2) r) on a sphere.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

EPS = 1e-4


def camera(scene):
    eye = np.asarray(scene["eye"], np.float64)
    fwd = np.asarray(scene["target"], np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(scene["up"], np.float64))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return eye, fwd, right, up


def primary_rays(scene):
    """Unit directions [W*H, 3] through the pixel centres, row-major from the top-left."""
    W, H = scene["width"], scene["height"]
    eye, fwd, right, up = camera(scene)
    th = np.tan(0.5 * scene["fov_y"])
    px, py = np.meshgrid(np.arange(W), np.arange(H))
    x = (2.0 * (px.ravel() + 0.5) / W - 1.0) * th * (W / H)
    y = (1.0 - 2.0 * (py.ravel() + 0.5) / H) * th
    d = fwd[None, :] + x[:, None] * right[None, :] + y[:, None] * up[None, :]
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def intersect(scene, o, d, tmin=EPS):
    """Closest hit beyond tmin of rays o + t d: (t, material, primitive), t =
    inf and material -1 on a miss, primitive -1 for the ground."""
    n = d.shape[0]
    o = np.broadcast_to(np.asarray(o, np.float64), (n, 3))
    best = np.full(n, np.inf)
    mat = np.full(n, -1, np.int64)
    prim = np.full(n, -2, np.int64)
    if scene.get("ground_material", -1) >= 0:
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (scene["ground_y"] - o[:, 1]) / d[:, 1]
        ok = (np.abs(d[:, 1]) > 1e-12) & (t > tmin) & (t < best)
        best[ok], mat[ok], prim[ok] = t[ok], scene["ground_material"], -1
    for s, (cx, cy, cz, r, m) in enumerate(scene["spheres"]):
        oc = o - np.array([cx, cy, cz])
        b = np.sum(oc * d, axis=1)
        c = np.sum(oc * oc, axis=1) - r * r
        disc = b * b - c
        q = np.sqrt(np.maximum(disc, 0.0))
        t = np.where(-b - q > tmin, -b - q, -b + q)
        ok = (disc >= 0.0) & (t > tmin) & (t < best)
        best[ok], mat[ok], prim[ok] = t[ok], m, s
    return best, mat, prim


def surface(scene, prim, p):
    """Shading frames [n, 3, 3] (rows t, b, n), u, v and the world-to-uv scale."""
    n = p.shape[0]
    N = np.zeros((n, 3))
    T = np.zeros((n, 3))
    u = np.zeros(n)
    v = np.zeros(n)
    s = np.zeros(n)
    g = prim == -1
    if np.any(g):
        inv = 1.0 / scene["ground_uv_scale"]
        N[g] = [0.0, 1.0, 0.0]
        T[g] = [1.0, 0.0, 0.0]
        u[g] = p[g, 0] * inv
        v[g] = p[g, 2] * inv
        s[g] = inv
    for k, (cx, cy, cz, r, _) in enumerate(scene["spheres"]):
        sel = prim == k
        if not np.any(sel):
            continue
        nn = (p[sel] - np.array([cx, cy, cz])) / r
        nn /= np.linalg.norm(nn, axis=1, keepdims=True)
        N[sel] = nn
        h = np.sqrt(nn[:, 0] ** 2 + nn[:, 2] ** 2)
        tt = np.stack([-nn[:, 2], np.zeros(len(nn)), nn[:, 0]], axis=1)
        pole = h * h <= 1e-12
        tt[~pole] /= h[~pole, None]
        tt[pole] = [1.0, 0.0, 0.0]
        T[sel] = tt
        u[sel] = np.arctan2(nn[:, 2], nn[:, 0]) / (2 * np.pi) + 0.5
        v[sel] = np.arccos(np.clip(nn[:, 1], -1.0, 1.0)) / np.pi
        s[sel] = 1.0 / (np.pi * np.sqrt(2.0) * r)
    B = np.cross(N, T)
    return np.stack([T, B, N], axis=1), u, v, s


def _vertices(scene, o, d, cone_before, lod_base_width):
    """Surface data where rays (o, d) first hit; cone width at the hit =
    cone_before + spread * t."""
    t, mat, prim = intersect(scene, o, d)
    hit = mat >= 0
    n = d.shape[0]
    o = np.broadcast_to(np.asarray(o, np.float64), (n, 3))
    out = {"material": mat, "t": t, "u": np.zeros(n), "v": np.zeros(n), "lod": np.zeros(n),
           "frame": np.zeros((n, 3, 3)), "view": np.zeros((n, 3)), "dir": d, "pos": np.zeros((n, 3)),
           "cone": np.zeros(n)}
    p = o[hit] + t[hit, None] * d[hit]
    F, u, v, s = surface(scene, prim[hit], p)
    cosv = np.abs(np.sum(F[:, 2, :] * d[hit], axis=1))
    spread = 2.0 * np.tan(0.5 * scene["fov_y"]) / scene["height"]
    cone = cone_before[hit] + spread * t[hit]
    fp = cone / np.maximum(cosv, 0.05) * s * lod_base_width
    out["u"][hit], out["v"][hit] = u, v
    out["lod"][hit] = np.log2(np.maximum(fp, 1e-6))
    out["frame"][hit] = F
    out["view"][hit] = np.einsum("nij,nj->ni", F, -d[hit])
    out["pos"][hit] = p
    out["cone"][hit] = cone
    return out


def gbuffer(scene, lod_base_width):
    d = primary_rays(scene)
    return _vertices(scene, camera(scene)[0], d, np.zeros(d.shape[0]), lod_base_width)


def _queries(u, v, lod, wi, wo):
    f = np.float32
    n = len(u)
    return {"u": u.astype(f), "v": v.astype(f), "lod": lod.astype(f), "xi": np.full(n, 0.5, f),
            "wix": wi[:, 0].astype(f), "wiy": wi[:, 1].astype(f), "wiz": wi[:, 2].astype(f),
            "wox": wo[:, 0].astype(f), "woy": wo[:, 1].astype(f), "woz": wo[:, 2].astype(f)}


def render_paths(scene, models, samplers, variates, lod_base_width, bounces):
    """Image [W*H, 3]: sky radiance where the primary ray leaves the scene;
    elsewhere the sum over the path's vertices (at most `bounces`) of its
    throughput times the two-sample MIS estimate of sky light there.
    models[k]: oracle.Model of material k (out_cosine set: the evaluation
    includes max(0, wi.z)); samplers[k]: its sampler layers; variates
    [bounces][pixels][5]."""
    g = gbuffer(scene, lod_base_width)
    L = scene["sky_radiance"]
    n = len(g["material"])
    rad = np.zeros((n, 3))
    rad[g["material"] < 0] = L
    thr = np.ones((n, 3))
    var = np.asarray(variates, np.float64).reshape(bounces, n, 5)
    for b in range(bounces):
        more = b + 1 < bounces
        ro = np.zeros((n, 3))
        rd = np.full((n, 3), np.nan)
        for k, (model, smp) in enumerate(zip(models, samplers)):
            idx = np.nonzero(g["material"] == k)[0]
            if idx.size == 0:
                continue
            u, v, lod, view = g["u"][idx], g["v"][idx], g["lod"][idx], g["view"][idx]
            r = var[b, idx]
            # light sample: cosine-weighted about the shading normal
            phi = 2.0 * np.pi * r[:, 4]
            dl = np.stack([np.sqrt(r[:, 3]) * np.cos(phi), np.sqrt(r[:, 3]) * np.sin(phi),
                           np.sqrt(np.maximum(1.0 - r[:, 3], 0.0))], axis=1)
            q = _queries(u, v, lod, view, dl)
            db, pb = O.sampler_sample(model, smp, q, r[:, :3])
            pbl = O.sampler_pdf(model, smp, q)
            f_b = O.eval(model, _queries(u, v, lod, db, view))
            f_l = O.eval(model, _queries(u, v, lod, dl, view))
            F = g["frame"][idx]
            off = 1e-3 * np.maximum(1.0, g["t"][idx])
            o = g["pos"][idx] + off[:, None] * F[:, 2, :]
            c = np.zeros((idx.size, 3))
            for dloc, f, own, p_b, p_l in ((db, f_b, pb, pb, np.maximum(db[:, 2], 0.0) / np.pi),
                                           (dl, f_l, dl[:, 2] / np.pi, pbl, dl[:, 2] / np.pi)):
                up = dloc[:, 2] > 0.0
                dw = np.einsum("nji,nj->ni", F, dloc)
                _, m_hit, _ = intersect(scene, o, dw)
                ok = up & (own > 0.0) & (m_hit < 0)
                w = np.where(ok, own * own / np.where(ok, p_b * p_b + p_l * p_l, 1.0), 0.0)
                a = np.where(ok, L * w / np.where(ok, own, 1.0), 0.0)
                c += a[:, None] * f
            rad[idx] += thr[idx] * c
            if more:
                go = (db[:, 2] > 0.0) & (pb > 0.0)
                sel = idx[go]
                thr[sel] *= f_b[go] / pb[go, None]
                ro[sel] = o[go]
                rd[sel] = np.einsum("nji,nj->ni", F[go], db[go])
        if not more:
            break
        live = np.isfinite(rd[:, 0])
        nxt = _vertices(scene, ro[live], rd[live], g["cone"][live], lod_base_width)
        g2 = {key: np.zeros_like(val) for key, val in g.items()}
        g2["material"] = np.full(n, -1, np.int64)
        for key in g2:
            g2[key][live] = nxt[key]
        g2["t"][~live] = np.inf
        g = g2
        if not np.any(g["material"] >= 0):
            break
    return rad


def render_direct(scene, models, samplers, variates, lod_base_width):
    """render_paths with one vertex: direct lighting."""
    return render_paths(scene, models, samplers, np.asarray(variates)[None], lod_base_width, 1)
