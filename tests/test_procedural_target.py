"""Closed-form pins of the procedural training target (workloads.synth
.ProceduralBRDF: Lambert + GGX specular with height-correlated Smith masking
and Schlick Fresnel), which the fits, the encoder and the albedo tests train
against.  Each check is an identity of the model, not a restatement of its
formula: a normalised distribution, Heitz's masking identity, Schlick's
endpoints, the bounds of the height-correlated shadowing term, reciprocity,
and the separation of the diffuse term."""
import numpy as np
import pytest
from scipy import integrate

import workloads as W

P = W.ProceduralBRDF


@pytest.mark.parametrize("alpha", [0.0025, 0.05, 0.3, 0.7, 1.0])
def test_ggx_ndf_is_normalised(alpha):
    # int over the hemisphere of D(h) cos(theta_h) dw = 1 (projected area of
    # the microsurface equals that of the macrosurface); in theta:
    # 2 pi int_0^{pi/2} D(theta) cos(theta) sin(theta) dtheta
    f = lambda th: 2.0 * np.pi * P.ggx_ndf(alpha, np.cos(th)) * np.cos(th) * np.sin(th)
    brk = [min(np.pi / 2, k * np.sqrt(alpha)) for k in (0.5, 1.0, 2.0, 4.0, 8.0)]
    val, err = integrate.quad(f, 0.0, np.pi / 2, points=brk, limit=500, epsabs=1e-13, epsrel=1e-11)
    assert abs(val - 1.0) < 1e-8, (alpha, val)


@pytest.mark.parametrize("alpha", [0.1, 0.3, 0.7, 1.0])
@pytest.mark.parametrize("theta_o", [0.0, 0.5, 1.0, 1.4])
def test_smith_masking_identity(alpha, theta_o):
    # Heitz (2014): G1(wo) int max(0, <wo, m>) D(m) dm = cos(theta_o), with
    # G1 = 1 / (1 + Lambda(wo)): pins Lambda against D
    wo = np.array([np.sin(theta_o), 0.0, np.cos(theta_o)])

    def inner(phi, th):
        m = np.array([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)])
        return max(0.0, float(wo @ m)) * P.ggx_ndf(alpha, np.cos(th)) * np.sin(th)

    val, _ = integrate.dblquad(inner, 0.0, np.pi / 2, 0.0, 2.0 * np.pi, epsabs=1e-10, epsrel=1e-8)
    g1 = 1.0 / (1.0 + P.smith_lambda(alpha, np.cos(theta_o)))
    assert abs(g1 * val - np.cos(theta_o)) < 1e-6, (alpha, theta_o, g1 * val, np.cos(theta_o))


def test_schlick_endpoints():
    for f0 in (0.0, 0.04, 0.5, 1.0):
        assert P.schlick(f0, 1.0) == pytest.approx(f0, abs=1e-15)   # normal incidence
        assert P.schlick(f0, 0.0) == pytest.approx(1.0, abs=1e-15)  # grazing
    c = np.linspace(0.0, 1.0, 101)
    assert np.all(np.diff(P.schlick(0.04, c)) <= 0.0)  # decreasing towards normal incidence


def _dirs(rng, n):
    return W.cosine_hemisphere(rng, n)


def test_height_correlated_shadowing_bounds():
    # 0 < G1(i) G1(o) <= G2 = 1 / (1 + Li + Lo) <= min(G1(i), G1(o)) <= 1
    rng = np.random.default_rng(5)
    ci, co = _dirs(rng, 20000)[2], _dirs(rng, 20000)[2]
    for alpha in (0.0025, 0.1, 0.5, 1.0):
        li, lo = P.smith_lambda(alpha, ci), P.smith_lambda(alpha, co)
        g2 = 1.0 / (1.0 + li + lo)
        g1i, g1o = 1.0 / (1.0 + li), 1.0 / (1.0 + lo)
        assert np.all(g2 > 0.0) and np.all(g2 <= 1.0)
        assert np.all(g2 <= np.minimum(g1i, g1o) + 1e-15)
        assert np.all(g2 >= g1i * g1o - 1e-15)
    assert P.smith_lambda(0.3, 1.0) == 0.0  # no masking at normal incidence


def test_normal_incidence_closed_form():
    # wi = wo = n: D = 1 / (pi alpha^2), G2 = 1, F = F0, so the specular part
    # is F0 / (4 pi alpha^2); the diffuse part is a / pi
    z = np.array([[0.0], [0.0], [1.0]])
    for r in (0.05, 0.3, 1.0):
        a = np.array([[0.25, 0.5, 0.75]])
        f = P.from_params(a, np.array([r]), z, z)
        alpha = r * r
        assert np.allclose(f, a / np.pi + 0.04 / (4.0 * np.pi * alpha * alpha), rtol=1e-12)


def test_reciprocity_and_diffuse_separation():
    rng = np.random.default_rng(6)
    target = P(np.random.default_rng(7))
    n = 5000
    u, v = rng.random(n), rng.random(n)
    wi, wo = _dirs(rng, n), _dirs(rng, n)
    f1 = target(u, v, wi, wo)
    f2 = target(u, v, wo, wi)
    assert np.allclose(f1, f2, rtol=1e-12, atol=0.0)
    a, r = target.params(u, v)
    assert np.all((a >= 0.05) & (a <= 0.95)) and np.all((r >= 0.05) & (r <= 1.0))
    # the albedo enters only through a / pi
    d = P.from_params(a + 0.1, r, wi, wo) - P.from_params(a, r, wi, wo)
    assert np.allclose(d, 0.1 / np.pi, rtol=1e-12)
    # nothing below the horizon
    below = wi.copy()
    below[2] = -below[2]
    assert np.all(P.from_params(a, r, below, wo) == 0.0)
