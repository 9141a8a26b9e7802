"""Pins of the oracle's importance-sampling proxy (Sec. 4.3, Appendix A):
closed forms of the activations, the textbook isotropic GGX half-vector
density as a special case (Walter et al. 2007), normalisation of both lobes by
quadrature over the sphere, the change of variables between half vectors and
outgoing directions checked by two independent quadratures, and a chi-square
test of the sample transform against the density."""
import numpy as np
import pytest

PI = np.pi


def _params(wd, mud, alpha, rho=0.0, mus=(0.0, 0.0)):
    ws = 1.0 - wd
    return np.array([wd, mud[0], mud[1], ws, alpha[0], alpha[1], rho, mus[0], mus[1]], np.float64)


def _sphere_grid(nc, nphi, upper=False):
    """Midpoint grid uniform in cos(theta) and phi; every cell has solid angle
    dcos * dphi."""
    lo = 0.0 if upper else -1.0
    c = lo + (np.arange(nc) + 0.5) * (1.0 - lo) / nc
    ph = (np.arange(nphi) + 0.5) * 2 * PI / nphi
    C, P = np.meshgrid(c, ph, indexing="ij")
    s = np.sqrt(1 - C * C)
    d = np.stack([s * np.cos(P), s * np.sin(P), C], axis=-1).reshape(-1, 3)
    return d, (1.0 - lo) / nc * 2 * PI / nphi


def test_activation_closed_forms(oracle):
    assert np.allclose(oracle.qtanh([0.0, 1.0, -1.0, 2.0, 5.0, -3.0]), [0.0, 0.75, -0.75, 1.0, 1.0, -1.0])
    assert np.allclose(oracle.qsinh([0.0, 1.0, -1.0, 2.0]), [0.0, 1.5, -1.5, 4.0])
    p = oracle.proxy_activate([0.3, 0.0, 1.0, -0.2, 0.0, 100.0, 1.0, -1.0, 0.5])
    e = np.exp([0.3, -0.2])
    assert np.isclose(p[0], e[0] / e.sum()) and np.isclose(p[0] + p[3], 1.0)
    assert np.isclose(p[4], 1e-3 + (1 - 1e-3) * 0.5) and np.isclose(p[5], 1.0)
    assert np.isclose(p[6], 0.99 * 0.75)
    assert np.allclose(p[[1, 2, 7, 8]], [0.0, 1.5, -1.5, 0.5 * 1.25])


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.0])
def test_isotropic_special_case_is_textbook_ggx(oracle, alpha):
    """M = diag(alpha, alpha, 1), no slope offset: the half-vector density is
    D_GGX(h) cos(theta_h), D_GGX = alpha^2 / (pi (cos^2 (alpha^2 - 1) + 1)^2)."""
    rng = np.random.default_rng(1)
    h = rng.normal(size=(500, 3))
    h[:, 2] = np.abs(h[:, 2])
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    p = _params(0.2, (0.0, 0.0), (alpha, alpha))
    got = oracle.proxy_pdf_h(p, h)
    c = h[:, 2]
    want = alpha ** 2 / (PI * (c * c * (alpha ** 2 - 1) + 1) ** 2) * c
    assert np.allclose(got, want, rtol=1e-12)


def test_diffuse_lobe_closed_form(oracle):
    rng = np.random.default_rng(2)
    wo = rng.normal(size=(300, 3))
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    p = _params(1.0, (0.0, 0.0), (0.5, 0.5))
    got = oracle.proxy_pdf(p, np.array([0.0, 0.6, 0.8]), wo)
    assert np.allclose(got, np.maximum(wo[:, 2], 0) / PI, rtol=1e-12)
    # tilted: density is cos(angle to n_d) / pi with n_d = normalize(-mu_x, -mu_y, 1)
    p2 = _params(1.0, (0.4, -0.7), (0.5, 0.5))
    nd = np.array([-0.4, 0.7, 1.0])
    nd /= np.linalg.norm(nd)
    got2 = oracle.proxy_pdf(p2, np.array([0.0, 0.0, 1.0]), wo)
    assert np.allclose(got2, np.maximum(wo @ nd, 0) / PI, rtol=1e-12)


PARAMS = [
    _params(0.3, (0.2, -0.1), (0.5, 0.8), rho=0.4, mus=(0.3, -0.2)),
    _params(0.6, (-0.5, 0.5), (0.9, 0.4), rho=-0.6, mus=(-0.4, 0.1)),
    _params(0.1, (0.0, 0.0), (0.35, 0.35), rho=0.0, mus=(0.5, 0.5)),
]


@pytest.mark.parametrize("p", PARAMS)
def test_specular_half_vector_density_integrates_to_one(oracle, p):
    d, dw = _sphere_grid(1500, 1500, upper=True)
    total = oracle.proxy_pdf_h(p, d).sum() * dw
    assert abs(total - 1.0) < 2e-4, total


@pytest.mark.parametrize("p", PARAMS)
def test_change_of_variables_between_half_vectors_and_directions(oracle, p):
    """Integral over outgoing directions of the full density = w_d + w_s x
    (half-vector mass with wi . h > 0), the second computed in half-vector
    space: two independent quadratures through the 1 / (4 |wo . h|)
    Jacobian."""
    wi = np.array([0.3, -0.2, 0.9])
    wi /= np.linalg.norm(wi)
    d, dw = _sphere_grid(1500, 1500)
    lhs = oracle.proxy_pdf(p, wi, d).sum() * dw
    h, dh = _sphere_grid(1500, 1500, upper=True)
    mass = (oracle.proxy_pdf_h(p, h) * (h @ wi > 0)).sum() * dh
    rhs = p[0] + p[3] * mass
    assert abs(lhs - rhs) < 5e-4, (lhs, rhs)


@pytest.mark.parametrize("p", PARAMS)
def test_sample_histogram_matches_density(oracle, p):
    """Chi-square of 200,000 samples over 12 x 24 (cos theta, phi) bins of the
    sphere against the density integrated over each bin.  Specular samples
    whose half vector faces away from wi carry no density (their reflected
    direction has normalize(wi + wo) below the surface) and are dropped, as
    the density omits them."""
    from scipy import stats
    wi = np.array([0.2, 0.1, 0.95])
    wi /= np.linalg.norm(wi)
    rng = np.random.default_rng(7)
    u = rng.random((200000, 3))
    wo, pdf = oracle.proxy_sample(p, wi, u)
    keep = (wo + wi)[:, 2] > 0
    spec = u[:, 2] >= p[0]
    keep |= ~spec
    wo = wo[keep]
    nc, nphi = 12, 24
    ci = np.clip(((wo[:, 2] + 1) / 2 * nc).astype(int), 0, nc - 1)
    pi_ = np.clip(((np.arctan2(wo[:, 1], wo[:, 0]) % (2 * PI)) / (2 * PI) * nphi).astype(int), 0, nphi - 1)
    obs = np.bincount(ci * nphi + pi_, minlength=nc * nphi).astype(float)
    sub = 40
    d, dw = _sphere_grid(nc * sub, nphi * sub)
    dens = oracle.proxy_pdf(p, wi, d).reshape(nc, sub, nphi, sub).sum(axis=(1, 3)).ravel() * dw
    exp = dens * len(u)
    mask = exp > 20
    chi2 = ((obs[mask] - exp[mask]) ** 2 / exp[mask]).sum()
    pval = stats.chi2.sf(chi2, mask.sum() - 1)
    assert pval > 1e-4, (chi2, mask.sum(), pval)
    # the density returned with each sample is the density at that direction
    assert np.allclose(pdf[keep], oracle.proxy_pdf(p, wi, wo), rtol=1e-12)


def test_sampler_network_layer_matches_numpy(oracle):
    """Zero hidden and output weights: the nine raw outputs are the output
    biases, so the parameters are their activations; a single ReLU layer with
    identity weights passes its inputs through (checked via the output)."""
    rng = np.random.default_rng(3)
    W0 = H0 = 8
    pyr = np.full((85, 8), 0.25, np.float16)
    dec = [(np.zeros((16, 14), np.float32), np.zeros(16, np.float32)),
           (np.zeros((16, 16), np.float32), np.zeros(16, np.float32)),
           (np.zeros((3, 16), np.float32), np.zeros(3, np.float32))]
    m = oracle.Model(W0, H0, 4, pyr, None, dec)
    b_out = rng.normal(size=9).astype(np.float32)
    layers = [(np.zeros((32, 11), np.float32), np.zeros(32, np.float32)),
              (np.zeros((32, 32), np.float32), np.zeros(32, np.float32)),
              (np.zeros((32, 32), np.float32), np.zeros(32, np.float32)),
              (np.zeros((9, 32), np.float32), b_out)]
    n = 5
    z = np.zeros(n, np.float32)
    q = dict(u=np.full(n, 0.3, np.float32), v=np.full(n, 0.6, np.float32), lod=np.full(n, 1.0, np.float32),
             wix=z, wiy=z, wiz=np.ones(n, np.float32), wox=z, woy=z, woz=np.ones(n, np.float32), xi=z)
    got = oracle.sampler_params(m, layers, q)
    want = oracle.proxy_activate(b_out.astype(np.float64))
    assert np.allclose(got, want[None, :], rtol=1e-15)
    # first layer reads (z, wi): pick z0 = 0.25 and wi_z = 1 into two units
    # that the output layer copies to mu_dx and mu_dy (qsinh(0.25), qsinh(1))
    W1 = np.zeros((32, 11), np.float32)
    W1[0, 0] = 1.0
    W1[1, 10] = 1.0
    I32 = np.eye(32, dtype=np.float32)
    W4 = np.zeros((9, 32), np.float32)
    W4[1, 0] = 1.0
    W4[2, 1] = 1.0
    layers2 = [(W1, np.zeros(32, np.float32)), (I32, np.zeros(32, np.float32)), (I32, np.zeros(32, np.float32)),
               (W4, np.zeros(9, np.float32))]
    got2 = oracle.sampler_params(m, layers2, q)
    assert np.allclose(got2[:, 1], 0.25 * 1.125) and np.allclose(got2[:, 2], 1.5)
