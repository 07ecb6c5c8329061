"""Oracle pins for the materials: the GGX microfacet BSDF (visible-normal
sampling, Smith height-correlated masking-shadowing, Schlick Fresnel) and the
Lambertian BSDF, checked against what the mathematics fixes rather than
against a retyped formula:

* a sampling pdf is a density: the pdf the evaluator returns integrates to 1
  over all directions (numerical quadrature over half vectors, whose measure
  dw_i = 4 (w_o . h) dw_h is geometry, not the BSDF); the part above the
  surface equals the fraction of samples the sampler keeps;
* the sampler draws from that density (chi-square over half-vector bins);
* the sampler's weight is f cos / pdf of the evaluator at the drawn direction;
* the mean weight equals the directional albedo, the integral of f cos by
  quadrature;
* Helmholtz reciprocity f(w_o, w_i) = f(w_i, w_o);
* a near-mirror surface reflects the Fresnel reflectance of its incidence
  angle (Schlick's form with F0 = albedo) and nothing else.
"""
import math

import numpy as np
import pytest

LAMBERT, GGX = 0, 1


def mat(kind, albedo, alpha=1.0):
    return np.array([kind, *albedo, alpha, 0, 0, 0], np.float32)


def wo_at(theta_deg, phi_deg=30.0):
    t, p = math.radians(theta_deg), math.radians(phi_deg)
    return np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])


def half_vector_grid(alpha, nt=1200, nphi=192):
    """Midpoint quadrature over the upper hemisphere of half vectors h.
    theta_h = atan(alpha tan(pi t / 2)) for t in (0, 1) crowds the nodes where
    a roughness-alpha lobe lives; the weights are the exact Jacobian of that
    substitution times sin(theta) dtheta dphi.  Returns h [nt, nphi, 3],
    the solid-angle weight of each node [nt, nphi], and t, phi."""
    t = (np.arange(nt) + 0.5) / nt
    x = 0.5 * math.pi * t
    th = np.arctan(alpha * np.tan(x))
    dth = alpha * 0.5 * math.pi / np.cos(x) ** 2 / (1.0 + (alpha * np.tan(x)) ** 2)
    phi = (np.arange(nphi) + 0.5) / nphi * 2 * math.pi
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    h = np.stack([st * np.cos(phi), st * np.sin(phi), np.broadcast_to(ct, (nt, nphi))], -1)
    w = (st * dth[:, None] / nt) * (2 * math.pi / nphi) * np.ones((1, nphi))
    return h, w, t, phi


def reflect_measure(wo, h, w):
    """wi = reflection of wo about h and the node's solid angle in wi:
    dw_i = 4 (wo . h) dw_h; nodes with wo . h <= 0 carry no weight."""
    c = h @ wo
    wi = 2.0 * c[..., None] * h - wo
    return wi, np.where(c > 0, 4.0 * c * w, 0.0)


GGX_CASES = [(a, th) for a in (0.05, 0.3, 0.7, 1.0) for th in (0.0, 30.0, 60.0, 80.0)]


@pytest.mark.parametrize("alpha,theta", GGX_CASES)
def test_ggx_pdf_is_a_density(orc, alpha, theta):
    # VNDF sampling reflects wo about a visible normal, so its pdf over the
    # whole sphere of wi (below-horizon reflections included, which the
    # sampler then rejects) integrates to exactly 1
    m = mat(GGX, (0.8, 0.5, 0.2), alpha)
    wo = wo_at(theta)
    h, w, _, _ = half_vector_grid(alpha)
    wi, dw = reflect_measure(wo, h.reshape(-1, 3), w.reshape(-1))
    _, pdf = orc.bsdf_eval(m, wo, wi)
    total = float(np.sum(pdf.astype(np.float64) * dw))
    assert abs(total - 1.0) < 2e-3, total
    # the part above the surface is the sampler's acceptance rate
    up = float(np.sum(np.where(wi[:, 2] > 0, pdf * dw, 0.0)))
    rng = np.random.default_rng(7)
    n = 200_000
    _, _, _, ok = orc.bsdf_sample(m, wo, rng.random((n, 2)))
    acc = ok.mean()
    sd = math.sqrt(max(up * (1 - up), 1e-12) / n)
    assert abs(acc - up) < 4.5 * sd + 1e-4, (acc, up)
    if theta == 0.0:
        # normal incidence: every normal is visible with weight D cos, and wi
        # stays above the surface exactly when theta_h < 45 degrees, whose
        # GGX probability is 1 / (1 + alpha^2) (tan^2 theta = alpha^2 u / (1 - u))
        assert abs(up - 1.0 / (1.0 + alpha * alpha)) < 1e-3, up


@pytest.mark.parametrize("alpha,theta", [(0.05, 0.0), (0.3, 30.0), (0.7, 60.0), (1.0, 80.0),
                                         (0.3, 75.0)])
def test_ggx_sampler_draws_from_its_pdf(orc, alpha, theta):
    # chi-square of the sampled half vectors against the evaluator's pdf
    # integrated over each bin; rejected samples form one more bin
    from scipy import stats
    m = mat(GGX, (0.9, 0.9, 0.9), alpha)
    wo = wo_at(theta)
    nt_b, nphi_b, kt, kp = 16, 12, 60, 16
    h, w, _, _ = half_vector_grid(alpha, nt_b * kt, nphi_b * kp)
    wi, dw = reflect_measure(wo, h.reshape(-1, 3), w.reshape(-1))
    _, pdf = orc.bsdf_eval(m, wo, wi)
    mass = np.where(wi[:, 2] > 0, pdf.astype(np.float64) * dw, 0.0)
    mass = mass.reshape(nt_b, kt, nphi_b, kp).sum(axis=(1, 3))
    n = 120_000
    rng = np.random.default_rng(11)
    swi, _, _, ok = orc.bsdf_sample(m, wo, rng.random((n, 2)))
    hs = swi[ok].astype(np.float64) + wo
    hs /= np.linalg.norm(hs, axis=1, keepdims=True)
    th = np.arccos(np.clip(hs[:, 2], -1, 1))
    t = np.arctan(np.tan(th) / alpha) / (0.5 * math.pi)
    ph = np.mod(np.arctan2(hs[:, 1], hs[:, 0]), 2 * math.pi)
    it = np.minimum((t * nt_b).astype(int), nt_b - 1)
    ip = np.minimum((ph / (2 * math.pi) * nphi_b).astype(int), nphi_b - 1)
    obs = np.zeros((nt_b, nphi_b))
    np.add.at(obs, (it, ip), 1.0)
    exp = np.append(mass.reshape(-1), max(1.0 - mass.sum(), 0.0)) * n
    obs = np.append(obs.reshape(-1), (~ok).sum())
    # pool bins with few expected samples into one
    small = exp < 20
    e = np.append(exp[~small], exp[small].sum())
    o = np.append(obs[~small], obs[small].sum())
    keep = e > 0
    chi2 = float(np.sum((o[keep] - e[keep]) ** 2 / e[keep]))
    dof = int(keep.sum()) - 1
    p = stats.chi2.sf(chi2, dof)
    assert p > 1e-4, (chi2, dof, p)


@pytest.mark.parametrize("alpha,theta", GGX_CASES)
def test_ggx_sample_weight_is_f_cos_over_pdf(orc, alpha, theta):
    m = mat(GGX, (0.8, 0.5, 0.2), alpha)
    wo = wo_at(theta)
    rng = np.random.default_rng(3)
    wi, wt, pdf, ok = orc.bsdf_sample(m, wo, rng.random((4000, 2)))
    assert ok.any()
    f, pe = orc.bsdf_eval(m, wo, wi[ok])
    # the evaluator re-derives h = normalize(wo + wi) from the float wi: a few
    # ulp of error in h, which the lobe D(h) amplifies by about 1 / alpha^2
    tol = 1e-6 / alpha**2 + 1e-6
    assert np.allclose(pdf[ok], pe, rtol=tol, atol=0)
    want = f * wi[ok, 2:3] / pe[:, None]
    assert np.allclose(wt[ok], want, rtol=tol, atol=1e-7)
    assert (wi[ok, 2] > 0).all() and not wt[~ok].any()


@pytest.mark.parametrize("alpha,theta", GGX_CASES)
def test_ggx_mean_weight_is_the_directional_albedo(orc, alpha, theta):
    m = mat(GGX, (0.8, 0.5, 0.2), alpha)
    wo = wo_at(theta)
    h, w, _, _ = half_vector_grid(alpha)
    wi, dw = reflect_measure(wo, h.reshape(-1, 3), w.reshape(-1))
    f, _ = orc.bsdf_eval(m, wo, wi)
    up = wi[:, 2] > 0
    albedo = np.sum(np.where(up[:, None], f * wi[:, 2:3] * dw[:, None], 0.0), axis=0)
    rng = np.random.default_rng(5)
    _, wt, _, _ = orc.bsdf_sample(m, wo, rng.random((200_000, 2)))
    mean = wt.astype(np.float64).mean(axis=0)
    sem = wt.astype(np.float64).std(axis=0) / math.sqrt(len(wt))
    assert np.all(np.abs(mean - albedo) < 4.5 * sem + 2e-4 * albedo + 1e-6), (mean, albedo, sem)
    # energy: a single-scattering microfacet model never reflects more than F
    assert np.all(albedo <= 1.0 + 1e-6)


def test_ggx_reciprocity(orc):
    rng = np.random.default_rng(9)
    n = 5000
    a = rng.normal(size=(n, 3))
    b = rng.normal(size=(n, 3))
    a[:, 2] = np.abs(a[:, 2])
    b[:, 2] = np.abs(b[:, 2])
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    for alpha in (0.1, 0.5, 1.0):
        m = mat(GGX, (0.7, 0.4, 0.1), alpha)
        fab, _ = orc.bsdf_eval(m, a, b)
        fba, _ = orc.bsdf_eval(m, b, a)
        assert np.allclose(fab, fba, rtol=1e-5, atol=0)


@pytest.mark.parametrize("theta", [0.0, 45.0, 75.0, 85.0])
def test_ggx_near_mirror_reflects_fresnel(orc, theta):
    # alpha -> 0: the microfacets are the macro surface, masking vanishes and
    # every sample is the mirror direction with weight F(cos theta_o),
    # Schlick's approximation with F0 = albedo (the material's reading)
    F0 = np.array([0.04, 0.5, 0.9])
    m = mat(GGX, F0, 1e-3)
    wo = wo_at(theta)
    rng = np.random.default_rng(1)
    wi, wt, _, ok = orc.bsdf_sample(m, wo, rng.random((2000, 2)))
    assert ok.all()
    mirror = np.array([-wo[0], -wo[1], wo[2]])
    # GGX's tail is heavy (P(theta_h > k alpha) = 1 / (1 + k^2)), so most
    # but not all samples sit within a few alpha of the mirror direction
    assert np.mean(wi @ mirror > 1 - 1e-4) > 0.9
    c = math.cos(math.radians(theta))
    F = F0 + (1 - F0) * (1 - c) ** 5
    assert np.allclose(wt.mean(axis=0), F, rtol=2e-3, atol=0), (wt.mean(axis=0), F)


def test_lambert_density_sampler_and_albedo(orc):
    alb = (0.7, 0.4, 0.1)
    m = mat(LAMBERT, alb)
    wo = wo_at(40.0)
    h, w, _, _ = half_vector_grid(1.0, 600, 128)   # any hemisphere grid serves
    dirs = h.reshape(-1, 3)
    f, pdf = orc.bsdf_eval(m, wo, dirs)
    dw = w.reshape(-1)
    assert abs(np.sum(pdf * dw) - 1.0) < 1e-3
    assert np.allclose(np.sum(f * dirs[:, 2:3] * dw[:, None], axis=0), alb, rtol=1e-3)
    rng = np.random.default_rng(2)
    wi, wt, p, ok = orc.bsdf_sample(m, wo, rng.random((20000, 2)))
    assert ok.mean() > 0.999 and np.allclose(wt[ok], alb)
    # cosine-distributed: E[cos theta] = 2/3, E[cos^2] = 1/2
    assert abs(wi[ok, 2].mean() - 2 / 3) < 0.01 and abs((wi[ok, 2] ** 2).mean() - 0.5) < 0.01
    _, pe = orc.bsdf_eval(m, wo, wi[ok])
    assert np.allclose(p[ok], pe, rtol=1e-6)
