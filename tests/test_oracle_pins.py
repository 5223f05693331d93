"""Pins of the CPU oracle to things other than itself: closed forms, library
routines, invariants, brute force and finite differences (CPU only).

The reflectivity conventions pinned here (media indexing, principal-branch
wavevectors, Nevot-Croce roughness, FWHM resolution) are the readings the
oracle's header lists for the Abeles formalism the paper names in Sec. 2.1.
"""
import math

import numpy as np
import pytest
import scipy.signal
import scipy.stats

import oracle
from paper_2509_06924_gb300 import workloads as W

FOURPI = 4 * math.pi
QGRID = np.logspace(np.log10(0.004), np.log10(0.35), 157)


def kz(q, rho, rho0=0.0, iota=0.0):
    """Wavevector in a medium, principal root with Im >= 0 (test's own)."""
    return np.sqrt((q / 2) ** 2 - FOURPI * (rho - rho0) + 1j * FOURPI * iota + 0j)


def fresnel_rough(ka, kb, sigma):
    return (ka - kb) / (ka + kb) * np.exp(-2 * ka * kb * sigma ** 2)


def one_layer(d, rho, iota, sig, front=0.0, back=2.07e-6, back_iota=0.0, scale=1.0, bkg=0.0):
    return W.pack([d], [front, rho, back], [iota, back_iota], sig, scale, bkg)


# --------------------------------------------------------------- quadrature
@pytest.mark.parametrize("K", [1, 2, 3, 5, 8, 13, 17, 21, 32, 48, 64])
def test_gauss_hermite_matches_numpy(K):
    x, w = oracle.gauss_hermite(K)
    xr, wr = np.polynomial.hermite.hermgauss(K)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-12 * max(1.0, np.abs(xr).max()))
    np.testing.assert_allclose(w, wr, rtol=1e-10, atol=1e-14 * wr.max())


@pytest.mark.parametrize("K", [17, 21])
def test_gauss_hermite_moments_exact(K):
    """Exact for polynomials of degree <= 2K-1: int x^(2m) e^(-x^2) = Gamma(m+1/2)."""
    x, w = oracle.gauss_hermite(K)
    for m in range(K):
        exact = math.gamma(m + 0.5)
        assert abs((w * x ** (2 * m)).sum() - exact) <= 1e-12 * exact * max(1, m)
        assert abs((w * x ** (2 * m + 1)).sum()) <= 1e-12 * math.gamma(m + 1.0) * max(1, m)
    assert abs(w.sum() - math.sqrt(math.pi)) < 1e-14


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("sigma", [0.0, 3.0, 12.0])
@pytest.mark.parametrize("iota", [0.0, 2e-8])
def test_bare_substrate_fresnel(sigma, iota):
    """n = 0: r = (k0-k1)/(k0+k1) exp(-2 k0 k1 sigma^2)."""
    p = W.pack([], [0.0, 2.07e-6], [iota], [sigma], 1.0, 0.0)
    r = oracle.amplitude(0, p, QGRID)
    ref = fresnel_rough(QGRID / 2 + 0j, kz(QGRID, 2.07e-6, iota=iota), sigma)
    np.testing.assert_allclose(r, ref, rtol=1e-12, atol=1e-15)


def test_fresnel_high_q_limit():
    """Far above the edge, R = 16 pi^2 drho^2 / Q^4 (1 + 16 pi drho / Q^2 + ...)
    (no roughness; expansion of the bare-substrate Fresnel coefficient)."""
    drho = 2.07e-6
    q = np.array([2.0, 4.0, 8.0])
    R = np.abs(oracle.amplitude(0, W.pack([], [0.0, drho], [0.0], [0.0], 1, 0), q)) ** 2
    ref = 16 * math.pi ** 2 * drho ** 2 / q ** 4 * (1 + 16 * math.pi * drho / q ** 2)
    np.testing.assert_allclose(R, ref, rtol=2e-8)


def test_critical_edge_and_total_reflection():
    """R = 1 below the backing's critical edge Q_c = sqrt(16 pi rho) for
    non-absorbing stacks, rough or not, with evanescent interior layers."""
    qc = math.sqrt(16 * math.pi * 2.07e-6)
    assert abs(qc - 0.0102) < 1e-4
    q = np.linspace(0.001, 0.98 * qc, 60)
    cases = [
        (0, W.pack([], [0.0, 2.07e-6], [0.0], [5.0], 1, 0)),
        (1, one_layer(300.0, 4.2e-6, 0.0, [5.0, 8.0])),
        (3, W.pack([120.0, 40.0, 600.0], [0.0, 6.0e-6, -0.5e-6, 3.0e-6, 2.07e-6], [0, 0, 0, 0],
                   [3.0, 7.0, 2.0, 11.0], 1, 0)),
    ]
    for n, p in cases:
        R = np.abs(oracle.amplitude(n, p, q)) ** 2
        np.testing.assert_allclose(R, 1.0, rtol=0, atol=1e-12)
    # just above the edge R drops below 1
    R = np.abs(oracle.amplitude(0, cases[0][1], np.array([1.05 * qc]))) ** 2
    assert R[0] < 0.9


@pytest.mark.parametrize("d", [35.0, 1470.0])
def test_one_layer_airy(d):
    """One layer: r = (r01 + r12 e^{2i k1 d}) / (1 + r01 r12 e^{2i k1 d})."""
    sig = [4.0, 9.0]
    p = one_layer(d, 4.24e-6, 3e-9, sig, back_iota=1e-9)
    k0 = QGRID / 2 + 0j
    k1 = kz(QGRID, 4.24e-6, iota=3e-9)
    k2 = kz(QGRID, 2.07e-6, iota=1e-9)
    r01, r12 = fresnel_rough(k0, k1, sig[0]), fresnel_rough(k1, k2, sig[1])
    ph = np.exp(2j * k1 * d)
    ref = (r01 + r12 * ph) / (1 + r01 * r12 * ph)
    np.testing.assert_allclose(oracle.amplitude(1, p, QGRID), ref, rtol=1e-10, atol=1e-14)


def test_two_layer_nested_airy_nonvacuum_fronting():
    """Two layers under a D2O-like fronting: nested Airy formula."""
    d = [80.0, 250.0]
    rho = [6.35e-6, 1.0e-6, 4.5e-6, 2.07e-6]
    iota = [5e-9, 0.0, 0.0]
    sig = [3.0, 6.0, 2.5]
    p = W.pack(d, rho, iota, sig, 1, 0)
    k = [kz(QGRID, rho[0], rho[0])] + [kz(QGRID, rho[j], rho[0], ([0.0] + iota)[j]) for j in (1, 2, 3)]
    r = [fresnel_rough(k[j], k[j + 1], sig[j]) for j in range(3)]
    e2 = np.exp(2j * k[2] * d[1])
    r1 = (r[1] + r[2] * e2) / (1 + r[1] * r[2] * e2)
    e1 = np.exp(2j * k[1] * d[0])
    ref = (r[0] + r1 * e1) / (1 + r[0] * r1 * e1)
    np.testing.assert_allclose(oracle.amplitude(2, p, QGRID), ref, rtol=1e-10, atol=1e-14)


def test_zero_roughness_limit_and_sigma_derivative():
    p0 = one_layer(200.0, 5e-6, 0.0, [0.0, 0.0])
    p1 = one_layer(200.0, 5e-6, 0.0, [1e-7, 1e-7])
    r0 = oracle.amplitude(1, p0, QGRID)
    r1 = oracle.amplitude(1, p1, QGRID)
    np.testing.assert_allclose(r1, r0, rtol=1e-12, atol=1e-16)
    sig0 = W.layout(1)["sigma"].start
    for idx in (sig0, sig0 + 1):
        _, dR = oracle.reflectivity_unsmeared(1, p0, QGRID, seed=idx)
        assert np.abs(dR).max() == 0.0


def test_fresnel_analytic_gradient():
    """Bare Si above the edge: R = rF^2 exp(-4 sigma^2 k0 k1), with
    dk1/drho1 = -2 pi / k1 and drF/dk1 = -2 k0/(k0+k1)^2."""
    sigma = 6.0
    q = np.linspace(0.02, 0.3, 40)
    p = W.pack([], [0.0, 2.07e-6], [0.0], [sigma], 1, 0)
    k0 = q / 2
    k1 = np.sqrt(k0 ** 2 - FOURPI * 2.07e-6)
    rF = (k0 - k1) / (k0 + k1)
    damp = np.exp(-4 * sigma ** 2 * k0 * k1)
    R = rF ** 2 * damp
    dR_dk1 = 2 * rF * (-2 * k0 / (k0 + k1) ** 2) * damp + R * (-4 * sigma ** 2 * k0)
    dR_drho1 = dR_dk1 * (-2 * math.pi / k1)
    dR_dsigma = R * (-8 * sigma * k0 * k1)
    L = W.layout(0)
    R_o, d_rho = oracle.reflectivity_unsmeared(0, p, q, seed=L["rho"].start + 1)
    _, d_sig = oracle.reflectivity_unsmeared(0, p, q, seed=L["sigma"].start)
    np.testing.assert_allclose(R_o, R, rtol=1e-12)
    np.testing.assert_allclose(d_rho, dR_drho1, rtol=1e-9)
    np.testing.assert_allclose(d_sig, dR_dsigma, rtol=1e-9)


# --------------------------------------------------------------- invariants
def test_split_layer_invariance():
    """Splitting a layer into two of identical SLD changes nothing, whatever
    the roughness put on the new interface (its Fresnel coefficient is 0)."""
    p1 = W.pack([100.0, 500.0, 60.0], [0.0, 3e-6, 5e-6, 1e-6, 2.07e-6], [1e-9, 2e-9, 0.0, 0.0],
                [4.0, 6.0, 3.0, 5.0], 1, 0)
    p2 = W.pack([100.0, 200.0, 300.0, 60.0], [0.0, 3e-6, 5e-6, 5e-6, 1e-6, 2.07e-6],
                [1e-9, 2e-9, 2e-9, 0.0, 0.0], [4.0, 6.0, 17.0, 3.0, 5.0], 1, 0)
    np.testing.assert_allclose(oracle.amplitude(4, p2, QGRID), oracle.amplitude(3, p1, QGRID),
                               rtol=1e-9, atol=1e-15)


def test_zero_thickness_layer_invariance():
    """A zero-thickness layer with smooth interfaces is invisible; so is one
    whose SLD equals its upper neighbour's, rough or not."""
    base = one_layer(400.0, 4.2e-6, 0.0, [5.0, 3.0])
    r = oracle.amplitude(1, base, QGRID)
    smooth = W.pack([400.0, 0.0], [0.0, 4.2e-6, 1.3e-6, 2.07e-6], [0.0, 0.0, 0.0], [5.0, 0.0, 0.0], 1, 0)
    np.testing.assert_allclose(oracle.amplitude(2, smooth, QGRID),
                               oracle.amplitude(1, one_layer(400.0, 4.2e-6, 0.0, [5.0, 0.0]), QGRID),
                               rtol=1e-10, atol=1e-15)
    same = W.pack([400.0, 0.0], [0.0, 4.2e-6, 4.2e-6, 2.07e-6], [0.0, 0.0, 0.0], [5.0, 9.0, 3.0], 1, 0)
    np.testing.assert_allclose(oracle.amplitude(2, same, QGRID), r, rtol=1e-10, atol=1e-15)


def test_common_sld_shift_invariance():
    """Only SLD differences matter: shifting all SLDs leaves R unchanged."""
    p = W.pack([150.0, 320.0], [1e-6, 3e-6, 5.5e-6, 2.07e-6], [1e-9, 0.0, 0.0], [3.0, 4.0, 5.0], 1, 0)
    q = p.copy()
    L = W.layout(2)
    q[L["rho"]] += 1.7e-6
    np.testing.assert_allclose(np.abs(oracle.amplitude(2, q, QGRID)), np.abs(oracle.amplitude(2, p, QGRID)),
                               rtol=1e-9, atol=1e-15)


def test_abeles_matches_parratt_many_stacks():
    rng = np.random.default_rng(7)
    for _ in range(25):
        n = int(rng.integers(1, 9))
        d, rho, iota, sig = rng.uniform(5, 700, n), rng.uniform(-0.5e-6, 6.5e-6, n), \
            rng.uniform(0, 2e-8, n), rng.uniform(0, 15, n + 1)
        p = W.pack(d, np.concatenate([[rng.choice([0, 6.35e-6])], rho, [2.07e-6]]),
                   np.concatenate([iota, [rng.uniform(0, 1e-9)]]), sig, 1, 0)
        a = oracle.amplitude(n, p, QGRID, form=0)
        b = oracle.amplitude(n, p, QGRID, form=1)
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-15)


def test_long_double_build_agrees():
    assert oracle.real_bytes("long") > 8
    p = W.pack([1470.0, 12.0], [0.0, 4.24e-6, 3.5e-6, 2.07e-6], [0.0, 0.0, 0.0], [11.4, 10.9, 3.2], 1, 1e-7)
    a = oracle.amplitude(2, p, QGRID)
    b = oracle.amplitude(2, p, QGRID, precision="long")
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-16)
    Q = QGRID.astype(np.float32).astype(np.float64)
    m = oracle.model(2, p, Q, 0.03 * Q, 21)
    mb = oracle.model(2, p, Q, 0.03 * Q, 21, precision="long")
    np.testing.assert_allclose(m, mb, rtol=1e-12)


# ---------------------------------------------------------------- smearing
@pytest.mark.parametrize("d,rel,K,tol", [(80.0, 0.05, 17, 1e-7), (300.0, 0.05, 21, 1e-5)])
def test_smearing_matches_brute_force_convolution(d, rel, K, tol):
    """GH smearing vs a 20001-point trapezoid convolution with the FWHM
    Gaussian exp(-4 ln2 (q-Q)^2 / dQ^2) over +-8 sigma."""
    p = one_layer(d, 4.2e-6, 0.0, [3.0, 5.0], scale=1.0, bkg=0.0)
    Qs = np.array([0.03, 0.06, 0.1, 0.2])
    dQ = rel * Qs
    m = oracle.model(1, p, Qs, dQ, K)
    for i, (Q, dq) in enumerate(zip(Qs, dQ)):
        sig = dq / (2 * math.sqrt(2 * math.log(2)))
        qq = np.linspace(Q - 8 * sig, Q + 8 * sig, 20001)
        g = np.exp(-4 * math.log(2) * (qq - Q) ** 2 / dq ** 2)
        R = oracle.reflectivity_unsmeared(1, p, qq)
        ref = np.trapezoid(g * R, qq) / np.trapezoid(g, qq)
        assert abs(m[i] - ref) <= tol * ref, (Q, m[i], ref)


def test_zero_resolution_is_unsmeared():
    p = one_layer(150.0, 4.2e-6, 0.0, [3.0, 5.0], scale=1.0, bkg=0.0)
    m = oracle.model(1, p, QGRID, np.zeros_like(QGRID), 17)
    np.testing.assert_allclose(m, oracle.reflectivity_unsmeared(1, p, QGRID), rtol=1e-14)


def test_scale_and_background():
    p = one_layer(150.0, 4.2e-6, 0.0, [3.0, 5.0], scale=1.0, bkg=0.0)
    p2 = one_layer(150.0, 4.2e-6, 0.0, [3.0, 5.0], scale=1.37, bkg=2.5e-7)
    a = oracle.model(1, p, QGRID, 0.04 * QGRID, 17)
    b = oracle.model(1, p2, QGRID, 0.04 * QGRID, 17)
    np.testing.assert_allclose(b, 1.37 * a + 2.5e-7, rtol=1e-13)


# -------------------------------------------------------------- likelihood
def test_loglik_is_gaussian_logpdf():
    p = one_layer(1470.0, 4.24e-6, 0.0, [11.4, 10.9], scale=1.048, bkg=1.05e-7)
    Q = W.log_grid(200, 0.005, 0.25).astype(np.float64)
    dQ = 0.03 * Q
    m = oracle.model(1, p, Q, dQ, 21)
    rng = np.random.default_rng(3)
    err = 0.05 * m
    Robs = m * np.exp(rng.normal(0, 0.05, m.size))
    ll, _ = oracle.loglik_grad(1, p, Q, dQ, Robs, err, 21, grad=False)
    ref = scipy.stats.norm.logpdf(Robs, loc=m, scale=err).sum()
    assert abs(ll - ref) <= 1e-10 * abs(ref)


# ---------------------------------------------------------------- gradient
@pytest.mark.parametrize("n", [0, 1, 3])
def test_dual_gradient_matches_central_differences(n):
    rng = np.random.default_rng(11 + n)
    d = rng.uniform(40, 400, n)
    # absorptions strictly positive: at iota = 0 below a critical edge the
    # principal branch makes d/d(iota) one-sided, which central FD cannot see
    p = W.pack(d, np.concatenate([[0.0], rng.uniform(1e-6, 6e-6, n), [2.07e-6]]),
               np.concatenate([rng.uniform(1e-9, 1e-8, n), [1e-9]]), rng.uniform(2, 9, n + 1), 1.02, 1.3e-7)
    Q = W.log_grid(60, 0.006, 0.25).astype(np.float64)
    dQ = 0.05 * Q
    m = oracle.model(n, p, Q, dQ, 17)
    Robs = m * np.exp(rng.normal(0, 0.05, m.size))
    err = 0.05 * m
    ll, g = oracle.loglik_grad(n, p, Q, dQ, Robs, err, 17)
    typ = W.typical_scale(n)
    fd = np.zeros_like(g)
    for i in range(p.size):
        h = 1e-6 * typ[i]
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fp, _ = oracle.loglik_grad(n, pp, Q, dQ, Robs, err, 17, grad=False)
        fm, _ = oracle.loglik_grad(n, pm, Q, dQ, Robs, err, 17, grad=False)
        fd[i] = (fp - fm) / (2 * h)
    scaled = np.abs((g - fd) * typ)
    assert scaled.max() <= 1e-5 * np.abs(g * typ).max(), (g, fd)
    # only SLD differences matter: the fronting-SLD gradient is minus the sum
    L = W.layout(n)
    grho = g[L["rho"]]
    assert abs(grho[0] + grho[1:].sum()) <= 1e-9 * np.abs(grho).max()


def test_rejects_bad_inputs():
    p = one_layer(100.0, 4e-6, 0.0, [3.0, 3.0])
    with pytest.raises(ValueError):
        oracle.amplitude(1, p, np.array([0.01, -0.02]))
    with pytest.raises(ValueError):
        oracle.loglik_grad(1, p, np.array([0.01]), np.array([0.0]), np.array([1.0]), np.array([0.0]), 17)
    bad = p.copy()
    bad[0] = np.nan
    with pytest.raises(ValueError):
        oracle.amplitude(1, bad, np.array([0.01]))


def test_batch_driver_matches_single_stack_calls():
    wl = W.make_workload("oled_cofit", n_stacks=2)
    ll, g = oracle.batch("grad", wl.n_layers, wl.params, wl.dataset, wl.q_off, wl.q, wl.dq,
                         wl.r_obs, wl.r_err, wl.n_quad)
    for s in range(wl.n_stacks):
        Q, dQ, Ro, e = wl.dataset_arrays(int(wl.dataset[s]))
        l1, g1 = oracle.loglik_grad(int(wl.n_layers[s]), wl.stack_params(s), Q, dQ, Ro, e, wl.n_quad)
        assert ll[s] == l1
        po = wl.par_off
        np.testing.assert_array_equal(g[po[s]:po[s + 1]], g1)


# ------------------------------------------------ resolution (smearing) scale
def test_resolution_derivative_fresnel_closed_form():
    """d loglik / d ln f (every dQ_i -> f dQ_i) for a bare rough-free
    substrate, written out here from the Fresnel amplitude: with k_0 = q/2,
    k_1 = sqrt(k_0^2 - 4 pi drho), dr/dk_0 = -8 pi drho / (k_1 (k_0 + k_1)^2),
    dR/dq = Re(conj(r) dr/dk_0) and dq_k/d ln f = sqrt(2) sigma_Q x_k."""
    drho, scale, bkg, K = 2.07e-6, 0.97, 2e-7, 17
    p = W.pack([], [0.0, drho], [0.0], [0.0], scale, bkg)
    Q = W.log_grid(80, 0.005, 0.3).astype(np.float64)   # spans the critical edge
    dQ = 0.05 * Q
    rng = np.random.default_rng(5)
    m = oracle.model(0, p, Q, dQ, K)
    Robs = m * np.exp(rng.normal(0, 0.05, m.size))
    err = 0.05 * m
    x, w = np.polynomial.hermite.hermgauss(K)
    sig = dQ / (2 * np.sqrt(2 * np.log(2)))
    q = Q[:, None] + np.sqrt(2) * sig[:, None] * x[None, :]
    k0 = q / 2
    k1 = np.sqrt(k0 ** 2 - FOURPI * drho + 0j)
    r = (k0 - k1) / (k0 + k1)
    dr = -2 * FOURPI * drho / (k1 * (k0 + k1) ** 2)
    dR = np.real(np.conj(r) * dr)
    S = (w / np.sqrt(np.pi) * np.abs(r) ** 2).sum(axis=1)
    dS = (w / np.sqrt(np.pi) * dR * np.sqrt(2) * sig[:, None] * x[None, :]).sum(axis=1)
    mm = scale * S + bkg
    ref = np.sum(-(mm - Robs) / err ** 2 * scale * dS)
    got = oracle.loglik_grad_res(0, p, Q, dQ, Robs, err, K)
    assert abs(got - ref) <= 1e-9 * np.sum(np.abs((mm - Robs) / err ** 2 * scale * dS))


@pytest.mark.parametrize("n", [1, 3])
def test_resolution_derivative_matches_central_differences(n):
    rng = np.random.default_rng(23 + n)
    p = W.pack(rng.uniform(60, 900, n), np.concatenate([[0.0], rng.uniform(1e-6, 6e-6, n), [2.07e-6]]),
               np.concatenate([rng.uniform(1e-9, 1e-8, n), [0.0]]), rng.uniform(2, 12, n + 1), 1.01, 1e-7)
    Q = W.log_grid(70, 0.005, 0.25).astype(np.float64)
    dQ = rng.uniform(0.02, 0.08, Q.size) * Q
    m = oracle.model(n, p, Q, dQ, 21)
    Robs = m * np.exp(rng.normal(0, 0.05, m.size))
    err = 0.05 * m
    g = oracle.loglik_grad_res(n, p, Q, dQ, Robs, err, 21)
    h = 1e-5
    fp, _ = oracle.loglik_grad(n, p, Q, dQ * np.exp(h), Robs, err, 21, grad=False, precision="long")
    fm, _ = oracle.loglik_grad(n, p, Q, dQ * np.exp(-h), Robs, err, 21, grad=False, precision="long")
    assert abs(g - (fp - fm) / (2 * h)) <= 1e-7 * abs(g)


def test_resolution_derivative_vanishes_without_smearing():
    p = one_layer(250.0, 4.5e-6, 1e-9, [4.0, 6.0], scale=1.0, bkg=1e-7)
    Q = W.log_grid(40, 0.006, 0.2).astype(np.float64)
    m = oracle.model(1, p, Q, np.zeros_like(Q), 17)
    assert oracle.loglik_grad_res(1, p, Q, np.zeros_like(Q), m * 1.03, 0.05 * m, 17) == 0.0


def test_batch_resolution_mode_matches_single_stack_calls():
    wl = W.make_workload("uneven", n_stacks=3)
    ll, g = oracle.batch("grad", wl.n_layers, wl.params, wl.dataset, wl.q_off, wl.q, wl.dq,
                         wl.r_obs, wl.r_err, wl.n_quad)
    ll3, g3, gr = oracle.batch("grad_res", wl.n_layers, wl.params, wl.dataset, wl.q_off, wl.q, wl.dq,
                               wl.r_obs, wl.r_err, wl.n_quad)
    np.testing.assert_array_equal(ll, ll3)
    np.testing.assert_array_equal(g, g3)
    for s in range(wl.n_stacks):
        Q, dQ, Ro, e = wl.dataset_arrays(int(wl.dataset[s]))
        assert gr[s] == oracle.loglik_grad_res(int(wl.n_layers[s]), wl.stack_params(s), Q, dQ, Ro, e, wl.n_quad)


# -------------------------------------------------------------- SLD profile
def test_sld_profile_sharp_steps_and_far_field():
    """sigma = 0: the profile is the media's SLDs between the interface
    depths; far outside it is the fronting and backing value."""
    d = [120.0, 35.0, 260.0]
    rho = [0.0, 4.1e-6, -0.4e-6, 2.9e-6, 2.07e-6]
    iota = [1e-8, 0.0, 3e-8, 0.0]
    p = W.pack(d, rho, iota, [0.0] * 4, 1.0, 0.0)
    edges = np.concatenate([[0.0], np.cumsum(d)])
    z = np.linspace(-50, 480, 531)
    r, i = oracle.sld_profile(3, p, z)
    medium = np.searchsorted(edges, z, side="right")   # 0 fronting .. 4 backing
    # the profile is rho_0 plus the steps: exact up to the rounding of that sum
    np.testing.assert_allclose(r, np.asarray(rho)[medium], rtol=0, atol=1e-20)
    np.testing.assert_allclose(i, np.concatenate([[0.0], iota])[medium], rtol=0, atol=1e-22)
    p2 = W.pack(d, rho, iota, [4.0, 9.0, 3.0, 6.0], 1.0, 0.0)
    r2, _ = oracle.sld_profile(3, p2, np.array([-400.0, 1200.0]))
    assert abs(r2[0] - rho[0]) < 1e-20 and abs(r2[1] - rho[-1]) < 1e-20


def test_sld_profile_single_interface_midpoint():
    p = W.pack([], [1.5e-6, 6.3e-6], [0.0], [7.0], 1.0, 0.0)
    r, _ = oracle.sld_profile(0, p, np.array([0.0, -7.0, 7.0]))
    assert abs(r[0] - (1.5e-6 + 6.3e-6) / 2) < 1e-21
    assert abs((r[1] - 1.5e-6) + (r[2] - 6.3e-6)) < 1e-21       # odd about the interface


def test_sld_profile_is_gaussian_smoothed_step_profile():
    """With one roughness on every interface the profile is the sharp profile
    convolved with a normal density of that width (brute-force sum on a fine
    grid), whatever the layer spacing."""
    d = [30.0, 8.0, 55.0]
    rho = [0.0, 5.2e-6, 1.1e-6, 3.4e-6, 2.07e-6]
    sig = 6.0
    sharp = W.pack(d, rho, [0.0] * 4, [0.0] * 4, 1.0, 0.0)
    rough = W.pack(d, rho, [0.0] * 4, [sig] * 4, 1.0, 0.0)
    h = 0.01
    # cell-centred samples: no sample sits on an interface depth
    zf = -150 + h * (np.arange(40000) + 0.5)
    step, _ = oracle.sld_profile(3, sharp, zf)
    t = h * np.arange(-6000, 6001)
    kern = np.exp(-0.5 * (t / sig) ** 2)
    kern /= kern.sum()
    conv = scipy.signal.fftconvolve(step, kern, mode="same")
    z = np.arange(-40.0, 130.0, 1.7)
    idx = np.round((z - zf[0]) / h).astype(int)
    r, _ = oracle.sld_profile(3, rough, zf[idx])
    np.testing.assert_allclose(r, conv[idx], rtol=0, atol=1e-6 * max(abs(x) for x in rho))
