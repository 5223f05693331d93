"""Pins of the CPU HMC reference (oracle/hmc.py): the leapfrog map against
the closed form of the harmonic oscillator, time reversibility and the
second-order energy error on a reflectivity posterior, the unconstrained
posterior's gradient against central differences, and the
Metropolis-Hastings decision at its limits (CPU only)."""
import numpy as np
import pytest

from oracle import hmc
from paper_2509_06924_gb300 import workloads as W


def test_leapfrog_is_the_harmonic_oscillator_map():
    """log pi = -u^2/2, unit mass: one leapfrog step is the linear map
    [[1 - e^2/2, e], [-e (1 - e^2/4), 1 - e^2/2]] on (u, p)."""
    def lg(u):
        return float(-0.5 * np.sum(u * u)), -u
    rng = np.random.default_rng(3)
    u0, p0 = rng.normal(size=4), rng.normal(size=4)
    for eps, L in ((0.1, 1), (0.3, 7), (1.2, 5)):
        A = np.array([[1 - eps ** 2 / 2, eps], [-eps * (1 - eps ** 2 / 4), 1 - eps ** 2 / 2]])
        AL = np.linalg.matrix_power(A, L)
        u, p, lp, g = hmc.leapfrog(lg, u0, p0, np.ones(4), eps, L)
        np.testing.assert_allclose(u, AL[0, 0] * u0 + AL[0, 1] * p0, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(p, AL[1, 0] * u0 + AL[1, 1] * p0, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(g, -u, rtol=0, atol=0)


def small_model(seed=7):
    """Two contrasts (D2O-like and air fronting) of a 2-layer film sharing
    the layers; scale per contrast; 7 free parameters."""
    rng = np.random.default_rng(seed)
    n = 2
    Q = W.log_grid(40, 0.008, 0.2).astype(np.float64)
    q_off = np.array([0, Q.size, 2 * Q.size])
    Qa = np.concatenate([Q, Q])
    dQ = 0.04 * Qa
    # free: d1, d2, rho1, rho2, sigma01, scale_c0, scale_c1
    lo = np.array([80.0, 20.0, 2e-6, 0.5e-6, 2.0, 0.9, 0.9])
    hi = np.array([200.0, 90.0, 6e-6, 3.0e-6, 9.0, 1.1, 1.1])
    truth = lo + (hi - lo) * rng.uniform(0.3, 0.7, lo.size)
    blocks_src, blocks_val = [], []
    for c, front in enumerate((6.35e-6, 0.0)):
        L = W.layout(n)
        src = -np.ones(4 * n + 6, np.int64)
        val = W.pack([0.0, 0.0], [front, 0.0, 0.0, 2.07e-6], [1e-9, 0.0, 0.0], [0.0, 4.0, 3.0], 0.0, 2e-7)
        rho0, sig0 = L["rho"].start, L["sigma"].start
        src[L["d"]] = [0, 1]
        src[rho0 + 1:rho0 + 3] = [2, 3]
        src[sig0] = 4
        src[L["scale"]] = 5 + c
        blocks_src.append(src)
        blocks_val.append(val)
    slot_src, slot_val = np.concatenate(blocks_src), np.concatenate(blocks_val)
    m0 = hmc.Model([n, n], [0, 1], slot_src, slot_val, lo, hi, q_off, Qa, dQ, np.ones(Qa.size),
                   np.ones(Qa.size), 17)
    u_t = np.log((truth - lo) / (hi - truth))
    import oracle
    m = oracle.batch("model", m0.n_layers, m0.packed(u_t), m0.dataset, q_off, Qa, dQ, None, None, 17)
    Robs = m * np.exp(rng.normal(0, 0.05, m.size))
    return hmc.Model([n, n], [0, 1], slot_src, slot_val, lo, hi, q_off, Qa, dQ, Robs, 0.05 * m, 17), u_t


def with_resolution(model, lo=0.6, hi=1.4):
    """The same model with one more free parameter: a resolution scale f of
    every dQ (both contrasts), prior [lo, hi]."""
    import oracle
    mod = hmc.Model(model.n_layers, model.dataset, model.slot_src, model.slot_val, np.append(model.lo, lo),
                    np.append(model.hi, hi), model.q_off, model.Q, model.dQ, model.Robs, model.err, model.K,
                    res_param=model.P)
    return mod


@pytest.mark.parametrize("res", [False, True])
def test_unconstrained_gradient_matches_central_differences(res):
    model, u_t = small_model()
    if res:
        model = with_resolution(model)
        u_t = np.append(u_t, 0.4)
    u = u_t + 0.3
    lp, g = model.logp_grad(u)
    for k in range(model.P):
        h = 1e-6
        e = np.zeros(model.P)
        e[k] = h
        fd = (model.logp_grad(u + e)[0] - model.logp_grad(u - e)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(g[k]))


def test_resolution_parameter_scales_every_dq():
    """log pi with a free resolution scale f equals the model without it,
    evaluated on the data with every dQ multiplied by f, plus the prior
    term of f."""
    model, u_t = small_model()
    mres = with_resolution(model)
    for uf in (-1.2, 0.0, 0.7):
        f = 0.6 + 0.8 / (1.0 + np.exp(-uf))
        lp, _ = mres.logp_grad(np.append(u_t, uf))
        scaled = hmc.Model(model.n_layers, model.dataset, model.slot_src, model.slot_val, model.lo, model.hi,
                           model.q_off, model.Q, f * model.dQ, model.Robs, model.err, model.K)
        lp0, _ = scaled.logp_grad(u_t)
        prior_f = -abs(uf) - 2.0 * np.log1p(np.exp(-abs(uf)))
        assert abs(lp - (lp0 + prior_f)) <= 1e-12 * abs(lp)


def test_packed_slots_tie_and_fix():
    model, u_t = small_model()
    th, _ = model.theta(u_t)
    p = model.packed(u_t)
    L = W.layout(2)
    d0, rho0 = L["d"].start, L["rho"].start
    assert p[d0] == th[0] and p[14 + d0] == th[0]                        # tied across contrasts
    assert p[L["scale"]] == th[5] and p[14 + L["scale"]] == th[6]        # per-contrast scale
    assert p[rho0] == 6.35e-6 and p[14 + rho0] == 0.0                    # fixed fronting


def test_reversibility_and_second_order_energy_error():
    model, u_t = small_model()
    rng = np.random.default_rng(1)
    inv_mass = np.ones(model.P)
    u0, p0 = u_t + 0.05 * rng.normal(size=model.P), rng.normal(size=model.P)
    u1, p1, _, _ = hmc.leapfrog(model.logp_grad, u0, p0, inv_mass, 2e-3, 6)
    ub, pb, _, _ = hmc.leapfrog(model.logp_grad, u1, -p1, inv_mass, 2e-3, 6)
    np.testing.assert_allclose(ub, u0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(-pb, p0, rtol=0, atol=1e-7)

    def dH(eps, L):
        lp0, _ = model.logp_grad(u0)
        u, p, lp, _ = hmc.leapfrog(model.logp_grad, u0, p0, inv_mass, eps, L)
        return (-lp + 0.5 * np.sum(p * p)) - (-lp0 + 0.5 * np.sum(p0 * p0))
    # same trajectory length, half the step: the energy error drops ~4x
    # (steps well inside the stability limit of this stiff posterior)
    r = dH(1e-3, 10) / dH(5e-4, 20)
    assert 3.5 < r < 4.5


@pytest.mark.parametrize("log_u,accept", [(-np.inf, True), (np.inf, False), (np.nan, False)])
def test_metropolis_decision_limits(log_u, accept):
    model, u_t = small_model()
    z = np.random.default_rng(2).normal(size=model.P)
    u, lp, acc, H0, H1 = hmc.hmc_step(model.logp_grad, u_t, z, log_u, np.ones(model.P), 2e-3, 3)
    assert acc == accept
    if not accept:
        np.testing.assert_array_equal(u, u_t)
        assert lp == model.logp_grad(u_t)[0]
