"""Pins of the CPU VI reference (oracle/vi.py): its single-sample estimates
against the closed-form ELBO of a Gaussian target, the zero-variance ELBO
when q equals the target, and its Adam update against torch.optim.Adam
(CPU only)."""
import numpy as np
import pytest

from oracle import vi


def gaussian_target(P, seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(P, P))
    A = B @ B.T + P * np.eye(P)                  # precision matrix
    return A, (lambda u: (float(-0.5 * u @ A @ u), -A @ u))


def random_phi(P, rng):
    mu = rng.normal(size=P)
    tri = np.zeros(vi.n_tri(P))
    idx = 0
    for i in range(P):
        for j in range(i + 1):
            tri[idx] = rng.normal(-0.5, 0.2) if i == j else 0.3 * rng.normal()
            idx += 1
    return mu, tri


@pytest.mark.parametrize("P", [1, 3, 6])
def test_design_average_is_the_exact_elbo_gradient(P):
    """For log pi = -u^T A u / 2 the loss is linear in e e^T, so averaging
    the single-sample estimates over e = +-sqrt(P) e_k (mean 0, second
    moment I) gives the exact expectation:
      ELBO = -(mu^T A mu + tr(L^T A L))/2 + sum log L_ii + P/2 + P/2 log 2 pi,
      d loss/d mu = A mu, d loss/d L_ij = (A L)_ij, d loss/d log L_ii = (A L)_ii L_ii - 1."""
    A, lg = gaussian_target(P, 10 + P)
    mu, tri = random_phi(P, np.random.default_rng(P))
    L = vi.unpack_L(tri, P)
    acc = np.zeros(P + tri.size)
    elbo = 0.0
    designs = [s * np.sqrt(P) * np.eye(P)[k] for k in range(P) for s in (1.0, -1.0)]
    for e in designs:
        el, gm, gt = vi.loss_grad(lg, mu, tri, e)
        acc += np.concatenate([gm, gt]) / len(designs)
        elbo += el / len(designs)
    AL = A @ L
    exact_elbo = -0.5 * (mu @ A @ mu + np.trace(L.T @ A @ L)) + np.sum(np.log(np.diag(L))) + P / 2 \
        + P / 2 * np.log(2 * np.pi)
    assert abs(elbo - exact_elbo) <= 1e-10 * abs(exact_elbo)
    np.testing.assert_allclose(acc[:P], A @ mu, rtol=1e-10, atol=1e-12)
    idx = P
    for i in range(P):
        for j in range(i + 1):
            want = AL[i, i] * L[i, i] - 1.0 if i == j else AL[i, j]
            assert abs(acc[idx] - want) <= 1e-10 * max(1.0, abs(want))
            idx += 1


def test_elbo_has_zero_variance_when_q_is_the_target():
    """q = N(0, Sigma) against log pi = -u^T Sigma^-1 u / 2: every draw gives
    the log normaliser P/2 log 2 pi + log det Sigma / 2."""
    P = 4
    A, lg = gaussian_target(P, 3)
    Sigma = np.linalg.inv(A)
    C = np.linalg.cholesky(Sigma)
    tri = np.zeros(vi.n_tri(P))
    idx = 0
    for i in range(P):
        for j in range(i + 1):
            tri[idx] = np.log(C[i, i]) if i == j else C[i, j]
            idx += 1
    logZ = P / 2 * np.log(2 * np.pi) + 0.5 * np.linalg.slogdet(Sigma)[1]
    rng = np.random.default_rng(4)
    for _ in range(5):
        el, _, _ = vi.loss_grad(lg, np.zeros(P), tri, rng.normal(size=P))
        assert abs(el - logZ) <= 1e-12 * max(1.0, abs(logZ))


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    x0 = rng.normal(size=7)
    grads = [rng.normal(size=7) for _ in range(6)]
    xt = torch.tensor(x0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([xt], lr=0.05, betas=(0.9, 0.999), eps=1e-8)
    x, m, v = x0.copy(), np.zeros(7), np.zeros(7)
    for t, g in enumerate(grads, start=1):
        opt.zero_grad()
        xt.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        x, m, v = vi.adam(x, g, m, v, t, 0.05)
        np.testing.assert_allclose(x, xt.detach().numpy(), rtol=1e-13, atol=1e-15)
