"""TEST INFRASTRUCTURE ONLY: plain CPU reference of one step of variational
inference for a co-fitted slab model (arXiv 2509.06924, Sec. 2.4 and the LED
fit of Sec. 4.2): a multivariate normal q(u; phi) = N(mu, L L^T) in the
unconstrained space of oracle/hmc.py, the single-sample reparameterised
estimate of the negative ELBO (Eqs. 22-24) and one Adam update of phi, for
many independent restarts.  Only the tests may import it.

phi of one restart: mu [P] and the lower triangle of L, packed row by row
((i, j <= i) at i (i + 1) / 2 + j) with the diagonal stored as log L_ii.
With a standard-normal draw e, u = mu + L e and
    loss = -log pi(u) + log q(u) = -log pi(u) - e^T e / 2 - sum_i log L_ii - P/2 log(2 pi),
whose gradient (e held fixed) is
    d loss / d mu = -g,   d loss / d L_ij = -g_i e_j (j < i),
    d loss / d log L_ii = -g_i e_i L_ii - 1,     g = d log pi / du at u.
Adam (Kingma and Ba) minimises the loss with the usual bias corrections.
The ELBO estimate returned is -loss.
"""
from __future__ import annotations

import numpy as np


def n_tri(P: int) -> int:
    return P * (P + 1) // 2


def unpack_L(tri, P):
    L = np.zeros((P, P))
    idx = 0
    for i in range(P):
        for j in range(i + 1):
            L[i, j] = np.exp(tri[idx]) if i == j else tri[idx]
            idx += 1
    return L


def loss_grad(logp_grad, mu, tri, e):
    """(ELBO estimate, d loss / d mu, d loss / d tri) of one restart."""
    P = mu.size
    L = unpack_L(tri, P)
    u = mu + L @ e
    lp, g = logp_grad(u)
    logdiag = np.array([tri[i * (i + 1) // 2 + i] for i in range(P)])
    elbo = lp + 0.5 * float(e @ e) + float(np.sum(logdiag)) + 0.5 * P * np.log(2 * np.pi)
    g_mu = -g
    g_tri = np.zeros_like(tri)
    idx = 0
    for i in range(P):
        for j in range(i + 1):
            g_tri[idx] = -g[i] * e[i] * L[i, i] - 1.0 if i == j else -g[i] * e[j]
            idx += 1
    return elbo, g_mu, g_tri


def adam(x, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t = 1, 2, ...) of parameters x with gradient grad;
    returns (x, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return x - lr * mh / (np.sqrt(vh) + eps), m, v


def vi_step(logp_grad, mu, tri, m, v, t, e, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One iteration of one restart: phi = (mu, tri) and the Adam moments m, v
    (ordered mu then tri).  Returns (mu, tri, m, v, ELBO estimate at the
    incoming phi)."""
    elbo, g_mu, g_tri = loss_grad(logp_grad, mu, tri, e)
    x = np.concatenate([mu, tri])
    grad = np.concatenate([g_mu, g_tri])
    x, m, v = adam(x, grad, m, v, t, lr, beta1, beta2, eps)
    P = mu.size
    return x[:P], x[P:], m, v, elbo
