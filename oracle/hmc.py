"""TEST INFRASTRUCTURE ONLY: plain CPU reference of one Hamiltonian Monte
Carlo step of a co-fitted slab model (arXiv 2509.06924, Sec. 2.3: leapfrog
integration, Eq. 7, over L steps of size dt with mass matrix M, then the
Metropolis-Hastings acceptance of Eq. 8; uniform box priors as in Tables 1-4;
sampling in an unconstrained space as Sec. 2.3.1 advises for bounded
parameters).  Only the tests may import it.

Model of one chain.  Free parameters theta_k (k < P) with uniform priors on
[lo_k, hi_k]; each contrast c of the chain is a stack whose packed slots
(layout d | rho | iota | sigma | scale | bkg) either copy a free parameter
(slot_src >= 0, parameters tied across contrasts) or hold a fixed value.
Sampling runs in the unconstrained coordinates u:
    theta_k = lo_k + (hi_k - lo_k) sigmoid(u_k),
    log pi(u) = sum_c loglik_c(theta(u)) + sum_k [log s_k + log(1 - s_k)],
the second sum being the uniform prior density times the Jacobian of the
map (up to the constant sum_k log(hi_k - lo_k) - log(hi_k - lo_k) = 0).
Optionally one free parameter (res_param) is a resolution scale f shared by
every contrast: each dataset's dQ_i becomes f dQ_i (the shared smearing
percentage of the LED co-fit, Sec. 4.2, is such an f when dQ_i = Q_i), and
d loglik / d f = (d loglik / d ln f) / f from the resolution derivative.

One step from u0 with standard-normal draws z (one per parameter) and a
uniform draw U (as log U), diagonal inverse mass m^-1, step eps, L steps:
    p = z / sqrt(m^-1);  H0 = -log pi(u0) + 1/2 sum p^2 m^-1
    p += eps/2 grad;  then L times: u += eps m^-1 p, p += eps grad (eps/2 on
    the last);  H1 likewise;  accept iff log U < H0 - H1 (NaN rejects).
Random numbers are inputs, so a GPU implementation can be compared draw for
draw.
"""
from __future__ import annotations

import numpy as np

import oracle


class Model:
    """n_layers, dataset: per contrast; slot_src/slot_val: per contrast,
    concatenated packed blocks; lo/hi: per free parameter; data: (q_off, Q,
    dQ, Robs, err) shared by all chains; K quadrature nodes."""

    def __init__(self, n_layers, dataset, slot_src, slot_val, lo, hi, q_off, Q, dQ, Robs, err, K, res_param=-1):
        self.n_layers = np.asarray(n_layers, np.int32)
        self.dataset = np.asarray(dataset, np.int32)
        self.slot_src = np.asarray(slot_src, np.int64)
        self.slot_val = np.asarray(slot_val, np.float64)
        self.lo = np.asarray(lo, np.float64)
        self.hi = np.asarray(hi, np.float64)
        self.q_off = np.asarray(q_off, np.int64)
        self.Q, self.dQ = np.asarray(Q, np.float64), np.asarray(dQ, np.float64)
        self.Robs, self.err = np.asarray(Robs, np.float64), np.asarray(err, np.float64)
        self.K = int(K)
        self.P = self.lo.size
        self.res_param = int(res_param)
        assert -1 <= self.res_param < self.P
        self.n_slots = int(np.sum(4 * self.n_layers + 6))
        assert self.slot_src.size == self.n_slots == self.slot_val.size

    def theta(self, u):
        s = 1.0 / (1.0 + np.exp(-u))
        return self.lo + (self.hi - self.lo) * s, s

    def packed(self, u):
        """Packed parameters of the chain's contrasts (concatenated)."""
        th, _ = self.theta(u)
        out = self.slot_val.copy()
        tied = self.slot_src >= 0
        out[tied] = th[self.slot_src[tied]]
        return out

    def logp_grad(self, u):
        """(log pi(u), d log pi / du) of one chain."""
        th, s = self.theta(u)
        p = self.packed(u)
        C = self.n_layers.size
        gt = np.zeros(self.P)                         # d loglik / d theta, tied slots summed
        if self.res_param >= 0:
            f = th[self.res_param]
            ll, g, gres = oracle.batch("grad_res", self.n_layers, p, self.dataset, self.q_off, self.Q,
                                       f * self.dQ, self.Robs, self.err, self.K)
            gt[self.res_param] = np.sum(gres) / f
        else:
            ll, g = oracle.batch("grad", self.n_layers, p, self.dataset, self.q_off, self.Q, self.dQ, self.Robs,
                                 self.err, self.K)
        tied = self.slot_src >= 0
        np.add.at(gt, self.slot_src[tied], g[tied])
        # log s + log(1 - s) = -|u| - 2 log(1 + e^-|u|)
        prior = np.sum(-np.abs(u) - 2.0 * np.log1p(np.exp(-np.abs(u))))
        grad = gt * (self.hi - self.lo) * s * (1.0 - s) + (1.0 - 2.0 * s)
        assert C == ll.size
        return float(np.sum(ll) + prior), grad


def leapfrog(logp_grad, u, p, inv_mass, eps, L):
    """L leapfrog steps from (u, p); returns (u, p, log pi, grad) at the end."""
    lp, g = logp_grad(u)
    p = p + 0.5 * eps * g
    for step in range(L):
        u = u + eps * inv_mass * p
        lp, g = logp_grad(u)
        p = p + (0.5 if step == L - 1 else 1.0) * eps * g
    return u, p, lp, g


def hmc_step(logp_grad, u0, z, log_unif, inv_mass, eps, L):
    """One HMC transition of one chain: returns (u, log pi(u), accepted,
    H0, H1) with u = u0 when rejected."""
    p0 = z / np.sqrt(inv_mass)
    lp0, _ = logp_grad(u0)
    H0 = -lp0 + 0.5 * np.sum(p0 * p0 * inv_mass)
    u1, p1, lp1, _ = leapfrog(logp_grad, u0, p0, inv_mass, eps, L)
    H1 = -lp1 + 0.5 * np.sum(p1 * p1 * inv_mass)
    acc = bool(log_unif < H0 - H1)          # False for NaN
    return (u1, lp1, True, H0, H1) if acc else (u0, lp0, False, H0, H1)
