"""Seeded synthetic workloads for the batched reflectivity path.

Input generation only: parameter draws, Q grids, resolutions, packing and
data-file I/O.  No reflectivity arithmetic lives here, so the CUDA library
and the CPU oracle can both be fed from this module.

The paper's datasets (D17 quartz film, ISIS OLED devices, refnx lipid
bilayer; Secs. 4.1, 4.2 and supplement S2) are not available, so every
workload is synthetic with the shapes of the paper's fits:

* ``film_1l``      1024 one-layer films on Si, 200 log-spaced Q in
                   [0.005, 0.3], dQ/Q = 5 % FWHM, 17 quadrature nodes.
* ``thick_oxide``  16384 thick (1000-3000 A) quartz-like films on Si,
                   400 Q in [0.005, 0.25], dQ/Q = 3 %, 21 nodes (the quartz
                   fit of Sec. 4.1, Tables 1-2).
* ``oled_cofit``   4096 chains x 3 contrasts of a 10-layer stack, Q lengths
                   150/220/300, dQ/Q = 5 %, 17 nodes (the LED co-fit of
                   Sec. 4.2, Tables 3-4).
* ``uneven``       10000 stacks with 1..20 layers, each with its own dataset
                   of 50..500 Q points and dQ/Q in [2 %, 8 %], 17 nodes.
* ``vi_step``      65536 reparameterised samples x 3 contrasts x 12 layers x
                   300 Q, dQ/Q = 5 %, 21 nodes (one VI/HMC gradient step).

Observed data: where ``tests/golden/data_<name>.txt`` exists it holds R_obs
and e written by a script that calls only the oracle (truth draw x
lognormal 5 % noise, e = 0.05 R_true).  Otherwise (``uneven``, whose 10000
datasets are too large to store) R_obs is a smooth stand-in envelope
min(1, (0.0102/Q)^4) x lognormal noise; it only has to have the right
magnitude, since the cost of the path does not depend on the data values.

Packed parameter layout of a stack with n layers (4n+6 float64 values):
``d[n] | rho[n+2] | iota[n+1] | sigma[n+1] | scale | bkg`` (thickness in A,
SLDs in absolute A^-2, roughness in A).
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np

SEED_BASE = 2509069240
CONFIG_IDS = {"film_1l": 1, "thick_oxide": 2, "oled_cofit": 3, "uneven": 4, "vi_step": 5}
GOLDEN_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")

SI_SLD = 2.07e-6
CONTRASTS = ((0.0, 2.07e-6), (6.35e-6, 2.07e-6), (0.0, 4.2e-6))  # fronting / backing SLD


def n_params(n: int) -> int:
    return 4 * n + 6


def layout(n: int) -> dict:
    """Slices of the packed parameter vector of an n-layer stack."""
    return {
        "d": slice(0, n),
        "rho": slice(n, 2 * n + 2),
        "iota": slice(2 * n + 2, 3 * n + 3),
        "sigma": slice(3 * n + 3, 4 * n + 4),
        "scale": 4 * n + 4,
        "bkg": 4 * n + 5,
    }


def pack(d, rho, iota, sigma, scale, bkg) -> np.ndarray:
    d = np.asarray(d, np.float64).ravel()
    n = d.size
    rho = np.asarray(rho, np.float64).ravel()
    iota = np.asarray(iota, np.float64).ravel()
    sigma = np.asarray(sigma, np.float64).ravel()
    assert rho.size == n + 2 and iota.size == n + 1 and sigma.size == n + 1
    return np.concatenate([d, rho, iota, sigma, [scale, bkg]])


def typical_scale(n: int) -> np.ndarray:
    """Per-parameter typical magnitudes (1 A, 1e-6 A^-2, 1e-8 A^-2, 1 A, 1,
    1e-7), the pre-scaling advice of Sec. 2.3.1, used to scale gradient
    errors (a gradient component times its typical scale)."""
    t = np.empty(n_params(n))
    L = layout(n)
    t[L["d"]] = 1.0
    t[L["rho"]] = 1e-6
    t[L["iota"]] = 1e-8
    t[L["sigma"]] = 1.0
    t[L["scale"]] = 1.0
    t[L["bkg"]] = 1e-7
    return t


@dataclasses.dataclass
class Workload:
    """A batch of stacks and datasets, host-side numpy arrays."""
    name: str
    n_layers: np.ndarray      # int32 [S]
    params: np.ndarray        # float64 [sum(4n+6)]
    dataset: np.ndarray       # int32 [S]
    q_off: np.ndarray         # int64 [D+1]
    q: np.ndarray             # float32 [Nq]
    dq: np.ndarray            # float32 [Nq] (FWHM)
    r_obs: np.ndarray         # float32 [Nq]
    r_err: np.ndarray         # float32 [Nq]
    n_quad: int

    @property
    def n_stacks(self) -> int:
        return int(self.n_layers.size)

    @property
    def n_datasets(self) -> int:
        return int(self.q_off.size - 1)

    @property
    def par_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(4 * self.n_layers.astype(np.int64) + 6)])

    @property
    def out_off(self) -> np.ndarray:
        lens = (self.q_off[1:] - self.q_off[:-1])[self.dataset]
        return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)

    @property
    def evals(self) -> int:
        """(stack x Q x quadrature node) evaluations of one pass."""
        return int(self.out_off[-1]) * self.n_quad

    def stack_params(self, s: int) -> np.ndarray:
        po = self.par_off
        return self.params[po[s]:po[s + 1]]

    def dataset_arrays(self, dsi: int):
        a, b = int(self.q_off[dsi]), int(self.q_off[dsi + 1])
        return self.q[a:b], self.dq[a:b], self.r_obs[a:b], self.r_err[a:b]

    def subset(self, stacks) -> "Workload":
        """The same datasets with a subset of the stacks."""
        stacks = np.asarray(stacks, dtype=np.int64)
        po = self.par_off
        params = np.concatenate([self.params[po[s]:po[s + 1]] for s in stacks]) if stacks.size else np.zeros(0)
        return dataclasses.replace(self, n_layers=self.n_layers[stacks].copy(), params=params,
                                   dataset=self.dataset[stacks].copy())


def log_grid(n: int, lo: float, hi: float) -> np.ndarray:
    return np.logspace(np.log10(lo), np.log10(hi), n).astype(np.float32)


# ---------------------------------------------------------------- draws ----
def _draw_film_1l(rng, S):
    d = rng.uniform(10, 300, S)
    rho1 = rng.uniform(1e-6, 6e-6, S)
    sig = rng.uniform(1, 10, (S, 2))
    return [pack([d[s]], [0.0, rho1[s], SI_SLD], [0.0, 0.0], sig[s], 1.0, 1e-7) for s in range(S)]


def _draw_thick_oxide(rng, S):
    d = rng.uniform(1000, 3000, S)
    rho1 = rng.normal(4.2e-6, 0.1e-6, S)
    sig = rng.uniform(2, 15, (S, 2))
    return [pack([d[s]], [0.0, rho1[s], SI_SLD], [0.0, 0.0], sig[s], 1.0, 1e-7) for s in range(S)]


def _draw_layers(rng, n):
    """Per-layer distributions of the multilayer workloads."""
    d = rng.uniform(50, 600, n)
    rho = rng.uniform(-0.5e-6, 6e-6, n)
    iota = rng.uniform(0, 1e-8, n)
    sig = rng.uniform(3, 20, n + 1)
    return d, rho, iota, sig


def _contrast_stacks(d, rho, iota, sig):
    out = []
    for front, back in CONTRASTS:
        out.append(pack(d, np.concatenate([[front], rho, [back]]), np.concatenate([iota, [0.0]]),
                        sig, 1.0, 1e-7))
    return out


# ------------------------------------------------------------- datasets ----
def _load_golden(name: str):
    path = os.path.join(GOLDEN_DIR, f"data_{name}.txt")
    if not os.path.exists(path):
        return None
    rows = np.loadtxt(path, comments="#", ndmin=2)
    ds = rows[:, 0].astype(np.int64)
    D = int(ds.max()) + 1
    q_off = np.zeros(D + 1, np.int64)
    for i in range(D):
        q_off[i + 1] = q_off[i] + int((ds == i).sum())
    cols = [rows[:, c].astype(np.float32) for c in range(1, 5)]
    return q_off, cols[0], cols[1], cols[2], cols[3]


def standin_data(rng, q: np.ndarray):
    """Data-shaped numbers with no model behind them (see module docstring)."""
    env = np.minimum(1.0, (0.0102 / q.astype(np.float64)) ** 4) + 1e-7
    r = env * np.exp(rng.normal(0, 0.05, q.size))
    return r.astype(np.float32), (0.05 * env).astype(np.float32)


def dataset_grids(name: str, rng=None):
    """Q / dQ grids of each dataset of a workload (without data)."""
    if name == "film_1l":
        qs = [log_grid(200, 0.005, 0.3)]
        rel = [0.05]
    elif name == "thick_oxide":
        qs = [log_grid(400, 0.005, 0.25)]
        rel = [0.03]
    elif name == "oled_cofit":
        qs = [log_grid(m, 0.005, 0.3) for m in (150, 220, 300)]
        rel = [0.05] * 3
    elif name == "vi_step":
        qs = [log_grid(300, 0.005, 0.3) for _ in range(3)]
        rel = [0.05] * 3
    else:
        raise KeyError(name)
    return qs, rel


def make_workload(name: str, n_stacks: int | None = None, seed_offset: int = 0,
                  data: str = "auto") -> Workload:
    """Build a workload.  ``n_stacks`` overrides the stack count (chains for
    the contrast workloads: stacks = 3 x chains there).  ``data``: 'auto'
    (golden file if present, else stand-in), 'standin', or 'none' (zeros)."""
    cfg = CONFIG_IDS[name]
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + cfg + 1000003 * seed_offset))
    if name == "uneven":
        S = 10000 if n_stacks is None else n_stacks
        n_layers = rng.integers(1, 21, S).astype(np.int32)
        nq = rng.integers(50, 501, S)
        rel = rng.uniform(0.02, 0.08, S)
        plist = []
        for s in range(S):
            d, rho, iota, sig = _draw_layers(rng, int(n_layers[s]))
            plist.append(pack(d, np.concatenate([[0.0], rho, [SI_SLD]]), np.concatenate([iota, [0.0]]),
                              sig, 1.0, 1e-7))
        q = [log_grid(int(m), 0.005, 0.3) for m in nq]
        dq = [(rel[s] * q[s].astype(np.float64)).astype(np.float32) for s in range(S)]
        dataset = np.arange(S, dtype=np.int32)
        q_off = np.concatenate([[0], np.cumsum([x.size for x in q])]).astype(np.int64)
        qa = np.concatenate(q) if S else np.zeros(0, np.float32)
        dqa = np.concatenate(dq) if S else np.zeros(0, np.float32)
        drng = np.random.Generator(np.random.PCG64(SEED_BASE + cfg + 77))
        if data == "none":
            r_obs, r_err = np.zeros_like(qa), np.ones_like(qa)
        else:
            r_obs, r_err = standin_data(drng, qa)
        return Workload(name, n_layers, np.concatenate(plist) if S else np.zeros(0), dataset, q_off,
                        qa, dqa, r_obs, r_err, 17)

    qs, rel = dataset_grids(name)
    K = {"film_1l": 17, "thick_oxide": 21, "oled_cofit": 17, "vi_step": 21}[name]
    if name in ("film_1l", "thick_oxide"):
        S = {"film_1l": 1024, "thick_oxide": 16384}[name] if n_stacks is None else n_stacks
        plist = (_draw_film_1l if name == "film_1l" else _draw_thick_oxide)(rng, S)
        n_layers = np.ones(S, np.int32)
        dataset = np.zeros(S, np.int32)
    else:
        chains = {"oled_cofit": 4096, "vi_step": 65536}[name] if n_stacks is None else n_stacks
        n = 10 if name == "oled_cofit" else 12
        plist = []
        for _ in range(chains):
            plist += _contrast_stacks(*_draw_layers(rng, n))
        n_layers = np.full(3 * chains, n, np.int32)
        dataset = np.tile(np.arange(3, dtype=np.int32), chains)
    q = np.concatenate(qs)
    dq = np.concatenate([(r * x.astype(np.float64)).astype(np.float32) for r, x in zip(rel, qs)])
    q_off = np.concatenate([[0], np.cumsum([x.size for x in qs])]).astype(np.int64)
    golden = _load_golden(name) if data == "auto" else None
    if golden is not None:
        g_off, gq, gdq, r_obs, r_err = golden
        assert np.array_equal(g_off, q_off) and np.array_equal(gq, q) and np.array_equal(gdq, dq), \
            f"golden data for {name} does not match its grids"
    elif data == "none":
        r_obs, r_err = np.zeros_like(q), np.ones_like(q)
    else:
        r_obs, r_err = standin_data(np.random.Generator(np.random.PCG64(SEED_BASE + cfg + 77)), q)
    params = np.concatenate(plist) if plist else np.zeros(0)
    return Workload(name, n_layers, params, dataset, q_off, q, dq, r_obs, r_err, K)


def truth_stacks(name: str):
    """The truth draw a golden data file is generated from: one stack per
    dataset (the contrasts of one chain for the co-fit workloads)."""
    cfg = CONFIG_IDS[name]
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + cfg + 424242))
    if name == "film_1l":
        return [1], _draw_film_1l(rng, 1)
    if name == "thick_oxide":
        return [1], _draw_thick_oxide(rng, 1)
    n = 10 if name == "oled_cofit" else 12
    return [n] * 3, _contrast_stacks(*_draw_layers(rng, n))


def cofit_sampler_model(name: str):
    """Sampler model of a co-fit workload ('oled_cofit' or 'vi_step'): the
    three contrasts share every layer's thickness, SLD, absorption and the
    roughnesses (tied slots); each contrast has its own free scale and
    background; fronting and backing SLDs and the backing absorption stay
    fixed.  Uniform priors: +-40 % (SLDs +-1.5e-6, absorption [0, 2e-8],
    roughness [1, 30], scale [0.8, 1.2], background [1e-8, 1e-6]) around the
    truth draw of the workload's data.  Returns (n_layers [3], dataset [3],
    slot_src, slot_val, lo, hi, u_truth)."""
    ns, stacks = truth_stacks(name)
    n = ns[0]
    L = layout(n)
    d0, r0, i0, s0 = L["d"].start, L["rho"].start, L["iota"].start, L["sigma"].start
    t = stacks[0]
    lo, hi, truth = [], [], []

    def free(lo_k, hi_k, v):
        lo.append(lo_k)
        hi.append(hi_k)
        truth.append(v)
        return len(lo) - 1
    shared = {}
    for j in range(n):
        shared[d0 + j] = free(0.6 * t[d0 + j], 1.4 * t[d0 + j], t[d0 + j])
        shared[r0 + 1 + j] = free(t[r0 + 1 + j] - 1.5e-6, t[r0 + 1 + j] + 1.5e-6, t[r0 + 1 + j])
        shared[i0 + j] = free(0.0, 2e-8, min(max(t[i0 + j], 1e-10), 1.99e-8))
    for j in range(n + 1):
        shared[s0 + j] = free(1.0, 30.0, t[s0 + j])
    src, val = [], []
    for c, st in enumerate(stacks):
        sc = free(0.8, 1.2, st[L["scale"]])
        bk = free(1e-8, 1e-6, st[L["bkg"]])
        s_c = -np.ones(4 * n + 6, np.int32)
        for slot, k in shared.items():
            s_c[slot] = k
        s_c[L["scale"]], s_c[L["bkg"]] = sc, bk
        src.append(s_c)
        val.append(np.asarray(st, np.float64))
    lo, hi, truth = np.array(lo), np.array(hi), np.array(truth)
    u_truth = np.log((truth - lo) / (hi - truth))
    return (np.array(ns, np.int32), np.arange(3, dtype=np.int32), np.concatenate(src), np.concatenate(val),
            lo, hi, u_truth)


def noise_rng(name: str):
    return np.random.Generator(np.random.PCG64(SEED_BASE + CONFIG_IDS[name] + 999331))


def write_data_file(name: str, q_off, q, dq, r_obs, r_err, header: str) -> str:
    path = os.path.join(GOLDEN_DIR, f"data_{name}.txt")
    with open(path, "w") as f:
        for line in header.strip().splitlines():
            f.write(f"# {line}\n")
        f.write("# columns: dataset Q[1/A] dQ_FWHM[1/A] R_obs e (float32 values, 9 significant digits)\n")
        for dsi in range(len(q_off) - 1):
            for i in range(int(q_off[dsi]), int(q_off[dsi + 1])):
                f.write(f"{dsi} {q[i]:.9g} {dq[i]:.9g} {r_obs[i]:.9g} {r_err[i]:.9g}\n")
    return path
