"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs, element by element.

Tolerances (per stack):
  smeared model m:   max |log m - log m_ref|              <= 2e-5
  log-likelihood:    |l - l_ref| / |l_ref|                <= 1e-5
  gradient:          ||(g - g_ref) * typ||_inf / ||g_ref * typ||_inf <= 1e-4
with typ = (1 A, 1e-6 A^-2, 1e-8 A^-2, 1 A, 1, 1e-7) per parameter class
(the pre-scaling advice of Sec. 2.3.1).  The model bound is twice the
log-likelihood's: a quadrature node within about 0.1 % (in k^2) of an
interior layer's critical edge loses digits to the cancellation of the
Parratt step above that layer (relative error ~ u k_0 / |k_j|), which the
smeared value keeps in part while the sum over Q points of the likelihood
averages it away.  A stack whose exact results move
by more than these bounds / 8 when its inputs are perturbed by one FP32
unit roundoff (oracle.perturbation_floor: an ill-conditioned stack, e.g.
a waveguide resonance sampled at its peak) is held to 8 times that response
instead: an FP32 evaluation cannot land closer than its own roundings allow.
The plain FP64 path is held to 1e-12 (log-likelihood; 1e-10 on films of up
to 5000 A), FP32 rounding of its float output (model) and 1e-5 (its
central-difference gradient).
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
import paper_2509_06924_gb300 as nr
from paper_2509_06924_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL_M, TOL_LL, TOL_G = 2e-5, 1e-5, 1e-4
COND = 8.0  # headroom over the oracle's own response to FP32-size input perturbations


def run_gpu(wl, precision="mixed", modes=("model", "loglik", "grad"), **kw):
    ctx = nr.Context(n_quad=wl.n_quad, precision=precision, **kw)
    b = nr.Batch.from_workload(wl)
    out = {}
    if "model" in modes:
        out["m"] = ctx.reflectivity(b).cpu().numpy().astype(np.float64)
    if "loglik" in modes:
        out["ll"] = ctx.loglik(b).cpu().numpy()
    if "grad" in modes:
        ll, g = ctx.loglik_grad(b)
        out["ll_g"], out["g"] = ll.cpu().numpy(), g.cpu().numpy()
    out["flags"] = ctx.device_status()
    ctx.close()
    return out


def run_oracle(wl, modes=("model", "grad")):
    out = {}
    if "model" in modes:
        out["m"] = oracle.batch("model", wl.n_layers, wl.params, wl.dataset, wl.q_off, wl.q, wl.dq, None, None,
                                wl.n_quad)
    if "grad" in modes:
        out["ll"], out["g"] = oracle.batch("grad", wl.n_layers, wl.params, wl.dataset, wl.q_off, wl.q, wl.dq,
                                           wl.r_obs, wl.r_err, wl.n_quad)
    return out


def grad_err(wl, g, g_ref, stacks=None):
    po = wl.par_off
    worst = 0.0
    for s in (range(wl.n_stacks) if stacks is None else stacks):
        typ = W.typical_scale(int(wl.n_layers[s]))
        a, b = g[po[s]:po[s + 1]] * typ, g_ref[po[s]:po[s + 1]] * typ
        den = np.max(np.abs(b))
        worst = max(worst, float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a))))
    return worst


def stack_errors(wl, gpu, ref):
    """Per-stack errors of the outputs present in both gpu and ref:
    'model' max |log m - log m_ref|, 'loglik' and 'loglik_g' (the gradient
    call's) |l - l_ref| / |l_ref|, 'grad' the scaled gradient error."""
    S = wl.n_stacks
    out = {}
    if "m" in gpu and "m" in ref:
        assert np.all(np.isfinite(gpu["m"]))
        e = np.abs(np.log(gpu["m"]) - np.log(ref["m"]))
        oo = wl.out_off
        out["model"] = np.array([e[oo[s]:oo[s + 1]].max() if oo[s + 1] > oo[s] else 0.0 for s in range(S)])
    if "ll" in gpu and "ll" in ref:
        out["loglik"] = np.abs(gpu["ll"] - ref["ll"]) / np.maximum(np.abs(ref["ll"]), 1e-300)
    if "g" in gpu and "g" in ref:
        out["loglik_g"] = np.abs(gpu["ll_g"] - ref["ll"]) / np.maximum(np.abs(ref["ll"]), 1e-300)
        out["grad"] = np.array([grad_err(wl, gpu["g"], ref["g"], [s]) for s in range(S)])
    return out


FLOOR_OF = {"model": "model", "loglik": "loglik", "loglik_g": "loglik", "grad": "grad"}


def check_bounds(wl, errs, tol):
    """Every stack within its base bound tol[kind], or, where the stack is
    ill-conditioned, within COND times the oracle's response to FP32-size
    input perturbations (computed for the stacks over the base bound only)."""
    over = sorted({s for k, e in errs.items() for s in np.flatnonzero(e > tol[k])})
    if not over:
        return
    sub = wl.subset(over)
    typ = np.concatenate([W.typical_scale(int(n)) for n in sub.n_layers])
    fl = oracle.perturbation_floor(sub.n_layers, sub.params, sub.dataset, sub.q_off, sub.q, sub.dq, sub.r_obs,
                                   sub.r_err, sub.n_quad, typ)
    for i, s in enumerate(over):
        for k, e in errs.items():
            bound = max(tol[k], COND * fl[FLOOR_OF[k]][i])
            assert e[s] <= bound, (f"stack {s} {k}: error {e[s]:.3e} above {tol[k]:.0e} and above {COND:g} x its "
                                   f"FP32 perturbation floor {fl[FLOOR_OF[k]][i]:.3e}")


def assert_parity(wl, gpu, ref, tol_m=TOL_M, tol_ll=TOL_LL, tol_g=TOL_G):
    assert gpu["flags"] == 0
    errs = stack_errors(wl, gpu, ref)
    check_bounds(wl, errs, {"model": tol_m, "loglik": tol_ll, "loglik_g": tol_ll, "grad": tol_g})


# ------------------------------------------------------------ workloads ----
# sizes the oracle finishes in seconds, spanning several CTA tiles and a
# ragged last tile (400 = 33 x 12 + 4 for K = 21, 200 = 13 x 15 + 5 for K = 17)
SMALL = [("film_1l", 96), ("thick_oxide", 128), ("oled_cofit", 8), ("uneven", 48), ("vi_step", 4)]


@pytest.mark.parametrize("name,S", SMALL)
def test_mixed_parity_small(name, S):
    wl = W.make_workload(name, n_stacks=S)
    assert_parity(wl, run_gpu(wl), run_oracle(wl))


@pytest.mark.parametrize("name,S", [("film_1l", 8), ("thick_oxide", 8), ("oled_cofit", 2), ("uneven", 10)])
def test_fp64_plain_parity(name, S):
    wl = W.make_workload(name, n_stacks=S)
    gpu = run_gpu(wl, precision="fp64")
    ref = run_oracle(wl)
    assert gpu["flags"] == 0
    # model output is float32: its rounding only
    np.testing.assert_allclose(gpu["m"], ref["m"], rtol=1.2e-7, atol=0)
    np.testing.assert_allclose(gpu["ll"], ref["ll"], rtol=1e-12)
    np.testing.assert_array_equal(gpu["ll"], gpu["ll_g"])
    # central differences with h = eps^(1/3) typ: truncation error
    assert grad_err(wl, gpu["g"], ref["g"]) <= 1e-5


# full-size workloads in the launch configuration the benchmark times;
# sampled stacks are compared with the oracle one by one
FULL = [("thick_oxide", 64), ("film_1l", 48), ("oled_cofit", 12), ("uneven", 12), ("vi_step", 6)]


@pytest.mark.parametrize("name,samples", FULL)
def test_mixed_parity_full_size_sampled(name, samples):
    wl = W.make_workload(name)
    gpu = run_gpu(wl, modes=("loglik", "grad"))
    assert gpu["flags"] == 0
    assert np.all(np.isfinite(gpu["g"])) and np.all(np.isfinite(gpu["ll_g"])) and np.all(np.isfinite(gpu["ll"]))
    rng = np.random.default_rng(20250906)
    stacks = np.sort(rng.choice(wl.n_stacks, size=min(samples, wl.n_stacks), replace=False))
    sub = wl.subset(stacks)
    ref = run_oracle(sub, modes=("model", "grad"))
    po, oo = wl.par_off, wl.out_off
    # the smeared model of the whole batch (nr_reflectivity), the sampled
    # stacks' slices taken on the device
    ctx = nr.Context(n_quad=wl.n_quad)
    m_all = ctx.reflectivity(nr.Batch.from_workload(wl))
    idx = torch.as_tensor(np.concatenate([np.arange(oo[s], oo[s + 1]) for s in stacks]), device=m_all.device)
    m = m_all[idx].cpu().numpy().astype(np.float64)
    assert ctx.device_status() == 0
    ctx.close()
    del m_all
    sel = {"m": m, "ll": gpu["ll"][stacks], "ll_g": gpu["ll_g"][stacks],
           "g": np.concatenate([gpu["g"][po[s]:po[s + 1]] for s in stacks])}
    check_bounds(sub, stack_errors(sub, sel, ref), {"model": TOL_M, "loglik": TOL_LL, "loglik_g": TOL_LL,
                                                   "grad": TOL_G})
    # a property that holds for every stack: only SLD differences matter,
    # so d/d rho_0 = -sum_j d/d rho_j
    for s in range(0, wl.n_stacks, max(1, wl.n_stacks // 4096)):
        n = int(wl.n_layers[s])
        gr = gpu["g"][po[s]:po[s + 1]][W.layout(n)["rho"]]
        assert abs(gr[0] + gr[1:].sum()) <= 1e-9 * np.abs(gr).max() + 1e-300


def test_full_size_is_deterministic():
    wl = W.make_workload("thick_oxide")
    ctx = nr.Context(n_quad=wl.n_quad)
    b = nr.Batch.from_workload(wl)
    ll1, g1 = ctx.loglik_grad(b)
    ll2, g2 = ctx.loglik_grad(b)
    assert torch.equal(ll1, ll2) and torch.equal(g1, g2)
    assert ctx.device_status() == 0


# ----------------------------------------------------------- edge cases ----
def custom_workload(stacks, datasets, K=17, data_from_oracle=True):
    """stacks: list of (n, packed params, dataset index); datasets: list of
    (Q, dQ) arrays.  Data: oracle model of the first stack on each dataset
    x 1.03, e = 5 %."""
    q_off = np.concatenate([[0], np.cumsum([len(q) for q, _ in datasets])]).astype(np.int64)
    q = np.concatenate([np.asarray(q, np.float32) for q, _ in datasets]) if datasets else np.zeros(0, np.float32)
    dq = np.concatenate([np.asarray(d, np.float32) for _, d in datasets]) if datasets else np.zeros(0, np.float32)
    r_obs = np.ones_like(q)
    r_err = np.full_like(q, 0.05)
    if data_from_oracle:
        for di in range(len(datasets)):
            a, b = int(q_off[di]), int(q_off[di + 1])
            owner = [s for s in stacks if s[2] == di]
            if owner and b > a:
                m = oracle.model(owner[0][0], owner[0][1], q[a:b], dq[a:b], K)
                r_obs[a:b] = (1.03 * m).astype(np.float32)
                r_err[a:b] = (0.05 * m).astype(np.float32)
    return W.Workload("custom", np.array([s[0] for s in stacks], np.int32),
                      np.concatenate([s[1] for s in stacks]), np.array([s[2] for s in stacks], np.int32),
                      q_off, q, dq, r_obs, r_err, K)


def rand_stack(rng, n, front=0.0, back=2.07e-6, d_range=(20, 400), absorbing=True):
    d = rng.uniform(*d_range, n)
    rho = rng.uniform(-0.5e-6, 6.5e-6, n)
    iota = rng.uniform(0, 1e-8, n) if absorbing else np.zeros(n)
    sig = rng.uniform(0, 15, n + 1)
    return W.pack(d, np.concatenate([[front], rho, [back]]), np.concatenate([iota, [0.0]]), sig,
                  rng.uniform(0.9, 1.1), rng.uniform(1e-8, 1e-6))


def test_bare_substrates_mixed_with_films():
    rng = np.random.default_rng(1)
    grid = (W.log_grid(123, 0.004, 0.3), 0.04 * W.log_grid(123, 0.004, 0.3))
    stacks = [(0, W.pack([], [0.0, 2.07e-6], [0.0], [4.0], 1.0, 1e-7), 0),
              (1, rand_stack(rng, 1), 0),
              (0, W.pack([], [6.35e-6, 2.07e-6], [1e-9], [0.0], 1.0, 5e-7), 0)]
    wl = custom_workload(stacks, [grid])
    assert_parity(wl, run_gpu(wl), run_oracle(wl))


def test_deep_stacks_every_bucket():
    rng = np.random.default_rng(2)
    grid = (W.log_grid(77, 0.005, 0.25), 0.05 * W.log_grid(77, 0.005, 0.25))
    ns = [2, 3, 5, 9, 13, 17, 20]           # one stack in every register bucket up to 20 layers
    stacks = [(n, rand_stack(rng, n), 0) for n in ns]
    wl = custom_workload(stacks, [grid])
    assert_parity(wl, run_gpu(wl), run_oracle(wl))


def test_stacks_deeper_than_the_workloads():
    """21..64 layers (beyond every workload), under the same bounds."""
    rng = np.random.default_rng(4)
    grid = (W.log_grid(77, 0.005, 0.25), 0.05 * W.log_grid(77, 0.005, 0.25))
    ns = [21, 33, 64]
    stacks = [(n, rand_stack(rng, n, d_range=(5, 60)), 0) for n in ns]
    wl = custom_workload(stacks, [grid])
    assert_parity(wl, run_gpu(wl), run_oracle(wl))


def test_empty_and_ragged_datasets():
    rng = np.random.default_rng(3)
    grids = [(np.zeros(0), np.zeros(0)),
             (W.log_grid(1, 0.05, 0.05), np.array([0.002])),
             (W.log_grid(253, 0.005, 0.3), 0.03 * W.log_grid(253, 0.005, 0.3)),
             (W.log_grid(13, 0.01, 0.2), 0.08 * W.log_grid(13, 0.01, 0.2))]
    stacks = [(1, rand_stack(rng, 1), 0), (2, rand_stack(rng, 2), 1), (3, rand_stack(rng, 3), 2),
              (1, rand_stack(rng, 1), 3), (4, rand_stack(rng, 4), 0)]
    wl = custom_workload(stacks, grids)
    gpu = run_gpu(wl)
    ref = run_oracle(wl)
    assert gpu["flags"] == 0
    # stacks on the empty dataset: loglik 0 and a zero gradient
    for s in (0, 4):
        assert gpu["ll_g"][s] == 0.0 and ref["ll"][s] == 0.0
        po = wl.par_off
        assert np.all(gpu["g"][po[s]:po[s + 1]] == 0.0)
    keep = [1, 2, 3]
    sub = wl.subset(keep)
    po = wl.par_off
    g = np.concatenate([gpu["g"][po[s]:po[s + 1]] for s in keep])
    assert grad_err(sub, g, run_oracle(sub, modes=("grad",))["g"]) <= TOL_G
    assert gpu["m"].size == int(wl.out_off[-1])
    e = np.max(np.abs(np.log(gpu["m"]) - np.log(ref["m"])))
    assert e <= TOL_M


@pytest.mark.parametrize("K", [1, 2, 32])
def test_quadrature_orders(K):
    wl = W.make_workload("film_1l", n_stacks=40)
    wl.n_quad = K
    assert_parity(wl, run_gpu(wl), run_oracle(wl))


# The 1- and 2-layer gradient buckets (n = 0, 1, 2) run two evaluations per
# thread when K >= 3; a warp's 64 evaluations straddle Q slots differently
# for every K.  Stacks with films denser than the substrate put nodes in the
# interior critical-edge band (the per-warp queue); the second dataset is
# dense around those edges.
@pytest.mark.parametrize("K", [3, 4, 5, 7, 13, 31])
def test_paired_gradient_kernel_orders_and_buckets(K):
    rng = np.random.default_rng(100 + K)
    q1, q2 = W.log_grid(61, 0.004, 0.3), W.log_grid(29, 0.008, 0.03)
    datasets = [(q1, 0.05 * q1), (q2, 0.06 * q2)]
    stacks = [(1, rand_stack(rng, 1), 0), (2, rand_stack(rng, 2), 1),
              (0, W.pack([], [0.0, 2.07e-6], [0.0], [3.0], 1.0, 1e-7), 0),
              (2, W.pack([300.0, 150.0], [0.0, 6.0e-6, 4.5e-6, 2.07e-6], [0.0, 0.0, 0.0], [3.0, 5.0, 4.0],
                         1.0, 1e-7), 1),
              (1, W.pack([900.0], [0.0, 5.0e-6, 2.07e-6], [2e-9, 0.0], [4.0, 6.0], 1.0, 1e-7), 1),
              (1, rand_stack(rng, 1), 1)]
    wl = custom_workload(stacks, datasets, K=K)
    ref_ll, ref_g, ref_r = oracle.batch("grad_res", wl.n_layers, wl.params, wl.dataset, wl.q_off, wl.q, wl.dq,
                                        wl.r_obs, wl.r_err, K)
    ref = {"ll": ref_ll, "g": ref_g, "m": run_oracle(wl, modes=("model",))["m"]}
    # model and log-likelihood run the paired forward kernels (the 1-layer
    # bucket and the runtime-n bucket with n = 0 and 2)
    assert_parity(wl, run_gpu(wl), ref)
    # several items per stack and a tile shorter than the widest, with the
    # resolution derivative through the same kernel
    ctx = nr.Context(n_quad=K, chunk_q=9, tile_q=5)
    ll, g, gr = (t.cpu().numpy() for t in ctx.loglik_grad_res(nr.Batch.from_workload(wl)))
    assert ctx.device_status() == 0
    ctx.close()
    assert np.max(np.abs(ll - ref_ll) / np.abs(ref_ll)) <= TOL_LL
    assert res_err(wl, g, gr, ref_g, ref_r) <= TOL_G


def test_zero_resolution_is_unsmeared():
    wl = W.make_workload("thick_oxide", n_stacks=16)
    wl.dq = np.zeros_like(wl.dq)
    assert_parity(wl, run_gpu(wl), run_oracle(wl))


def test_quartz_posterior_stack_from_table1():
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "quartz_table1.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    p = W.pack([vals["thick_quartz"], vals["thick_oxide"]],
               [vals["sld_air"], vals["sld_quartz"], vals["sld_oxide"], vals["sld_si"]], [0.0, 0.0, 0.0],
               [vals["rough_air_quartz"], vals["rough_quartz_oxide"], vals["rough_oxide_si"]],
               vals["scale"], vals["bkg"])
    q = W.log_grid(300, 0.006, 0.2)
    wl = custom_workload([(2, p, 0)], [(q, 0.02 * q.astype(np.float64))], K=21)
    assert_parity(wl, run_gpu(wl), run_oracle(wl))


def test_chunked_matches_unchunked():
    wl = W.make_workload("oled_cofit", n_stacks=4)
    a = run_gpu(wl)
    b = run_gpu(wl, chunk_q=24, tile_q=5)
    np.testing.assert_array_equal(a["m"], b["m"])
    np.testing.assert_allclose(b["ll_g"], a["ll_g"], rtol=1e-12)
    assert grad_err(wl, b["g"], a["g"]) <= 1e-6
    assert_parity(wl, b, run_oracle(wl))


def test_chunk_choice_follows_the_makespan_estimate():
    """Whole stacks where one wave of them nearly fills the GPU (the
    one-layer film: 1024 stacks, 760 resident CTAs; a chunk's fixed cost
    outweighs the shorter tail), Q-range chunks where a few deep stacks
    would leave most CTAs idle; every Q point is covered exactly once
    either way, so the chunked plan keeps parity."""
    film = W.make_workload("film_1l")
    ctx = nr.Context(n_quad=film.n_quad)
    bf = nr.Batch.from_workload(film)
    groups = ctx.plan_groups(bf, grad=True)
    assert sum(g["items"] for g in groups) == film.n_stacks
    wl = W.make_workload("vi_step", n_stacks=4)             # 12 stacks of 12 layers x 300 Q
    ctx2 = nr.Context(n_quad=wl.n_quad)
    b = nr.Batch.from_workload(wl)
    groups = ctx2.plan_groups(b, grad=True)
    assert sum(g["items"] for g in groups) > 4 * wl.n_stacks
    ctx.close()
    ctx2.close()
    assert_parity(wl, run_gpu(wl), run_oracle(wl))


def test_host_memory_calls_match_device_calls():
    wl = W.make_workload("uneven", n_stacks=20)
    ctx = nr.Context(n_quad=wl.n_quad)
    bd = nr.Batch.from_workload(wl)
    bh = nr.Batch.from_workload(wl, device="cpu", pin=True)
    lld, gd = ctx.loglik_grad(bd)
    llh, gh = ctx.loglik_grad(bh)
    assert not llh.is_cuda
    assert torch.equal(lld.cpu(), llh) and torch.equal(gd.cpu(), gh)
    assert torch.equal(ctx.reflectivity(bd).cpu(), ctx.reflectivity(bh))
    assert torch.equal(ctx.loglik(bd).cpu(), ctx.loglik(bh))


def test_autograd_function_backward_is_the_exact_gradient():
    wl = W.make_workload("film_1l", n_stacks=12)
    ctx = nr.Context(n_quad=wl.n_quad)
    b = nr.Batch.from_workload(wl)
    params = b.params.clone().requires_grad_(True)
    ll = nr.loglik_autograd(params, ctx, b)
    w = torch.linspace(0.5, 2.0, wl.n_stacks, dtype=torch.float64, device=ll.device)
    (ll * w).sum().backward()
    _, g = ctx.loglik_grad(b)
    per = torch.as_tensor(4 * wl.n_layers.astype(np.int64) + 6, device=g.device)
    torch.testing.assert_close(params.grad, g * torch.repeat_interleave(w, per), rtol=0, atol=0)


def test_device_data_errors_raise_flags_not_faults():
    wl = W.make_workload("film_1l", n_stacks=3)
    ctx = nr.Context(n_quad=wl.n_quad)
    b = nr.Batch.from_workload(wl)
    bad_err = b.r_err.clone()
    bad_err[5] = 0.0
    ll = ctx.loglik(nr.Batch(b.n_layers, b.dataset, b.q_off, b.params, b.q, b.dq, b.r_obs, bad_err))
    assert ctx.device_status() & nr.NR_FLAG_BAD_ERR
    assert not torch.isfinite(ll).all()
    bad_p = b.params.clone()
    bad_p[3] = float("nan")
    ctx.loglik_grad(b.with_params(bad_p))
    assert ctx.device_status() & nr.NR_FLAG_NONFINITE_PARAM
    bad_q = b.dq.clone()
    bad_q[0] = 10.0    # nodes at q <= 0
    m = ctx.reflectivity(nr.Batch(b.n_layers, b.dataset, b.q_off, b.params, b.q, bad_q))
    assert ctx.device_status() & nr.NR_FLAG_BAD_Q
    assert not torch.isfinite(m[0])
    # the context stays usable and clean afterwards
    ll2, _ = ctx.loglik_grad(b)
    assert ctx.device_status() == 0 and torch.isfinite(ll2).all()


def test_metadata_validation():
    wl = W.make_workload("film_1l", n_stacks=2)
    ctx = nr.Context(n_quad=wl.n_quad)
    b = nr.Batch.from_workload(wl)
    for bad in (dict(n_layers=np.array([1, 65], np.int32)), dict(dataset=np.array([0, 1], np.int32)),
                dict(q_off=np.array([0, -1], np.int64))):
        fields = dict(n_layers=b.n_layers, dataset=b.dataset, q_off=b.q_off)
        fields.update(bad)
        bb = nr.Batch(fields["n_layers"], fields["dataset"], fields["q_off"], b.params, b.q, b.dq, b.r_obs, b.r_err)
        with pytest.raises(nr.NRError) as ei:
            ctx.loglik(bb)
        assert ei.value.status == nr.NR_EINVAL
    with pytest.raises(nr.NRError):
        ctx.loglik(nr.Batch(b.n_layers, b.dataset, b.q_off, b.params, b.q, b.dq))  # no data
    # an empty batch is fine
    e = nr.Batch(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(1, np.int64), b.params[:0], b.q[:0], b.dq[:0],
                 b.r_obs[:0], b.r_err[:0])
    ll, g = ctx.loglik_grad(e)
    assert ll.numel() == 0 and g.numel() == 0


def test_plan_before_capture_and_graph_replay():
    wl = W.make_workload("thick_oxide", n_stacks=64)
    ctx = nr.Context(n_quad=wl.n_quad)
    b = nr.Batch.from_workload(wl)
    ctx.plan(b)
    ll = torch.empty(wl.n_stacks, dtype=torch.float64, device="cuda")
    g = torch.empty(b.params.numel(), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.loglik_grad(b, ll_out=ll, grad_out=g, stream=s)
    torch.cuda.synchronize()
    ref_ll, ref_g = ll.clone(), g.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        ctx.loglik_grad(b, ll_out=ll, grad_out=g, stream=s)
    ll.zero_()
    g.zero_()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(ll, ref_ll) and torch.equal(g, ref_g)


# ---------------------------------------------- resolution-scale derivative
def res_err(wl, g, gr, g_ref, gr_ref):
    """The resolution derivative as one more gradient component (typical
    scale 1, like the model scale): max over stacks of the scaled error over
    the stack's largest scaled component."""
    po = wl.par_off
    worst = 0.0
    for s in range(wl.n_stacks):
        typ = W.typical_scale(int(wl.n_layers[s]))
        ref = np.append(g_ref[po[s]:po[s + 1]] * typ, gr_ref[s])
        got = np.append(g[po[s]:po[s + 1]] * typ, gr[s])
        worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    return worst


@pytest.mark.parametrize("name,S,kw", [("thick_oxide", 48, {}), ("film_1l", 40, {}), ("oled_cofit", 4, {}),
                                       ("uneven", 24, {}), ("vi_step", 2, {}),
                                       ("oled_cofit", 3, {"chunk_q": 40, "tile_q": 3})])
def test_resolution_derivative_parity(name, S, kw):
    wl = W.make_workload(name, n_stacks=S)
    ctx = nr.Context(n_quad=wl.n_quad, **kw)
    b = nr.Batch.from_workload(wl)
    ll, g, gr = (t.cpu().numpy() for t in ctx.loglik_grad_res(b))
    ll0, g0 = (t.cpu().numpy() for t in ctx.loglik_grad(b))
    assert ctx.device_status() == 0
    ctx.close()
    ref_ll, ref_g, ref_r = oracle.batch("grad_res", wl.n_layers, wl.params, wl.dataset, wl.q_off, wl.q, wl.dq,
                                        wl.r_obs, wl.r_err, wl.n_quad)
    assert np.all(np.isfinite(gr))
    assert np.max(np.abs(ll - ref_ll) / np.abs(ref_ll)) <= TOL_LL
    assert res_err(wl, g, gr, ref_g, ref_r) <= TOL_G
    # the log-likelihood and parameter gradient are those of nr_loglik_grad
    assert np.max(np.abs(ll - ll0) / np.abs(ll0)) <= 1e-6
    assert grad_err(wl, g, g0) <= 1e-5


def test_resolution_derivative_host_batch_and_fp64_refusal():
    wl = W.make_workload("thick_oxide", n_stacks=6)
    ctx = nr.Context(n_quad=wl.n_quad)
    lld, gd, rd = ctx.loglik_grad_res(nr.Batch.from_workload(wl))
    llh, gh, rh = ctx.loglik_grad_res(nr.Batch.from_workload(wl, device="cpu", pin=True))
    assert not rh.is_cuda
    assert torch.equal(rd.cpu(), rh) and torch.equal(gd.cpu(), gh)
    ctx.close()
    ctx64 = nr.Context(n_quad=wl.n_quad, precision="fp64")
    with pytest.raises(nr.NRError):
        ctx64.loglik_grad_res(nr.Batch.from_workload(wl))
    ctx64.close()


# ------------------------------------------------------------- SLD profiles
def profile_ref(wl, z):
    po = wl.par_off
    rho = np.zeros((wl.n_stacks, z.size))
    iota = np.zeros((wl.n_stacks, z.size))
    for s in range(wl.n_stacks):
        rho[s], iota[s] = oracle.sld_profile(int(wl.n_layers[s]), wl.params[po[s]:po[s + 1]], z.astype(np.float64))
    return rho, iota


@pytest.mark.parametrize("name,S", [("thick_oxide", 16), ("oled_cofit", 9), ("uneven", 40), ("vi_step", 6)])
def test_sld_profile_parity(name, S):
    wl = W.make_workload(name, n_stacks=S)
    depth = max(float(np.sum(wl.stack_params(s)[:int(wl.n_layers[s])])) for s in range(S))
    z = np.linspace(-60.0, depth + 60.0, 1037).astype(np.float32)   # ragged against the 256-thread sweep
    ctx = nr.Context(n_quad=wl.n_quad)
    b = nr.Batch.from_workload(wl)
    rho, iota = ctx.sld_profile(b, torch.as_tensor(z, device="cuda"))
    assert ctx.device_status() == 0
    rho, iota = rho.cpu().numpy(), iota.cpu().numpy()
    ref_r, ref_i = profile_ref(wl, z)
    for s in range(S):
        scale_r = np.max(np.abs(ref_r[s]))
        scale_i = max(np.max(np.abs(ref_i[s])), 1e-12)
        assert np.max(np.abs(rho[s] - ref_r[s])) <= 2e-6 * scale_r
        assert np.max(np.abs(iota[s] - ref_i[s])) <= 2e-6 * scale_i
    ctx.close()


def test_sld_profile_sharp_steps_host_batch_and_flags():
    d = [120.0, 35.0]
    rho = [0.0, 4.1e-6, -0.4e-6, 2.07e-6]
    stacks = [(2, W.pack(d, rho, [1e-8, 0.0, 0.0], [0.0, 0.0, 0.0], 1.0, 0.0), 0),
              (0, W.pack([], [0.0, 2.07e-6], [0.0], [3.0], 1.0, 0.0), 0)]
    q = W.log_grid(10, 0.01, 0.2)
    wl = custom_workload(stacks, [(q, 0.05 * q.astype(np.float64))])
    z = np.array([-10.0, 0.0, 119.0, 120.0, 154.0, 155.0, 400.0], np.float32)
    ctx = nr.Context(n_quad=wl.n_quad)
    rho_d, iota_d = ctx.sld_profile(nr.Batch.from_workload(wl), torch.as_tensor(z, device="cuda"))
    rho_h, iota_h = ctx.sld_profile(nr.Batch.from_workload(wl, device="cpu", pin=True), torch.as_tensor(z))
    assert torch.equal(rho_d.cpu(), rho_h) and torch.equal(iota_d.cpu(), iota_h)
    # sharp steps: the deeper medium's value from the interface depth on
    np.testing.assert_allclose(rho_h[0].numpy(), [0.0, 4.1e-6, 4.1e-6, -0.4e-6, -0.4e-6, 2.07e-6, 2.07e-6],
                               rtol=0, atol=2e-12)
    assert abs(float(rho_h[1, 1]) - 2.07e-6 / 2) < 1e-12
    assert ctx.device_status() == 0
    bad = wl.params.copy()
    bad[0] = np.nan
    wl_bad = custom_workload([(2, bad[:14], 0)], [(q, 0.05 * q.astype(np.float64))], data_from_oracle=False)
    ctx.sld_profile(nr.Batch.from_workload(wl_bad), torch.as_tensor(z, device="cuda"))
    assert ctx.device_status() & nr.NR_FLAG_NONFINITE_PARAM
    ctx.close()


# ------------------------------------------------------- on-device HMC step
def sampler_setup(C=8, seed=7, res=False):
    """A two-contrast co-fit sampler and its CPU reference; res: one more
    free parameter, the resolution scale f of every dQ (prior [0.6, 1.4])."""
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_hmc import small_model, with_resolution
    from oracle import hmc
    model, u_t = small_model(seed)
    if res:
        model = with_resolution(model)
        u_t = np.append(u_t, 0.4)
    # the device holds the data as float32: the reference uses the same values
    f32 = lambda a: np.asarray(a, np.float32)
    ref = hmc.Model(model.n_layers, model.dataset, model.slot_src, model.slot_val, model.lo, model.hi,
                    model.q_off, f32(model.Q), f32(model.dQ), f32(model.Robs), f32(model.err), model.K,
                    res_param=model.res_param)
    ctx = nr.Context(n_quad=model.K)
    dev = lambda a: torch.as_tensor(f32(a), device="cuda")
    smp = nr.Sampler(ctx, C, model.n_layers, model.dataset, model.q_off, dev(model.Q), dev(model.dQ),
                     dev(model.Robs), dev(model.err), model.slot_src, model.slot_val, model.lo, model.hi,
                     res_param=model.res_param)
    rng = np.random.default_rng(seed + 1)
    u = u_t[None, :] + 0.2 * rng.normal(size=(C, model.P))
    return ctx, smp, ref, u, rng


@pytest.mark.parametrize("res", [False, True])
def test_sampler_logp_grad_parity(res):
    ctx, smp, ref, u, _ = sampler_setup(res=res)
    lp, g = smp.logp_grad(torch.as_tensor(u, device="cuda"))
    lp, g = lp.cpu().numpy(), g.cpu().numpy()
    for c in range(u.shape[0]):
        lr, gr = ref.logp_grad(u[c])
        assert abs(lp[c] - lr) <= 1e-5 * abs(lr)
        assert np.max(np.abs(g[c] - gr)) <= 1e-4 * np.max(np.abs(gr))
    smp.close()
    ctx.close()


@pytest.mark.parametrize("res", [False, True])
def test_hmc_step_parity_and_graph_replay(res):
    C, P_eps, L = 8, 4e-4, 6
    ctx, smp, ref, u, rng = sampler_setup(C, res=res)
    z = rng.normal(size=(C, ref.P))
    inv_mass = np.full(ref.P, 1.0)
    # first half of the chains must accept, the rest reject: decisions that
    # do not hinge on rounding; both branches of every kernel path run
    log_u = np.where(np.arange(C) < C // 2, -np.inf, np.inf)
    ud = torch.as_tensor(u, device="cuda")
    lp, acc = smp.hmc_step(ud, torch.as_tensor(z, device="cuda"), torch.as_tensor(log_u, device="cuda"),
                           torch.as_tensor(inv_mass, device="cuda"), P_eps, L)
    assert ctx.device_status() == 0
    ug, lp, acc = ud.cpu().numpy(), lp.cpu().numpy(), acc.cpu().numpy()
    from oracle import hmc
    for c in range(C):
        ur, lr, ar, H0, H1 = hmc.hmc_step(ref.logp_grad, u[c], z[c], log_u[c], inv_mass, P_eps, L)
        assert bool(acc[c]) == ar
        assert abs(lp[c] - lr) <= 1e-5 * abs(lr)
        # L leapfrog steps amplify the gradient's relative error by ~eps^2 L^2 |d2 log pi|
        assert np.max(np.abs(ug[c] - ur)) <= 1e-6 + 1e-6 * np.max(np.abs(ur))
    # the same step as a captured CUDA graph reproduces the eager result
    u2 = torch.as_tensor(u, device="cuda")
    zt, lt, mt = (torch.as_tensor(a, device="cuda") for a in (z, log_u, inv_mass))
    lp2 = torch.empty(C, dtype=torch.float64, device="cuda")
    acc2 = torch.empty(C, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        smp.hmc_step(u2, zt, lt, mt, P_eps, L, lp2, acc2, stream=s)    # warm-up (plans stay cached)
    torch.cuda.synchronize()
    u2.copy_(torch.as_tensor(u, device="cuda"))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        smp.hmc_step(u2, zt, lt, mt, P_eps, L, lp2, acc2, stream=s)
    u2.copy_(torch.as_tensor(u, device="cuda"))
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(u2.cpu(), torch.as_tensor(ug)) and torch.equal(acc2.cpu(), torch.as_tensor(acc))
    smp.close()
    ctx.close()


def test_sampler_rejects_bad_models():
    ctx = nr.Context(n_quad=17)
    q = torch.ones(4, device="cuda")
    with pytest.raises(nr.NRError):      # slot source out of range
        nr.Sampler(ctx, 2, [0], [0], [0, 4], q, q, q, q, [5, -1, -1, -1, -1, -1], [0.0] * 6, [0.0], [1.0])
    with pytest.raises(nr.NRError):      # empty prior box
        nr.Sampler(ctx, 2, [0], [0], [0, 4], q, q, q, q, [0, -1, -1, -1, -1, -1], [0.0] * 6, [1.0], [1.0])
    ctx.close()


# ---------------------------------------------- variational-inference step
def test_vi_step_parity_and_graph_replay():
    from oracle import vi
    R = 6
    ctx, smp, ref, u_c, rng = sampler_setup(R, seed=11)
    P = ref.P
    nphi = nr.vi_phi_size(P)
    phi = np.zeros((R, nphi))
    phi[:, :P] = u_c                                   # mu: the chains' starting points
    for r in range(R):                                 # L = 0.1 I plus a little correlation
        idx = P
        for i in range(P):
            for j in range(i + 1):
                phi[r, idx] = np.log(0.1) if i == j else 0.02 * rng.normal()
                idx += 1
    m0 = 0.01 * np.abs(rng.normal(size=(R, nphi)))
    v0 = 0.001 * np.abs(rng.normal(size=(R, nphi)))
    eps = rng.normal(size=(R, P))
    t0 = 4                                             # iterations already done
    dev = lambda a: torch.as_tensor(a, device="cuda")
    ph, m, v, t = dev(phi), dev(m0), dev(v0), dev(np.array([t0], np.int32))
    elbo = smp.vi_step(ph, m, v, t, dev(eps), lr=0.05)
    assert ctx.device_status() == 0 and int(t.item()) == t0 + 1
    ph, m, v, elbo = ph.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy(), elbo.cpu().numpy()
    for r in range(R):
        mu_r, tri_r, m_r, v_r, el_r = vi.vi_step(ref.logp_grad, phi[r, :P], phi[r, P:], m0[r], v0[r], t0 + 1,
                                                 eps[r], 0.05)
        assert abs(elbo[r] - el_r) <= 1e-5 * abs(el_r)
        # the gradient carries the mixed path's ~1e-5 relative error; Adam's
        # step is lr * mhat / sqrt(vhat): its error stays a small fraction of lr
        np.testing.assert_allclose(ph[r], np.concatenate([mu_r, tri_r]), rtol=0, atol=2e-3 * 0.05)
        # Adam's first moment carries the gradient's error: held to the
        # gradient bound, 1e-4 of the largest gradient term (1 - beta1) g
        assert np.max(np.abs(m[r] - m_r)) <= 1e-4 * np.max(np.abs(m_r - 0.9 * m0[r]))
    # a captured iteration replays with the device counter advancing
    ph2, m2, v2, t2, e2 = dev(phi), dev(m0), dev(v0), dev(np.array([t0], np.int32)), dev(eps)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        smp.vi_step(ph2, m2, v2, t2, e2, stream=s)
    torch.cuda.synchronize()
    ph2.copy_(dev(phi)); m2.copy_(dev(m0)); v2.copy_(dev(v0)); t2.fill_(t0)
    graph = torch.cuda.CUDAGraph()
    el2 = torch.empty(R, dtype=torch.float64, device="cuda")
    with torch.cuda.graph(graph, stream=s):
        smp.vi_step(ph2, m2, v2, t2, e2, elbo_out=el2, stream=s)
    ph2.copy_(dev(phi)); m2.copy_(dev(m0)); v2.copy_(dev(v0)); t2.fill_(t0)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert int(t2.item()) == t0 + 2
    smp.close()
    ctx.close()


@pytest.mark.parametrize("name,S", [("uneven", 40), ("thick_oxide", 64), ("oled_cofit", 6), ("film_1l", 48)])
def test_autotuned_plan_keeps_parity(name, S):
    """nr_plan with autotune = 1 times the candidate launch shapes (paired or
    one-evaluation kernel, widest tile or half) per register bucket and keeps
    the fastest; whatever it picks matches the oracle."""
    wl = W.make_workload(name, n_stacks=S)
    ctx = nr.Context(n_quad=wl.n_quad, autotune=True)
    b = nr.Batch.from_workload(wl)
    ctx.plan(b)
    info = ctx.plan_info(b)
    assert info["tile_q"] >= 1 and info["grid_ctas"] >= 1 and info["launches"] >= 1
    gpu = {"m": ctx.reflectivity(b).cpu().numpy().astype(np.float64), "ll": ctx.loglik(b).cpu().numpy()}
    ll, g = ctx.loglik_grad(b)
    gpu["ll_g"], gpu["g"] = ll.cpu().numpy(), g.cpu().numpy()
    gpu["flags"] = ctx.device_status()
    ctx.close()
    assert_parity(wl, gpu, run_oracle(wl))


# ------------------------------------------------- failure injection ------
def test_alloc_failure_leaves_context_usable():
    """An allocation failure (injected on the host: nr_debug_fail_allocs,
    no cudaMalloc is called) surfaces as NR_ENOMEM, and the same context
    completes the plan and the call afterwards."""
    wl = W.make_workload("oled_cofit", n_stacks=4)
    try:
        nr.debug_fail_allocs(1)                # the context's status word
        with pytest.raises(nr.NRError) as err:
            nr.Context(n_quad=wl.n_quad)
        assert err.value.status == nr.NR_ENOMEM
        nr.debug_fail_allocs(0)
        ctx = nr.Context(n_quad=wl.n_quad)
        b = nr.Batch.from_workload(wl)
        nr.debug_fail_allocs(2)                # the new plan's work-list buffers
        with pytest.raises(nr.NRError) as err:
            ctx.loglik_grad(b)
        assert err.value.status == nr.NR_ENOMEM
    finally:
        nr.debug_fail_allocs(0)
    ll, g = ctx.loglik_grad(b)
    assert ctx.device_status() == 0
    ref = run_oracle(wl, modes=("grad",))
    assert np.max(np.abs(ll.cpu().numpy() - ref["ll"]) / np.abs(ref["ll"])) <= TOL_LL
    assert grad_err(wl, g.cpu().numpy(), ref["g"]) <= TOL_G
    ctx.close()


DEBUG_CASES = (("thick_oxide", 64), ("oled_cofit", 8), ("uneven", 40))
DEBUG_CHILD = r"""
import sys
import numpy as np
import paper_2509_06924_gb300 as nr
from paper_2509_06924_gb300 import _build, workloads as W
assert nr.debug_build_selected() and nr.library_path() == _build.DEBUG_LIB
out = {}
for name, S in %r:
    wl = W.make_workload(name, n_stacks=S)
    ctx = nr.Context(n_quad=wl.n_quad)
    b = nr.Batch.from_workload(wl)
    out[name + "_m"] = ctx.reflectivity(b).cpu().numpy().astype(np.float64)
    ll, g = ctx.loglik_grad(b)
    f0 = ctx.device_status()
    ctx.debug_poison_plan(b, True)
    ctx.loglik_grad(b)
    f1 = ctx.device_status()
    ctx.debug_poison_plan(b, False)
    ll2, g2 = ctx.loglik_grad(b)
    f2 = ctx.device_status()
    ctx.close()
    out[name + "_ll"], out[name + "_g"] = ll.cpu().numpy(), g.cpu().numpy()
    out[name + "_ll2"], out[name + "_g2"] = ll2.cpu().numpy(), g2.cpu().numpy()
    out[name + "_flags"] = np.array([f0, f1, f2])
np.savez(sys.argv[1], **out)
""" % (DEBUG_CASES,)


def test_debug_build_reports_a_corrupted_plan(tmp_path):
    """The NR_DEBUG library (device bounds checks that set a status flag and
    skip the access instead of trapping), run in a child process with
    NR_DEBUG=1: on clean batches of the one-layer, rolled and per-bucket
    kernels it raises no flag and keeps parity with the oracle; a plan whose
    first work item names a stack one past the batch (nr_debug_poison_plan)
    gives NR_FLAG_DEBUG_BOUNDS and no fault; restored, the same plan
    reproduces the clean results."""
    import subprocess
    import sys
    from paper_2509_06924_gb300 import _build
    _build.build_debug()
    out = str(tmp_path / "debug.npz")
    r = subprocess.run([sys.executable, "-c", DEBUG_CHILD, out], cwd=ROOT, capture_output=True, text=True,
                       timeout=900, env={**os.environ, "NR_DEBUG": "1"})
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    d = np.load(out)
    for name, S in DEBUG_CASES:
        assert list(d[name + "_flags"]) == [0, nr.NR_FLAG_DEBUG_BOUNDS, 0], name
        wl = W.make_workload(name, n_stacks=S)
        gpu = {"m": d[name + "_m"], "ll_g": d[name + "_ll"], "g": d[name + "_g"], "flags": 0}
        assert_parity(wl, gpu, run_oracle(wl))
        np.testing.assert_allclose(d[name + "_ll2"], d[name + "_ll"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(d[name + "_g2"], d[name + "_g"], rtol=1e-12, atol=1e-300)


def test_strong_absorbers_thick_layers_and_total_reflection():
    """Outside the workloads' ranges: absorption up to 1e-6 A^-2 (a strong
    neutron absorber; the workloads stop at 1e-8), layers up to 5000 A
    (layer phases up to 1500 rad at the top of the Q range, deep into the
    sin/cos table's reduction), Q from well below the backing's critical
    edge (total reflection, evanescent layers) and roughness up to 25 A.
    The same conditioning-aware bounds."""
    rng = np.random.default_rng(77)
    q = W.log_grid(240, 0.004, 0.3)
    stacks = []
    for t in range(12):
        n = 1 + t % 4
        d = rng.uniform(500.0, 5000.0, n)
        rho = np.concatenate([[0.0], rng.uniform(-0.5e-6, 7e-6, n), [(2.07e-6, 6.36e-6)[t % 2]]])
        iota = np.concatenate([rng.choice([0.0, 1e-7, 1e-6], n), [0.0]])
        sig = rng.uniform(0.0, 25.0, n + 1)
        stacks.append((n, W.pack(d, rho, iota, sig, 1.0, 1e-7), 0))
    wl = custom_workload(stacks, [(q, 0.03 * q)], K=17)
    gpu, ref = run_gpu(wl), run_oracle(wl)
    assert_parity(wl, gpu, ref)
    # the plain FP64 path (Parratt, against the oracle's Abeles product):
    # phases of 1e3 rad carry ~1e-13 relative rounding, amplified by the
    # fringes of thick films
    fp = run_gpu(wl, precision="fp64", modes=("loglik",))
    np.testing.assert_allclose(fp["ll"], ref["ll"], rtol=1e-10)


def test_waveguide_resonance_stacks():
    """A 520-700 A low-SLD layer between two 300 A high-SLD layers guides
    neutrons between the critical edges of its neighbours: sharp resonances
    whose gradient is most sensitive to rounding (the first stack's exact
    gradient moves by 7e-5 of its largest component under one-unit-roundoff
    input perturbations).  Dense Q over the guided range, 21 nodes; the
    scaled gradient error must stay within 5e-5 here, half the general bound."""
    q = W.log_grid(160, 0.006, 0.03)
    stacks = []
    for d_core, rho_hi in ((600.0, 6.0e-6), (600.0, 5.3e-6), (520.0, 6.3e-6), (700.0, 5.8e-6)):
        stacks.append((3, W.pack([300.0, d_core, 300.0], [0.0, rho_hi, 1.0e-6, rho_hi, 2.07e-6],
                                 [1e-9, 2e-10, 1e-9, 0.0], [4.0, 3.0, 3.0, 5.0], 1.0, 1e-7), 0))
    wl = custom_workload(stacks, [(q, 0.05 * q)], K=21)
    gpu, ref = run_gpu(wl), run_oracle(wl)
    assert_parity(wl, gpu, ref)
    assert grad_err(wl, gpu["g"], ref["g"]) <= 5e-5
