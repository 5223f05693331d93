"""nr_loglik_grad_noalloc: the log-likelihood + gradient call for hosts that
may not allocate device memory (a plug-in inside an application that owns
every allocation, a real-time loop that must stay out of the allocator).
Called through the C ABI, twice in a row on different batches (the calls
share one fixed device array), and compared with nr_loglik_grad within the
parity tolerances of the GPU tests.  Collected last so that a stop-at-first-
failure run has already run every other test."""
import ctypes

import numpy as np
import pytest

import paper_2509_06924_gb300 as nr
from paper_2509_06924_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_LL, TOL_G = 1e-5, 1e-4


def call_noalloc(batch, K, stream=None):
    lib = nr.load_library()
    ll = torch.full((batch.n_stacks,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full((batch.params.numel(),), float("nan"), dtype=torch.float64, device="cuda")
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    cb = batch._c()
    s = torch.cuda.current_stream() if stream is None else stream
    st = lib.nr_loglik_grad_noalloc(ctypes.byref(cb), K, ctypes.c_void_p(ll.data_ptr()),
                                    ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(flags.data_ptr()),
                                    ctypes.c_void_p(s.cuda_stream))
    assert st == nr.NR_OK, lib.nr_last_error()
    torch.cuda.synchronize()
    return ll.cpu().numpy(), g.cpu().numpy(), int(flags.item())


def scaled_grad_err(wl, g, g_ref):
    po = wl.par_off
    worst = 0.0
    for s in range(wl.n_stacks):
        typ = W.typical_scale(int(wl.n_layers[s]))
        a, b = g[po[s]:po[s + 1]] * typ, g_ref[po[s]:po[s + 1]] * typ
        worst = max(worst, float(np.max(np.abs(a - b)) / np.max(np.abs(b))))
    return worst


def test_noalloc_matches_nr_loglik_grad_on_two_calls_in_a_row():
    # two different batches back to back: thin-film stacks (1-layer bucket)
    # then stacks of 1..20 layers (several buckets), so the second call must
    # fully replace what the first left in the shared array
    for name, S in (("thick_oxide", 300), ("uneven", 40)):
        wl = W.make_workload(name, n_stacks=S)
        b = nr.Batch.from_workload(wl)
        ll, g, flags = call_noalloc(b, wl.n_quad)
        ctx = nr.Context(n_quad=wl.n_quad)
        ll_ref, g_ref = ctx.loglik_grad(b)
        ll_ref, g_ref = ll_ref.cpu().numpy(), g_ref.cpu().numpy()
        ctx.close()
        assert flags == 0
        assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
        assert np.max(np.abs(ll - ll_ref) / np.abs(ll_ref)) <= TOL_LL
        assert scaled_grad_err(wl, g, g_ref) <= TOL_G


def test_noalloc_rejects_oversized_and_host_batches():
    lib = nr.load_library()
    S = nr.NOALLOC_MAX_STACKS + 1
    n_layers = np.ones(S, np.int32)
    dataset = np.zeros(S, np.int32)
    q_off = np.array([0, 4], np.int64)
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    params = torch.zeros(10 * S, dtype=torch.float64, device="cuda")
    b = nr.Batch(n_layers, dataset, q_off, params, dummy, dummy, dummy, dummy)
    cb = b._c()
    out = torch.zeros(S, dtype=torch.float64, device="cuda")
    st = lib.nr_loglik_grad_noalloc(ctypes.byref(cb), 17, ctypes.c_void_p(out.data_ptr()), None, None, None)
    assert st == nr.NR_EINVAL
    assert b"NR_NOALLOC_MAX_STACKS" in lib.nr_last_error()
    wl = W.make_workload("film_1l", n_stacks=2)
    hb = nr.Batch.from_workload(wl, device="cpu")
    cb = hb._c()
    st = lib.nr_loglik_grad_noalloc(ctypes.byref(cb), 17, None, None, None, None)
    assert st == nr.NR_EINVAL


def test_noalloc_warm_call_allocates_no_device_memory():
    # the property the entry point exists for: once the library's module is
    # loaded, a call changes neither the device's free memory nor torch's
    # allocator
    wl = W.make_workload("oled_cofit", n_stacks=8)
    b = nr.Batch.from_workload(wl)
    ll = torch.empty(wl.n_stacks, dtype=torch.float64, device="cuda")
    g = torch.empty(b.params.numel(), dtype=torch.float64, device="cuda")
    flags = torch.empty(1, dtype=torch.int32, device="cuda")
    nr.loglik_grad_noalloc(b, wl.n_quad, ll, g, flags)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    a0, r0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for _ in range(2):
        nr.loglik_grad_noalloc(b, wl.n_quad, ll, g, flags)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == (a0, r0)
    assert int(flags.item()) == 0 and bool(torch.isfinite(ll).all())


def test_noalloc_full_array_matches_nr_loglik_grad():
    # exactly NR_NOALLOC_MAX_STACKS stacks: the shared array is full
    S = nr.NOALLOC_MAX_STACKS
    wl = W.make_workload("thick_oxide", n_stacks=S)
    b = nr.Batch.from_workload(wl)
    ll, g, flags = call_noalloc(b, wl.n_quad)
    ctx = nr.Context(n_quad=wl.n_quad)
    ll_ref, g_ref = ctx.loglik_grad(b)
    ll_ref, g_ref = ll_ref.cpu().numpy(), g_ref.cpu().numpy()
    ctx.close()
    assert flags == 0
    assert np.max(np.abs(ll - ll_ref) / np.abs(ll_ref)) <= TOL_LL
    assert scaled_grad_err(wl, g, g_ref) <= TOL_G


def test_noalloc_error_flags_are_cleared_then_raised():
    lib = nr.load_library()
    wl = W.make_workload("film_1l", n_stacks=8)
    bad = wl.r_err.copy()
    bad[5] = 0.0                                 # e <= 0: NR_FLAG_BAD_ERR, never a trap
    bb = nr.Batch.from_arrays(wl.n_layers, wl.dataset, wl.q_off, wl.params, wl.q, wl.dq, wl.r_obs, bad)
    _, _, flags = call_noalloc(bb, wl.n_quad)
    assert flags & nr.NR_FLAG_BAD_ERR
    # without a flags buffer the status goes to the library's own word and the
    # call still succeeds
    ll = torch.empty(wl.n_stacks, dtype=torch.float64, device="cuda")
    cb = bb._c()
    st = lib.nr_loglik_grad_noalloc(ctypes.byref(cb), wl.n_quad, ctypes.c_void_p(ll.data_ptr()), None, None,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == nr.NR_OK
    torch.cuda.synchronize()
    # a clean batch afterwards: the flags word starts at zero again
    ll, g, flags = call_noalloc(nr.Batch.from_workload(wl), wl.n_quad)
    assert flags == 0 and np.all(np.isfinite(ll)) and np.all(np.isfinite(g))


def test_noalloc_refuses_stream_capture():
    lib = nr.load_library()
    wl = W.make_workload("film_1l", n_stacks=4)
    b = nr.Batch.from_workload(wl)
    call_noalloc(b, wl.n_quad)                   # set-up on this device, eager
    ll = torch.empty(wl.n_stacks, dtype=torch.float64, device="cuda")
    cb = b._c()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        ll.zero_()                               # the graph holds something
        st = lib.nr_loglik_grad_noalloc(ctypes.byref(cb), wl.n_quad, ctypes.c_void_p(ll.data_ptr()), None, None,
                                        ctypes.c_void_p(s.cuda_stream))
    assert st == nr.NR_EINVAL
    assert b"captured" in lib.nr_last_error()
    # the library and the device stay usable
    ll2, _, flags = call_noalloc(b, wl.n_quad)
    assert flags == 0 and np.all(np.isfinite(ll2))


def test_noalloc_binding_checks_output_buffers():
    wl = W.make_workload("film_1l", n_stacks=4)
    b = nr.Batch.from_workload(wl)
    short = torch.empty(wl.n_stacks - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        nr.loglik_grad_noalloc(b, wl.n_quad, short, None)
    with pytest.raises(ValueError):
        nr.loglik_grad_noalloc(b, wl.n_quad, None, torch.empty(b.params.numel(), dtype=torch.float32,
                                                               device="cuda"))
    ll = torch.empty(wl.n_stacks, dtype=torch.float64, device="cuda")
    nr.loglik_grad_noalloc(b, wl.n_quad, ll, None)  # either output may be left out
    torch.cuda.synchronize()
    assert bool(torch.isfinite(ll).all())
