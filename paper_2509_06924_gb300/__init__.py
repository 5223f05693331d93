"""GB300-native batched neutron reflectometry: the forward reflectivity model,
its Gaussian log-likelihood and the exact gradient of that log-likelihood
(arXiv 2509.06924: Abeles forward model, Sec. 2.1; refjax kernel interface and
smearing, Sec. 3; chi^2 / Gaussian likelihood, Eq. 25 and Sec. 2.1), for many
parameter samples at once, as HMC and variational inference need them.

This module is the thin Python binding of the C-ABI library ``libnr.so``
(include/nr.h): it marshals numpy / torch buffers into the C structs and
calls the library; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: without the compiled library (or without
a CUDA device) the calls raise.

    import paper_2509_06924_gb300 as nr
    ctx = nr.Context(n_quad=21)                       # NR_MIXED precision
    batch = nr.Batch.from_workload(wl, device="cuda")  # device tensors
    ll, grad = ctx.loglik_grad(batch)                 # torch float64 on device
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

from . import _build

NR_OK, NR_EINVAL, NR_ENOMEM, NR_ECUDA, NR_ETIMEOUT, NR_ENONFINITE = range(6)
NR_MIXED, NR_FP64_PLAIN = 0, 1
NR_MEM_DEVICE, NR_MEM_HOST = 0, 1
NR_FLAG_NONFINITE_PARAM, NR_FLAG_BAD_Q, NR_FLAG_BAD_ERR, NR_FLAG_DEBUG_BOUNDS = 1, 2, 4, 8
MAX_LAYERS = 64
MAX_QUAD = 32
EXPORTS = ("nr_create", "nr_destroy", "nr_last_error", "nr_plan", "nr_reflectivity", "nr_loglik",
           "nr_loglik_grad", "nr_loglik_grad_res", "nr_sld_profile", "nr_device_status", "nr_quadrature",
           "nr_plan_info", "nr_loglik_grad_noalloc", "nr_sampler_create", "nr_sampler_destroy",
           "nr_sampler_logp_grad", "nr_hmc_step", "nr_vi_step", "nr_plan_groups", "nr_tune_cache_get",
           "nr_tune_cache_put", "nr_debug_fail_allocs", "nr_debug_poison_plan")
NOALLOC_MAX_STACKS = 16384


class NRError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"nr status {status}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("n_quad", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("tile_q", ctypes.c_int32), ("chunk_q", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("serial", ctypes.c_int32)]


class CBatch(ctypes.Structure):
    _fields_ = [("n_stacks", ctypes.c_int32), ("n_datasets", ctypes.c_int32),
                ("n_layers", ctypes.c_void_p), ("dataset", ctypes.c_void_p), ("q_off", ctypes.c_void_p),
                ("memory", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("params", ctypes.c_void_p), ("q", ctypes.c_void_p), ("dq", ctypes.c_void_p),
                ("r_obs", ctypes.c_void_p), ("r_err", ctypes.c_void_p)]


class CCofitModel(ctypes.Structure):
    _fields_ = [("n_chains", ctypes.c_int32), ("n_contrasts", ctypes.c_int32), ("n_free", ctypes.c_int32),
                ("n_layers", ctypes.c_void_p), ("dataset", ctypes.c_void_p), ("n_datasets", ctypes.c_int32),
                ("q_off", ctypes.c_void_p), ("q", ctypes.c_void_p), ("dq", ctypes.c_void_p),
                ("r_obs", ctypes.c_void_p), ("r_err", ctypes.c_void_p), ("slot_src", ctypes.c_void_p),
                ("slot_val", ctypes.c_void_p), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
                ("res_param", ctypes.c_int32)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("paired", ctypes.c_int32), ("tile_q", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("ms", ctypes.c_double)]


class CAdam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


_LIB = None
_LIB_LOCK = threading.Lock()


def debug_build_selected() -> bool:
    """NR_DEBUG=1 in the environment selects the NR_DEBUG library (device
    bounds checks that set NR_FLAG_DEBUG_BOUNDS) for this process."""
    return os.environ.get("NR_DEBUG") == "1"


def library_path() -> str:
    return _build.DEBUG_LIB if debug_build_selected() else _build.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libnr.so, or its NR_DEBUG variant (building it first when it is
    missing or stale)."""
    global _LIB
    with _LIB_LOCK:
        if _LIB is None:
            path = library_path()
            if build_if_missing:
                _build.build_debug() if debug_build_selected() else _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"the CUDA library {path} is missing; run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            vp, i32, i64p = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.nr_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Options)]
            lib.nr_create.restype = ctypes.c_int
            lib.nr_destroy.argtypes = [vp]
            lib.nr_destroy.restype = None
            lib.nr_last_error.argtypes = []
            lib.nr_last_error.restype = ctypes.c_char_p
            lib.nr_plan.argtypes = [vp, ctypes.POINTER(CBatch)]
            lib.nr_reflectivity.argtypes = [vp, ctypes.POINTER(CBatch), vp, vp]
            lib.nr_loglik.argtypes = [vp, ctypes.POINTER(CBatch), vp, vp]
            lib.nr_loglik_grad.argtypes = [vp, ctypes.POINTER(CBatch), vp, vp, vp]
            lib.nr_device_status.argtypes = [vp, vp, i32p]
            lib.nr_quadrature.argtypes = [i32, dp, dp]
            lib.nr_plan_info.argtypes = [vp, ctypes.POINTER(CBatch), i64p, i32p, i32p, i32p, i32p]
            lib.nr_loglik_grad_noalloc.argtypes = [ctypes.POINTER(CBatch), i32, vp, vp, vp, vp]
            lib.nr_loglik_grad_res.argtypes = [vp, ctypes.POINTER(CBatch), vp, vp, vp, vp]
            lib.nr_sld_profile.argtypes = [vp, ctypes.POINTER(CBatch), vp, i32, vp, vp, vp]
            lib.nr_sampler_create.argtypes = [vp, ctypes.POINTER(CCofitModel), ctypes.POINTER(vp)]
            lib.nr_sampler_destroy.argtypes = [vp]
            lib.nr_sampler_destroy.restype = None
            lib.nr_sampler_logp_grad.argtypes = [vp, vp, vp, vp, vp]
            lib.nr_hmc_step.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, i32, vp, vp, vp]
            lib.nr_vi_step.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(CAdam), vp, vp]
            lib.nr_plan_groups.argtypes = [vp, ctypes.POINTER(CBatch), i32, i32, i32p, i32p, i32p, i32p, i32p,
                                           i32p]
            lib.nr_tune_cache_get.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(TuneEntry)]
            lib.nr_tune_cache_put.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(TuneEntry)]
            lib.nr_debug_fail_allocs.argtypes = [i32]
            lib.nr_debug_poison_plan.argtypes = [vp, ctypes.POINTER(CBatch), i32]
            for name in EXPORTS:
                if name not in ("nr_destroy", "nr_last_error", "nr_sampler_destroy"):
                    getattr(lib, name).restype = ctypes.c_int
            _LIB = lib
        return _LIB


def _check(status: int) -> None:
    if status != NR_OK:
        raise NRError(status, load_library(False).nr_last_error().decode(errors="replace"))


def quadrature(K: int):
    """The library's K-point Gauss-Hermite rule for exp(-x^2) (host call)."""
    x = np.zeros(K)
    w = np.zeros(K)
    _check(load_library().nr_quadrature(K, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return x, w


@dataclasses.dataclass
class Batch:
    """A batch of stacks: host metadata (numpy) plus bulk arrays that are
    either torch tensors on a CUDA device or (pinned) host tensors."""
    n_layers: np.ndarray
    dataset: np.ndarray
    q_off: np.ndarray
    params: object
    q: object
    dq: object
    r_obs: object = None
    r_err: object = None

    @property
    def n_stacks(self) -> int:
        return int(self.n_layers.size)

    @property
    def n_datasets(self) -> int:
        return int(self.q_off.size - 1)

    @property
    def on_host(self) -> bool:
        return not self.params.is_cuda

    @property
    def total_out(self) -> int:
        lens = (self.q_off[1:] - self.q_off[:-1])[self.dataset]
        return int(lens.sum())

    @staticmethod
    def from_arrays(n_layers, dataset, q_off, params, q, dq, r_obs=None, r_err=None, device="cuda",
                    pin: bool = False) -> "Batch":
        import torch
        dev = torch.device(device)

        def t(a, dt):
            if a is None:
                return None
            x = torch.as_tensor(np.ascontiguousarray(a), dtype=dt)
            if dev.type == "cuda":
                return x.to(dev)
            return x.pin_memory() if pin else x

        return Batch(np.ascontiguousarray(n_layers, dtype=np.int32), np.ascontiguousarray(dataset, dtype=np.int32),
                     np.ascontiguousarray(q_off, dtype=np.int64), t(params, torch.float64), t(q, torch.float32),
                     t(dq, torch.float32), t(r_obs, torch.float32), t(r_err, torch.float32))

    @staticmethod
    def from_workload(wl, device="cuda", pin: bool = False) -> "Batch":
        return Batch.from_arrays(wl.n_layers, wl.dataset, wl.q_off, wl.params, wl.q, wl.dq, wl.r_obs, wl.r_err,
                                 device=device, pin=pin)

    def with_params(self, params) -> "Batch":
        return dataclasses.replace(self, params=params)

    def _c(self) -> CBatch:
        def ptr(x):
            return None if x is None else x.data_ptr()
        for name in ("params", "q", "dq", "r_obs", "r_err"):
            x = getattr(self, name)
            if x is not None and not x.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
        p = self.params
        import torch
        if p.dtype != torch.float64:
            raise TypeError("params must be float64")
        return CBatch(self.n_stacks, self.n_datasets, self.n_layers.ctypes.data, self.dataset.ctypes.data,
                      self.q_off.ctypes.data, NR_MEM_HOST if self.on_host else NR_MEM_DEVICE, 0,
                      ptr(p), ptr(self.q), ptr(self.dq), ptr(self.r_obs), ptr(self.r_err))


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """One library context (quadrature rule, precision, plan cache) on the
    current CUDA device."""

    def __init__(self, n_quad: int = 17, precision: str = "mixed", autotune: bool = False, tile_q: int = 0,
                 chunk_q: int = 0, grid_ctas: int = 0, serial: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2509_06924_gb300 needs a CUDA device (no CPU fallback)")
        self._lib = load_library()
        prec = {"mixed": NR_MIXED, "fp64": NR_FP64_PLAIN}[precision]
        opt = Options(n_quad, prec, 1, int(autotune), tile_q, chunk_q, grid_ctas, int(serial))
        h = ctypes.c_void_p()
        _check(self._lib.nr_create(ctypes.byref(h), ctypes.byref(opt)))
        self._h = h
        self.n_quad = n_quad
        self.precision = precision
        self.device = torch.cuda.current_device()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, batch: Batch) -> None:
        cb = batch._c()
        _check(self._lib.nr_plan(self._h, ctypes.byref(cb)))

    def plan_info(self, batch: Batch) -> dict:
        cb = batch._c()
        ev = ctypes.c_int64()
        tq, cq, gr, la = (ctypes.c_int32() for _ in range(4))
        _check(self._lib.nr_plan_info(self._h, ctypes.byref(cb), ctypes.byref(ev), ctypes.byref(tq),
                                      ctypes.byref(cq), ctypes.byref(gr), ctypes.byref(la)))
        return {"evals": ev.value, "tile_q": tq.value, "chunk_q": cq.value, "grid_ctas": gr.value,
                "launches": la.value}

    def plan_groups(self, batch: Batch, grad: bool = True) -> list:
        """The launches of one compute call on this batch (one per register
        bucket): layer capacity, paired kernel or not, tile, grid, items."""
        cb = batch._c()
        cnt = ctypes.c_int32()
        _check(self._lib.nr_plan_groups(self._h, ctypes.byref(cb), int(grad), 0, ctypes.byref(cnt), None, None,
                                        None, None, None))
        n = cnt.value
        arrs = [(ctypes.c_int32 * max(n, 1))() for _ in range(5)]
        _check(self._lib.nr_plan_groups(self._h, ctypes.byref(cb), int(grad), n, ctypes.byref(cnt), *arrs))
        keys = ("nmax", "paired", "tile_q", "grid", "items")
        return [{k: int(a[i]) for k, a in zip(keys, arrs)} for i in range(n)]

    def _alloc(self, batch: Batch, n, dtype, out=None):
        import torch
        if out is not None:
            return out
        if batch.on_host:
            return torch.empty(n, dtype=dtype).pin_memory()
        return torch.empty(n, dtype=dtype, device=batch.params.device)

    def reflectivity(self, batch: Batch, out=None, stream=None):
        """Smeared model m = scale * S(Q) + bkg, float32 [sum of dataset lengths]."""
        import torch
        r = self._alloc(batch, batch.total_out, torch.float32, out)
        cb = batch._c()
        _check(self._lib.nr_reflectivity(self._h, ctypes.byref(cb), ctypes.c_void_p(r.data_ptr()),
                                         _stream_handle(stream)))
        return r

    def loglik(self, batch: Batch, out=None, stream=None):
        """Gaussian log-likelihood per stack, float64 [S]."""
        import torch
        ll = self._alloc(batch, batch.n_stacks, torch.float64, out)
        cb = batch._c()
        _check(self._lib.nr_loglik(self._h, ctypes.byref(cb), ctypes.c_void_p(ll.data_ptr()),
                                   _stream_handle(stream)))
        return ll

    def loglik_grad(self, batch: Batch, ll_out=None, grad_out=None, stream=None):
        """(loglik [S], gradient packed like params), float64."""
        import torch
        ll = self._alloc(batch, batch.n_stacks, torch.float64, ll_out)
        g = self._alloc(batch, batch.params.numel(), torch.float64, grad_out)
        cb = batch._c()
        _check(self._lib.nr_loglik_grad(self._h, ctypes.byref(cb), ctypes.c_void_p(ll.data_ptr()),
                                        ctypes.c_void_p(g.data_ptr()), _stream_handle(stream)))
        return ll, g

    def loglik_grad_res(self, batch: Batch, ll_out=None, grad_out=None, res_out=None, stream=None):
        """(loglik [S], gradient packed like params, d loglik / d ln f [S]),
        float64, f a common scale of every dQ of a stack's dataset (f = 1)."""
        import torch
        ll = self._alloc(batch, batch.n_stacks, torch.float64, ll_out)
        g = self._alloc(batch, batch.params.numel(), torch.float64, grad_out)
        r = self._alloc(batch, batch.n_stacks, torch.float64, res_out)
        cb = batch._c()
        _check(self._lib.nr_loglik_grad_res(self._h, ctypes.byref(cb), ctypes.c_void_p(ll.data_ptr()),
                                            ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                            _stream_handle(stream)))
        return ll, g, r

    def sld_profile(self, batch: Batch, z, rho_out=None, iota_out=None, stream=None):
        """(rho(z), iota(z)) of every stack, float32 [S, nz]: error-function
        interfaces of width sigma_j at depths z_j = d_1 + ... + d_j.  z: a
        float32 tensor in the batch's memory kind."""
        import torch
        nz = int(z.numel())
        rho = self._alloc(batch, batch.n_stacks * nz, torch.float32, rho_out)
        iota = self._alloc(batch, batch.n_stacks * nz, torch.float32, iota_out)
        cb = batch._c()
        _check(self._lib.nr_sld_profile(self._h, ctypes.byref(cb), ctypes.c_void_p(z.data_ptr()), nz,
                                        ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(iota.data_ptr()),
                                        _stream_handle(stream)))
        return rho.view(batch.n_stacks, nz), iota.view(batch.n_stacks, nz)

    def debug_poison_plan(self, batch: Batch, on: bool) -> None:
        """Testing hook of NR_DEBUG builds (nr_debug_poison_plan): corrupt
        (on) or restore (off) the first work item of the batch's gradient
        plan."""
        cb = batch._c()
        _check(self._lib.nr_debug_poison_plan(self._h, ctypes.byref(cb), int(bool(on))))

    def device_status(self, stream=None) -> int:
        """Synchronise and return (and clear) the sticky NR_FLAG_* word."""
        f = ctypes.c_int32()
        st = self._lib.nr_device_status(self._h, _stream_handle(stream), ctypes.byref(f))
        if st not in (NR_OK, NR_ENONFINITE):
            _check(st)
        return int(f.value)


class Sampler:
    """On-device HMC over n_chains chains of a co-fitted model (nr_sampler_*,
    nr_hmc_step).  Per contrast: n_layers, dataset (index into the datasets
    given by q_off and the device tensors q, dq, r_obs, r_err); per packed
    slot of the concatenated contrasts: slot_src (free parameter or -1) and
    slot_val (fixed value); per free parameter: uniform prior bounds lo, hi;
    res_param: the free parameter that scales every dQ (-1: none).
    States u are unconstrained: theta = lo + (hi - lo) sigmoid(u)."""

    def __init__(self, ctx: Context, n_chains: int, n_layers, dataset, q_off, q, dq, r_obs, r_err, slot_src,
                 slot_val, lo, hi, res_param: int = -1):
        import numpy as np
        self._lib = ctx._lib
        self._ctx = ctx                                   # the sampler lives in the context
        self._keep = [np.ascontiguousarray(n_layers, np.int32), np.ascontiguousarray(dataset, np.int32),
                      np.ascontiguousarray(q_off, np.int64), np.ascontiguousarray(slot_src, np.int32),
                      np.ascontiguousarray(slot_val, np.float64), np.ascontiguousarray(lo, np.float64),
                      np.ascontiguousarray(hi, np.float64)]
        self._data = (q, dq, r_obs, r_err)                # referenced by the sampler
        nl, ds, qo, src, val, lo_, hi_ = self._keep
        self.n_chains, self.n_free = int(n_chains), int(lo_.size)
        m = CCofitModel(self.n_chains, nl.size, self.n_free, nl.ctypes.data, ds.ctypes.data, qo.size - 1,
                        qo.ctypes.data, q.data_ptr(), dq.data_ptr(), r_obs.data_ptr(), r_err.data_ptr(),
                        src.ctypes.data, val.ctypes.data, lo_.ctypes.data, hi_.ctypes.data, int(res_param))
        h = ctypes.c_void_p()
        _check(self._lib.nr_sampler_create(ctx._h, ctypes.byref(m), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nr_sampler_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def logp_grad(self, u, stream=None):
        """(log pi [C], d log pi / du [C, P]) at u [C, P] (float64, device)."""
        import torch
        lp = torch.empty(self.n_chains, dtype=torch.float64, device=u.device)
        g = torch.empty_like(u)
        _check(self._lib.nr_sampler_logp_grad(self._h, ctypes.c_void_p(u.data_ptr()),
                                              ctypes.c_void_p(lp.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                              _stream_handle(stream)))
        return lp, g

    def hmc_step(self, u, z, log_unif, inv_mass, eps: float, n_leapfrog: int, logp_out=None, accepted_out=None,
                 stream=None):
        """One HMC transition of every chain, in place on u [C, P]; returns
        (log pi [C], accepted [C] int32).  z: standard-normal draws [C, P];
        log_unif: log of uniform draws [C]; inv_mass: [P]."""
        import torch
        lp = logp_out if logp_out is not None else torch.empty(self.n_chains, dtype=torch.float64,
                                                                device=u.device)
        acc = accepted_out if accepted_out is not None else torch.empty(self.n_chains, dtype=torch.int32,
                                                                        device=u.device)
        _check(self._lib.nr_hmc_step(self._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                     ctypes.c_void_p(log_unif.data_ptr()), ctypes.c_void_p(inv_mass.data_ptr()),
                                     float(eps), int(n_leapfrog), ctypes.c_void_p(lp.data_ptr()),
                                     ctypes.c_void_p(acc.data_ptr()), _stream_handle(stream)))
        return lp, acc

    def vi_step(self, phi, adam_m, adam_v, t, eps, lr=0.05, beta1=0.9, beta2=0.999, eps_adam=1e-8,
                elbo_out=None, stream=None):
        """One variational-inference iteration of every restart (the sampler's
        chains): phi [R, P + P(P+1)/2] (mu, then the packed lower triangle of L
        with log L_ii on its diagonal), Adam moments adam_m, adam_v of the same
        shape, t a device int32 iteration counter, eps [R, P] standard-normal
        draws.  Updates phi, the moments and t in place; returns the
        single-sample ELBO estimates [R] at the incoming phi."""
        import torch
        elbo = elbo_out if elbo_out is not None else torch.empty(self.n_chains, dtype=torch.float64,
                                                                  device=phi.device)
        opt = CAdam(lr, beta1, beta2, eps_adam)
        _check(self._lib.nr_vi_step(self._h, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(adam_m.data_ptr()),
                                    ctypes.c_void_p(adam_v.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                    ctypes.c_void_p(eps.data_ptr()), ctypes.byref(opt),
                                    ctypes.c_void_p(elbo.data_ptr()), _stream_handle(stream)))
        return elbo


def tune_cache_get(path: str, key: str):
    """One entry of an autotune cache file (dict), or None when absent."""
    e = TuneEntry()
    if load_library().nr_tune_cache_get(path.encode(), key.encode(), ctypes.byref(e)) != NR_OK:
        return None
    return {"paired": e.paired, "tile_q": e.tile_q, "ctas_per_sm": e.ctas_per_sm, "ms": e.ms}


def tune_cache_put(path: str, key: str, paired: int, tile_q: int, ctas_per_sm: int, ms: float = 0.0) -> None:
    """Write one entry of an autotune cache file (host only)."""
    e = TuneEntry(int(paired), int(tile_q), int(ctas_per_sm), 0, float(ms))
    _check(load_library().nr_tune_cache_put(path.encode(), key.encode(), ctypes.byref(e)))


def debug_fail_allocs(count: int) -> None:
    """Testing hook: the next `count` device allocations of the library fail
    as out-of-memory (NR_ENOMEM) without calling cudaMalloc."""
    _check(load_library().nr_debug_fail_allocs(int(count)))


def vi_phi_size(P: int) -> int:
    """Entries of one restart's variational parameters: mu [P] and the packed
    lower triangle of L [P (P + 1) / 2]."""
    return P + P * (P + 1) // 2


def loglik_grad_noalloc(batch: Batch, n_quad: int, ll_out, grad_out, flags_out=None, stream=None) -> None:
    """Log-likelihood and gradient through nr_loglik_grad_noalloc, for hosts
    that may not allocate device memory: the caller passes device outputs
    (and optionally a device int32 for the error flags); the library
    allocates nothing.  Either output may be None (not computed into).  The
    C ABI cannot see buffer sizes, so they are checked here: ll_out holds at
    least n_stacks float64 values, grad_out at least params.numel(), both
    contiguous on the batch's device."""
    import torch

    def dev_ptr(t, name, dtype, numel):
        if t is None:
            return None
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == batch.params.device):
            raise ValueError(f"{name} must be a CUDA tensor on the batch's device")
        if t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
            raise ValueError(f"{name} must be a contiguous {dtype} tensor of at least {numel} elements")
        return t.data_ptr()

    if batch.on_host:
        raise ValueError("nr_loglik_grad_noalloc takes device-memory batches only")
    p_ll = dev_ptr(ll_out, "ll_out", torch.float64, batch.n_stacks)
    p_g = dev_ptr(grad_out, "grad_out", torch.float64, batch.params.numel())
    p_f = dev_ptr(flags_out, "flags_out", torch.int32, 1)
    cb = batch._c()
    _check(load_library().nr_loglik_grad_noalloc(
        ctypes.byref(cb), n_quad, ctypes.c_void_p(p_ll), ctypes.c_void_p(p_g), ctypes.c_void_p(p_f),
        _stream_handle(stream)))


def _autograd_function():
    import torch

    class NRLogLik(torch.autograd.Function):
        """loglik(params) with the library's exact gradient as backward:
        forward calls nr_loglik_grad once and keeps the gradient."""

        @staticmethod
        def forward(ctx_, params, nr_ctx, batch):
            ll, g = nr_ctx.loglik_grad(batch.with_params(params.detach().contiguous()))
            ctx_.save_for_backward(g)
            ctx_.layout = (batch.n_layers, batch.n_stacks)
            return ll

        @staticmethod
        def backward(ctx_, grad_ll):
            (g,) = ctx_.saved_tensors
            n_layers, _ = ctx_.layout
            per = torch.as_tensor(4 * n_layers.astype(np.int64) + 6, device=g.device)
            scale = torch.repeat_interleave(grad_ll, per)
            return g * scale, None, None

    return NRLogLik


_NRLogLik = None


def loglik_autograd(params, ctx: Context, batch: Batch):
    """Differentiable per-stack log-likelihood (torch.autograd)."""
    global _NRLogLik
    if _NRLogLik is None:
        _NRLogLik = _autograd_function()
    return _NRLogLik.apply(params, ctx, batch)
