"""TEST INFRASTRUCTURE ONLY: ctypes wrapper around the plain CPU oracle
(``nr_oracle.c``) for the batched neutron-reflectivity model of
arXiv 2509.06924 (Abeles forward model, Sec. 2.1; Gaussian smearing, Sec. 3;
Gaussian likelihood / chi^2, Sec. 2.1 and Eq. 25; exact gradient, Sec. 3).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the C source is compiled here with gcc into ``oracle/_build``.

Every function takes and returns float64 numpy arrays.  ``precision="long"``
selects the long-double build of the same source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[str, ctypes.CDLL] = {}

MAX_LAYERS = 64


def _lib_path(precision: str) -> str:
    return os.path.join(_BUILD, "liboracle_ld.so" if precision == "long" else "liboracle.so")


def build(force: bool = False) -> None:
    """Compile both oracle builds (double and long double) with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    for precision, extra in (("double", []), ("long", ["-DNR_ORACLE_LONG"])):
        out = _lib_path(precision)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra, _SRC, "-o", out + ".tmp", "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)  # without OpenMP
        os.replace(out + ".tmp", out)


def _lib(precision: str = "double") -> ctypes.CDLL:
    with _LOCK:
        if precision not in _LIBS:
            build()
            lib = ctypes.CDLL(_lib_path(precision))
            D = ctypes.POINTER(ctypes.c_double)
            I32 = ctypes.POINTER(ctypes.c_int32)
            I64 = ctypes.POINTER(ctypes.c_int64)
            c_int = ctypes.c_int
            lib.oracle_gauss_hermite.argtypes = [c_int, D, D]
            lib.oracle_amplitude.argtypes = [c_int, D, c_int, D, c_int, D, D]
            lib.oracle_reflectivity_unsmeared_d.argtypes = [c_int, D, c_int, D, c_int, D, D]
            lib.oracle_model.argtypes = [c_int, D, c_int, D, D, c_int, c_int, D]
            lib.oracle_loglik_grad.argtypes = [c_int, D, c_int, D, D, D, D, c_int, D, D]
            lib.oracle_loglik_grad_res.argtypes = [c_int, D, c_int, D, D, D, D, c_int, D]
            lib.oracle_sld_profile.argtypes = [c_int, D, c_int, D, D, D]
            lib.oracle_batch.argtypes = [c_int, c_int, I32, D, I32, c_int, I64, D, D, D, D,
                                         c_int, c_int, D, D, D]
            _LIBS[precision] = lib
        return _LIBS[precision]


def _d(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(status: int, what: str) -> None:
    if status != 0:
        raise ValueError(f"oracle {what} failed with status {status}")


def max_threads() -> int:
    return int(_lib().oracle_max_threads())


def real_bytes(precision: str = "double") -> int:
    return int(_lib(precision).oracle_real_bytes())


def gauss_hermite(K: int, precision: str = "double"):
    """Nodes/weights of the K-point Gauss-Hermite rule for exp(-x^2)."""
    x = np.zeros(K)
    w = np.zeros(K)
    _check(_lib(precision).oracle_gauss_hermite(K, _d(x), _d(w)), "gauss_hermite")
    return x, w


def amplitude(n: int, params, q, form: int = 0, precision: str = "double") -> np.ndarray:
    """Unsmeared complex amplitude r(q); form 0 = Abeles matrix, 1 = Parratt."""
    p, q = _f64(params), _f64(q)
    re, im = np.zeros(q.size), np.zeros(q.size)
    _check(_lib(precision).oracle_amplitude(n, _d(p), q.size, _d(q), form, _d(re), _d(im)),
           "amplitude")
    return re + 1j * im


def reflectivity_unsmeared(n: int, params, q, seed: int = -1, precision: str = "double"):
    """R(q) = |r|^2 and, if seed >= 0, dR/d params[seed] (exact, dual numbers)."""
    p, q = _f64(params), _f64(q)
    R, dR = np.zeros(q.size), np.zeros(q.size)
    _check(_lib(precision).oracle_reflectivity_unsmeared_d(n, _d(p), q.size, _d(q), seed,
                                                          _d(R), _d(dR)), "unsmeared")
    return (R, dR) if seed >= 0 else R


def model(n: int, params, Q, dQ, K: int, form: int = 0, precision: str = "double") -> np.ndarray:
    """Smeared model m = scale * S(Q) + bkg of one stack."""
    p, Q, dQ = _f64(params), _f64(Q), _f64(dQ)
    m = np.zeros(Q.size)
    _check(_lib(precision).oracle_model(n, _d(p), Q.size, _d(Q), _d(dQ), K, form, _d(m)), "model")
    return m


def loglik_grad(n: int, params, Q, dQ, Robs, err, K: int, grad: bool = True,
                precision: str = "double"):
    """(loglik, gradient or None) of one stack."""
    p, Q, dQ, Robs, err = _f64(params), _f64(Q), _f64(dQ), _f64(Robs), _f64(err)
    ll = np.zeros(1)
    g = np.zeros(4 * n + 6) if grad else None
    _check(_lib(precision).oracle_loglik_grad(n, _d(p), Q.size, _d(Q), _d(dQ), _d(Robs), _d(err), K,
                                              _d(ll), _d(g) if grad else None), "loglik_grad")
    return float(ll[0]), g


def loglik_grad_res(n: int, params, Q, dQ, Robs, err, K: int, precision: str = "double") -> float:
    """d loglik / d ln f of one stack, where every dQ_i is scaled by f (at
    f = 1): the derivative in a shared resolution (smearing) scale."""
    p, Q, dQ, Robs, err = _f64(params), _f64(Q), _f64(dQ), _f64(Robs), _f64(err)
    out = np.zeros(1)
    _check(_lib(precision).oracle_loglik_grad_res(n, _d(p), Q.size, _d(Q), _d(dQ), _d(Robs), _d(err), K,
                                                  _d(out)), "loglik_grad_res")
    return float(out[0])


def sld_profile(n: int, params, z, precision: str = "double"):
    """(rho(z), iota(z)) of one stack: interface steps smoothed by the
    Gaussian roughness (error-function profile), depth z in A from the
    fronting/first-layer interface."""
    p, z = _f64(params), _f64(z)
    rho, iota = np.zeros(z.size), np.zeros(z.size)
    _check(_lib(precision).oracle_sld_profile(n, _d(p), z.size, _d(z), _d(rho), _d(iota)), "sld_profile")
    return rho, iota


def batch(mode: str, n_layers, params, dataset, q_off, Q, dQ, Robs, err, K: int,
          n_threads: int = 0, precision: str = "double"):
    """Batch driver.  mode: 'model' -> m [sum of dataset lengths over stacks];
    'loglik' -> ll [n_stacks]; 'grad' -> (ll, grad packed like params);
    'grad_res' -> (ll, grad, d ll / d ln(resolution scale) [n_stacks])."""
    nl = np.ascontiguousarray(n_layers, dtype=np.int32)
    ds = np.ascontiguousarray(dataset, dtype=np.int32)
    qo = np.ascontiguousarray(q_off, dtype=np.int64)
    p, Q, dQ = _f64(params), _f64(Q), _f64(dQ)
    Robs = _f64(Robs if Robs is not None else np.zeros_like(Q))
    err = _f64(err if err is not None else np.ones_like(Q))
    S = nl.size
    lens = (qo[1:] - qo[:-1])[ds] if S else np.zeros(0, np.int64)
    m = np.zeros(int(lens.sum()) if mode == "model" else max(S, 1) if mode == "grad_res" else 1)
    ll = np.zeros(max(S, 1))
    g = np.zeros(p.size if mode in ("grad", "grad_res") else 1)
    code = {"model": 0, "loglik": 1, "grad": 2, "grad_res": 3}[mode]
    st = _lib(precision).oracle_batch(
        code, S, nl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _d(p),
        ds.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(qo.size - 1),
        qo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _d(Q), _d(dQ), _d(Robs), _d(err),
        K, n_threads, _d(m), _d(ll), _d(g))
    _check(st, "batch")
    if mode == "model":
        return m
    if mode == "loglik":
        return ll[:S]
    if mode == "grad_res":
        return ll[:S], g, m[:S]
    return ll[:S], g


def perturbation_floor(n_layers, params, dataset, q_off, Q, dQ, Robs, err, K: int, typ, n_pert: int = 3,
                       seed: int = 0x5EED, n_threads: int = 0) -> dict:
    """How far the exact results of each stack move when every input
    parameter is perturbed by at most one FP32 unit roundoff: p_t = p (1 +
    2^-24 u_t), u_t uniform in [-1, 1] per parameter, t = 1..n_pert.  Per
    stack, the largest over t of
      'loglik': |l_t - l| / |l|,
      'model':  max_i |log m_t,i - log m_i| (the smeared model),
      'grad':   ||(g_t - g) typ||_inf / ||g typ||_inf,
    with typ packed like params.  An evaluation in FP32 arithmetic cannot be
    expected to land closer to the exact result than this response: its own
    roundings act as perturbations of the same size.  Condition estimate
    for the parity bounds; not part of the method."""
    nl = np.ascontiguousarray(n_layers, dtype=np.int32)
    p = _f64(params)
    typ = _f64(typ)
    S = nl.size
    po = np.concatenate([[0], np.cumsum(4 * nl.astype(np.int64) + 6)])
    lens = (np.asarray(q_off)[1:] - np.asarray(q_off)[:-1])[np.asarray(dataset)]
    oo = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ll0, g0 = batch("grad", nl, p, dataset, q_off, Q, dQ, Robs, err, K, n_threads=n_threads)
    m0 = batch("model", nl, p, dataset, q_off, Q, dQ, None, None, K, n_threads=n_threads)
    rng = np.random.default_rng(seed)
    f_ll, f_m, f_g = np.zeros(S), np.zeros(S), np.zeros(S)
    for _ in range(n_pert):
        pt = p * (1.0 + 2.0 ** -24 * rng.uniform(-1.0, 1.0, p.size))
        ll, g = batch("grad", nl, pt, dataset, q_off, Q, dQ, Robs, err, K, n_threads=n_threads)
        m = batch("model", nl, pt, dataset, q_off, Q, dQ, None, None, K, n_threads=n_threads)
        for s in range(S):
            f_ll[s] = max(f_ll[s], abs(ll[s] - ll0[s]) / abs(ll0[s]))
            a, b = po[s], po[s + 1]
            den = np.max(np.abs(g0[a:b] * typ[a:b]))
            if den > 0:
                f_g[s] = max(f_g[s], float(np.max(np.abs((g[a:b] - g0[a:b]) * typ[a:b])) / den))
            if oo[s + 1] > oo[s]:
                f_m[s] = max(f_m[s], float(np.max(np.abs(np.log(m[oo[s]:oo[s + 1]]) - np.log(m0[oo[s]:oo[s + 1]])))))
    return {"loglik": f_ll, "model": f_m, "grad": f_g}
