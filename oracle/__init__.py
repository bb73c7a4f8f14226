"""Plain FP64 CPU oracle for the matrix-element workflow of arXiv:2106.12631.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may load
this package.  The CUDA path never imports it, and it imports nothing from the
CUDA path: the only thing both sides share is the seeded input generator in
``paper_2106_12631_gb300.inputs``.

The C++ source (``mg_oracle.cpp``) evaluates, for every event, the plain
definition of the tree-level squared matrix element (Sec. 2 of the paper):
all Feynman diagrams, all helicity combinations and all explicit colour
assignments, with explicit 4x4 Dirac matrices and explicit SU(3) generators.
RAMBO (Sec. 3, random numbers -> momenta) follows Kleiss, Stirling and Ellis.

Pins: see ``tests/test_oracle_*.py`` (closed forms, Dirac/SU(3) identities,
RAMBO invariants and volumes, Ward identity, Lorentz, parity and Bose
invariance, finite differences for the dual-number gradient).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NPAR = {1: 4, 2: 4, 3: 5, 4: 6}


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O3, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off",
           "-pthread", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("mz", ctypes.c_double), ("wz", ctypes.c_double),
                ("alpha_inv", ctypes.c_double), ("sw2", ctypes.c_double),
                ("mt", ctypes.c_double), ("wt", ctypes.c_double),
                ("alpha_s", ctypes.c_double)]


def params(**over) -> Params:
    from paper_2106_12631_gb300.inputs import SM_PARAMS
    d = dict(SM_PARAMS)
    d.update(over)
    return Params(**{k: float(d[k]) for k, _ in Params._fields_})


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            pp = ctypes.POINTER(Params)
            L.oracle_process_info.argtypes = [ctypes.c_int, ip, ip, ip, ip]
            L.oracle_rambo.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, dp,
                                       ctypes.c_int, pp, dp, dp]
            L.oracle_me.argtypes = [ctypes.c_int, ctypes.c_long, dp, pp, dp, dp, ctypes.c_int]
            L.oracle_amplitudes.argtypes = [ctypes.c_int, dp, ctypes.c_int, pp, dp,
                                            ctypes.c_int, dp, ctypes.c_int]
            L.oracle_colour_gram.argtypes = [ctypes.c_int, dp, ctypes.c_int]
            L.oracle_chain_colour_matrix.argtypes = [ctypes.c_int, dp, ctypes.c_int]
            L.oracle_su3.argtypes = [dp, dp]
            L.oracle_wavefunction.argtypes = [ctypes.c_int, dp, ctypes.c_double,
                                              ctypes.c_int, dp]
            L.oracle_gamma.argtypes = [dp]
            L.oracle_me_grad.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, dp,
                                         ctypes.c_int, pp, dp, dp, ctypes.c_int]
            L.oracle_event_sum.argtypes = [ctypes.c_long, dp, dp, dp]
            L.oracle_colour_flow_info.argtypes = [ctypes.c_int, ip, dp]
            L.oracle_colour_flows.argtypes = [ctypes.c_int, ctypes.c_long, dp, pp, dp, ctypes.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _chk(rc: int, what: str):
    if rc < 0:
        raise ValueError(f"oracle {what} failed with status {rc}")
    return rc


def process_info(proc: int) -> dict:
    a, b, c, d = (ctypes.c_int() for _ in range(4))
    _chk(lib().oracle_process_info(proc, a, b, c, d), "process_info")
    return {"npar": a.value, "nhel": b.value, "ndiagrams": c.value, "namplitudes": d.value}


def rambo(proc: int, rnd: np.ndarray, ecm: float, prm: Params | None = None):
    """rnd: (nrows, nevt) uniforms -> (mom (npar, 4, nevt), wgt (nevt,))."""
    rnd = np.ascontiguousarray(rnd, dtype=np.float64)
    nrows, nevt = rnd.shape
    prm = prm or params()
    mom = np.zeros((NPAR[proc], 4, nevt))
    wgt = np.zeros(nevt)
    _chk(lib().oracle_rambo(proc, nevt, ecm, _p(rnd), nrows, ctypes.byref(prm), _p(mom), _p(wgt)),
         "rambo")
    return mom, wgt


def me(proc: int, mom: np.ndarray, prm: Params | None = None, per_helicity: bool = False,
       nthreads: int = 1):
    """mom: (npar, 4, nevt) -> me (nevt,) [and per-helicity (nhel, nevt)]."""
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    nevt = mom.shape[2]
    prm = prm or params()
    out = np.zeros(nevt)
    ph = np.zeros((1 << NPAR[proc], nevt)) if per_helicity else None
    _chk(lib().oracle_me(proc, nevt, _p(mom), ctypes.byref(prm), _p(out),
                         _p(ph) if ph is not None else None, nthreads), "me")
    return (out, ph) if per_helicity else out


def amplitudes(proc: int, mom1: np.ndarray, h: int, prm: Params | None = None,
               pol_override: np.ndarray | None = None, pol_leg: int = -1) -> np.ndarray:
    """Per-diagram amplitudes (four-gluon vertices split in three terms) for one event."""
    mom1 = np.ascontiguousarray(mom1, dtype=np.float64).reshape(-1)
    prm = prm or params()
    cap = 512
    buf = np.zeros(2 * cap)
    ov = None
    if pol_override is not None:
        ov = np.ascontiguousarray(np.stack([np.real(pol_override), np.imag(pol_override)], -1)
                                  .reshape(-1), dtype=np.float64)
    n = _chk(lib().oracle_amplitudes(proc, _p(mom1), h, ctypes.byref(prm),
                                     _p(ov) if ov is not None else None, pol_leg, _p(buf), cap),
             "amplitudes")
    return buf[: 2 * n:2] + 1j * buf[1: 2 * n:2]


def colour_gram(proc: int) -> np.ndarray:
    cap = 512 * 512
    buf = np.zeros(2 * cap)
    n = _chk(lib().oracle_colour_gram(proc, _p(buf), cap), "colour_gram")
    z = buf[: 2 * n * n:2] + 1j * buf[1: 2 * n * n:2]
    return z.reshape(n, n)


def chain_colour_matrix(ng: int) -> np.ndarray:
    cap = 24 * 24
    buf = np.zeros(2 * cap)
    n = _chk(lib().oracle_chain_colour_matrix(ng, _p(buf), cap), "chain_colour_matrix")
    z = buf[: 2 * n * n:2] + 1j * buf[1: 2 * n * n:2]
    return z.reshape(n, n)


def su3():
    T = np.zeros(8 * 3 * 3 * 2)
    f = np.zeros(512)
    lib().oracle_su3(_p(T), _p(f))
    T = T.reshape(8, 3, 3, 2)
    return T[..., 0] + 1j * T[..., 1], f.reshape(8, 8, 8)


def wavefunction(kind: str, p: np.ndarray, m: float, lam: int) -> np.ndarray:
    k = {"u": 0, "v": 1, "eps": 2}[kind]
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(8)
    _chk(lib().oracle_wavefunction(k, _p(p), m, lam, _p(out)), "wavefunction")
    return out[0::2] + 1j * out[1::2]


def gamma() -> np.ndarray:
    g = np.zeros(5 * 16 * 2)
    lib().oracle_gamma(_p(g))
    g = g.reshape(5, 4, 4, 2)
    return g[..., 0] + 1j * g[..., 1]


def me_grad(proc: int, rnd: np.ndarray, ecm: float, prm: Params | None = None,
            nthreads: int = 1):
    """Forward-mode dual-number gradient d(me)/d(rnd): (me (nevt,), grad (nrows, nevt))."""
    rnd = np.ascontiguousarray(rnd, dtype=np.float64)
    nrows, nevt = rnd.shape
    prm = prm or params()
    out = np.zeros(nevt)
    grad = np.zeros((nrows, nevt))
    _chk(lib().oracle_me_grad(proc, nevt, ecm, _p(rnd), nrows, ctypes.byref(prm), _p(out),
                              _p(grad), nthreads), "me_grad")
    return out, grad


def event_sum(me_: np.ndarray, wgt: np.ndarray) -> np.ndarray:
    me_ = np.ascontiguousarray(me_, dtype=np.float64)
    wgt = np.ascontiguousarray(wgt, dtype=np.float64)
    out = np.zeros(3)
    _chk(lib().oracle_event_sum(me_.shape[0], _p(me_), _p(wgt), _p(out)), "event_sum")
    return out


def colour_flow_info(proc: int):
    """(number of colour flows, residual of the projection of the diagrams'
    colour tensors onto the colour chains)."""
    n, r = ctypes.c_int(), ctypes.c_double()
    _chk(lib().oracle_colour_flow_info(proc, n, ctypes.byref(r)), "colour_flow_info")
    return n.value, r.value


def colour_flows(proc: int, mom: np.ndarray, prm: Params | None = None, nthreads: int = 1) -> np.ndarray:
    """Colour-flow amplitudes J_s of every helicity: complex (nhel, nflow, nevt); the
    full-colour amplitude is sum_s J_s (T^{a_s1} .. T^{a_sk})_{i_top j_antitop}."""
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    nevt = mom.shape[2]
    nf, _ = colour_flow_info(proc)
    prm = prm or params()
    out = np.zeros((1 << NPAR[proc], nf, nevt, 2))
    _chk(lib().oracle_colour_flows(proc, nevt, _p(mom), ctypes.byref(prm), _p(out), nthreads), "colour_flows")
    return out[..., 0] + 1j * out[..., 1]


def choose_colour(jf: np.ndarray, mask: np.ndarray, u: np.ndarray) -> np.ndarray:
    """One colour flow per event with probability w_s / sum_t w_t, w_s = sum over the
    good helicities of |J_s|^2: the first flow whose running sum exceeds u * sum
    (the last flow if rounding leaves none); -1 where the sum is zero."""
    good = np.nonzero(np.asarray(mask))[0]
    w = np.zeros(jf.shape[1:])
    for h in good:
        w += np.abs(jf[h]) ** 2
    out = np.full(jf.shape[2], -1, dtype=np.int32)
    for e in range(jf.shape[2]):
        tot = sum(w[s, e] for s in range(w.shape[0]))
        if tot <= 0.0:
            continue
        target, run = u[e] * tot, 0.0
        out[e] = w.shape[0] - 1
        for s in range(w.shape[0]):
            run += w[s, e]
            if run > target:
                out[e] = s
                break
    return out


# ---- cross section and unweighting (Sec. 3: the run's weighted events give the
# cross section; unweighting keeps events with probability x / max x) ----------
HBARC2_PB = 0.3893793721e9  # (hbar c)^2 in pb GeV^2


def cross_section(proc: int, ecm: float, me_: np.ndarray, wgt: np.ndarray) -> np.ndarray:
    """(sigma, error) in pb: sigma = (hbar c)^2 (2 pi)^(4 - 3 n) / (2 s) mean(w me),
    the Monte Carlo error from the sample variance (flux of massless beams,
    w = RAMBO's flat phase-space weight without (2 pi) factors)."""
    nf = NPAR[proc] - 2
    sums = event_sum(me_, wgt)
    n = sums[2]
    mean = sums[0] / n
    var = (sums[1] / n - mean * mean) * n / (n - 1) if n > 1 else 0.0
    norm = HBARC2_PB * (2 * np.pi) ** (4 - 3 * nf) / (2 * ecm * ecm)
    return np.array([norm * mean, norm * np.sqrt(max(var, 0.0) / n)])


def unweight(me_: np.ndarray, wgt: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Hit-or-miss: indices i (increasing) with u_i * max_j x_j < x_i, x = w me."""
    x = np.asarray(wgt, dtype=np.float64) * np.asarray(me_, dtype=np.float64)
    if x.size == 0:
        return np.zeros(0, dtype=np.int64)
    xmax = x.max()
    return np.nonzero(np.asarray(u, dtype=np.float64) * xmax < x)[0].astype(np.int64)



def choose_helicity(ph: np.ndarray, mask: np.ndarray, u: np.ndarray) -> np.ndarray:
    """One helicity per event with probability |M_h|^2 / sum over the good h.

    Inverse-CDF sampling over the good helicities (mask != 0) in increasing
    index order: the first h whose running sum exceeds u * sum (the last good
    one if rounding leaves none); -1 where the sum is zero.  ph: (nhel, nevt).
    """
    ph = np.asarray(ph, dtype=np.float64)
    good = np.nonzero(np.asarray(mask))[0]
    out = np.full(ph.shape[1], -1, dtype=np.int32)
    for e in range(ph.shape[1]):
        tot = sum(ph[h, e] for h in good)
        if tot <= 0.0:
            continue
        target, run = u[e] * tot, 0.0
        out[e] = good[-1]
        for h in good:
            run += ph[h, e]
            if run > target:
                out[e] = h
                break
    return out
