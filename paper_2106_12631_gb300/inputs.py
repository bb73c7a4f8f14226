"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds no matrix-element or phase-space arithmetic: only the
uniform random numbers the workflow starts from (the paper's toy workflow
draws them with cuRAND, "four per particle", Sec. 3) and the fixed physics
inputs of the four workloads.

Uniforms come from a counter-based SplitMix64 generator (Steele, Lea and
Flood, OOPSLA 2014): the value for event ``i`` and row ``k`` depends only on
``(seed, i, k)``, so any event of a large batch can be regenerated alone:

    key  = mix64(seed)
    z    = mix64(key + (i * 64 + k + 1) * 0x9E3779B97F4A7C15)   (mod 2^64)
    u    = ((z >> 11) + 0.5) * 2^-53          in the open interval (0, 1)

with mix64(x) = SplitMix64's finaliser (xor-shift 30 / multiply
0xBF58476D1CE4E5B9 / xor-shift 27 / multiply 0x94D049BB133111EB / xor-shift 31).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
ROW_STRIDE = 64  # counter slots reserved per event

# Standard-Model inputs of the workloads (GeV units)
SM_PARAMS = dict(mz=91.188, wz=2.441, alpha_inv=132.507, sw2=0.2222,
                 mt=173.0, wt=1.491, alpha_s=0.118)

# The five workloads: process id, centre-of-mass energy, events, random rows
#   1 e+e- -> mu+mu- (photon + Z), 2 gg -> t tbar, 3 gg -> t tbar g, 4 gg -> t tbar g g
WORKLOADS = {
    "ee_mumu": dict(index=1, proc=1, ecm=500.0, nevt=16384, nrows=8),
    "gg_tt": dict(index=2, proc=2, ecm=1500.0, nevt=1 << 20, nrows=8),
    "gg_ttg": dict(index=3, proc=3, ecm=1500.0, nevt=1 << 20, nrows=12),
    "gg_ttgg": dict(index=4, proc=4, ecm=1500.0, nevt=1 << 20, nrows=16),
    "gg_ttg_grad": dict(index=5, proc=3, ecm=1500.0, nevt=1 << 18, nrows=16),
}
SEED_BASE = 2106126310
FILTER_SEED_OFFSET = 1000


def seed_of(workload: str) -> int:
    return SEED_BASE + WORKLOADS[workload]["index"]


def filter_seed_of(workload: str) -> int:
    return seed_of(workload) + FILTER_SEED_OFFSET


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniforms(seed: int, nrows: int, nevt: int, first_event: int = 0) -> np.ndarray:
    """(nrows, nevt) float64 uniforms in (0, 1) for events first_event .. first_event+nevt-1."""
    if nrows > ROW_STRIDE:
        raise ValueError("at most %d rows per event" % ROW_STRIDE)
    with np.errstate(over="ignore"):
        key = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        ev = np.arange(first_event, first_event + nevt, dtype=np.uint64)
        out = np.empty((nrows, nevt), dtype=np.float64)
        for k in range(nrows):
            ctr = ev * np.uint64(ROW_STRIDE) + np.uint64(k + 1)
            z = _mix64(key + ctr * GOLDEN)
            out[k] = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    return out


def uniforms_at(seed: int, nrows: int, events: np.ndarray) -> np.ndarray:
    """Uniforms for an arbitrary list of event indices: (nrows, len(events))."""
    events = np.asarray(events, dtype=np.int64)
    cols = [uniforms(seed, nrows, 1, int(e))[:, 0] for e in events]
    return np.stack(cols, axis=1) if cols else np.zeros((nrows, 0))
