"""Small test-only helpers: Minkowski products, Lorentz transformations and
the parity bars shared by the test files."""
import numpy as np

# FP64 path: 1e-12 relative per event; on events whose own FP64 conditioning
# is worse, 4 d_rot (d_rot: oracle_conditioning below), never above 1e-9.
FP64_REL = 1e-12
FP64_CAP = 1e-9
# mixed path (FP32 amplitudes, FP64 propagator invariants and sums): stated bound
MIXED_MAX_REL = 1e-4
MIXED_P999_REL = 1e-5
MIXED_MEDIAN_REL = 1e-6


def fp64_tol(d_rot):
    """Per-event FP64 bar: 1e-12, or 4 d_rot on ill-conditioned events, at most 1e-9."""
    return np.minimum(np.maximum(FP64_REL, 4 * np.asarray(d_rot)), FP64_CAP)


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def boost(p, beta):
    """Pure boost of four-vectors p[..., 4 on axis 0] by velocity beta (3-vector)."""
    b = np.asarray(beta, dtype=float)
    b2 = b @ b
    g = 1.0 / np.sqrt(1.0 - b2)
    bp = b[0] * p[1] + b[1] * p[2] + b[2] * p[3]
    out = np.empty_like(p)
    out[0] = g * (p[0] + bp)
    for k in range(3):
        out[k + 1] = p[k + 1] + ((g - 1.0) * bp / b2 + g * p[0]) * b[k]
    return out


def rotate(p, axis, angle):
    """Rotation of the spatial part about a unit axis (Rodrigues)."""
    k = np.asarray(axis, dtype=float)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K
    out = p.copy()
    out[1:] = np.tensordot(R, p[1:], axes=(1, 0))
    return out


def two_body(ecm, m, cth, phi):
    """Beams along +-z and a back-to-back final pair of mass m at angles (cth, phi):
    exactly on shell up to one rounding, independent of any phase-space generator."""
    n = len(cth)
    e = ecm / 2.0
    k = np.sqrt(e * e - m * m)
    sth = np.sqrt(1.0 - cth ** 2)
    mom = np.zeros((4, 4, n))
    mom[0] = np.array([e, 0.0, 0.0, e])[:, None]
    mom[1] = np.array([e, 0.0, 0.0, -e])[:, None]
    d = np.stack([sth * np.cos(phi), sth * np.sin(phi), cth])
    mom[2, 0] = e
    mom[2, 1:] = k * d
    mom[3, 0] = e
    mom[3, 1:] = -k * d
    return mom


def rambo_gamma(rnd, nfin):
    """Lorentz factor Q0/M of the unconstrained massless system RAMBO boosts back
    to rest; its rounding is amplified by about gamma^2 (condition estimate)."""
    Q = np.zeros((4, rnd.shape[1]))
    for i in range(nfin):
        c = 2 * rnd[4 * i] - 1
        s = np.sqrt(1 - c * c)
        f = 2 * np.pi * rnd[4 * i + 1]
        e = -np.log(rnd[4 * i + 2] * rnd[4 * i + 3])
        Q += np.stack([e, e * s * np.cos(f), e * s * np.sin(f), e * c])
    return Q[0] / np.sqrt(mdot(Q, Q))


ROTATIONS = (([0.3, 0.5, 0.8], 0.77), ([-0.6, 0.2, 0.1], 2.3))


def oracle_conditioning(orc, proc, mom, prm=None, nthreads=8):
    """Sensitivity of the FP64 oracle to rounding-level changes of the momenta:
    the largest relative change of me under exact rotations of the event (a
    rotation only re-rounds the inputs).  Events near a collinear or soft
    limit cancel strongly between diagrams and show large values."""
    me0 = orc.me(proc, mom, prm, nthreads=nthreads)
    worst = np.zeros_like(me0)
    for axis, ang in ROTATIONS:
        mr = np.ascontiguousarray(np.stack([rotate(mom[l], axis, ang) for l in range(mom.shape[0])]))
        worst = np.maximum(worst, np.abs(orc.me(proc, mr, prm, nthreads=nthreads) / me0 - 1))
    return me0, worst

