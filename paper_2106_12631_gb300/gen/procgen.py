"""Restricted process generator: Feynman diagrams -> straight-line CUDA.

For each of the four processes of the paper's benchmarks (Sec. 2 and Table 1:
e+e- -> mu+mu-, gg -> t tbar, gg -> t tbar g, gg -> t tbar g g) this script
enumerates the tree-level Feynman diagrams, decomposes their colour factors
into colour flows (the colour-flow method of Sec. 2: each diagram's amplitude
is added, with a coefficient, to the dual amplitudes J_sigma of the flows it
contributes to), computes the colour matrix of the flows, and emits one
straight-line device function per process that evaluates every J_sigma for
one helicity combination from external wavefunctions, internal currents and
vertex amplitudes (the three routine categories of Sec. 2 / Fig. 1).

Design (independent of the CPU oracle, which uses explicit colour tensors):

* All momenta are taken outgoing.  The antitop (QCD processes) or the mu-
  (e+e- -> mu+mu-) is the root leg; every other leg subset S gets the list
  of off-shell currents whose external legs are exactly S; each unordered
  partition into 2 (or 3, four-gluon vertex) parts is visited once.  With the
  antitop as root, the fermion line never closes into a gluon, so every
  diagram's colour factor is a product, along the quark line, of matrices
  M built from gluon sub-trees by nested commutators:
      external gluon a        M = T^a
      three-gluon vertex      M = -i [M1, M2]          (f^{abx} T^x = -i [T^a, T^b])
      four-gluon term 0/1/2   M = -[[M1,M2],M3] / -[[M1,M3],M2] / -[[M2,M3],M1]
  Expanding the commutators gives the diagram's coefficient on each colour
  chain (T^{a_s1} ... T^{a_sn})_{i j} exactly (powers of i, integers).
* The colour matrix C_{st} = sum over colours of chain_s conj(chain_t) is
  computed with explicit Gell-Mann matrices and reconstructed as exact
  rationals (common denominator, integer numerators).
* Conventions: Peskin & Schroeder Feynman rules (quark-gluon i g gamma^mu T^a,
  three-gluon g f^abc [...], four-gluon -i g^2 [...], fermion propagator
  i(p/ + m)/(p^2 - m^2 + i m Gamma), Feynman-gauge vector propagator
  -i g^{mu nu}/(p^2 - M^2 + i M Gamma)).  The Z propagator's q^mu q^nu term
  is dropped: it vanishes on the massless lepton currents.

Run ``python -m paper_2106_12631_gb300.gen`` to regenerate ``csrc/gen/``.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# process definitions
# ---------------------------------------------------------------------------
# line kinds: "g" gluon, "A" photon, "Z", ("row", fl) flowing-out fermion
# (u-bar / v-bar), ("col", fl) flowing-in fermion (u / v); fl in {"t","e","mu"}


@dataclass
class LegSpec:
    name: str
    kind: object
    incoming: bool
    particle: bool
    mass: str  # "0" or "mt"


@dataclass
class ProcSpec:
    pid: int
    name: str
    legs: list
    root: int
    hel_avg: int
    col_avg: int
    sym: int


PROCS = {
    1: ProcSpec(1, "ee_mumu", [
        LegSpec("e+", ("row", "e"), True, False, "0"),
        LegSpec("e-", ("col", "e"), True, True, "0"),
        LegSpec("mu+", ("col", "mu"), False, False, "0"),
        LegSpec("mu-", ("row", "mu"), False, True, "0")], root=3, hel_avg=4, col_avg=1, sym=1),
    2: ProcSpec(2, "gg_tt", [
        LegSpec("g", "g", True, True, "0"), LegSpec("g", "g", True, True, "0"),
        LegSpec("t", ("row", "t"), False, True, "mt"),
        LegSpec("t~", ("col", "t"), False, False, "mt")], root=3, hel_avg=4, col_avg=64, sym=1),
    3: ProcSpec(3, "gg_ttg", [
        LegSpec("g", "g", True, True, "0"), LegSpec("g", "g", True, True, "0"),
        LegSpec("t", ("row", "t"), False, True, "mt"),
        LegSpec("t~", ("col", "t"), False, False, "mt"),
        LegSpec("g", "g", False, True, "0")], root=3, hel_avg=4, col_avg=64, sym=1),
    4: ProcSpec(4, "gg_ttgg", [
        LegSpec("g", "g", True, True, "0"), LegSpec("g", "g", True, True, "0"),
        LegSpec("t", ("row", "t"), False, True, "mt"),
        LegSpec("t~", ("col", "t"), False, False, "mt"),
        LegSpec("g", "g", False, True, "0"), LegSpec("g", "g", False, True, "0")],
        root=3, hel_avg=4, col_avg=64, sym=2),
}


def _is_row(k):
    return isinstance(k, tuple) and k[0] == "row"


def _is_col(k):
    return isinstance(k, tuple) and k[0] == "col"


# ---------------------------------------------------------------------------
# symbolic colour: polynomials in non-commuting generators T^{a_g}
# represented as {tuple(gluon legs in order): complex coefficient}
# ---------------------------------------------------------------------------
def cmul(x, y):
    out = {}
    for kx, vx in x.items():
        for ky, vy in y.items():
            k = kx + ky
            out[k] = out.get(k, 0) + vx * vy
    return {k: v for k, v in out.items() if v != 0}


def cadd(x, y, s=1):
    out = dict(x)
    for k, v in y.items():
        out[k] = out.get(k, 0) + s * v
    return {k: v for k, v in out.items() if v != 0}


def cscale(x, s):
    return {k: v * s for k, v in x.items() if v * s != 0}


def comm(x, y):
    return cadd(cmul(x, y), cmul(y, x), -1)


# ---------------------------------------------------------------------------
# diagram enumeration
# ---------------------------------------------------------------------------
@dataclass
class Cur:
    idx: int
    legs: frozenset
    kind: object              # line kind of the current
    vertex: str               # "ext", "qqg_row", "qqg_col", "ggg", "gggg0/1/2", "ffa", "ffz", ...
    children: tuple = ()
    colour: dict = field(default_factory=dict)  # gluon currents: matrix rep M; fermion: line product
    n4: int = 0               # four-gluon vertices below
    nz4: int = 0              # ... with term != 0


@dataclass
class Amp:
    vertex: str               # "ffv_t", "ffv_a", "ffz"
    row: int                  # current indices (row fermion, col fermion, boson)
    col: int
    bos: int
    colour: dict
    counted: bool             # first member of its four-gluon family


class Process:
    def __init__(self, spec: ProcSpec):
        self.spec = spec
        self.n = len(spec.legs)
        self.cur = []
        self.by_legs = {}
        self.amps = []
        rest = frozenset(i for i in range(self.n) if i != spec.root)
        self._currents(rest)
        self._amplitudes(rest)

    # ---- currents -------------------------------------------------------
    def _new(self, **kw):
        c = Cur(idx=len(self.cur), **kw)
        self.cur.append(c)
        return c.idx

    def _currents(self, S):
        if S in self.by_legs:
            return self.by_legs[S]
        out = []
        if len(S) == 1:
            (leg,) = S
            L = self.spec.legs[leg]
            col = {(leg,): 1} if L.kind == "g" else ({(): 1} if isinstance(L.kind, tuple) else {})
            out.append(self._new(legs=S, kind=L.kind, vertex="ext", children=(leg,), colour=col))
            self.by_legs[S] = out
            return out
        items = sorted(S)
        first = items[0]
        others = items[1:]
        # two-part partitions: the part holding `first` is S1
        for r in range(0, len(others)):
            for sub in itertools.combinations(others, r):
                S1 = frozenset((first,) + sub)
                S2 = S - S1
                if not S2:
                    continue
                for a in self._currents(S1):
                    for b in self._currents(S2):
                        out.extend(self._join2(S, a, b))
        # three-part partitions (four-gluon vertex)
        for r1 in range(0, len(others)):
            for sub1 in itertools.combinations(others, r1):
                S1 = frozenset((first,) + sub1)
                R = sorted(S - S1)
                if len(R) < 2:
                    continue
                f2 = R[0]
                for r2 in range(0, len(R) - 1):
                    for sub2 in itertools.combinations(R[1:], r2):
                        S2 = frozenset((f2,) + sub2)
                        S3 = frozenset(R) - S2
                        if not S3:
                            continue
                        for a in self._currents(S1):
                            for b in self._currents(S2):
                                for c in self._currents(S3):
                                    out.extend(self._join3(S, a, b, c))
        self.by_legs[S] = out
        return out

    def _join2(self, S, ia, ib):
        A, B = self.cur[ia], self.cur[ib]
        made = []
        for x, y in ((A, B), (B, A)):
            if x is B and A.kind == B.kind:
                continue
            kx, ky = x.kind, y.kind
            n4, nz4 = x.n4 + y.n4, x.nz4 + y.nz4
            if kx == "g" and ky == "g" and x is A:
                col = cscale(comm(x.colour, y.colour), -1j)
                made.append(self._new(legs=S, kind="g", vertex="ggg", children=(x.idx, y.idx),
                                      colour=col, n4=n4, nz4=nz4))
            elif _is_row(kx) and ky == "g" and kx[1] == "t":
                made.append(self._new(legs=S, kind=kx, vertex="qqg_row", children=(x.idx, y.idx),
                                      colour=cmul(x.colour, y.colour), n4=n4, nz4=nz4))
            elif _is_col(kx) and ky == "g" and kx[1] == "t":
                made.append(self._new(legs=S, kind=kx, vertex="qqg_col", children=(x.idx, y.idx),
                                      colour=cmul(y.colour, x.colour), n4=n4, nz4=nz4))
            elif _is_row(kx) and _is_col(ky) and kx[1] == ky[1] and kx[1] != "t":
                for bos in ("A", "Z"):
                    made.append(self._new(legs=S, kind=bos, vertex="ff" + bos.lower() + "_cur",
                                          children=(x.idx, y.idx), colour={(): 1}, n4=n4, nz4=nz4))
            elif _is_row(kx) and _is_col(ky) and kx[1] == "t":
                raise NotImplementedError("quark line closing into a gluon: choose a quark root")
        return made

    def _join3(self, S, ia, ib, ic):
        A, B, C = self.cur[ia], self.cur[ib], self.cur[ic]
        if not (A.kind == B.kind == C.kind == "g"):
            return []
        m1, m2, m3 = A.colour, B.colour, C.colour
        cols = [cscale(comm(comm(m1, m2), m3), -1), cscale(comm(comm(m1, m3), m2), -1),
                cscale(comm(comm(m2, m3), m1), -1)]
        made = []
        n4 = 1 + A.n4 + B.n4 + C.n4
        nz = A.nz4 + B.nz4 + C.nz4
        for t in range(3):
            made.append(self._new(legs=S, kind="g", vertex="gggg%d" % t, children=(ia, ib, ic),
                                  colour=cols[t], n4=n4, nz4=nz + (t != 0)))
        return made

    # ---- amplitudes at the root -------------------------------------------
    def _amplitudes(self, rest):
        spec = self.spec
        rk = spec.legs[spec.root].kind
        root_cur = self._new(legs=frozenset([spec.root]), kind=rk, vertex="ext",
                             children=(spec.root,), colour={(): 1})
        self.root_cur = root_cur
        items = sorted(rest)
        for r in range(1, len(items)):
            for sub in itertools.combinations(items, r):
                S1 = frozenset(sub)
                S2 = rest - S1
                for a in self._currents(S1):
                    for b in self._currents(S2):
                        A, B = self.cur[a], self.cur[b]
                        if B.kind == "g" and _is_row(A.kind) and _is_col(rk) and A.kind[1] == "t":
                            # quark line: row (top end) . T^b . root column
                            self.amps.append(Amp("ffv_t", a, root_cur, b, cmul(A.colour, B.colour),
                                                 A.nz4 + B.nz4 == 0))
                        elif B.kind in ("A", "Z") and _is_col(A.kind) and _is_row(rk) \
                                and A.kind[1] == rk[1]:
                            self.amps.append(Amp("ffv_a" if B.kind == "A" else "ffz", root_cur, a, b,
                                                 {(): 1}, True))

    @property
    def ndiagrams(self):
        return sum(1 for a in self.amps if a.counted)

    def gluon_legs(self):
        return [i for i, L in enumerate(self.spec.legs) if L.kind == "g"]


# ---------------------------------------------------------------------------
# colour flows and colour matrix
# ---------------------------------------------------------------------------
def gell_mann():
    lam = np.zeros((8, 3, 3), complex)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / math.sqrt(3)
    return lam / 2


def chain_matrix(ng: int):
    """C_{st} for the ng! chains in lexicographic permutation order, as (numerators, den)."""
    T = gell_mann()
    perms = list(itertools.permutations(range(ng)))
    # tensor of each chain over (a_1..a_ng, i, j)
    ch = []
    for p in perms:
        acc = np.zeros((8,) * ng + (3, 3), complex)
        for a in itertools.product(range(8), repeat=ng):
            M = np.eye(3, dtype=complex)
            for k in p:
                M = M @ T[a[k]]
            acc[a] = M
        ch.append(acc.reshape(-1))
    ch = np.array(ch)
    C = ch @ ch.conj().T
    assert np.max(np.abs(C.imag)) < 1e-10
    C = C.real
    den = 8 * 3 ** ng  # SU(3) chain traces are rationals with denominators 2^a 3^b
    num = np.rint(C * den)
    assert np.max(np.abs(num - C * den)) < 1e-8, "colour matrix not rational with denominator 8 3^n"
    num = num.astype(np.int64)
    g = int(np.gcd.reduce(np.append(num.reshape(-1), den)))
    return perms, num // g, den // g


def colour_flows(proc: Process):
    """Coefficient of every amplitude on every chain; returns (perms, coef[namp][nflow])."""
    gl = proc.gluon_legs()
    ng = len(gl)
    if ng == 0:
        return [()], np.ones((len(proc.amps), 1), complex)
    perms = list(itertools.permutations(range(ng)))
    index = {tuple(gl[k] for k in p): i for i, p in enumerate(perms)}
    coef = np.zeros((len(proc.amps), len(perms)), complex)
    for d, a in enumerate(proc.amps):
        for word, v in a.colour.items():
            coef[d, index[word]] += v
    return perms, coef


# ---------------------------------------------------------------------------
# CUDA emission
# ---------------------------------------------------------------------------
def _cpx(z):
    z = complex(z)
    return "cx<R>(R(%r), R(%r))" % (z.real, z.imag)


# Floating-point operations of each device routine as written in
# csrc/helas.cuh (complex add 2, complex multiply 6, real x complex 2; an FMA
# counts as 2).  External wavefunctions include their square roots and
# divisions as one operation each.
FLOPS = {
    "ixxxxx": 45, "oxxxxx": 45, "vxxxxx": 20,
    "FFV1_0": 96, "FFV2_4_0": 104,
    "FFV1_1": 148, "FFV1_2": 148, "FFV1P0_3": 106, "FFV2_4_3": 114,
    "VVV1P0_1": 176, "VVVV1P0_1": 142, "VVVV3P0_1": 142, "VVVV4P0_1": 142,
    "VVV1_0": 168, "VVVV_0": 136,
    # amputated currents (no propagator) and the contraction sum_i X_i Y_i
    "FFV1_2A": 72, "FFV1_1A": 72, "FFV1P0_3A": 80, "FFV2_4_3A": 96, "VVV1P0_1A": 158, "VVVV_A": 124,
    "DOT4": 30, "W4ADD": 8,
    "jamp": 2,
}


def colour_sum_sym_flops(cnum) -> int:
    """J^dagger C J / CDEN with the symmetric form: per row the diagonal term
    (2 multiplies), two multiply-adds per non-zero upper entry, the row's
    re/im products into the sum (4), and the final scale."""
    nc = cnum.shape[0]
    upper = sum(1 for i in range(nc) for j in range(i + 1, nc) if cnum[i, j] != 0)
    return 2 * nc + 4 * upper + 4 * nc + 1


def colour_sum_flops(cnum) -> int:
    """Real colour sum J^dagger C J with C = CNUM / CDEN on CUDA cores: per row
    two FMAs per non-zero entry, then re/im products, the row sum and the scale."""
    nz = int(np.count_nonzero(cnum))
    return 4 * nz + 4 * cnum.shape[0] + 1


LOCK_EVERY = 8  # routine calls between CTA-wide lockstep points


class Emitter:
    """Straight-line device code for one process."""

    def __init__(self, proc: Process):
        self.p = proc
        self.spec = proc.spec
        self.perms, self.coef = colour_flows(proc)
        ng = len(proc.gluon_legs())
        if ng:
            _, self.cnum, self.cden = chain_matrix(ng)
        else:
            self.cnum, self.cden = np.ones((1, 1), np.int64), 1
        self.mom = []        # momentum table entries: (legs tuple) all-outgoing sums
        self.mom_index = {}
        self.props = []      # (mom index, kind)
        self.prop_index = {}

    def momentum(self, legs):
        """Momentum-table entry of the outgoing sum over `legs`.  A leg set that
        contains the root leg is expressed through its complement, K_S = -K_S',
        so that every momentum and invariant is formed from the same legs as in
        the root-form program (momenta conserve only up to rounding)."""
        root = self.p.spec.root
        if root in legs:
            comp = tuple(sorted(set(range(self.p.n)) - set(legs)))
            key = ("neg", comp)
        else:
            key = tuple(sorted(legs))
        if key not in self.mom_index:
            self.mom_index[key] = len(self.mom)
            self.mom.append(key)
        return self.mom_index[key]

    def prop(self, legs, kind):
        key = (tuple(sorted(legs)), kind)
        if key not in self.prop_index:
            self.prop_index[key] = len(self.props)
            self.props.append((self.momentum(legs), kind))
        return self.prop_index[key]

    def _current_code(self, c, var):
        """One line of device code computing current c (children already emitted)."""
        p, spec = self.p, self.spec
        v = var[c.idx]
        if c.vertex == "ext":
            leg = c.children[0]
            L = spec.legs[leg]
            m = "cp.mt" if L.mass == "mt" else "R(0)"
            pm = "K + %d" % (4 * self.momentum_phys(leg))
            h = "hel[%d]" % leg
            if L.kind == "g":
                return "  const W4<R> %s = vxxxxx<R>(%s, %s, %d);" % (v, pm, h, 1 if L.incoming else -1)
            if _is_col(L.kind):
                return "  const W4<R> %s = ixxxxx<R>(%s, %s, %s, %d);" % (v, pm, m, h, 1 if L.particle else -1)
            return "  const W4<R> %s = oxxxxx<R>(%s, %s, %s, %d);" % (v, pm, m, h, 1 if L.particle else -1)
        ch = [var[i] for i in c.children]
        if c.vertex == "ggg":
            a, b = p.cur[c.children[0]], p.cur[c.children[1]]
            k1, k2 = self.momentum(a.legs), self.momentum(b.legs)
            pr = self.prop(c.legs, "g")
            return ("  const W4<R> %s = VVV1P0_1<R>(%s, %s, K + %d, K + %d, cp.gs, prop[%d]);"
                    % (v, ch[0], ch[1], 4 * k1, 4 * k2, pr))
        if c.vertex.startswith("gggg"):
            fn = ("VVVV1P0_1", "VVVV3P0_1", "VVVV4P0_1")[int(c.vertex[-1])]
            pr = self.prop(c.legs, "g")
            return "  const W4<R> %s = %s<R>(%s, %s, %s, cp.gs2, prop[%d]);" % (v, fn, ch[0], ch[1], ch[2], pr)
        if c.vertex in ("qqg_row", "qqg_col"):
            k = self.momentum(c.legs)
            pr = self.prop(c.legs, "t")
            fn = "FFV1_2" if c.vertex == "qqg_row" else "FFV1_1"
            return ("  const W4<R> %s = %s<R>(%s, %s, cp.gs, K + %d, cp.mt, prop[%d]);"
                    % (v, fn, ch[0], ch[1], 4 * k, pr))
        if c.vertex == "ffa_cur":
            pr = self.prop(c.legs, "A")
            return "  const W4<R> %s = FFV1P0_3<R>(%s, %s, cp.ee, prop[%d]);" % (v, ch[0], ch[1], pr)
        if c.vertex == "ffz_cur":
            pr = self.prop(c.legs, "Z")
            return ("  const W4<R> %s = FFV2_4_3<R>(%s, %s, cp.gz, cp.gzl, cp.gzr, prop[%d]);"
                    % (v, ch[0], ch[1], pr))
        raise ValueError(c.vertex)

    def _deps(self, i, out):
        """All currents (transitively) needed by current i, children first."""
        c = self.p.cur[i]
        if c.vertex != "ext":
            for ch in c.children:
                self._deps(ch, out)
        if i not in out:
            out[i] = None
        return out

    def schedule(self):
        """Order amplitudes so consecutive ones share currents; each current is
        emitted just before its first use, which keeps the live set small."""
        p = self.p
        need = [list(self._deps(a.row, self._deps(a.bos, self._deps(a.col, {})))) for a in p.amps]
        uses = {}
        for d, n in enumerate(need):
            for i in n:
                uses[i] = uses.get(i, 0) + 1
        done = set()
        order = []
        left = set(range(len(p.amps)))
        live = set()
        while left:
            def cost(d):
                new = sum(1 for i in need[d] if i not in done)
                frees = sum(1 for i in need[d] if i in live and uses[i] == 1)
                return (new - frees, d)
            d = min(left, key=cost)
            left.discard(d)
            order.append(d)
            for i in need[d]:
                if i not in done:
                    done.add(i)
                    live.add(i)
                uses[i] -= 1
                if uses[i] == 0:
                    live.discard(i)
        return order, need

    def emit(self) -> str:
        p = self.p
        order, need = self.schedule()
        var = {}
        self.flops = 0
        ncalls = 0
        body = ["  cx<R> amp;"]
        for d in order:
            a = p.amps[d]
            for i in need[d]:
                if i not in var:
                    var[i] = "w%d" % i
                    line = self._current_code(p.cur[i], var)
                    self.flops += FLOPS[line.split("=")[1].split("<")[0].strip()]
                    body.append(line)
                    ncalls += 1
                    if ncalls % LOCK_EVERY == 0:
                        body.append("  Lock::sync();")
            if a.vertex == "ffv_t":
                body.append("  amp = FFV1_0<R>(%s, %s, %s, cp.gs);" % (var[a.row], var[a.col], var[a.bos]))
            elif a.vertex == "ffv_a":
                body.append("  amp = FFV1_0<R>(%s, %s, %s, cp.ee);" % (var[a.row], var[a.col], var[a.bos]))
            else:
                body.append("  amp = FFV2_4_0<R>(%s, %s, %s, cp.gz, cp.gzl, cp.gzr);"
                            % (var[a.row], var[a.col], var[a.bos]))
            self.flops += FLOPS["FFV2_4_0" if a.vertex == "ffz" else "FFV1_0"]
            ncalls += 1
            if ncalls % LOCK_EVERY == 0:
                body.append("  Lock::sync();")
            for s_ in np.nonzero(self.coef[d])[0]:
                body.append("  " + self._accum(s_, self.coef[d, s_]))
                self.flops += FLOPS["jamp"]
        self.ncurrents = len(var)
        self.body = body
        return "\n".join(body)

    def momentum_phys(self, leg):
        key = ("phys", leg)
        if key not in self.mom_index:
            self.mom_index[key] = len(self.mom)
            self.mom.append(key)
        return self.mom_index[key]

    @staticmethod
    def _accum(s, z):
        z = complex(z)
        if z == 1:
            return "J.add(%d, amp);" % s
        if z == -1:
            return "J.sub(%d, amp);" % s
        if z == 1j:
            return "J.addi(%d, amp);" % s
        if z == -1j:
            return "J.subi(%d, amp);" % s
        raise ValueError("colour-flow coefficient %r outside {+-1, +-i}" % z)


GRAD_PROCS = (2, 3)  # processes with a generated adjoint


class GradEmitter:
    """Reverse-mode (adjoint) program for one process: forward diagram program
    for one helicity, colour sum, then the adjoint of every step in reverse
    order.  Momentum-table and propagator adjoints are routed directly to the
    final-state legs' momentum adjoints pb[4 * leg + mu] (beams are constant)."""

    def __init__(self, em: "Emitter"):
        self.em = em
        self.p = em.p

    def _route(self, mom_index, kb, lines, sign=1):
        """pb += d(momentum entry)/d(p_leg) . kb for the final-state legs."""
        key = self.em.mom[mom_index]
        spec = self.p.spec
        if key[0] == "phys":
            legs = [(key[1], 1)]
        elif key[0] == "neg":
            legs = [(l, 1 if spec.legs[l].incoming else -1) for l in key[1]]
        else:
            legs = [(l, -1 if spec.legs[l].incoming else 1) for l in key]
        for leg, sg in legs:
            if leg < 2:
                continue
            sgn = sg * sign
            for mu in range(4):
                lines.append("    pb[%d] %s= %s[%d];" % (4 * leg + mu, "+" if sgn > 0 else "-", kb, mu))

    def emit(self) -> str:
        em, p = self.em, self.p
        order, need = em.schedule()
        var, cur_order = {}, []
        fwd = ["    cx<R> J[NCOLOR];", "    #pragma unroll", "    for (int s = 0; s < NCOLOR; ++s) J[s] = cx<R>(R(0), R(0));",
               "    cx<R> amp;"]
        accum = {1: "J[%d] += amp;", -1: "J[%d] -= amp;", 1j: "J[%d] += mul_i(amp);", -1j: "J[%d] -= mul_i(amp);"}
        for d in order:
            a = p.amps[d]
            for i in need[d]:
                if i not in var:
                    var[i] = "w%d" % i
                    fwd.append("  " + em._current_code(p.cur[i], var))
                    cur_order.append(i)
            fwd.append("    amp = FFV1_0<R>(%s, %s, %s, cp.gs);" % (var[a.row], var[a.col], var[a.bos]))
            for s_ in np.nonzero(em.coef[d])[0]:
                fwd.append("    " + accum[complex(em.coef[d, s_])] % s_)
        nc = em.coef.shape[1]
        body = list(fwd)
        # colour sum and its adjoint Jb = 2 C J / den
        body.append("    R m2 = R(0);")
        body.append("    cx<R> Jb[NCOLOR];")
        for i in range(nc):
            tr = " + ".join("R(%d) * J[%d].re" % (int(em.cnum[i, j]), j) for j in range(nc) if em.cnum[i, j] != 0)
            ti = " + ".join("R(%d) * J[%d].im" % (int(em.cnum[i, j]), j) for j in range(nc) if em.cnum[i, j] != 0)
            body.append("    { const R tr = %s, ti = %s; m2 += J[%d].re * tr + J[%d].im * ti;"
                        " Jb[%d] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }" % (tr, ti, i, i, i))
        body.append("    m2 /= R(CDEN);")
        for i in cur_order:
            body.append("    W4<R> %sb = w4_zero<R>();" % var[i])
        body.append("    cx<R> propb[NPROP];")
        body.append("    #pragma unroll")
        body.append("    for (int j = 0; j < NPROP; ++j) propb[j] = cx<R>(R(0), R(0));")
        conjc = {1: "", -1: "-", 1j: "mul_mi", -1j: "mul_i"}
        for d in reversed(order):
            a = p.amps[d]
            terms = []
            for s_ in np.nonzero(em.coef[d])[0]:
                z = complex(em.coef[d, s_])
                terms.append({1: "Jb[%d]", -1: "-Jb[%d]", 1j: "mul_mi(Jb[%d])", -1j: "mul_i(Jb[%d])"}[z] % s_)
            body.append("    { const cx<R> ab = %s;" % " + ".join(terms))
            body.append("      FFV1_0_adj<R>(%s, %s, %s, cp.gs, ab, %sb, %sb, %sb); }"
                        % (var[a.row], var[a.col], var[a.bos], var[a.row], var[a.col], var[a.bos]))
        for i in reversed(cur_order):
            c = p.cur[i]
            v = var[i]
            if c.vertex == "ext":
                continue
            ch = [var[j] for j in c.children]
            if c.vertex == "ggg":
                A, B = p.cur[c.children[0]], p.cur[c.children[1]]
                k1, k2 = em.momentum(A.legs), em.momentum(B.legs)
                pr = em.prop(c.legs, "g")
                body.append("    { R kb1[4] = {R(0), R(0), R(0), R(0)}, kb2[4] = {R(0), R(0), R(0), R(0)};")
                body.append("      VVV1P0_1_adj<R>(%s, %s, K + %d, K + %d, cp.gs, prop[%d], %sb, %sb, %sb, kb1, kb2, propb[%d]);"
                            % (ch[0], ch[1], 4 * k1, 4 * k2, pr, v, ch[0], ch[1], pr))
                self._route(k1, "kb1", body)
                self._route(k2, "kb2", body)
                body.append("    }")
            elif c.vertex.startswith("gggg"):
                fn = ("VVVV1P0_1_adj", "VVVV3P0_1_adj", "VVVV4P0_1_adj")[int(c.vertex[-1])]
                pr = em.prop(c.legs, "g")
                body.append("    %s<R>(%s, %s, %s, cp.gs2, prop[%d], %sb, %sb, %sb, %sb, propb[%d]);"
                            % (fn, ch[0], ch[1], ch[2], pr, v, ch[0], ch[1], ch[2], pr))
            elif c.vertex == "qqg_row":
                k = em.momentum(c.legs)
                pr = em.prop(c.legs, "t")
                body.append("    { R kb[4] = {R(0), R(0), R(0), R(0)};")
                body.append("      FFV1_2_adj<R>(%s, %s, cp.gs, K + %d, cp.mt, prop[%d], %sb, %sb, %sb, kb, propb[%d]);"
                            % (ch[0], ch[1], 4 * k, pr, v, ch[0], ch[1], pr))
                self._route(k, "kb", body)
                body.append("    }")
            else:
                raise ValueError("no adjoint for %s" % c.vertex)
        # propagators
        kinds = {"g": 0, "t": 1, "A": 2, "Z": 3}
        for j, (mi, kind) in enumerate(em.props):
            body.append("    { R kb[4] = {R(0), R(0), R(0), R(0)};")
            body.append("      prop_adj<R>(prop[%d], %s, K + %d, propb[%d], kb);"
                        % (j, "true" if kind == "t" else "false", 4 * mi, j))
            self._route(mi, "kb", body)
            body.append("    }")
        # external wavefunctions (final-state legs only: beams are constant)
        spec = p.spec
        for i in cur_order:
            c = p.cur[i]
            if c.vertex != "ext":
                continue
            leg = c.children[0]
            if leg < 2:
                continue
            L = spec.legs[leg]
            kind = 2 if L.kind == "g" else (0 if _is_col(L.kind) else 1)
            ns = (1 if L.incoming else -1) if L.kind == "g" else (1 if L.particle else -1)
            m = "cp.mt" if L.mass == "mt" else "R(0)"
            pm = em.momentum_phys(leg)
            body.append("    { R kb[4] = {R(0), R(0), R(0), R(0)};")
            body.append("      external_adj<R>(%d, K + %d, %s, hel[%d], %d, %sb, kb);"
                        % (kind, 4 * pm, m, leg, ns, var[i]))
            self._route(pm, "kb", body)
            body.append("    }")
        body.append("    return m2;")
        return "\n".join(body)


def bf16_colour_image(cnum) -> np.ndarray:
    """B operand of the tensor-core colour sum: B[n][k] = cnum[k][n] in BF16,
    laid out in the canonical K-major no-swizzle layout (8-row x 16-byte core
    matrices; K-adjacent core matrices 128 bytes apart, 8-row groups KP*16
    bytes apart), as little-endian 32-bit words."""
    nc = cnum.shape[0]
    kp = (nc + 15) // 16 * 16
    img = np.zeros(kp * kp, dtype=np.uint16)  # NP = KP rows
    for n in range(kp):
        for k in range(kp):
            v = np.float32(cnum[k, n] if (n < nc and k < nc) else 0)
            bits = int(np.array([v], dtype=np.float32).view(np.uint32)[0])
            if bits & 0xFFFF:
                raise ValueError("colour numerator %r not exact in BF16" % float(v))
            off = (n >> 3) * (kp // 8) * 128 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2
            img[off // 2] = bits >> 16
    return img.view(np.uint32)


def generate(pid: int) -> str:
    proc = Process(PROCS[pid])
    em = Emitter(proc)
    # physical momenta first so that external legs have fixed slots
    for leg in range(proc.n):
        em.momentum_phys(leg)
    body = em.emit()
    spec = proc.spec
    ncol = em.coef.shape[1]
    nflow_used = int(np.count_nonzero(np.any(em.coef != 0, axis=0)))
    assert nflow_used == ncol
    coefs = set(complex(z) for z in em.coef.reshape(-1) if z != 0)
    out = []
    out.append("// GENERATED by paper_2106_12631_gb300/gen/procgen.py -- do not edit.")
    out.append("// Process %d: %s (%s)" % (pid, spec.name, " ".join(L.name for L in spec.legs)))
    out.append("// %d Feynman diagrams (%d amplitude terms), %d colour flows, %d wavefunctions"
               % (proc.ndiagrams, len(proc.amps), ncol, em.ncurrents))
    out.append("// colour-flow coefficients used: %s" % sorted(coefs, key=lambda z: (z.real, z.imag)))
    out.append("#pragma once")
    out.append("namespace mg {")
    sp = SharedProgram(proc, em)
    out.extend(sp.emit_tables(pid))
    img = bf16_colour_image(em.cnum)
    out.append("// colour-matrix numerators as the BF16 B operand of the tensor-core colour sum")
    out.append("static __device__ __align__(16) const uint32_t kColourB%d[%d] = {%s};"
               % (pid, img.size, ", ".join("0x%08x" % int(w) for w in img)))
    out.append("struct Proc%d {" % pid)
    out.append("  static constexpr int NPAR = %d;" % proc.n)
    out.append("  static constexpr int NHEL = %d;" % (1 << proc.n))
    out.append("  static constexpr int NCOLOR = %d;" % ncol)
    out.append("  static constexpr int NDIAGRAMS = %d;" % proc.ndiagrams)
    out.append("  static constexpr int NAMPS = %d;" % len(proc.amps))
    out.extend(sp.struct_lines(pid))
    out.append("  static constexpr int NMOM = %d;" % len(em.mom))
    out.append("  static constexpr int NPROP = %d;" % len(em.props))
    out.append("  static constexpr int NFINAL = %d;" % (proc.n - 2))
    out.append("  // floating-point operations per helicity: diagram program, CUDA-core colour sum")
    out.append("  static constexpr long FLOPS_AMP = %d;" % em.flops)
    out.append("  static constexpr long FLOPS_CSUM = %d;" % colour_sum_flops(em.cnum))
    out.append("  static constexpr double NORM = 1.0 / %d.0;  // 1/(helicity avg x colour avg x symmetry)"
               % (spec.hel_avg * spec.col_avg * spec.sym))
    # momentum table: for each entry, the legs (signs: incoming legs enter as -p)
    mrows = []
    for key in em.mom:
        mask = 0
        sign = 0
        if key[0] == "phys":
            mask = 1 << key[1]
            sgn_mask = 0
            kind = 0
        elif key[0] == "neg":
            # -(sum of outgoing momenta of the complement): incoming legs enter as +p
            for leg in key[1]:
                mask |= 1 << leg
            sgn_mask = sum(1 << leg for leg in key[1] if not spec.legs[leg].incoming)
            kind = 1
        else:
            for leg in key:
                mask |= 1 << leg
            sgn_mask = sum(1 << leg for leg in key if spec.legs[leg].incoming)
            kind = 1
        mrows.append("{%d, %d, %d}" % (kind, mask, sgn_mask))
    out.append("  // momentum table: {0 physical / 1 all-outgoing sum, leg mask, mask of legs entering as -p}")
    out.append("  static __host__ __device__ constexpr int mom(int j, int k) {")
    out.append("    constexpr int t[NMOM][3] = {%s};" % ", ".join(mrows))
    out.append("    return t[j][k];")
    out.append("  }")
    prows = []
    kinds = {"g": 0, "t": 1, "A": 2, "Z": 3}
    for (mi, kind) in em.props:
        prows.append("{%d, %d}" % (mi, kinds[kind]))
    out.append("  // propagators: {momentum entry, 0 gluon / 1 top / 2 photon / 3 Z}")
    out.append("  static __host__ __device__ constexpr int prop(int j, int k) {")
    out.append("    constexpr int t[NPROP][2] = {%s};" % ", ".join(prows))
    out.append("    return t[j][k];")
    out.append("  }")
    pof = [[-1, -1] for _ in em.mom]
    for pi, (mi, _) in enumerate(em.props):
        slot = pof[mi].index(-1)  # at most two lines (photon and Z) share one momentum
        pof[mi][slot] = pi
    out.append("  // propagator entries formed from each momentum entry (-1: none)")
    out.append("  static __host__ __device__ constexpr int mom_prop(int j, int k) {")
    out.append("    constexpr int t[NMOM][2] = {%s};" % ", ".join("{%d, %d}" % tuple(r) for r in pof))
    out.append("    return t[j][k];")
    out.append("  }")
    out.append("  static __device__ __forceinline__ const uint32_t* colour_bf16_image() { return kColourB%d; }" % pid)
    out.append("  // colour matrix = CNUM / CDEN (real symmetric)")
    out.append("  static constexpr int CDEN = %d;" % em.cden)
    out.append("  static __host__ __device__ constexpr int cnum(int i, int j) {")
    out.append("    constexpr int t[NCOLOR][NCOLOR] = {%s};"
               % ", ".join("{" + ", ".join(str(int(x)) for x in row) + "}" for row in em.cnum))
    out.append("    return t[i][j];")
    out.append("  }")
    out.append("  // Dual amplitudes J_s of one helicity combination (hel[k] = +-1), accumulated")
    out.append("  // through J.add/sub/addi/subi(s, amp) (J_s += amp, -amp, i amp, -i amp);")
    out.append("  // Lock::sync() marks points where a CTA may re-align its warps.")
    out.append("  template <class R, class Acc, class Lock>")
    out.append("  static __device__ __forceinline__ void amplitudes(const R* __restrict__ K,"
               " const cx<R>* __restrict__ prop, const int* hel, const Couplings<R>& cp, Acc& J) {")
    out.append("    J.zero();")
    out.append(body)
    out.append("  }")
    out.append("  static constexpr bool HAS_GRAD = %s;" % ("true" if pid in GRAD_PROCS else "false"))
    if pid in GRAD_PROCS:
        out.append("  // |M_h|^2 of one helicity (colour summed) and its gradient with respect to the")
        out.append("  // physical momenta of the final-state legs, accumulated into pb[4 * leg + mu]")
        out.append("  template <class R>")
        out.append("  static __device__ __forceinline__ R amplitudes_grad(const R* __restrict__ K,"
                   " const cx<R>* __restrict__ prop, const int* hel, const Couplings<R>& cp, R* pb) {")
        out.append(GradEmitter(em).emit())
        out.append("  }")
    out.append("};")
    out.append("}  // namespace mg")
    return "\n".join(out) + "\n"


def summary(pid: int) -> dict:
    proc = Process(PROCS[pid])
    em = Emitter(proc)
    for leg in range(proc.n):
        em.momentum_phys(leg)
    em.emit()
    sp = SharedProgram(proc, em)
    sp.emit_tables(pid)
    return dict(flops_amp=em.flops, flops_csum=colour_sum_flops(em.cnum),
                flops_csum_sym=colour_sum_sym_flops(em.cnum), ncurrents=em.ncurrents,
                hs_flops_items=sp.flops_items, hs_flops_amp_hel=sp.flops_amps_hel, hs_ncur=len(sp.order),
                hs_nslots=sp.nslots, hs_nx=len(sp.xoff), hs_xcap=sp.xcap, hs_nxchunk=len(sp.chunks),
                ndiagrams=proc.ndiagrams, namps=len(proc.amps), ncolor=em.coef.shape[1],
                nmom=len(em.mom), nprop=len(em.props), coef=em.coef, cnum=em.cnum, cden=em.cden,
                perms=em.perms, gluon_legs=proc.gluon_legs())


# ---------------------------------------------------------------------------
# Helicity-shared program: every off-shell current is evaluated once per
# helicity combination of ITS OWN legs (2^|S| variants per event instead of
# once per event helicity), and every diagram's amplitude is formed at the
# vertex that needs the cheapest set of such currents.
# ---------------------------------------------------------------------------
# Any vertex of a tree diagram gives the same amplitude (the same product of
# vertex factors and propagators).  Seen from a vertex n of the antitop-rooted
# tree, the branch towards the root is the "complement" current U(n):
#   at a quark-line vertex (row r, gluon g | col U):  U(r) = col current (g, U),
#                                                      U(g) = gluon from the pair (r, U)
#   at a three-gluon vertex (c0, c1 | P):              U(c0) = ggg(c1, P), U(c1) = ggg(P, c0)
#     (cyclic order kept, so f^abc and the Lorentz factor keep their orientation)
#   at a four-gluon term t (c0, c1, c2 | P):           U(ck) = term t with leg k as output
# The colour coefficients stay those of the antitop-rooted form.
#
# The amplitude at a vertex is multilinear in its operands, so with operand k
# left out it is a plain contraction  A = sum_i X_i Y_i  of Y = operand k with
# the AMPUTATED current X of the other operands (the same vertex without its
# propagator; vectors stored with a lower index).  X depends only on the
# helicities of its own legs: it is built once per event and helicity variant,
# like the currents, and each event helicity pays only the contraction
# (30 flops) instead of a full vertex (96 to 168 flops).  The generator picks
# the vertex and the left-out operand of every amplitude together.

SHARED_COST = {"ext": 40, "ggg": FLOPS["VVV1P0_1"], "gggg": FLOPS["VVVV1P0_1"], "qqg_row": FLOPS["FFV1_2"],
               "col": FLOPS["FFV1_1"], "pair": FLOPS["FFV1P0_3"], "ffa_cur": FLOPS["FFV1P0_3"],
               "ffz_cur": FLOPS["FFV2_4_3"],
               "arow": FLOPS["FFV1_2A"], "acol": FLOPS["FFV1_1A"], "apair": FLOPS["FFV1P0_3A"],
               "apair_e": FLOPS["FFV1P0_3A"], "azpair": FLOPS["FFV2_4_3A"], "aggg": FLOPS["VVV1P0_1A"],
               "agggg": FLOPS["VVVV_A"]}

# operands that may be left out of each amplitude form (lepton amplitudes:
# the boson only, so that the couplings stay in one amputated pair current)
EXCLUDE = {"ffv": (0, 1, 2), "ffv_a": (2,), "ffz": (2,), "vvv": (0, 1, 2),
           "vvvv0": (0, 1, 2, 3), "vvvv1": (0, 1, 2, 3), "vvvv2": (0, 1, 2, 3)}

# four-gluon term t: L_t = (A_a.A_b)(A_c.A_d) - (A_e.A_f)(A_g.A_h), legs 0..3
VVVV_PAIRS = {0: (((0, 2), (1, 3)), ((0, 3), (1, 2))),
              1: (((0, 1), (2, 3)), ((0, 3), (1, 2))),
              2: (((0, 1), (2, 3)), ((0, 2), (1, 3)))}


class SharedProgram:
    SLOT_BUDGET = 768  # current + amputated-chunk variant slots per event (FP32: 8 events in 192 KB)
    # amputated-chunk slots per event are rounded up to a multiple of this: a
    # 256-thread CTA of 4 events x 64 helicities then builds a chunk in whole
    # rounds of one item per thread (gg -> t t~ g g: 4 chunks of 192 slots,
    # 12 rounds, instead of 176 x 4 + 64 in 13)
    CHUNK_QUANTUM = 64
    CUR_CAP = 416      # current variant slots per event

    def __init__(self, proc: Process, emitter: "Emitter"):
        self.p = proc
        self.em = emitter
        self.n = proc.n
        self._legs = {}
        self._closure = {}
        self._cands()
        self._choose()
        self._layout()

    # ---- descriptors -------------------------------------------------------
    def legs(self, d):
        s = self._legs.get(d)
        if s is not None:
            return s
        if d[0] == "N":
            s = frozenset(self.p.cur[d[1]].legs)
        else:
            s = frozenset()
            for x in d[2:]:
                if isinstance(x, tuple):
                    s |= self.legs(x)
        self._legs[d] = s
        return s

    def kind(self, d):
        if d[0] == "N":
            v = self.p.cur[d[1]].vertex
            return "gggg" if v.startswith("gggg") else v
        return d[1]

    def inputs(self, d):
        if d[0] == "N":
            c = self.p.cur[d[1]]
            return [] if c.vertex == "ext" else [("N", ch) for ch in c.children]
        return [x for x in d[2:] if isinstance(x, tuple)]

    def closure(self, d):
        """d and every current it is built from."""
        c = self._closure.get(d)
        if c is None:
            c = frozenset([d]).union(*[self.closure(x) for x in self.inputs(d)])
            self._closure[d] = c
        return c

    def nvar(self, d):
        return 1 << len(self.legs(d))

    @staticmethod
    def xdesc(kind, args, k):
        """Amputated current of the operands of amplitude (kind, args) other than k."""
        if kind == "ffv":
            r, c, b = args
            return {0: ("X", "acol", b, c), 1: ("X", "arow", r, b), 2: ("X", "apair", r, c)}[k]
        if kind == "ffv_a":
            return ("X", "apair_e", args[0], args[1])
        if kind == "ffz":
            return ("X", "azpair", args[0], args[1])
        if kind == "vvv":
            c0, c1, u = args
            return {2: ("X", "aggg", c0, c1), 0: ("X", "aggg", c1, u), 1: ("X", "aggg", u, c0)}[k]
        t = int(kind[-1])
        return ("X", "agggg", t, k) + tuple(None if i == k else a for i, a in enumerate(args))

    # ---- candidate evaluation points -------------------------------------------
    def _cands(self):
        p = self.p
        top = ("N", p.root_cur)
        self.cands = []
        for a in p.amps:
            A, B = ("N", a.row), ("N", a.bos)
            if a.vertex != "ffv_t":  # leptons: the root-form amplitude only
                opts = [(a.vertex, (("N", a.row), ("N", a.col), ("N", a.bos)))]
            else:
                opts = [("ffv", (A, top, B))]
                stack = [(a.row, ("U", "col", B, top)), (a.bos, ("U", "pair", A, top))]
                while stack:
                    n, U = stack.pop()
                    c = p.cur[n]
                    if c.vertex == "ext":
                        continue
                    ch = [("N", x) for x in c.children]
                    if c.vertex == "qqg_row":
                        r, g = ch
                        opts.append(("ffv", (r, U, g)))
                        stack.append((c.children[0], ("U", "col", g, U)))
                        stack.append((c.children[1], ("U", "pair", r, U)))
                    elif c.vertex == "ggg":
                        c0, c1 = ch
                        opts.append(("vvv", (c0, c1, U)))
                        stack.append((c.children[0], ("U", "ggg", c1, U)))
                        stack.append((c.children[1], ("U", "ggg", U, c0)))
                    elif c.vertex.startswith("gggg"):
                        t = int(c.vertex[-1])
                        opts.append(("vvvv%d" % t, (ch[0], ch[1], ch[2], U)))
                        for k in range(3):
                            others = tuple(x for j, x in enumerate(ch) if j != k)
                            stack.append((c.children[k], ("U", "gggg", t, k) + others + (U,)))
            # every vertex form with every operand that may be left out
            full = []
            for kind, args in opts:
                for k in EXCLUDE[kind]:
                    X = self.xdesc(kind, args, k)
                    cl = frozenset().union(*[self.closure(x) for x in self.inputs(X)], self.closure(args[k]))
                    full.append((kind, args, k, X, cl))
            self.cands.append(full)

    def _choose(self):
        """Greedy choice of (vertex, left-out operand) per amplitude minimising the
        per-event cost: the shared currents and amputated currents once per event,
        plus, per event helicity, the contractions — an amplitude whose amputated
        current and colour flows (up to a phase) match another's joins its
        contraction (8 flops instead of 30 + 2 per flow) — with current slots capped."""
        refc, xref, kref = {}, {}, {}
        state = {"cost": 0, "slots": 0}
        nhel = 1 << self.n
        pats, nflows = [], []
        for di in range(len(self.cands)):
            flows = []
            for s_ in np.nonzero(self.em.coef[di])[0]:
                z = complex(self.em.coef[di, s_])
                flows.append(int(s_) | ({1: 0, -1: 1, 1j: 2, -1j: 3}[z] << 6))
            pats.append(min(self._rotate(flows, r) for r in range(4)))
            nflows.append(len(flows))
        di_of = {}
        for di, opts in enumerate(self.cands):
            for o in opts:
                di_of[id(o)] = di

        def hel_cost(di, first):
            return FLOPS["W4ADD"] + (FLOPS["DOT4"] - FLOPS["W4ADD"] + FLOPS["jamp"] * nflows[di] if first else 0)

        def cost_cur(d):
            return SHARED_COST[self.kind(d)] * self.nvar(d)

        def apply(opt, s):
            _, _, _, X, cl = opt
            for d in cl:
                r = refc.get(d, 0)
                if (r == 0 and s > 0) or (r == 1 and s < 0):
                    state["cost"] += s * cost_cur(d)
                    state["slots"] += s * self.nvar(d)
                refc[d] = r + s
            r = xref.get(X, 0)
            if (r == 0 and s > 0) or (r == 1 and s < 0):
                state["cost"] += s * SHARED_COST[X[1]] * self.nvar(X)
            xref[X] = r + s
            di = di_of[id(opt)]
            key = (X, pats[di])
            r = kref.get(key, 0)
            state["cost"] += s * nhel * hel_cost(di, (r == 0 and s > 0) or (r == 1 and s < 0))
            kref[key] = r + s

        def added(opt):
            _, _, _, X, cl = opt
            c = sl = 0
            for d in cl:
                if refc.get(d, 0) == 0:
                    c += cost_cur(d)
                    sl += self.nvar(d)
            if xref.get(X, 0) == 0:
                c += SHARED_COST[X[1]] * self.nvar(X)
            di = di_of[id(opt)]
            c += nhel * hel_cost(di, kref.get((X, pats[di]), 0) == 0)
            over = max(0, state["slots"] + sl - self.CUR_CAP)
            return c + over * 10 ** 7

        def run(start):
            for k in list(refc):
                refc[k] = 0
            for k in list(xref):
                xref[k] = 0
            for k in list(kref):
                kref[k] = 0
            state["cost"] = state["slots"] = 0
            choice = list(start)
            for di, opts in enumerate(self.cands):
                apply(opts[choice[di]], +1)
            for _ in range(8):
                changed = False
                for di, opts in enumerate(self.cands):
                    apply(opts[choice[di]], -1)
                    best = min(range(len(opts)), key=lambda i: (added(opts[i]), i))
                    if best != choice[di]:
                        changed = True
                    choice[di] = best
                    apply(opts[best], +1)
                if not changed:
                    break
            return state["cost"], choice

        # start: root form, the largest operand left out (a start from a greedy
        # cover of the amplitudes by (amputated current, flow pattern) keys, i.e.
        # the most merged contractions, converges to the same choice)
        start = []
        for opts in self.cands:
            start.append(max(range(len(opts)), key=lambda i: (opts[i][0] == opts[0][0] and opts[i][1] == opts[0][1],
                                                             len(self.legs(opts[i][1][opts[i][2]])))))
        choice = run(start)[1]
        self.choice = choice
        self.flops_event = state["cost"]

    # ---- currents, amputated currents, chunks --------------------------------------
    def _layout(self):
        need = set()
        xs = []
        for opts, ci in zip(self.cands, self.choice):
            need |= opts[ci][4]
            if opts[ci][3] not in xs:
                xs.append(opts[ci][3])
        self.level = {}
        for d in sorted(need, key=lambda d: len(self.closure(d))):
            ins = self.inputs(d)
            self.level[d] = 0 if not ins else 1 + max(self.level[x] for x in ins)
        self.order = sorted(need, key=lambda d: (self.level[d], self.kind(d), sorted(self.legs(d)), repr(d)))
        self.cid = {d: i for i, d in enumerate(self.order)}
        self.offset = {}
        off = 0
        for d in self.order:
            self.offset[d] = off
            off += self.nvar(d)
        self.nslots = off
        # amputated currents, packed into chunks that share one buffer
        xs.sort(key=lambda X: (X[1], sorted(self.legs(X)), repr(X)))
        total = sum(self.nvar(X) for X in xs)
        # two chunk buffers when it takes more than one chunk (the kernel builds
        # chunk c + 1 while it contracts chunk c)
        cap = (self.SLOT_BUDGET - self.nslots) // 2
        cap = -(-cap // self.CHUNK_QUANTUM) * self.CHUNK_QUANTUM
        self.xcap = total if total <= self.SLOT_BUDGET - self.nslots else cap
        assert self.xcap >= max(self.nvar(X) for X in xs), "no room for an amputated current"
        self.xchunk, self.xoff, self.chunks = {}, {}, [[]]
        used = 0
        for X in xs:
            if used + self.nvar(X) > self.xcap:
                self.chunks.append([])
                used = 0
            self.xchunk[X] = len(self.chunks) - 1
            self.xoff[X] = used
            self.chunks[-1].append(X)
            used += self.nvar(X)

    def variant(self, d, hel_bits):
        """Variant index of current d for an event helicity (bit l of hel_bits = leg l is +1)."""
        v = 0
        for k, l in enumerate(sorted(self.legs(d))):
            v |= ((hel_bits >> l) & 1) << k
        return v

    def sub_variant(self, child, parent, v):
        """Variant of `child` inside variant v of `parent` (child legs subset of parent legs)."""
        pl = sorted(self.legs(parent))
        bits = 0
        for k, l in enumerate(pl):
            bits |= ((v >> k) & 1) << l
        return self.variant(child, bits)

    # ---- device tables ------------------------------------------------------------
    HS_TYPES = {"ixxxxx": 0, "oxxxxx": 1, "vxxxxx": 2, "row": 3, "col": 4, "pair": 5, "zcur": 6,
                "ggg": 7, "gggg": 8, "arow": 9, "acol": 10, "apair": 11, "azpair": 12, "aggg": 13, "agggg": 14}

    def _canon_prop_legs(self, legs):
        """The invariant of an internal line, formed from the side without the
        root leg (as in the root-form program)."""
        root = self.p.spec.root
        return frozenset(range(self.n)) - legs if root in legs else legs

    def _gggg_positions(self, d):
        """(term, output position, {position: operand}) of a four-gluon current."""
        xs = self.inputs(d)
        if d[0] == "N":
            return int(self.p.cur[d[1]].vertex[-1]), 3, {0: xs[0], 1: xs[1], 2: xs[2]}
        if d[0] == "U":
            term, outpos = d[2], d[3]
            o1, o2, U = d[4], d[5], d[6]
            rest = [q for q in range(3) if q != outpos]
            return term, outpos, {rest[0]: o1, rest[1]: o2, 3: U}
        term, outpos = d[2], d[3]
        return term, outpos, {q: d[4 + q] for q in range(4) if q != outpos}

    def _item(self, d, v):
        """One variant of a current or amputated current:
        (type, a, b, c, flag, out, in[3], k0, k1, prop)."""
        em, spec = self.em, self.p.spec
        out = (self.xoff[d] if d[0] == "X" else self.offset[d]) + v
        ins = [0] * 3
        a = b = c = flag = 0
        k0 = k1 = prop = 0
        kind = self.kind(d)
        xs = self.inputs(d)
        slot = lambda x: self.offset[x] + self.sub_variant(x, d, v)
        legs = self.legs(d)
        if kind == "ext":
            leg = self.p.cur[d[1]].children[0]
            L = spec.legs[leg]
            hel = 1 if v else -1
            k0 = em.momentum_phys(leg)
            flag = 1 if L.mass == "mt" else 0
            if L.kind == "g":
                t, c = self.HS_TYPES["vxxxxx"], (1 if L.incoming else -1)
            elif _is_col(L.kind):
                t, c = self.HS_TYPES["ixxxxx"], (1 if L.particle else -1)
            else:
                t, c = self.HS_TYPES["oxxxxx"], (1 if L.particle else -1)
            a, b = leg, hel
        elif kind in ("qqg_row", "arow"):
            t = self.HS_TYPES["row" if kind == "qqg_row" else "arow"]
            ins[0], ins[1] = slot(xs[0]), slot(xs[1])   # (row, gluon)
            if kind == "qqg_row":
                k0 = em.momentum(legs)
                prop = em.prop(self._canon_prop_legs(legs), "t")
        elif kind in ("col", "acol"):
            t = self.HS_TYPES[kind]
            g, U = xs
            ins[0], ins[1] = slot(U), slot(g)   # FFV1_1(fi = U, v = g)
            if kind == "col":
                k0 = em.momentum(legs)
                prop = em.prop(self._canon_prop_legs(legs), "t")
        elif kind in ("pair", "apair", "apair_e"):
            t = self.HS_TYPES["pair" if kind == "pair" else "apair"]
            r, U = xs
            ins[0], ins[1] = slot(r), slot(U)   # FFV1P0_3(fo = r, fi = U)
            a = 1 if kind == "apair_e" else 0
            if kind == "pair":
                prop = em.prop(self._canon_prop_legs(legs), "g")
        elif kind == "azpair":
            t = self.HS_TYPES["azpair"]
            ins[0], ins[1] = slot(xs[0]), slot(xs[1])
        elif kind in ("ffa_cur", "ffz_cur"):
            t = self.HS_TYPES["pair" if kind == "ffa_cur" else "zcur"]
            ins[0], ins[1] = slot(xs[0]), slot(xs[1])
            a = 1  # coupling: e
            prop = em.prop(self._canon_prop_legs(legs), "A" if kind == "ffa_cur" else "Z")
        elif kind in ("ggg", "aggg"):
            t = self.HS_TYPES[kind]
            ins[0], ins[1] = slot(xs[0]), slot(xs[1])
            k0, k1 = em.momentum(self.legs(xs[0])), em.momentum(self.legs(xs[1]))
            if kind == "ggg":
                prop = em.prop(self._canon_prop_legs(legs), "g")
        elif kind in ("gggg", "agggg"):
            t = self.HS_TYPES[kind]
            # each of the term's two products pairs the output position with an
            # operand X_j and dots the other two: o = X_0 (X_1 . W) - X_1 (X_0 . W),
            # W the third operand; in = {X_0, X_1, W}
            term, outpos, pos = self._gggg_positions(d)
            xs_ = []
            for pair in VVVV_PAIRS[term]:
                (p0, p1), (p2, p3) = pair
                if outpos in (p0, p1):
                    xs_.append(p1 if outpos == p0 else p0)
                else:
                    xs_.append(p3 if outpos == p2 else p2)
            assert len(xs_) == 2 and xs_[0] != xs_[1]
            (w_,) = [q for q in pos if q not in xs_]
            ins[0], ins[1], ins[2] = slot(pos[xs_[0]]), slot(pos[xs_[1]]), slot(pos[w_])
            if kind == "gggg":
                prop = em.prop(self._canon_prop_legs(legs), "g")
        else:
            raise ValueError(kind)
        return (t, a, b, c, flag, out, ins, k0, k1, prop)

    def emit_tables(self, pid: int) -> list:
        nh = 1 << self.n
        items, level_start = [], []
        cur_level = -1
        for d in self.order:
            if self.level[d] != cur_level:
                cur_level = self.level[d]
                level_start.append(len(items))
            for v in range(self.nvar(d)):
                items.append(self._item(d, v))
        level_start.append(len(items))
        xitem_start = []
        for chunk in self.chunks:
            xitem_start.append(len(items))
            for X in chunk:
                for v in range(self.nvar(X)):
                    items.append(self._item(X, v))
        xitem_start.append(len(items))
        # amplitudes by chunk, then by amputated current (loaded once per run) and operand
        patterns = {}
        amps = []
        for di, (opts, ci) in enumerate(zip(self.cands, self.choice)):
            kind, args, k, X, _ = opts[ci]
            Y = args[k]
            assert self.legs(X) | self.legs(Y) == frozenset(range(self.n)) and not self.legs(X) & self.legs(Y)
            flows = []
            for s_ in np.nonzero(self.em.coef[di])[0]:
                z = complex(self.em.coef[di, s_])
                code = {1: 0, -1: 1, 1j: 2, -1j: 3}[z]
                flows.append(int(s_) | (code << 6))
            key = tuple(flows)
            if key not in patterns:
                patterns[key] = len(patterns)
            xset = sum(1 << l for l in self.legs(X))
            amps.append((self.xchunk[X], self.xoff[X], self.offset[Y], patterns[key], xset, flows))
        amps.sort()
        assert len(patterns) < 256 and self.nslots < 65536 and self.xcap < 65536
        self.patterns = patterns
        self.amp_list = amps
        self.groups = self._merge_groups(amps)
        xamp_start = [0] * (len(self.chunks) + 1)
        for c in range(len(self.chunks)):
            xamp_start[c + 1] = xamp_start[c] + sum(1 for a in amps if a[0] == c)
        out = []
        self._exact_flops(items, amps)
        self.tables = dict(nitems=len(items), level_start=level_start, xitem_start=xitem_start,
                           xamp_start=xamp_start, namps=len(amps), ncur=len(self.order), nx=len(self.xoff))
        out.append("// helicity-shared program: %d currents in %d levels (%d variant slots), %d amputated"
                   " currents in %d chunk(s) of <= %d slots, %d amplitudes; %d flops per event (all helicities)"
                   % (len(self.order), len(level_start) - 1, self.nslots, len(self.xoff), len(self.chunks),
                      self.xcap, len(amps), self.flops_items + nh * self.flops_amps_hel))
        out.append("static __device__ const HsItem kHsItems%d[%d] = {%s};" % (
            pid, len(items), ", ".join("{%d, {%s}, %d, %d, %d, %d, %d, %d, %d, %d}" % (
                o, ", ".join(map(str, ins)), t, a, b, c, flag, k0, k1, pr)
                for (t, a, b, c, flag, o, ins, k0, k1, pr) in items)))
        out.append("static __constant__ int kHsXItem%d[%d] = {%s};  // item ranges of the amputated chunks"
                   % (pid, len(xitem_start), ", ".join(map(str, xitem_start))))
        # variant of every leg set S for every event helicity h: the bits of the
        # legs of S in ascending order, leg l being +1 when bit n-1-l of h is set
        var = []
        for S in range(1 << self.n):
            for ih in range(nh):
                v = k = 0
                for l in range(self.n):
                    if S >> l & 1:
                        v |= ((ih >> (self.n - 1 - l)) & 1) << k
                        k += 1
                var.append(v)
        out.append("static __device__ __align__(16) const uint8_t kHsVar%d[%d] = {%s};  // [leg set][helicity]"
                   % (pid, len(var), ", ".join(map(str, var))))
        return out

    def _exact_flops(self, items, amps):
        """Operation count: current and amputated-current variants per event,
        contractions + flow sums per helicity."""
        item_flops = {0: FLOPS["ixxxxx"], 1: FLOPS["oxxxxx"], 2: FLOPS["vxxxxx"], 3: FLOPS["FFV1_2"],
                      4: FLOPS["FFV1_1"], 5: FLOPS["FFV1P0_3"], 6: FLOPS["FFV2_4_3"], 7: FLOPS["VVV1P0_1"],
                      8: FLOPS["VVVV1P0_1"], 9: FLOPS["FFV1_2A"], 10: FLOPS["FFV1_1A"], 11: FLOPS["FFV1P0_3A"],
                      12: FLOPS["FFV2_4_3A"], 13: FLOPS["VVV1P0_1A"], 14: FLOPS["VVVV_A"]}
        self.flops_items = sum(item_flops[it[0]] for it in items)
        groups = self._merge_groups(amps)
        self.flops_amps_hel = sum(FLOPS["DOT4"] + FLOPS["jamp"] * len(g["flows"]) + FLOPS["W4ADD"] * (len(g["ys"]) - 1)
                                  for g in groups)

    def struct_lines(self, pid: int) -> list:
        t = self.tables

        def table_fn(name, vals):
            return ["  static __host__ __device__ constexpr int %s(int i) {" % name,
                    "    constexpr int t[%d] = {%s};" % (len(vals), ", ".join(map(str, vals))),
                    "    return t[i];",
                    "  }"]
        return [
            "  // helicity-shared program (tables above)",
            "  static constexpr int HS_NSLOT = %d;   // current variant slots per event" % self.nslots,
            "  static constexpr int HS_XCAP = %d;    // amputated-current slots per event and chunk" % self.xcap,
            "  static constexpr int HS_NXCHUNK = %d;" % len(self.chunks),
            "  static constexpr int HS_XBUFS = %d;   // chunk buffers" % (1 if len(self.chunks) == 1 else 2),
            "  static constexpr int HS_NITEM = %d;" % t["nitems"],
            "  static constexpr int HS_NLEVEL = %d;" % (len(t["level_start"]) - 1),
            "  static constexpr int HS_NAMP = %d;" % t["namps"],
            "  static constexpr int HS_NCUR = %d;" % t["ncur"],
            "  static constexpr int HS_NX = %d;" % t["nx"],
            "  // operations: current variants per event, contractions + flow sums per helicity",
            "  static constexpr long HS_FLOPS_ITEMS = %d;" % self.flops_items,
            "  static constexpr long HS_FLOPS_AMP_HEL = %d;" % self.flops_amps_hel,
            "  // item ranges of the current levels and of the amputated chunks; amplitude ranges of the chunks",
        ] + table_fn("hs_level", t["level_start"]) + [
            "  static __device__ __forceinline__ int hs_xitem(int c) { return kHsXItem%d[c]; }" % pid,
            "  static __device__ __forceinline__ const uint8_t* hs_variants() { return kHsVar%d; }" % pid,
            "  static __device__ __forceinline__ const HsItem* hs_items() { return kHsItems%d; }" % pid,
        ] + self._contract_code() + self._contract_adj_code()

    @staticmethod
    def _rotate(flows, r):
        """Colour-flow coefficients times i^r (codes: 0 +1, 1 -1, 2 +i, 3 -i)."""
        times_i = {0: 2, 2: 1, 1: 3, 3: 0}
        out = []
        for f in flows:
            c = f >> 6
            for _ in range(r):
                c = times_i[c]
            out.append((f & 63) | (c << 6))
        return tuple(sorted(out))

    def _merge_groups(self, amps):
        """Amplitudes of one chunk with the same amputated current X whose colour
        flows agree up to a phase i^r contract once:
            sum_k (X . Y_k) i^{r_k} P = X . (sum_k i^{r_k} Y_k) P."""
        groups = []
        index = {}
        for (ch, xo, yo, pat, xset, flows) in amps:
            base = None
            for r in range(4):
                key = (ch, xo, self._rotate(flows, r))
                if key in index:
                    base = index[key], (4 - r) % 4  # flows = i^{-r} P
                    break
            if base is None:
                index[(ch, xo, tuple(sorted(flows)))] = len(groups)
                groups.append(dict(ch=ch, xo=xo, xset=xset, flows=list(flows), ys=[(yo, 0)]))
            else:
                groups[base[0]]["ys"].append((yo, base[1]))
        return groups

    def _contract_adj_code(self) -> list:
        """Adjoint of hs_contract for one (event, helicity): from Jb_s = dL/dJ_s
        (Wirtinger: dL/dRe + i dL/dIm) each group's Ab = sum_s conj(c_s) Jb_s;
        Xb += conj(Y) Ab (registers, one atomic add per amputated current) and
        Yb_k = conj(phase_k) conj(X) Ab added atomically into the operands' slots."""
        nh = 1 << self.n
        ALL = (1 << self.n) - 1
        cj = {0: "Jb[%d]", 1: "-Jb[%d]", 2: "mul_mi(Jb[%d])", 3: "mul_i(Jb[%d])"}  # conj(c) Jb
        ph = {0: "Yb", 1: "w4_mul_mi(Yb)", 2: "w4_neg(Yb)", 3: "w4_mul_i(Yb)"}      # conj(i^r) Yb
        def lane_mask(legs):
            """lane bits of a warp whose helicity bits are those of `legs` (lane
            bit b = helicity bit b = leg n-1-b; a warp spans helicity bits 0..4)"""
            m = 0
            for b in range(min(5, self.n)):
                if (self.n - 1 - b) in legs:
                    m |= 1 << b
            return m

        # with at most 32 helicities an event's helicities are all in one warp, so
        # after the warp sum the first lane of the slot's group is its only writer
        one_warp = self.n <= 5

        def add(target, slot, value, mask):
            # full: lanes = consecutive helicities of one event, all good: sum the
            # lanes sharing the slot first (reduce-scatter), each component added
            # once per warp (a plain add when the warp holds every helicity of
            # the event, else atomic)
            return ["          if (full) {",
                    "            w4_warp_reduce_add<%du, %s>(%s, %s, %s, lane, act);"
                    % (mask, "false" if one_warp else "true", value, target, slot),
                    "          } else {",
                    "            %s.atomic_add(%s, %s);" % (target, slot, value),
                    "          }"]

        def xb_add(xo, mask):
            return (["          if constexpr ((PASS & 2) != 0) {"]
                    + ["  " + ln for ln in add("xbb", "%d + vx" % xo, "Xb", mask)] + ["          }"])

        lines = ["  // adjoint of hs_contract: Jb -> atomic adds into curb (operands) and xbb (amputated);",
                 "  // full = the warp's lanes are consecutive helicities of its event(s), all good;",
                 "  // act = this lane has an (event, helicity) (lanes without one add zeros)",
                 "  // PASS bit 0: the operand adjoints Yb (read X); bit 1: the amputated-current",
                 "  // adjoints Xb (read Y), so that Xb can overwrite X in a second pass",
                 "  template <int PASS, class R, class CUR, class XB>",
                 "  static __device__ __forceinline__ void hs_contract_adj(int c, const CUR& cur, const XB& xb,"
                 " const uint8_t* __restrict__ vt, const cx<R>* Jb, const CUR& curb, const XB& xbb, bool full,"
                 " int lane, bool act) {",
                 "    switch (c) {"]
        for c in range(len(self.chunks)):
            lines.append("      case %d: {" % c)
            last_x = None
            last_mask = 0
            for g in self.groups:
                if g["ch"] != c:
                    continue
                xlegs = set(l for l in range(self.n) if g["xset"] >> l & 1)
                if g["xo"] != last_x:
                    if last_x is not None:
                        lines += xb_add(last_x, last_mask)
                        lines.append("        }")
                    lines.append("        {")
                    lines.append("          const int vx = vt[%d];" % (g["xset"] * nh))
                    lines.append("          const W4<R> X = xb[%d + vx];" % g["xo"])
                    lines.append("          W4<R> Xb = w4_zero<R>();")
                    last_x = g["xo"]
                    last_mask = lane_mask(set(range(self.n)) - xlegs)
                yv = (ALL ^ g["xset"]) * nh
                ab = " + ".join(cj[f >> 6] % (f & 63) for f in g["flows"])
                lines.append("          {")
                lines.append("            const int vy = vt[%d];" % yv)
                lines.append("            W4<R> Y = cur[%d + vy];" % g["ys"][0][0])
                acc = {0: "w4_add", 1: "w4_addi", 2: "w4_sub", 3: "w4_subi"}
                for (yo, r) in g["ys"][1:]:
                    lines.append("            Y = %s(Y, cur[%d + vy]);" % (acc[r], yo))
                lines.append("            const cx<R> ab = %s;" % ab)
                lines.append("            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);")
                lines.append("            if constexpr ((PASS & 1) != 0) {")
                lines.append("              const W4<R> Yb = w4_conj_scale(X, ab);")
                for (yo, r) in g["ys"]:
                    lines += ["    " + ln for ln in add("curb", "%d + vy" % yo, ph[r], lane_mask(xlegs))]
                lines.append("            }")
                lines.append("          }")
            if last_x is not None:
                lines += xb_add(last_x, last_mask)
                lines.append("        }")
            lines.append("      } break;")
        lines += ["      default: break;", "    }", "  }"]
        return lines

    def _contract_code(self) -> list:
        """Contractions of one chunk for one (event, helicity), straight-line: every
        operand offset and variant-table entry is a constant, so the loads of
        successive amplitudes are independent; each (merged) amplitude goes
        straight into its colour flows J_s (+amp, -amp, +i amp, -i amp); the
        contraction of an amplitude with a single flow accumulates into it."""
        nh = 1 << self.n
        ALL = (1 << self.n) - 1
        ops = {r: "flow_add<%d>(J[%%d], a);" % r for r in range(4)}
        acc = {0: "w4_add", 1: "w4_addi", 2: "w4_sub", 3: "w4_subi"}  # Y_sum += i^r Y
        lines = ["  // A = sum_i X_i Y_i for the amplitudes of chunk c: X = xb[X slot + variant],",
                 "  // Y = cur[Y slot + variant], variant of a leg set S for this helicity = vt[S * NHEL];",
                 "  // amplitudes with the same X and colour flows equal up to a phase share one",
                 "  // contraction with the phase-weighted sum of their Y;",
                 "  // HS_LOCKSTEP(m, n) between amputated currents (amplitudes m and n of the chunk",
                 "  // start the previous and the next one)",
                 "  template <class R, class CUR, class XB>",
                 "  static __device__ __forceinline__ void hs_contract(int c, const CUR& cur, const XB& xb,"
                 " const uint8_t* __restrict__ vt, cx<R>* J) {",
                 "    switch (c) {"]
        for c in range(len(self.chunks)):
            lines.append("      case %d: {" % c)
            last_x = None
            n = prev = 0
            for g in self.groups:
                if g["ch"] != c:
                    continue
                if g["xo"] != last_x and n > 0:
                    lines.append("        }")
                    lines.append("        HS_LOCKSTEP(%d, %d);" % (prev, n))
                    prev = n
                    last_x = None
                n += len(g["ys"])
                if g["xo"] != last_x:
                    lines.append("        {")
                    lines.append("          const W4<R> X = xb[%d + vt[%d]];" % (g["xo"], g["xset"] * nh))
                    last_x = g["xo"]
                yv = (ALL ^ g["xset"]) * nh
                flows = " ".join(ops[f >> 6] % (f & 63) for f in g["flows"])
                one = len(g["flows"]) == 1  # a single flow: the contraction accumulates into it
                if one:
                    f = g["flows"][0]
                    into = "dot4_acc<%d>(J[%d], X, %%s);" % (f >> 6, f & 63)
                if len(g["ys"]) == 1:
                    y = "cur[%d + vt[%d]]" % (g["ys"][0][0], yv)
                    if one:
                        lines.append("          " + into % y)
                    else:
                        lines.append("          { const cx<R> a = dot4(X, %s); %s }" % (y, flows))
                else:
                    y0 = g["ys"][0][0]
                    lines.append("          {")
                    lines.append("            W4<R> Y = cur[%d + vt[%d]];" % (y0, yv))
                    for (yo, r) in g["ys"][1:]:
                        lines.append("            Y = %s(Y, cur[%d + vt[%d]]);" % (acc[r], yo, yv))
                    if one:
                        lines.append("            " + into % "Y")
                    else:
                        lines.append("            const cx<R> a = dot4(X, Y); %s" % flows)
                    lines.append("          }")
            if last_x is not None:
                lines.append("        }")
            lines.append("      } break;")
        lines += ["      default: break;", "    }", "  }"]
        return lines
