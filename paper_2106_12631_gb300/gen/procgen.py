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
    "jamp": 2,
}


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
    return dict(flops_amp=em.flops, flops_csum=colour_sum_flops(em.cnum), ncurrents=em.ncurrents,
                hs_flops_items=sp.flops_items, hs_flops_amp_hel=sp.flops_amps_hel, hs_ncur=len(sp.order),
                hs_nslots=sp.nslots,
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

SHARED_COST = {"ext": 40, "ggg": FLOPS["VVV1P0_1"], "gggg": FLOPS["VVVV1P0_1"], "qqg_row": FLOPS["FFV1_2"],
               "col": FLOPS["FFV1_1"], "pair": FLOPS["FFV1P0_3"], "ffa_cur": FLOPS["FFV1P0_3"],
               "ffz_cur": FLOPS["FFV2_4_3"]}
SHARED_AMP = {"ffv": FLOPS["FFV1_0"], "vvv": FLOPS["VVV1_0"], "vvvv": FLOPS["VVVV_0"], "ffv_a": FLOPS["FFV1_0"],
              "ffz": FLOPS["FFV2_4_0"]}

# four-gluon term t: L_t = (A_a.A_b)(A_c.A_d) - (A_e.A_f)(A_g.A_h), legs 0..3
VVVV_PAIRS = {0: (((0, 2), (1, 3)), ((0, 3), (1, 2))),
              1: (((0, 1), (2, 3)), ((0, 3), (1, 2))),
              2: (((0, 1), (2, 3)), ((0, 2), (1, 3)))}


class SharedProgram:
    def __init__(self, proc: Process, emitter: "Emitter"):
        self.p = proc
        self.em = emitter
        self.n = proc.n
        self._cands()
        self._choose()
        self._currents()

    # ---- descriptors -------------------------------------------------------
    def legs(self, d):
        if d[0] == "N":
            return frozenset(self.p.cur[d[1]].legs)
        s = frozenset()
        for x in d[2:]:
            if isinstance(x, tuple):
                s |= self.legs(x)
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

    def deps(self, d, out):
        if d in out:
            return
        for x in self.inputs(d):
            self.deps(x, out)
        out[d] = None

    # ---- candidate evaluation points -------------------------------------------
    def _cands(self):
        p = self.p
        top = ("N", p.root_cur)
        self.cands = []
        for a in p.amps:
            A, B = ("N", a.row), ("N", a.bos)
            if a.vertex != "ffv_t":  # leptons: the root-form amplitude only
                self.cands.append([(a.vertex, (("N", a.row), ("N", a.col), ("N", a.bos)))])
                continue
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
            self.cands.append(opts)

    SLOT_CAP = 384  # variant slots per event (shared memory: 12 KB in FP32, 24 KB in FP64)

    def _cost(self, choice):
        need = {}
        amp = 0
        for opts, ci in zip(self.cands, choice):
            kind, args = opts[ci]
            amp += SHARED_AMP["vvvv" if kind.startswith("vvvv") else kind] * (1 << self.n)
            for x in args:
                self.deps(x, need)
        cur = sum(SHARED_COST[self.kind(d)] * (1 << len(self.legs(d))) for d in need)
        slots = sum(1 << len(self.legs(d)) for d in need)
        over = max(0, slots - self.SLOT_CAP)
        return cur + amp + over * 10 ** 7

    def _choose(self):
        choice = [0] * len(self.cands)
        for _ in range(4):
            changed = False
            for di in range(len(self.cands)):
                best = None
                for ci in range(len(self.cands[di])):
                    choice[di] = ci
                    t = self._cost(choice)
                    if best is None or t < best[0]:
                        best = (t, ci)
                if choice[di] != best[1]:
                    changed = True
                choice[di] = best[1]
            if not changed:
                break
        self.choice = choice
        self.flops_event = self._cost(choice)

    # ---- currents and their variants ------------------------------------------
    def _currents(self):
        need = {}
        for opts, ci in zip(self.cands, self.choice):
            for x in opts[ci][1]:
                self.deps(x, need)
        self.order = list(need)                    # children before parents
        self.cid = {d: i for i, d in enumerate(self.order)}
        self.level = {}
        for d in self.order:
            ins = self.inputs(d)
            self.level[d] = 0 if not ins else 1 + max(self.level[x] for x in ins)
        self.order.sort(key=lambda d: self.level[d])
        self.cid = {d: i for i, d in enumerate(self.order)}
        self.offset = {}
        off = 0
        for d in self.order:
            self.offset[d] = off
            off += 1 << len(self.legs(d))
        self.nslots = off

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
                "ggg": 7, "gggg": 8}
    AMP_TYPES = {"ffv": 0, "ffv_a": 1, "ffz": 2, "vvv": 3, "vvvv0": 4, "vvvv1": 5, "vvvv2": 6}

    def _canon_prop_legs(self, legs):
        """The invariant of an internal line, formed from the side without the
        root leg (as in the root-form program)."""
        root = self.p.spec.root
        return frozenset(range(self.n)) - legs if root in legs else legs

    def _item(self, d, v):
        """One current variant: (type, a, b, c, flag, out, in[6], k0, k1, prop)."""
        em, spec = self.em, self.p.spec
        out = self.offset[d] + v
        ins = [0] * 6
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
        elif kind == "qqg_row":
            t = self.HS_TYPES["row"]
            ins[0], ins[1] = slot(xs[0]), slot(xs[1])
            k0 = em.momentum(legs)
            prop = em.prop(self._canon_prop_legs(legs), "t")
        elif kind == "col":
            t = self.HS_TYPES["col"]
            g, U = xs
            ins[0], ins[1] = slot(U), slot(g)   # FFV1_1(fi = U, v = g)
            k0 = em.momentum(legs)
            prop = em.prop(self._canon_prop_legs(legs), "t")
        elif kind == "pair":
            t = self.HS_TYPES["pair"]
            r, U = xs
            ins[0], ins[1] = slot(r), slot(U)   # FFV1P0_3(fo = r, fi = U)
            prop = em.prop(self._canon_prop_legs(legs), "g")
        elif kind in ("ffa_cur", "ffz_cur"):
            t = self.HS_TYPES["pair" if kind == "ffa_cur" else "zcur"]
            ins[0], ins[1] = slot(xs[0]), slot(xs[1])
            a = 1  # coupling: e
            prop = em.prop(self._canon_prop_legs(legs), "A" if kind == "ffa_cur" else "Z")
        elif kind == "ggg":
            t = self.HS_TYPES["ggg"]
            ins[0], ins[1] = slot(xs[0]), slot(xs[1])
            k0, k1 = em.momentum(self.legs(xs[0])), em.momentum(self.legs(xs[1]))
            prop = em.prop(self._canon_prop_legs(legs), "g")
        elif kind == "gggg":
            t = self.HS_TYPES["gggg"]
            if d[0] == "N":
                term = int(self.p.cur[d[1]].vertex[-1])
                pos = {0: xs[0], 1: xs[1], 2: xs[2]}
                outpos = 3
            else:
                term, outpos = d[2], d[3]
                o1, o2, U = d[4], d[5], d[6]
                rest = [q for q in range(3) if q != outpos]
                pos = {rest[0]: o1, rest[1]: o2, 3: U}
            for j, pair in enumerate(VVVV_PAIRS[term]):
                (p0, p1), (p2, p3) = pair
                if outpos in (p0, p1):
                    X = p1 if outpos == p0 else p0
                    Y, Z = p2, p3
                else:
                    X = p3 if outpos == p2 else p2
                    Y, Z = p0, p1
                ins[3 * j + 0], ins[3 * j + 1], ins[3 * j + 2] = slot(pos[X]), slot(pos[Y]), slot(pos[Z])
            prop = em.prop(self._canon_prop_legs(legs), "g")
        else:
            raise ValueError(kind)
        return (t, a, b, c, flag, out, ins, k0, k1, prop)

    def emit_tables(self, pid: int) -> list:
        em = self.em
        nh = 1 << self.n
        items, level_start = [], []
        cur_level = -1
        for d in self.order:
            if self.level[d] != cur_level:
                cur_level = self.level[d]
                level_start.append(len(items))
            for v in range(1 << len(self.legs(d))):
                items.append(self._item(d, v))
        level_start.append(len(items))
        # amplitudes, sorted so that consecutive ones share operands
        amps = []
        for di, (opts, ci) in enumerate(zip(self.cands, self.choice)):
            kind, args = opts[ci]
            ops = [self.cid[x] for x in args]
            ks = [em.momentum(self.legs(x)) for x in args] if kind == "vvv" else [0, 0, 0]
            flows = []
            for s_ in np.nonzero(self.em.coef[di])[0]:
                z = complex(self.em.coef[di, s_])
                code = {1: 0, -1: 1, 1j: 2, -1j: 3}[z]
                flows.append(int(s_) | (code << 6))
            amps.append((self.AMP_TYPES[kind], ops, ks, flows))
        amps.sort(key=lambda a: (a[1], a[0]))
        patterns = {}
        groups = {}
        for t, ops, ks, flows in amps:
            key = tuple(flows)
            if key not in patterns:
                patterns[key] = len(patterns)
            o = list(ops) + [0] * (4 - len(ops))
            groups.setdefault(t, []).append("{%d, %d, {%s}, {%s}}" % (
                t, patterns[key], ", ".join(map(str, o)), ", ".join(map(str, ks[:3]))))
        self.patterns = patterns
        self.groups = {t: len(rows) for t, rows in groups.items()}
        self.amp_list = [(t, list(ops), ks, flows) for t, ops, ks, flows in amps]
        amp_rows = []
        for t in sorted(groups):
            amp_rows.extend(groups[t])
        # slot of every current for every event helicity index
        slot = []
        for d in self.order:
            row = []
            for ih in range(nh):
                bits = 0
                for l in range(self.n):
                    bits |= ((ih >> (self.n - 1 - l)) & 1) << l
                row.append(self.offset[d] + self.variant(d, bits))
            slot.append(row)
        out = []
        self._exact_flops(items, amps)
        out.append("// helicity-shared program: %d currents in %d levels, %d variant slots, %d amplitudes,"
                   " %d flops per event (all helicities)" % (len(self.order), len(level_start) - 1, self.nslots,
                                                            len(amps), self.flops_items + nh * self.flops_amps_hel))
        out.append("static __device__ const HsItem kHsItems%d[%d] = {%s};" % (
            pid, len(items), ", ".join("{%d, %d, %d, %d, %d, %d, {%s}, %d, %d, %d}" % (
                t, a, b, c, flag, o, ", ".join(map(str, ins)), k0, k1, pr)
                for (t, a, b, c, flag, o, ins, k0, k1, pr) in items)))
        out.append("static __constant__ HsAmp kHsAmps%d[%d] = {%s};  // grouped by type"
                   % (pid, len(amp_rows), ", ".join(amp_rows)))
        out.append("static __device__ const uint16_t kHsSlot%d[%d][%d] = {%s};" % (
            pid, len(self.order), nh, ", ".join("{" + ", ".join(map(str, r)) + "}" for r in slot)))
        self.tables = dict(nitems=len(items), level_start=level_start, namps=len(amps), ncur=len(self.order))
        return out

    def _exact_flops(self, items, amps):
        """Operation count: current variants per event, amplitudes + flow sums per helicity."""
        item_flops = {0: FLOPS["ixxxxx"], 1: FLOPS["oxxxxx"], 2: FLOPS["vxxxxx"], 3: FLOPS["FFV1_2"],
                      4: FLOPS["FFV1_1"], 5: FLOPS["FFV1P0_3"], 6: FLOPS["FFV2_4_3"], 7: FLOPS["VVV1P0_1"],
                      8: FLOPS["VVVV1P0_1"]}
        amp_flops = {0: FLOPS["FFV1_0"], 1: FLOPS["FFV1_0"], 2: FLOPS["FFV2_4_0"], 3: FLOPS["VVV1_0"],
                     4: FLOPS["VVVV_0"], 5: FLOPS["VVVV_0"], 6: FLOPS["VVVV_0"]}
        self.flops_items = sum(item_flops[it[0]] for it in items)
        self.flops_amps_hel = sum(amp_flops[t] + FLOPS["jamp"] * len(fl) for t, _, _, fl in amps)

    def struct_lines(self, pid: int) -> list:
        t = self.tables
        return [
            "  // helicity-shared program (tables above)",
            "  static constexpr int HS_NSLOT = %d;" % self.nslots,
            "  static constexpr int HS_NITEM = %d;" % t["nitems"],
            "  static constexpr int HS_NLEVEL = %d;" % (len(t["level_start"]) - 1),
            "  static constexpr int HS_NAMP = %d;" % t["namps"],
            "  static constexpr int HS_NCUR = %d;" % t["ncur"],
            "  // operations: current variants per event, amplitudes + flow sums per helicity",
            "  static constexpr long HS_FLOPS_ITEMS = %d;" % self.flops_items,
            "  static constexpr long HS_FLOPS_AMP_HEL = %d;" % self.flops_amps_hel,
            "  static __host__ __device__ constexpr int hs_level(int l) {",
            "    constexpr int t[%d] = {%s};" % (len(t["level_start"]), ", ".join(map(str, t["level_start"]))),
            "    return t[l];",
            "  }",
            "  static __device__ __forceinline__ const HsItem* hs_items() { return kHsItems%d; }" % pid,
            "  static __device__ __forceinline__ const HsAmp* hs_amps() { return kHsAmps%d; }" % pid,
            "  static __device__ __forceinline__ const uint16_t* hs_slots() { return &kHsSlot%d[0][0]; }" % pid,
        ] + self._flow_switch() + (self._amp_unrolled(pid) if self.AMP_UNROLL else self._amp_loops(pid))

    AMP_UNROLL = False  # straight-line amplitude phase instead of per-type loops

    def _amp_unrolled(self, pid: int) -> list:
        calls = {0: "FFV1_0<R>(%s, %s, %s, cp.gs)", 1: "FFV1_0<R>(%s, %s, %s, cp.ee)",
                 2: "FFV2_4_0<R>(%s, %s, %s, cp.gz, cp.gzl, cp.gzr)"}
        lines = ["  template <class R>",
                 "  static __device__ __forceinline__ void hs_amplitudes(const W4<R>* __restrict__ cur,"
                 " const uint16_t* __restrict__ sl, const R* __restrict__ K, const Couplings<R>& cp, cx<R>* J) {",
                 "    cx<R> amp;"]
        ops = {0: "J[%d] += amp;", 1: "J[%d] -= amp;", 2: "J[%d] += mul_i(amp);", 3: "J[%d] -= mul_i(amp);"}
        for ia, (t, o, ks, flows) in enumerate(self.amp_list):
            if ia % 4 == 0 and ia:
                lines.append("    __syncwarp();  // bounds load hoisting (live ranges)")
            lines.append("    {")
            names = []
            for j, c in enumerate(o):
                lines.append("      const W4<R> x%d = cur[sl[%d * NHEL]];" % (j, c))
                names.append("x%d" % j)
            if t in calls:
                lines.append("      amp = " + calls[t] % tuple(names[:3]) + ";")
            elif t == 3:
                lines.append("      amp = VVV1_0<R>(%s, %s, %s, K + %d, K + %d, K + %d, cp.gs);" % (
                    names[0], names[1], names[2], 4 * ks[0], 4 * ks[1], 4 * ks[2]))
            else:
                lines.append("      amp = VVVV_0<R>(%d, %s, %s, %s, %s, cp.gs2);" % (t - 4, *names[:4]))
            lines.append("      " + " ".join(ops[f >> 6] % (f & 63) for f in flows))
            lines.append("    }")
        lines.append("  }")
        return lines

    def _amp_loops(self, pid: int) -> list:
        """Amplitude phase: one loop per amplitude type over its (constant-memory)
        table; an operand is reloaded only when it changes (uniform branch)."""
        calls = {0: "FFV1_0<R>(o0, o1, o2, cp.gs)", 1: "FFV1_0<R>(o0, o1, o2, cp.ee)",
                 2: "FFV2_4_0<R>(o0, o1, o2, cp.gz, cp.gzl, cp.gzr)",
                 3: "VVV1_0<R>(o0, o1, o2, K + 4 * a.k[0], K + 4 * a.k[1], K + 4 * a.k[2], cp.gs)",
                 4: "VVVV_0<R>(0, o0, o1, o2, o3, cp.gs2)", 5: "VVVV_0<R>(1, o0, o1, o2, o3, cp.gs2)",
                 6: "VVVV_0<R>(2, o0, o1, o2, o3, cp.gs2)"}
        lines = ["  // amplitudes of one (event, helicity): operands cur[sl[c * NHEL]], flows into J",
                 "  template <class R>",
                 "  static __device__ __forceinline__ void hs_amplitudes(const W4<R>* __restrict__ cur,"
                 " const uint16_t* __restrict__ sl, const R* __restrict__ K, const Couplings<R>& cp, cx<R>* J) {",
                 "    W4<R> o0, o1, o2, o3;"]
        start = 0
        for t in sorted(self.groups):
            n = self.groups[t]
            nops = 4 if t >= 4 else 3
            lines.append("    {  // type %d: %d amplitudes" % (t, n))
            lines.append("      int l0 = -1, l1 = -1;")
            lines.append("      for (int d = %d; d < %d; ++d) {" % (start, start + n))
            lines.append("        const HsAmp a = kHsAmps%d[d];" % pid)
            lines.append("        if (a.op[0] != l0) { o0 = cur[sl[a.op[0] * NHEL]]; l0 = a.op[0]; }")
            lines.append("        if (a.op[1] != l1) { o1 = cur[sl[a.op[1] * NHEL]]; l1 = a.op[1]; }")
            lines.append("        o2 = cur[sl[a.op[2] * NHEL]];")
            if nops == 4:
                lines.append("        o3 = cur[sl[a.op[3] * NHEL]];")
            lines.append("        hs_flows<R>(a.pat, %s, J);" % calls[t])
            lines.append("      }")
            lines.append("    }")
            start += n
        lines.append("  }")
        return lines

    def _flow_switch(self) -> list:
        """J_s +=, -=, += i, -= i amp for the colour flows of amplitude pattern `pat`."""
        ops = {0: "J[%d] += amp;", 1: "J[%d] -= amp;", 2: "J[%d] += mul_i(amp);", 3: "J[%d] -= mul_i(amp);"}
        lines = ["  static constexpr int HS_NPAT = %d;" % len(self.patterns),
                 "  // colour-flow updates of each amplitude pattern: J_s += amp, -amp, i amp, -i amp",
                 "  template <class R>",
                 "  static __device__ __forceinline__ void hs_flows(int pat, cx<R> amp, cx<R>* J) {",
                 "    switch (pat) {"]
        for key, pat in sorted(self.patterns.items(), key=lambda kv: kv[1]):
            lines.append("      case %d: %s break;" % (pat, " ".join(ops[f >> 6] % (f & 63) for f in key)))
        lines += ["      default: break;", "    }", "  }"]
        return lines

