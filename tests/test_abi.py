"""Host-side checks of the C ABI and of the process generator (no GPU needed).

* libmg.so loads and exports every function include/mg.h declares; so does
  libmg_cpu.so for include/mg_cpu.h.
* Process descriptions and host-side argument validation (these return before
  any CUDA call).
* The generated CUDA headers are up to date with the generator.
* The generator's diagram counts, colour-flow coefficients and colour matrix
  agree with the paper's counts and with the oracle's explicit-SU(3) chain
  matrix (two independent constructions).
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2106_12631_gb300 import mg
    return mg.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "mg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(mg_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def test_cpu_build_exports_its_header():
    from paper_2106_12631_gb300 import cpu_simd
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "mg_cpu.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"^\s*int\s+(mgc_\w+)\s*\(", text, flags=re.M)))
    assert names == ["mgc_lanes", "mgc_sigmakin"]
    L = cpu_simd.lib()
    for n in names:
        assert hasattr(L, n), n
    assert L.mgc_sigmakin(0, 1, None, None, 0, None, None, 1) == -2
    assert L.mgc_sigmakin(1, 1, None, None, 0, None, None, 1) == -1
    assert L.mgc_sigmakin(1, 0, None, None, 1, None, None, 1) == 0


def test_process_info():
    from paper_2106_12631_gb300 import mg
    want = {1: (4, 16, 1, 2, 8), 2: (4, 16, 2, 3, 8), 3: (5, 32, 6, 16, 12), 4: (6, 64, 24, 123, 16)}
    for p, (npar, nhel, ncol, ndiag, nrand) in want.items():
        info = mg.process_info(p)
        assert (info["npar"], info["nhel"], info["ncolor"], info["ndiagrams"], info["nrand"]) == \
            (npar, nhel, ncol, ndiag, nrand)
    assert mg.process_info(4)["mass"] == [0, 0, 173.0, 173.0, 0, 0]


def test_host_side_validation(L):
    vp = ctypes.c_void_p
    fake = 0x10000  # never dereferenced: every call below fails validation first
    assert L.mg_sigmakin(0, 1, vp(fake), vp(fake), vp(fake), 0, None) == -2
    assert L.mg_sigmakin(1, -5, vp(fake), vp(fake), vp(fake), 0, None) == -1
    assert L.mg_sigmakin(1, 3, vp(fake + 4), vp(fake), vp(fake), 0, None) == -3
    assert L.mg_sigmakin(1, 3, None, vp(fake), vp(fake), 0, None) == -1
    assert L.mg_sigmakin(1, 0, None, None, None, 0, None) == 0  # empty batch is a no-op
    assert L.mg_sigmakin(1, 3, vp(fake), vp(fake), vp(fake), 99, None) == -1
    L.mg_rambo.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, vp, ctypes.c_int, vp, vp, vp]
    assert L.mg_rambo(4, 8, 300.0, vp(fake), 16, vp(fake), vp(fake), None) == -1
    assert L.mg_rambo(4, 8, 1500.0, vp(fake), 12, vp(fake), vp(fake), None) == -1
    assert L.mg_rambo(4, 0, 1500.0, None, 16, None, None, None) == 0
    L.mg_event_sum_scratch_bytes.restype = ctypes.c_int64
    assert L.mg_event_sum_scratch_bytes(ctypes.c_int64(-1)) == -1
    L.mg_status_string.restype = ctypes.c_char_p
    assert L.mg_status_string(-3) == b"device pointer not 16-byte aligned"


def test_params_roundtrip():
    from paper_2106_12631_gb300 import mg
    old = mg.get_params()
    assert old["mt"] == 173.0 and old["alpha_s"] == 0.118
    mg.set_params(mt=172.5)
    assert mg.get_params()["mt"] == 172.5
    with pytest.raises(mg.MGError):
        mg.set_params(sw2=1.5)
    mg.set_params(**old)
    assert mg.get_params() == old


def test_generated_code_up_to_date():
    from paper_2106_12631_gb300.gen.__main__ import main
    assert main(check=True) == 0


@pytest.mark.parametrize("pid,ndiag,ncol", [(1, 2, 1), (2, 3, 2), (3, 16, 6), (4, 123, 24)])
def test_generator_counts_and_coefficients(pid, ndiag, ncol):
    from paper_2106_12631_gb300.gen import procgen
    s = procgen.summary(pid)
    assert s["ndiagrams"] == ndiag and s["ncolor"] == ncol
    vals = set(complex(z) for z in s["coef"].reshape(-1) if z != 0)
    assert vals <= {1, -1, 1j, -1j}
    # every amplitude contributes to at least one flow, every flow gets amplitudes
    assert np.all(np.any(s["coef"] != 0, axis=1)) and np.all(np.any(s["coef"] != 0, axis=0))


@pytest.mark.parametrize("ng", [2, 3, 4])
def test_generator_colour_matrix_matches_oracle(orc, ng):
    from paper_2106_12631_gb300.gen import procgen
    perms, num, den = procgen.chain_matrix(ng)
    C = orc.chain_colour_matrix(ng).real
    np.testing.assert_allclose(num / den, C, rtol=0, atol=1e-12)
    assert np.all(np.diag(num) * 3 ** ng == den * 3 * 4 ** ng)


@pytest.mark.parametrize("pid", [1, 2, 3, 4])
def test_generator_merged_contractions_keep_every_amplitude(pid):
    """Amplitudes merged into one contraction (same amputated current X, colour
    flows equal up to a phase i^r) each keep their own flows: i^r times the
    group's pattern, and every amplitude appears in exactly one group."""
    from paper_2106_12631_gb300.gen import procgen
    proc = procgen.Process(procgen.PROCS[pid])
    em = procgen.Emitter(proc)
    for leg in range(proc.n):
        em.momentum_phys(leg)
    em.emit()
    sp = procgen.SharedProgram(proc, em)
    sp.emit_tables(pid)
    remaining = [(a[0], a[1], a[2], tuple(sorted(a[5]))) for a in sp.amp_list]
    for g in sp.groups:
        for yo, r in g["ys"]:
            remaining.remove((g["ch"], g["xo"], yo, sp._rotate(g["flows"], r)))
    assert remaining == []


def shared_program(pid):
    from paper_2106_12631_gb300.gen import procgen
    proc = procgen.Process(procgen.PROCS[pid])
    em = procgen.Emitter(proc)
    for leg in range(proc.n):
        em.momentum_phys(leg)
    em.emit()
    sp = procgen.SharedProgram(proc, em)
    sp.emit_tables(pid)
    return sp


@pytest.mark.parametrize("pid", [1, 2, 3, 4])
def test_generator_chunks_fill_whole_rounds(pid):
    """Amputated-current chunks: every amputated current in exactly one chunk,
    within the chunk capacity; with several chunks the capacity is a multiple
    of the chunk quantum, and for gg -> t t~ g g all four chunks are full
    (192 slots per event: three rounds of the 4-event, 256-thread CTA)."""
    sp = shared_program(pid)
    sizes = [sum(sp.nvar(X) for X in c) for c in sp.chunks]
    assert sorted(X for c in sp.chunks for X in c) == sorted(sp.xoff)
    assert max(sizes) <= sp.xcap
    if len(sp.chunks) > 1:
        assert sp.xcap % sp.CHUNK_QUANTUM == 0
    if pid == 4:
        assert sizes == [192] * 4


@pytest.mark.parametrize("pid", [3, 4])
def test_generator_four_gluon_items_three_operands(pid):
    """A four-gluon item names its three distinct operand slots {X_0, X_1, W}
    and the kernels form X_0 (X_1 . W) - X_1 (X_0 . W).  Against the two
    products read off the vertex's pairings (each pairs the output with one
    operand X_j and dots the other two: X_0 (Y_0 . Z_0) - X_1 (Y_1 . Z_1)),
    evaluated on random complex vectors per slot: equal for every variant."""
    from paper_2106_12631_gb300.gen import procgen
    sp = shared_program(pid)
    rng = np.random.default_rng(pid)
    eta = np.array([1.0, -1.0, -1.0, -1.0])

    def vdot(a, b):
        return np.sum(eta * a * b)

    n = 0
    for d in list(sp.order) + list(sp.xoff):
        if sp.kind(d) not in ("gggg", "agggg"):
            continue
        term, outpos, pos = sp._gggg_positions(d)
        for v in range(sp.nvar(d)):
            ins = sp._item(d, v)[6]
            assert len(set(ins)) == 3
            six = []
            for (p0, p1), (p2, p3) in procgen.VVVV_PAIRS[term]:
                if outpos in (p0, p1):
                    x, y, z = (p1 if outpos == p0 else p0), p2, p3
                else:
                    x, y, z = (p3 if outpos == p2 else p2), p0, p1
                six += [sp.offset[pos[q]] + sp.sub_variant(pos[q], d, v) for q in (x, y, z)]
            V = {s: rng.normal(size=4) + 1j * rng.normal(size=4) for s in set(six) | set(ins)}
            old = V[six[0]] * vdot(V[six[1]], V[six[2]]) - V[six[3]] * vdot(V[six[4]], V[six[5]])
            new = V[ins[0]] * vdot(V[ins[1]], V[ins[2]]) - V[ins[1]] * vdot(V[ins[0]], V[ins[2]])
            np.testing.assert_allclose(new, old, rtol=1e-12, atol=1e-12)
            n += 1
    assert n > 0
