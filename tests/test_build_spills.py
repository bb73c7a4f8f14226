"""Register budget of the default SIGMAKIN kernels (no GPU needed: ptxas only).

The helicity-shared kernels run at a fixed number of CTAs per SM, so the
register count per thread is capped (126 for gg -> t t~ g g at two 256-thread
CTAs per SM, 80 for gg -> t t~ g at three), and a change anywhere in their
code or arguments can push them into spilling to local memory, which cost
gg -> t t~ g 8 % once.  The default kernels of the four processes, in both
precisions, must compile without spills or local stack.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import tempfile

import pytest

from paper_2106_12631_gb300 import build as B

pytestmark = pytest.mark.slow


def ptxas_report(src: str) -> dict:
    """ptxas -v report per compiled entry: name -> (stack bytes, spill stores, spill loads)."""
    with tempfile.TemporaryDirectory() as d:
        cmd = [B.nvcc(), *B.ARCH, *B.FLAGS, "-Xptxas", "-v", "-c", src, "-o", os.path.join(d, "x.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, name = {}, None
    for ln in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\w+)'", ln)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", ln)
        if m and name:
            out[name] = tuple(int(x) for x in m.groups())
            name = None
    return out


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_default_kernels_do_not_spill():
    srcs = [os.path.join(B.CSRC, f) for f in ("sigmakin_p1.cu", "sigmakin_p2.cu", "sigmakin_p3.cu", "sigmakin_p4.cu",
                                               "sigmakin_p3_fp64.cu", "sigmakin_p4_fp64.cu")]
    with cf.ThreadPoolExecutor(len(srcs)) as ex:
        reports = list(ex.map(ptxas_report, srcs))
    checked = 0
    for rep in reports:
        for name, (stack, st, ld) in rep.items():
            # the helicity-shared kernel with the CUDA-core colour sum (template
            # argument CS = 0): the default of MG_MIXED below 48 colour flows and of MG_FP64
            if "sigmakin_hs_kernel" in name and ("EfLi0E" in name or "EdLi0E" in name):
                assert (stack, st, ld) == (0, 0, 0), (name, stack, st, ld)
                checked += 1
    assert checked >= 6, checked


LAYOUT_PROBE = r'''
#include "sigmakin_hs.cuh"
#include "gen/proc3.cuh"
#include "gen/proc4.cuh"
#include <cstdio>
template <class P, class R, int CS> void show(const char* name) {
  using L = mg::HsLayout<P, R, CS>;
  std::printf("%s %zu %d\n", name, (size_t)L::bytes, mg::HsCfg<P, R>::CTAS);
}
int main() {
  show<mg::Proc4, float, 0>("p4_simt");
  show<mg::Proc4, float, 1>("p4_tc");
  show<mg::Proc3, float, 0>("p3_simt");
  return 0;
}
'''


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_layouts_admit_their_ctas_per_sm():
    """The helicity-shared FP32 kernels are tuned for a fixed number of CTAs per
    SM (two for gg -> t t~ g g, three for gg -> t t~ g): their shared memory
    plus the 1 KB the GPU reserves per CTA must fit the SM's 228 KB that many
    times, for the CUDA-core and the tcgen05 colour sum alike (a layout
    1 KB too large halves the resident warps)."""
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "probe.cu"), os.path.join(d, "probe")
        with open(src, "w") as f:
            f.write(LAYOUT_PROBE)
        r = subprocess.run([B.nvcc(), *B.ARCH, "-std=c++17", "--expt-relaxed-constexpr", "-I", B.CSRC,
                            "-I", os.path.join(os.path.dirname(B.CSRC), "..", "include"), src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    sm_bytes, reserved = 233472, 1024
    seen = 0
    for ln in out:
        if not ln.strip():
            continue
        name, nbytes, ctas = ln.split()
        assert (int(nbytes) + reserved) * int(ctas) <= sm_bytes, (name, nbytes, ctas)
        seen += 1
    assert seen == 3
