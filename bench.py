"""Throughput of the matrix-element hot path on GB300 (one JSON line on stdout).

A step is one pass of the whole path over one batch of seeded synthetic
events of gg -> t t~ g g at sqrt(s) = 1500 GeV (2^20 events per GPU):
  RAMBO on the 16 filter events -> helicity filter -> RAMBO on the batch ->
  SIGMAKIN (mixed precision by default) -> FP64 event sum.
The random numbers are resident in HBM before the timed region.  The
per-step working set (random numbers 128 MiB + momenta 192 MiB + outputs) is
larger than the 126 MB L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
benchmark) on the host cores on a bounded sample of the same workload.
Under torchrun every rank processes its own 2^20 events (weak scaling);
rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "gg_ttgg"
METRIC = "matrix elements/sec on 1 GB300 (gg->ttgg), mixed-precision vs FP64 at stated rel. error"
UNIT = "ME/s"
FP32_LANES_PER_SM = 128
SMS = 152
SM_MAX_MHZ = 2070.0

# DRAM traffic of the mixed gg -> t t~ g g SIGMAKIN kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch over 2^18 events,
# scaled by events; it reads the momenta once and writes |M|^2), valid only
# while the kernel sources are the ones captured.
SIGMAKIN_TRAFFIC = {"bytes_per_event": 192.69, "sources_sha1": "ceea71af37bc050e8c44025841035afdf399fe92"}
# Tensor-pipe activity of the tcgen05 colour-sum variant from the same kind of
# capture (sm__pipe_tensor_cycles_active, fraction of its peak), valid while
# the kernel sources are the ones captured.
TC_TENSOR_PIPE = {"frac": 0.0167, "sources_sha1": "ceea71af37bc050e8c44025841035afdf399fe92"}
SIGMAKIN_SOURCES = ["paper_2106_12631_gb300/csrc/" + f for f in
                    ("sigmakin_hs.cuh", "sigmakin_launch.cuh", "sigmakin.cuh", "helas.cuh", "colour_tc.cuh",
                     "mg_types.cuh", "process.cuh", "gen/proc4.cuh")]


def sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in SIGMAKIN_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "mixed_simt", "mixed_tc", "fp64", "mixed_unrolled",
                                                        "fp64_unrolled"])
    ap.add_argument("--nevt", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-others", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="SIGMAKIN throughput against the number of events per launch (no step, one JSON line)")
    return ap.parse_args()


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def shard_first_event(rank: int, nevt: int) -> int:
    """First event index of a rank's batch: ranks take disjoint, contiguous
    ranges of the counter-based random stream (weak scaling)."""
    return rank * nevt


def max_over_ranks(seconds: float, world: int, dev) -> float:
    """The job's time: the slowest rank's."""
    if world == 1:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(sums, world: int):
    """The path's one exchange: the event sums (sum w me, sum (w me)^2, N) of
    all ranks, added in place."""
    if world > 1:
        import torch
        torch.distributed.all_reduce(sums, op=torch.distributed.ReduceOp.SUM)
    return sums


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def rel_err_stats(x, ref) -> dict:
    """Per-event relative error |x / ref - 1| over all events: max, median,
    99.99th percentile, non-finite results, and the events above 1e-5 (the
    stated bound of the mixed path's 99.9th percentile) and above 1e-12 (the FP64
    bar)."""
    import numpy as np
    import torch
    x = x.cpu().numpy() if isinstance(x, torch.Tensor) else np.asarray(x)
    ref = ref.cpu().numpy() if isinstance(ref, torch.Tensor) else np.asarray(ref)
    bad = ~np.isfinite(x)
    rel = np.where(bad, np.inf, np.abs(x / ref - 1))
    return {"max": float(rel.max()), "median": float(np.median(rel)), "p99.99": float(np.quantile(rel, 0.9999)),
            "nonfinite": int(bad.sum()), "above_1e-5": int((rel > 1e-5).sum()),
            "above_1e-12": int((rel > 1e-12).sum()), "events": int(rel.size)}


def measure_other_workloads(mg, I, dev, stream, reps: int = 3) -> dict:
    """ME/s of SIGMAKIN (FP64 and mixed) for e+e- -> mu+mu-, gg -> t t~, gg -> t t~ g,
    and of the adjoint gradient of gg -> t t~ g (2^18 events, 16 random rows)."""
    import torch

    def time_it(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    out = {}
    for name in ("ee_mumu", "gg_tt", "gg_ttg", "gg_ttg_grad"):
        w = I.WORKLOADS[name]
        proc, nevt, nr, ecm = w["proc"], w["nevt"], w["nrows"], w["ecm"]
        rnd = torch.from_numpy(I.uniforms(I.seed_of(name), nr, nevt)).to(dev)
        frnd = torch.from_numpy(I.uniforms(I.filter_seed_of(name), nr, 16)).to(dev)
        mask = mg.filter_helicities(proc, mg.rambo(proc, frnd, ecm)[0])
        mom, _ = mg.rambo(proc, rnd, ecm)
        me = torch.empty(nevt, dtype=torch.float64, device=dev)
        res = {"events": nevt, "good_helicities": int(mask.sum().item())}
        if name == "gg_ttg_grad":
            grad = torch.empty((nr, nevt), dtype=torch.float64, device=dev)
            for mode in ("mixed", "fp64"):
                t = time_it(lambda: mg.sigmakin_grad(proc, rnd, ecm, mask, mode=mode, grad=grad, me=me,
                                                     stream=stream))
                res[mode] = {"value": nevt / t, "unit": "gradients/s", "ms": 1e3 * t}
        else:
            me_by_mode = {}
            for mode in ("mixed", "fp64"):
                t = time_it(lambda: mg.sigmakin(proc, mom, mask, mode=mode, me=me, stream=stream))
                res[mode] = {"value": nevt / t, "unit": UNIT, "sigmakin_ms": 1e3 * t}
                me_by_mode[mode] = me.clone()
            res["mixed_vs_fp64_rel_err"] = rel_err_stats(me_by_mode["mixed"], me_by_mode["fp64"])
        if name == "ee_mumu":
            # the paper's own e+e- -> mu+mu- point: 2^19 events per launch, past the
            # plateau in events in flight (16384 events leave the GPU mostly idle)
            big = 1 << 19
            rnd_b = torch.from_numpy(I.uniforms(I.seed_of(name), nr, big)).to(dev)
            mom_b, _ = mg.rambo(proc, rnd_b, ecm)
            me_b = torch.empty(big, dtype=torch.float64, device=dev)
            res["events_2^19"] = {}
            for mode in ("mixed", "fp64"):
                t = time_it(lambda: mg.sigmakin(proc, mom_b, mask, mode=mode, me=me_b, stream=stream))
                res["events_2^19"][mode] = {"value": big / t, "unit": UNIT, "sigmakin_ms": 1e3 * t}
            del rnd_b, mom_b, me_b
        out[name] = res
    return out


def measure_generation(mg, proc, ecm, nevt, seed, mom, wgt, me, sums, stream, hbm_gbs, mask, mode, reps=3):
    import torch

    def time_it(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    from paper_2106_12631_gb300 import inputs as I
    rnd = torch.from_numpy(I.uniforms(seed, 16, nevt)).to(mom.device)
    mom2, wgt2 = torch.empty_like(mom), torch.empty_like(wgt)
    t_buf = time_it(lambda: mg.rambo(proc, rnd, ecm, mom=mom2, wgt=wgt2, stream=stream))
    t_seed = time_it(lambda: mg.rambo_seeded(proc, nevt, ecm, seed, 0, mom=mom2, wgt=wgt2, stream=stream))
    idx = torch.empty(nevt, dtype=torch.int64, device=mom.device)
    cnt = torch.empty(1, dtype=torch.int64, device=mom.device)
    scratch = torch.empty(mg.unweight_scratch_bytes(nevt) // 8 + 2, dtype=torch.float64, device=mom.device)
    t_uw = time_it(lambda: mg.unweight(me, wgt, seed, 0, idx=idx, count=cnt, scratch=scratch, stream=stream))
    kept = int(cnt.item())
    xs = mg.cross_section(proc, ecm, sums, stream=stream).cpu().numpy()
    scr = torch.empty(mg.event_sum_scratch_bytes(nevt) // 8 + 2, dtype=torch.float64, device=mom.device)
    out3 = torch.empty(3, dtype=torch.float64, device=mom.device)
    t_sum = time_it(lambda: mg.event_sum(me, wgt, out=out3, scratch=scr, stream=stream))
    uw_bytes = 3 * 16 * nevt + 8 * kept  # (w, me) read by three passes, kept indices written
    # the batched entry point for an external integrator: the same events as an
    # array of structures, alone and with a helicity and a colour flow chosen per event
    mom_aos = mom.permute(2, 0, 1).contiguous()
    me_b = torch.empty_like(me)
    hel_b = torch.empty(nevt, dtype=torch.int32, device=mom.device)
    col_b = torch.empty(nevt, dtype=torch.int32, device=mom.device)
    ws = torch.empty(mg.batch_workspace_bytes(proc, nevt) // 8 + 2, dtype=torch.float64, device=mom.device)
    t_batch = time_it(lambda: mg.matrix_elements_batch(proc, mom_aos, mask, mode=mode, me=me_b, workspace=ws,
                                                       stream=stream))
    choose = "unrolled" not in mode  # the choices come with the helicity-shared kernels
    t_choice = time_it(lambda: mg.matrix_elements_batch(proc, mom_aos, mask, mode=mode, hel_rnd=rnd[0], col_rnd=rnd[1],
                                                        me=me_b, hel=hel_b, col=col_b, workspace=ws,
                                                        stream=stream)) if choose else None
    t_sig = time_it(lambda: mg.sigmakin(proc, mom, mask, mode=mode, me=me_b, stream=stream))
    # RAMBO and SIGMAKIN in one kernel (no momentum buffer) against the two kernels
    wgt_b = torch.empty_like(wgt)
    fusable = "unrolled" not in mode
    t_two = time_it(lambda: (mg.rambo(proc, rnd, ecm, mom=mom2, wgt=wgt2, stream=stream),
                             mg.sigmakin(proc, mom2, mask, mode=mode, me=me_b, stream=stream)))
    t_fused = time_it(lambda: mg.sigmakin_rambo(proc, rnd, ecm, mask, mode=mode, me=me_b, wgt=wgt_b,
                                                stream=stream)) if fusable else None
    del mom_aos, ws
    return {"events": nevt,
            "rambo_device_rng_ms": 1e3 * t_seed, "rambo_buffered_ms": 1e3 * t_buf,
            "unweight_ms": 1e3 * t_uw, "unweight_kept": kept,
            "unweight_gbs": uw_bytes / t_uw / 1e9,
            "unweight_hbm_frac": (uw_bytes / t_uw / 1e9) / hbm_gbs if hbm_gbs else None,
            "cross_section_pb": float(xs[0]), "cross_section_err_pb": float(xs[1]),
            "batch_aos_ms": 1e3 * t_batch,
            "batch_aos_with_choices_ms": 1e3 * t_choice if t_choice is not None else None, "sigmakin_soa_ms": 1e3 * t_sig,
            "rambo_then_sigmakin_ms": 1e3 * t_two,
            "rambo_sigmakin_fused_ms": 1e3 * t_fused if t_fused is not None else None,
            "rooflines": {
                "event_sum": {"bound": "hbm", "achieved": 16 * nevt / t_sum / 1e9, "peak": hbm_gbs,
                              "unit": "GB/s", "frac": (16 * nevt / t_sum / 1e9) / hbm_gbs if hbm_gbs else None,
                              "ms": 1e3 * t_sum, "bytes_per_event": 16},
                "unweight": {"bound": "hbm", "achieved": uw_bytes / t_uw / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                             "frac": (uw_bytes / t_uw / 1e9) / hbm_gbs if hbm_gbs else None,
                             "ms": 1e3 * t_uw, "bytes_per_event": 48}}}


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo; Arm hosts name the part by its ids)."""
    import platform
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return platform.machine()
    for key in ("model name", "Hardware", "CPU part"):
        for ln in info.splitlines():
            if ln.startswith(key):
                return "%s %s: %s" % (platform.machine(), key, ln.split(":", 1)[1].strip())
    return platform.machine()


def sweep_events_per_launch() -> dict:
    """ME/s of SIGMAKIN against the events of one launch (the paper's throughput
    against the grid size): e+e- -> mu+mu- and gg -> t t~ g g, mixed and FP64,
    inputs resident, CUDA events, three launches after one warm-up."""
    import torch

    from paper_2106_12631_gb300 import inputs as I
    from paper_2106_12631_gb300 import mg
    dev = torch.device("cuda", 0)
    out = {"metric": "SIGMAKIN ME/s against events per launch", "unit": UNIT, "points": {}}
    plan = {("ee_mumu", "mixed"): range(10, 23, 2), ("ee_mumu", "fp64"): range(10, 23, 2),
            ("gg_ttgg", "mixed"): range(8, 22, 1), ("gg_ttgg", "fp64"): range(8, 19, 2)}
    for (name, mode), ks in plan.items():
        w = I.WORKLOADS[name]
        proc, nr, ecm = w["proc"], w["nrows"], w["ecm"]
        frnd = torch.from_numpy(I.uniforms(I.filter_seed_of(name), nr, 16)).to(dev)
        mask = mg.filter_helicities(proc, mg.rambo(proc, frnd, ecm)[0])
        nmax = 1 << max(ks)
        mom, _ = mg.rambo(proc, torch.from_numpy(I.uniforms(I.seed_of(name), nr, nmax)).to(dev), ecm)
        me = torch.empty(nmax, dtype=torch.float64, device=dev)
        pts = []
        for k in ks:
            n = 1 << k
            m = mom[:, :, :n].contiguous()
            mg.sigmakin(proc, m, mask, mode=mode, me=me[:n])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(3):
                mg.sigmakin(proc, m, mask, mode=mode, me=me[:n])
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3 / 3
            pts.append({"events": n, "ms": 1e3 * t, "value": n / t})
        out["points"]["%s_%s" % (name, mode)] = pts
    return out


def cpu_simd_rates(seed: int, threads: int) -> dict:
    """The SIMD CPU build of the same program (libmg_cpu.so) on the host cores,
    gg -> t t~ g g on a bounded sample: ME/s per precision."""
    import oracle
    from paper_2106_12631_gb300 import cpu_simd
    from paper_2106_12631_gb300 import inputs as I
    frnd = I.uniforms(I.filter_seed_of(WORKLOAD), 16, 16)
    fmom, _ = oracle.rambo(4, frnd, 1500.0)
    _, ph = oracle.me(4, fmom, per_helicity=True, nthreads=threads)
    mask = (abs(ph).max(axis=1) > 0).astype("int32")
    out = {"kind": "SIMD CPU build of the helicity-shared program", "cores": threads}
    for prec, n in (("fp32", 16384), ("fp64", 8192)):
        rnd = I.uniforms(seed, 16, n)
        mom, _ = oracle.rambo(4, rnd, 1500.0)
        cpu_simd.sigmakin(4, mom[:, :, :256].copy(), mask, prec, nthreads=threads)  # warm-up
        t0 = time.perf_counter()
        cpu_simd.sigmakin(4, mom, mask, prec, nthreads=threads)
        dt = time.perf_counter() - t0
        out[prec] = {"value": n / dt, "unit": UNIT, "lanes": cpu_simd.lanes(prec),
                     "sample": "%d gg->ttgg events, %.2f s wall" % (n, dt)}
    return out


def cpu_oracle_rate(nevt_sample: int, seed: int, threads: int):
    """Oracle ME/s on the host cores for a bounded sample (RAMBO + |M|^2, FP64)."""
    import numpy as np

    import oracle
    from paper_2106_12631_gb300 import inputs as I
    oracle.build()
    rnd = I.uniforms(seed, 16, nevt_sample)
    oracle.me(4, oracle.rambo(4, rnd[:, :2], 1500.0)[0])  # colour set-up outside the timing
    t0 = time.perf_counter()
    mom, _ = oracle.rambo(4, rnd, 1500.0)
    oracle.me(4, mom, nthreads=threads)
    dt = time.perf_counter() - t0
    return nevt_sample / dt, dt


# seeded sample per workload for the error against the oracle (the workload's
# first events; about a second of oracle time on the host cores in all)
ORACLE_ERROR_SAMPLE = (("ee_mumu", 4096), ("gg_tt", 4096), ("gg_ttg", 4096), ("gg_ttgg", 1024))


def oracle_error_stats(mg, dev, cores: int) -> dict:
    """Relative error of the GPU's FP64 and mixed-precision |M|^2 against the
    FP64 oracle, per workload, on a seeded sample: the oracle's own RAMBO
    momenta go to both sides, the GPU uses its own helicity filter."""
    import torch

    import oracle
    from paper_2106_12631_gb300 import inputs as I
    oracle.build()
    out = {}
    for name, n in ORACLE_ERROR_SAMPLE:
        w = I.WORKLOADS[name]
        proc, nr, ecm = w["proc"], w["nrows"], w["ecm"]
        mom, _ = oracle.rambo(proc, I.uniforms(I.seed_of(name), nr, n), ecm)
        t0 = time.perf_counter()
        me_o = oracle.me(proc, mom, nthreads=cores)
        dt = time.perf_counter() - t0
        frnd = torch.from_numpy(I.uniforms(I.filter_seed_of(name), nr, 16)).to(dev)
        mask = mg.filter_helicities(proc, mg.rambo(proc, frnd, ecm)[0])
        mom_d = torch.from_numpy(mom).to(dev)
        res = {"events": n, "oracle_s": dt}
        for mode in ("fp64", "mixed"):
            res[mode] = rel_err_stats(mg.sigmakin(proc, mom_d, mask, mode=mode), me_o)
        out[name] = res
    return out


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    from paper_2106_12631_gb300 import inputs as I
    cores = os.cpu_count() or 1
    sample = 2048
    seed = I.seed_of(WORKLOAD)
    for _ in range(args.warmup):
        cpu_oracle_rate(256, seed, cores)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = cpu_oracle_rate(sample, seed, cores)
        rates.append(r)
        times.append(dt)
    value = sample * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64 uniforms -> RAMBO)",
        "config": {"workload": "gg->ttgg tree-level |M|^2, RAMBO 4-body at 1500 GeV, FP64 CPU oracle",
                   "events_per_step": sample, "nevt_full": args.nevt},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d events of the gg->ttgg workload per step (RAMBO + all 64 "
                                   "helicities, explicit colour), std::thread over %d cores" % (sample, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.sweep:
        if rank == 0:
            print(json.dumps(sweep_events_per_launch()))
        return
    import numpy as np
    import torch

    from paper_2106_12631_gb300 import inputs as I
    from paper_2106_12631_gb300 import mg
    from paper_2106_12631_gb300.gen import procgen

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    proc, ecm, nevt = 4, 1500.0, args.nevt
    seed = I.seed_of(WORKLOAD)
    # inputs resident in HBM: this rank's own event range
    rnd = torch.from_numpy(I.uniforms(seed, 16, nevt, first_event=shard_first_event(rank, nevt))).to(dev)
    frnd = torch.from_numpy(I.uniforms(I.filter_seed_of(WORKLOAD), 16, 16)).to(dev)
    info = mg.process_info(proc)
    mom = torch.empty((info["npar"], 4, nevt), dtype=torch.float64, device=dev)
    wgt = torch.empty(nevt, dtype=torch.float64, device=dev)
    fmom = torch.empty((info["npar"], 4, 16), dtype=torch.float64, device=dev)
    fwgt = torch.empty(16, dtype=torch.float64, device=dev)
    mask = torch.empty(info["nhel"], dtype=torch.int32, device=dev)
    me = torch.empty(nevt, dtype=torch.float64, device=dev)
    out = torch.empty(3, dtype=torch.float64, device=dev)
    scratch = torch.empty(mg.event_sum_scratch_bytes(nevt) // 8 + 2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    kernel_launches_per_step = 6  # rambo(filter), filter, rambo, sigmakin, event_sum x2

    # the helicity filter runs on a high-priority stream next to the batch's
    # RAMBO: its few long CTAs take SMs as RAMBO's short CTAs retire.
    # Consecutive steps alternate between two streams, each with its own
    # momentum, weight, matrix-element, event-sum and mask buffers, so one
    # step's RAMBO can fill the tail of the previous step's SIGMAKIN; every
    # step still runs the filter, RAMBO, SIGMAKIN and the event sum of its batch.
    filt = torch.cuda.Stream(priority=-1)
    pipes = [stream, torch.cuda.Stream()]
    bufs = [(mom, wgt, me, out, scratch, mask),
            (torch.empty_like(mom), torch.empty_like(wgt), torch.empty_like(me), torch.empty_like(out),
             torch.empty_like(scratch), torch.empty_like(mask))]
    mask_ready = [torch.cuda.Event() for _ in range(2)]
    mask_free = [torch.cuda.Event() for _ in range(2)]

    def step(k, mode):
        b = k & 1
        st = pipes[b]
        mom_b, wgt_b, me_b, out_b, scr_b, mask_b = bufs[b]
        filt.wait_event(mask_free[b])  # the SIGMAKIN two steps back has read this mask
        mg.rambo(proc, frnd, ecm, mom=fmom, wgt=fwgt, stream=filt)
        mg.filter_helicities(proc, fmom, mask=mask_b, stream=filt)
        mask_ready[b].record(filt)
        mg.rambo(proc, rnd, ecm, mom=mom_b, wgt=wgt_b, stream=st)
        st.wait_event(mask_ready[b])
        mg.sigmakin(proc, mom_b, mask_b, mode=mode, me=me_b, stream=st)
        mask_free[b].record(st)
        mg.event_sum(me_b, wgt_b, out=out_b, scratch=scr_b, stream=st)

    def run_steps(mode, n):
        pipes[1].wait_stream(stream)
        filt.wait_stream(stream)
        for k in range(n):
            step(k, mode)
        stream.wait_stream(pipes[1])
        stream.wait_stream(filt)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(mode, steps):
        run_steps(mode, args.warmup)
        torch.cuda.synchronize()
        barrier()
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        t0.record(stream)
        run_steps(mode, steps)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        total = t0.elapsed_time(t1) / 1e3
        # SIGMAKIN's own launch duration (for the roofline and the comparison
        # lines): in the pipelined steps a launch's events would also cover the
        # wait for the previous step's kernel, so the kernel is timed right
        # after the steps, alone, back to back on one stream, on the same inputs
        for a, b in kev:
            a.record(stream)
            mg.sigmakin(proc, mom, mask, mode=mode, me=me, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        kern = [a.elapsed_time(b) / 1e3 for a, b in kev]
        return max_over_ranks(total, world, dev), kern

    clocks = ClockSampler(local)
    clocks.start()
    total, kern = timed(args.mode, args.steps)
    clk = clocks.stop()
    me_main = me.clone()
    sums = out.clone()
    ngood = int(mask.sum().item())
    value = world * nevt * args.steps / total

    # the same step with the per-helicity unrolled kernel (every helicity recomputes its currents)
    unrolled = None
    if args.mode in ("mixed", "fp64") and not args.no_others:
        tu, ku = timed(args.mode + "_unrolled", max(1, min(args.steps, 2)))
        unrolled = {"mode": args.mode + "_unrolled", "value": world * nevt * max(1, min(args.steps, 2)) / tu,
                    "unit": UNIT, "sigmakin_ms": 1e3 * statistics.mean(ku)}

    # the same step with the colour sum on the tensor cores (split-BF16 tcgen05)
    tensor_core = None
    if args.mode == "mixed" and not args.no_others:
        tt, kt = timed("mixed_tc", max(1, min(args.steps, 2)))
        tensor_core = {"mode": "mixed_tc", "value": world * nevt * max(1, min(args.steps, 2)) / tt, "unit": UNIT,
                       "sigmakin_ms": 1e3 * statistics.mean(kt),
                       "tensor_pipe_active": TC_TENSOR_PIPE["frac"] if TC_TENSOR_PIPE["sources_sha1"] == sources_sha1()
                       else None,
                       "tensor_pipe_source": "ncu sm__pipe_tensor_cycles_active of one 2^18-event launch"}

    # SIGMAKIN split in two kernels per chunk (currents, then amplitudes), the
    # chunks' launches replayed from a CUDA graph; same momenta and mask
    kernel_split = None
    if args.mode in ("mixed", "fp64") and not args.no_others:
        smode = "mixed_simt" if args.mode == "mixed" else "fp64"  # gg -> t t~ g g: CUDA-core colour sum
        ws = torch.empty(mg.sigmakin_split_workspace_bytes(proc, smode, nevt) // 8 + 2, dtype=torch.float64,
                         device=dev)
        me_s = torch.empty_like(me)
        mg.sigmakin_split(proc, mom, mask, mode=smode, me=me_s, workspace=ws, stream=stream)  # graph capture
        torch.cuda.synchronize()
        ns = max(1, min(args.steps, 3))
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(ns):
            mg.sigmakin_split(proc, mom, mask, mode=smode, me=me_s, workspace=ws, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        ts = a0.elapsed_time(a1) / 1e3 / ns
        kernel_split = {"mode": smode, "value": world * nevt / ts, "unit": UNIT, "sigmakin_ms": 1e3 * ts,
                        "workspace_mib": ws.numel() * 8 / 2 ** 20,
                        "identical_to_single_kernel": bool(torch.equal(me_s, me_main))}
        del ws, me_s

    fp64 = None
    if not args.no_fp64 and args.mode != "fp64":
        t64, k64 = timed("fp64", max(1, min(args.steps, 2)))
        me64 = me.clone()
        fp64 = {"value": world * nevt * max(1, min(args.steps, 2)) / t64, "unit": UNIT,
                "sigmakin_ms": 1e3 * statistics.mean(k64),
                "mixed_vs_fp64_rel_err": rel_err_stats(me_main, me64)}

    # event generation from the step's weighted events: device-RNG RAMBO (vs the
    # buffered one), cross section, hit-or-miss unweighting (CUDA events)
    generation = None
    if not args.no_others:
        generation = measure_generation(mg, proc, ecm, nevt, seed, mom, wgt, me, out, stream,
                                        measured_peaks().get("hbm_gbs"), mask, args.mode)

    # the other workloads (SIGMAKIN or the adjoint alone, inputs resident, CUDA events)
    others = {} if args.no_others else measure_other_workloads(mg, I, dev, stream)

    # end to end through the library's host-buffer entry point (mg_pipeline_host):
    # every step copies the batch's random numbers from pinned host memory, runs
    # RAMBO + SIGMAKIN + the event sum, and copies me and the event sum back.
    # Consecutive steps alternate between two streams, workspaces and host
    # output buffers, so one step's copies overlap the previous step's kernels.
    # Each step's helicity mask comes from its own 16 filter events, drawn and
    # filtered on the device (mg_rambo_seeded, mg_filter_helicities) on the
    # high-priority stream one step ahead, into one of two mask buffers.
    rnd_h = torch.from_numpy(I.uniforms(seed, 16, nevt, first_event=shard_first_event(rank, nevt))).pin_memory()
    me_hs = [torch.empty(nevt, dtype=torch.float64).pin_memory() for _ in range(2)]
    sums_hs = [torch.empty(3, dtype=torch.float64).pin_memory() for _ in range(2)]
    wss = [torch.empty(mg.pipeline_workspace_bytes(proc, nevt, 16) // 8 + 2, dtype=torch.float64, device=dev)
           for _ in range(2)]
    pipes = [stream, torch.cuda.Stream()]
    masks = [torch.empty_like(mask) for _ in range(2)]
    mask_ready = [torch.cuda.Event() for _ in range(2)]
    mask_free = [torch.cuda.Event() for _ in range(2)]
    fseed = I.filter_seed_of(WORKLOAD)

    def filter_e2e(k):
        b = k & 1
        filt.wait_event(mask_free[b])  # the pipeline two steps back has read this mask
        mg.rambo_seeded(proc, 16, ecm, fseed, 0, mom=fmom, wgt=fwgt, stream=filt)
        mg.filter_helicities(proc, fmom, mask=masks[b], stream=filt)
        mask_ready[b].record(filt)

    def steps_e2e(n):
        pipes[1].wait_stream(stream)
        filt.wait_stream(stream)
        filter_e2e(0)
        for k in range(n):
            if k + 1 < n:
                filter_e2e(k + 1)
            b = k & 1
            pipes[b].wait_event(mask_ready[b])
            mg.pipeline_host(proc, rnd_h, ecm, masks[b], mode=args.mode, me_host=me_hs[b], sums_host=sums_hs[b],
                             workspace=wss[b], stream=pipes[b])
            mask_free[b].record(pipes[b])
        stream.wait_stream(pipes[1])

    steps_e2e(args.warmup)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps_e2e(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    te2e = e0.elapsed_time(e1) / 1e3
    te2e = max_over_ranks(te2e, world, dev)
    e2e_same = bool(torch.equal(me_hs[(args.steps - 1) & 1], me_main.cpu()))
    sum_over_ranks(sums, world)
    e2e = {"value": world * nevt * args.steps / te2e, "unit": UNIT,
           "h2d_bytes_per_step": 8 * rnd_h.numel(),
           "d2h_bytes_per_step": 8 * nevt + 8 * 3,
           "api": "mg_pipeline_host (host rnd in; host me and event sum out), filter on the device; "
                  "steps alternate between two streams",
           "me_identical_to_device_step": e2e_same}
    del wss

    # roofline of the dominant kernel (SIGMAKIN): FP32 CUDA-core arithmetic.
    # Algorithmic flops per event of the helicity-shared kernel: every current
    # variant once per event, then per good helicity its amplitudes and colour sum.
    s = procgen.summary(proc)
    flops_per_me = s["hs_flops_items"] + ngood * (s["hs_flops_amp_hel"] + s["flops_csum_sym"])
    ksec = statistics.mean(kern)
    achieved = flops_per_me * nevt / ksec / 1e12
    peak32 = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    traffic = None
    if args.mode == "mixed" and SIGMAKIN_TRAFFIC["bytes_per_event"] and \
            SIGMAKIN_TRAFFIC["sources_sha1"] == sources_sha1():
        traffic = SIGMAKIN_TRAFFIC["bytes_per_event"] * nevt
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak32, "unit": "TFLOP/s",
                "frac": achieved / peak32, "traffic": traffic,
                "kernel": "sigmakin_hs_kernel<Proc4,%s>" % {"mixed": "float,SIMT", "mixed_simt": "float,SIMT",
                                                            "mixed_tc": "float,TC", "fp64": "double,SIMT"}.get(
                                                                args.mode, args.mode),
                "flops_per_me": flops_per_me,
                "flops_per_me_per_helicity_unshared": s["flops_amp"] + s["flops_csum"],
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.mode != "fp64" else "f64",
        "data": "synthetic (seeded SplitMix64 uniforms -> RAMBO)",
        "config": {"workload": "gg->ttgg tree-level |M|^2, 2^20 events/GPU, RAMBO 4-body at 1500 GeV, "
                               "mt=173 wt=1.491 alpha_s=0.118",
                   "mode": args.mode, "events_per_gpu": nevt, "good_helicities": ngood,
                   "l2": "inputs larger than L2 (336 MiB per step), no flush",
                   "steps": "filter, RAMBO, SIGMAKIN and event sum per step; consecutive steps on two streams",
                   "parallelism": "dp%d (independent event batches)" % world},
        "sigmakin_ms": 1e3 * ksec,
        "fp64": fp64,
        "unrolled": unrolled,
        "tensor_core_colour_sum": tensor_core,
        "kernel_split": kernel_split,
        "other_workloads": others,
        "event_generation": generation,
        "event_sum": [float(x) for x in sums.cpu().numpy()],
        "roofline": roofline,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": kernel_launches_per_step * args.steps,
    }
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rate, dt = cpu_oracle_rate(8192, seed, cores)
        rate1, dt1 = cpu_oracle_rate(512, seed, 1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "8192 gg->ttgg events (RAMBO + |M|^2 over all 64 helicities, "
                                          "explicit colour), FP64, %.1f s wall" % dt,
                                "single_thread": {"value": rate1, "unit": UNIT,
                                                  "sample": "512 events, %.1f s wall" % dt1},
                                "cpu": cpu_model()}
        line["cpu_simd"] = cpu_simd_rates(seed, cores)
        line["rel_err_vs_oracle"] = oracle_error_stats(mg, dev, cores)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
