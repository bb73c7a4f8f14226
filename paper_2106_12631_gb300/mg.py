"""Python binding of the C ABI in include/mg.h (argument marshalling only).

Every computation runs in libmg.so's CUDA kernels; this module checks tensor
shapes, dtypes, devices and contiguity, passes raw pointers and the current
torch stream, and turns status codes into exceptions.  There is no CPU path:
if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

MG_FP64, MG_MIXED, MG_MIXED_SIMT, MG_FP64_UNROLLED, MG_MIXED_UNROLLED, MG_MIXED_TC = 0, 1, 2, 3, 4, 5
MODES = {"fp64": MG_FP64, "mixed": MG_MIXED, "mixed_simt": MG_MIXED_SIMT, "fp64_unrolled": MG_FP64_UNROLLED,
         "mixed_unrolled": MG_MIXED_UNROLLED, "mixed_tc": MG_MIXED_TC}
PROCS = {"ee_mumu": 1, "gg_tt": 2, "gg_ttg": 3, "gg_ttgg": 4}

_lock = threading.Lock()
_lib = None


class MGError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib().mg_status_string(status).decode()
        if status == -5:
            msg += " (cudaError %d)" % lib().mg_last_cuda_error()
        super().__init__("%s: %s" % (what, msg))
        self.status = status


class ProcessInfo(ctypes.Structure):
    _fields_ = [("npar", ctypes.c_int), ("nhel", ctypes.c_int), ("ncolor", ctypes.c_int),
                ("ndiagrams", ctypes.c_int), ("namplitudes", ctypes.c_int), ("nrand", ctypes.c_int),
                ("mass", ctypes.c_double * 8)]


class Params(ctypes.Structure):
    _fields_ = [("mz", ctypes.c_double), ("wz", ctypes.c_double), ("alpha_inv", ctypes.c_double),
                ("sw2", ctypes.c_double), ("mt", ctypes.c_double), ("wt", ctypes.c_double),
                ("alpha_s", ctypes.c_double)]


def lib():
    """Load libmg.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.mg_get_process_info.argtypes = [i32, ctypes.POINTER(ProcessInfo)]
            L.mg_set_params.argtypes = [ctypes.POINTER(Params)]
            L.mg_get_params.argtypes = [ctypes.POINTER(Params)]
            L.mg_rambo.argtypes = [i32, i64, ctypes.c_double, vp, i32, vp, vp, vp]
            L.mg_filter_helicities.argtypes = [i32, i64, vp, vp, vp]
            L.mg_sigmakin.argtypes = [i32, i64, vp, vp, vp, i32, vp]
            L.mg_sigmakin_grad.argtypes = [i32, i64, ctypes.c_double, vp, i32, vp, vp, vp, vp, i32, vp]
            L.mg_event_sum_scratch_bytes.argtypes = [i64]
            L.mg_event_sum_scratch_bytes.restype = i64
            L.mg_event_sum.argtypes = [i64, vp, vp, vp, vp, i64, vp]
            u64 = ctypes.c_uint64
            L.mg_rambo_seeded.argtypes = [i32, i64, ctypes.c_double, u64, i64, vp, vp, vp]
            L.mg_cross_section.argtypes = [i32, ctypes.c_double, vp, vp, vp]
            L.mg_unweight_scratch_bytes.argtypes = [i64]
            L.mg_unweight_scratch_bytes.restype = i64
            L.mg_unweight.argtypes = [i64, vp, vp, u64, i64, vp, vp, vp, i64, vp]
            L.mg_sigmakin_split_workspace_bytes.argtypes = [i32, i32, i64]
            L.mg_sigmakin_split_workspace_bytes.restype = i64
            L.mg_sigmakin_split.argtypes = [i32, i64, vp, vp, i32, vp, vp, i64, vp]
            L.mg_batch_workspace_bytes.argtypes = [i32, i64]
            L.mg_batch_workspace_bytes.restype = i64
            L.mg_matrix_elements_batch.argtypes = [i32, i64, vp, vp, i32, vp, vp, vp, vp, vp, vp, i64, vp]
            L.mg_event_sum_noalloc_max_events.argtypes = []
            L.mg_event_sum_noalloc_max_events.restype = i64
            L.mg_event_sum_noalloc.argtypes = [i64, vp, vp, vp, vp]
            L.mg_pipeline_workspace_bytes.argtypes = [i32, i64, i32]
            L.mg_pipeline_workspace_bytes.restype = i64
            L.mg_pipeline_host.argtypes = [i32, i64, ctypes.c_double, vp, i32, vp, i32, vp, vp, vp, vp, i64, vp]
            L.mg_sigmakin_rambo.argtypes = [i32, i64, ctypes.c_double, vp, i32, vp, i32, vp, vp, vp]
            L.mg_sigmakin_seeded.argtypes = [i32, i64, ctypes.c_double, u64, i64, vp, i32, vp, vp, vp]
            L.mg_status_string.argtypes = [i32]
            L.mg_status_string.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise MGError(status, what)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, name: str, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t.data_ptr()


def _ws(t: torch.Tensor):
    """(device pointer, bytes) of a caller workspace tensor."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("workspace must be a contiguous CUDA tensor")
    return t.data_ptr(), t.numel() * t.element_size()


def _proc(proc) -> int:
    return PROCS[proc] if isinstance(proc, str) else int(proc)


def process_info(proc) -> dict:
    info = ProcessInfo()
    _check(lib().mg_get_process_info(_proc(proc), ctypes.byref(info)), "mg_get_process_info")
    return {"npar": info.npar, "nhel": info.nhel, "ncolor": info.ncolor, "ndiagrams": info.ndiagrams,
            "namplitudes": info.namplitudes, "nrand": info.nrand, "mass": list(info.mass)[: info.npar]}


def get_params() -> dict:
    p = Params()
    _check(lib().mg_get_params(ctypes.byref(p)), "mg_get_params")
    return {k: getattr(p, k) for k, _ in Params._fields_}


def set_params(**kw):
    d = get_params()
    d.update(kw)
    _check(lib().mg_set_params(ctypes.byref(Params(**d))), "mg_set_params")


def rambo(proc, rnd: torch.Tensor, ecm: float, mom=None, wgt=None, stream=None):
    """rnd (nrows, nevt) float64 CUDA -> (mom (npar, 4, nevt), wgt (nevt,))."""
    p = _proc(proc)
    nrows, nevt = rnd.shape
    npar = process_info(p)["npar"]
    if mom is None:
        mom = torch.empty((npar, 4, nevt), dtype=torch.float64, device=rnd.device)
    if wgt is None:
        wgt = torch.empty((nevt,), dtype=torch.float64, device=rnd.device)
    _check(lib().mg_rambo(p, nevt, float(ecm), _dev(rnd, torch.float64, "rnd"), nrows,
                          _dev(mom, torch.float64, "mom", (npar, 4, nevt)),
                          _dev(wgt, torch.float64, "wgt", (nevt,)), _stream(stream)), "mg_rambo")
    return mom, wgt


def rambo_seeded(proc, nevt: int, ecm: float, seed: int, first_event: int = 0, mom=None, wgt=None, device=None,
                 stream=None):
    """RAMBO with the uniforms drawn on the device (counter-based, as inputs.uniforms)."""
    p = _proc(proc)
    npar = process_info(p)["npar"]
    dev = device if device is not None else (mom.device if mom is not None else torch.device("cuda"))
    if mom is None:
        mom = torch.empty((npar, 4, nevt), dtype=torch.float64, device=dev)
    if wgt is None:
        wgt = torch.empty((nevt,), dtype=torch.float64, device=dev)
    _check(lib().mg_rambo_seeded(p, nevt, float(ecm), seed & 0xFFFFFFFFFFFFFFFF, first_event,
                                 _dev(mom, torch.float64, "mom", (npar, 4, nevt)),
                                 _dev(wgt, torch.float64, "wgt", (nevt,)), _stream(stream)), "mg_rambo_seeded")
    return mom, wgt


def cross_section(proc, ecm: float, sums: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """(sigma, error) in pb on the device from the event sums of mg_event_sum."""
    if out is None:
        out = torch.empty((2,), dtype=torch.float64, device=sums.device)
    _check(lib().mg_cross_section(_proc(proc), float(ecm), _dev(sums, torch.float64, "sums", (3,)),
                                  _dev(out, torch.float64, "out", (2,)), _stream(stream)), "mg_cross_section")
    return out


def unweight_scratch_bytes(nevt: int) -> int:
    return int(lib().mg_unweight_scratch_bytes(nevt))


def unweight(me: torch.Tensor, wgt: torch.Tensor, seed: int, first_event: int = 0, idx=None, count=None,
             scratch=None, stream=None):
    """Hit-or-miss unweighting: (idx (nevt,) int64 with the kept indices first, count (1,) int64)."""
    nevt = me.shape[0]
    if idx is None:
        idx = torch.empty((max(nevt, 1),), dtype=torch.int64, device=me.device)
    if idx.numel() < nevt:
        raise ValueError("idx must hold nevt entries")
    if count is None:
        count = torch.empty((1,), dtype=torch.int64, device=me.device)
    nb = unweight_scratch_bytes(nevt)
    if scratch is None:
        scratch = torch.empty((max(nb, 16) + 7) // 8, dtype=torch.float64, device=me.device)
    _check(lib().mg_unweight(nevt, _dev(me, torch.float64, "me", (nevt,)), _dev(wgt, torch.float64, "wgt", (nevt,)),
                             seed & 0xFFFFFFFFFFFFFFFF, first_event, _dev(idx, torch.int64, "idx"),
                             _dev(count, torch.int64, "count", (1,)), scratch.data_ptr(),
                             scratch.numel() * scratch.element_size(), _stream(stream)), "mg_unweight")
    return idx, count


def batch_workspace_bytes(proc, nevt: int) -> int:
    return int(lib().mg_batch_workspace_bytes(_proc(proc), nevt))


def matrix_elements_batch(proc, mom_aos: torch.Tensor, mask: torch.Tensor, mode="mixed", hel_rnd=None, col_rnd=None,
                          me=None, hel=None, col=None, workspace=None, stream=None):
    """mom_aos (nevt, npar, 4) float64 CUDA -> me (nevt,), or (me, hel, col) when hel_rnd or
    col_rnd (nevt,) uniforms are given (a choice not asked for is None)."""
    p = _proc(proc)
    nevt, npar = mom_aos.shape[0], process_info(p)["npar"]
    if me is None:
        me = torch.empty((nevt,), dtype=torch.float64, device=mom_aos.device)
    if hel_rnd is not None and hel is None:
        hel = torch.empty((nevt,), dtype=torch.int32, device=mom_aos.device)
    if col_rnd is not None and col is None:
        col = torch.empty((nevt,), dtype=torch.int32, device=mom_aos.device)
    nb = batch_workspace_bytes(p, nevt)
    if workspace is None:
        workspace = torch.empty(((max(nb, 16) + 7) // 8,), dtype=torch.float64, device=mom_aos.device)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    opt = lambda t, dt, name: _dev(t, dt, name, (nevt,)) if t is not None else None
    _check(lib().mg_matrix_elements_batch(
        p, nevt, _dev(mom_aos, torch.float64, "mom_aos", (nevt, npar, 4)),
        _dev(mask, torch.int32, "mask", (process_info(p)["nhel"],)), m,
        opt(hel_rnd, torch.float64, "hel_rnd"), opt(col_rnd, torch.float64, "col_rnd"),
        _dev(me, torch.float64, "me", (nevt,)), opt(hel, torch.int32, "hel"), opt(col, torch.int32, "col"),
        *_ws(workspace), _stream(stream)),
        "mg_matrix_elements_batch")
    if hel_rnd is None and col_rnd is None:
        return me
    return me, hel, col


def sigmakin_split_workspace_bytes(proc, mode, nevt: int) -> int:
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    return int(lib().mg_sigmakin_split_workspace_bytes(_proc(proc), m, nevt))


def sigmakin_split(proc, mom: torch.Tensor, mask: torch.Tensor, mode="mixed_simt", me=None, workspace=None,
                   stream=None) -> torch.Tensor:
    """The kernel-split variant of sigmakin (currents, then amplitudes, per chunk, in a CUDA graph)."""
    p = _proc(proc)
    nevt = mom.shape[2]
    if me is None:
        me = torch.empty((nevt,), dtype=torch.float64, device=mom.device)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    if workspace is None:
        nb = max(sigmakin_split_workspace_bytes(p, m, nevt), 16)
        workspace = torch.empty(((nb + 7) // 8,), dtype=torch.float64, device=mom.device)
    info = process_info(p)
    _check(lib().mg_sigmakin_split(p, nevt, _dev(mom, torch.float64, "mom", (info["npar"], 4, nevt)),
                                   _dev(mask, torch.int32, "mask", (info["nhel"],)), m,
                                   _dev(me, torch.float64, "me", (nevt,)), *_ws(workspace), _stream(stream)),
           "mg_sigmakin_split")
    return me


def filter_helicities(proc, mom: torch.Tensor, mask=None, stream=None) -> torch.Tensor:
    p = _proc(proc)
    info = process_info(p)
    if mask is None:
        mask = torch.empty((info["nhel"],), dtype=torch.int32, device=mom.device)
    nevt = mom.shape[2]
    _check(lib().mg_filter_helicities(p, nevt, _dev(mom, torch.float64, "mom", (info["npar"], 4, nevt)),
                                      _dev(mask, torch.int32, "mask", (info["nhel"],)), _stream(stream)),
           "mg_filter_helicities")
    return mask


def sigmakin(proc, mom: torch.Tensor, mask: torch.Tensor, mode="mixed", me=None, stream=None) -> torch.Tensor:
    p = _proc(proc)
    info = process_info(p)
    nevt = mom.shape[2]
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    if me is None:
        me = torch.empty((nevt,), dtype=torch.float64, device=mom.device)
    _check(lib().mg_sigmakin(p, nevt, _dev(mom, torch.float64, "mom", (info["npar"], 4, nevt)),
                             _dev(mask, torch.int32, "mask", (info["nhel"],)),
                             _dev(me, torch.float64, "me", (nevt,)), m, _stream(stream)), "mg_sigmakin")
    return me


def _me_wgt(nevt, device, me, wgt):
    if me is None:
        me = torch.empty((nevt,), dtype=torch.float64, device=device)
    if wgt is None:
        wgt = torch.empty((nevt,), dtype=torch.float64, device=device)
    return me, wgt


def sigmakin_rambo(proc, rnd: torch.Tensor, ecm: float, mask: torch.Tensor, mode="mixed", me=None, wgt=None,
                   stream=None):
    """RAMBO and SIGMAKIN in one kernel: rnd (nrows, nevt) float64 CUDA -> (me, wgt),
    equal to rambo() followed by sigmakin()."""
    p = _proc(proc)
    nrows, nevt = rnd.shape
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    me, wgt = _me_wgt(nevt, rnd.device, me, wgt)
    _check(lib().mg_sigmakin_rambo(p, nevt, float(ecm), _dev(rnd, torch.float64, "rnd"), nrows,
                                   _dev(mask, torch.int32, "mask", (process_info(p)["nhel"],)), m,
                                   _dev(me, torch.float64, "me", (nevt,)), _dev(wgt, torch.float64, "wgt", (nevt,)),
                                   _stream(stream)), "mg_sigmakin_rambo")
    return me, wgt


def sigmakin_seeded(proc, nevt: int, ecm: float, seed: int, mask: torch.Tensor, mode="mixed", first_event: int = 0,
                    me=None, wgt=None, stream=None):
    """RAMBO with device-drawn uniforms and SIGMAKIN in one kernel -> (me, wgt),
    equal to rambo_seeded() followed by sigmakin()."""
    p = _proc(proc)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    me, wgt = _me_wgt(nevt, mask.device, me, wgt)
    _check(lib().mg_sigmakin_seeded(p, nevt, float(ecm), seed & 0xFFFFFFFFFFFFFFFF, first_event,
                                    _dev(mask, torch.int32, "mask", (process_info(p)["nhel"],)), m,
                                    _dev(me, torch.float64, "me", (nevt,)), _dev(wgt, torch.float64, "wgt", (nevt,)),
                                    _stream(stream)), "mg_sigmakin_seeded")
    return me, wgt


def sigmakin_grad(proc, rnd: torch.Tensor, ecm: float, mask: torch.Tensor, mode="mixed", gout=None, grad=None,
                  me=None, stream=None):
    """d me / d rnd (times gout) for every event: (grad (nrows, nevt), me (nevt,))."""
    p = _proc(proc)
    nrows, nevt = rnd.shape
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    if grad is None:
        grad = torch.empty((nrows, nevt), dtype=torch.float64, device=rnd.device)
    if me is None:
        me = torch.empty((nevt,), dtype=torch.float64, device=rnd.device)
    g = _dev(gout, torch.float64, "gout", (nevt,)) if gout is not None else None
    _check(lib().mg_sigmakin_grad(p, nevt, float(ecm), _dev(rnd, torch.float64, "rnd"), nrows,
                                  _dev(mask, torch.int32, "mask", (process_info(p)["nhel"],)), g,
                                  _dev(grad, torch.float64, "grad", (nrows, nevt)),
                                  _dev(me, torch.float64, "me", (nevt,)), m, _stream(stream)), "mg_sigmakin_grad")
    return grad, me


class MatrixElement(torch.autograd.Function):
    """me = SIGMAKIN(RAMBO(rnd)) with a backward pass through the adjoint kernel.

    forward(rnd (nrows, nevt) float64 CUDA, proc, ecm, mask, mode) -> me (nevt,)
    backward: grad_rnd = grad_me * d me / d rnd (mg_sigmakin_grad)."""

    @staticmethod
    def forward(ctx, rnd, proc, ecm, mask, mode="mixed"):
        mom, _ = rambo(proc, rnd.contiguous(), ecm)
        me = sigmakin(proc, mom, mask, mode=mode)
        ctx.save_for_backward(rnd, mask)
        ctx.args = (proc, ecm, mode)
        return me

    @staticmethod
    def backward(ctx, grad_me):
        rnd, mask = ctx.saved_tensors
        proc, ecm, mode = ctx.args
        grad, _ = sigmakin_grad(proc, rnd.contiguous(), ecm, mask, mode=mode,
                                gout=grad_me.contiguous().to(torch.float64))
        return grad, None, None, None, None


def matrix_element(rnd: torch.Tensor, proc, ecm: float, mask: torch.Tensor, mode="mixed") -> torch.Tensor:
    """Differentiable me(rnd) (see MatrixElement)."""
    return MatrixElement.apply(rnd, proc, ecm, mask, mode)


def event_sum_scratch_bytes(nevt: int) -> int:
    return int(lib().mg_event_sum_scratch_bytes(nevt))


def event_sum(me: torch.Tensor, wgt: torch.Tensor, out=None, scratch=None, stream=None) -> torch.Tensor:
    nevt = me.shape[0]
    if out is None:
        out = torch.empty((3,), dtype=torch.float64, device=me.device)
    nb = event_sum_scratch_bytes(nevt)
    if scratch is None:
        scratch = torch.empty((max(nb, 16) + 7) // 8, dtype=torch.float64, device=me.device)
    _check(lib().mg_event_sum(nevt, _dev(me, torch.float64, "me", (nevt,)),
                              _dev(wgt, torch.float64, "wgt", (nevt,)), _dev(out, torch.float64, "out", (3,)),
                              scratch.data_ptr(), scratch.numel() * scratch.element_size(), _stream(stream)),
           "mg_event_sum")
    return out


def event_sum_noalloc(me: torch.Tensor, wgt: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """event_sum without caller scratch (fixed library-owned array; see include/mg.h)."""
    nevt = me.shape[0]
    if out is None:
        out = torch.empty((3,), dtype=torch.float64, device=me.device)
    _check(lib().mg_event_sum_noalloc(nevt, _dev(me, torch.float64, "me", (nevt,)),
                                      _dev(wgt, torch.float64, "wgt", (nevt,)),
                                      _dev(out, torch.float64, "out", (3,)), _stream(stream)),
           "mg_event_sum_noalloc")
    return out


def pipeline_workspace_bytes(proc, nevt: int, nrows: int) -> int:
    return int(lib().mg_pipeline_workspace_bytes(_proc(proc), nevt, nrows))


def pipeline_host(proc, rnd_host: torch.Tensor, ecm: float, mask: torch.Tensor, mode="mixed", me_host=None,
                  wgt_host=None, sums_host=None, workspace=None, stream=None):
    """Host random numbers -> (H2D) RAMBO -> SIGMAKIN -> (D2H) host me (and wgt, and the
    event sum into sums_host[3] if given).  Async on the stream; synchronise before reading
    the host buffers.  rnd_host should be pinned."""
    p = _proc(proc)
    if rnd_host.is_cuda or rnd_host.dtype != torch.float64 or not rnd_host.is_contiguous():
        raise ValueError("rnd_host must be a contiguous float64 CPU tensor")
    nrows, nevt = rnd_host.shape
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    if me_host is None:
        me_host = torch.empty((nevt,), dtype=torch.float64, pin_memory=True)
    for t, name, n in ((me_host, "me_host", nevt), (wgt_host, "wgt_host", nevt), (sums_host, "sums_host", 3)):
        if t is not None and (t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n):
            raise ValueError("%s must be a contiguous float64 CPU tensor of %d values" % (name, n))
    nb = pipeline_workspace_bytes(p, nevt, nrows)
    if workspace is None:
        workspace = torch.empty(((nb + 7) // 8,), dtype=torch.float64, device=mask.device)
    _check(lib().mg_pipeline_host(p, nevt, float(ecm), rnd_host.data_ptr(), nrows,
                                  _dev(mask, torch.int32, "mask", (process_info(p)["nhel"],)), m,
                                  me_host.data_ptr(),
                                  wgt_host.data_ptr() if wgt_host is not None else None,
                                  sums_host.data_ptr() if sums_host is not None else None,
                                  *_ws(workspace),
                                  _stream(stream)), "mg_pipeline_host")
    return me_host


def library_path() -> str:
    return os.path.abspath(_build.LIB)
