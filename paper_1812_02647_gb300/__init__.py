"""Python binding of the GB300 harmonic-sum library (``include/harmonic_sum.h``).

Argument marshalling only: every step of the harmonic sum runs in the library's CUDA kernels.
PyTorch supplies device memory and the current stream.  The module-level ``hs_*`` functions mirror
the C entry points one to one; ``HarmonicSum`` and ``HarmonicSumFn`` are conveniences on top.

Importing builds the library in place if it is missing or stale (nvcc required) and raises if it
cannot be built or loaded: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

STD, MAX, FBIN, GREEDY = 1, 2, 4, 8
VARIANTS = {"std": STD, "max": MAX, "fbin": FBIN, "greedy": GREEDY}
VARIANT_NAMES = {v: k for k, v in VARIANTS.items()}
F32, F16, BF16 = 0, 1, 2
DTYPE_NAMES = {F32: "f32", F16: "f16", BF16: "bf16"}
FLAG_OUT_ALL_H = 1
FLAG_STAGED_SPANS = 2
FLAG_MAX_WINDOW0 = 4
FLAG_POW2_STAGES = 8
FLAG_GREEDY_FIXED1 = 16
FLAG_CHECK_TIMEOUT = 32
HMAX_1D, HMAX_2D = 32, 16

OK, ERR_INVALID, ERR_ALIGN, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, 1, 2, 3, 4, 5, 6
WARN_CAND_OVERFLOW = 100

CANDIDATE_DTYPE = np.dtype([("spectrum", "<u4"), ("bin", "<u4"), ("snr", "<f4"), ("z", "<i2"), ("h", "u1"),
                            ("variant", "u1")])

_P = ctypes.c_void_p


class PlanDesc(ctypes.Structure):
    _fields_ = [("variants", ctypes.c_int), ("hmax", ctypes.c_int), ("dtype", ctypes.c_int),
                ("max_bins", ctypes.c_int64), ("nz", ctypes.c_int), ("z_min", ctypes.c_int),
                ("threshold", ctypes.c_float), ("cand_capacity", ctypes.c_int64), ("flags", ctypes.c_int)]


class Out(ctypes.Structure):
    _fields_ = [("best_snr", _P), ("best_h", _P), ("path", _P), ("all_h", _P), ("cand", _P), ("cand_count", _P)]


class Out2d(ctypes.Structure):
    _fields_ = [("best_snr", _P), ("best_h", _P), ("best_snr_n", _P), ("best_h_n", _P), ("best_z_n", _P),
                ("cand", _P), ("cand_count", _P)]


class HSError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__("%s%s" % (where + ": " if where else "", hs_status_string(status)))


def _load():
    path = _build.build()
    lib = ctypes.CDLL(path)
    I, I64, U32, SZ = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
    sig = {
        "hs_status_string": ([I], ctypes.c_char_p),
        "hs_version": ([], I),
        "hs_plan_create": ([ctypes.POINTER(_P), ctypes.POINTER(PlanDesc)], I),
        "hs_plan_destroy": ([_P], I),
        "hs_plan_set_calibration": ([_P, I, _P, _P], I),
        "hs_noise_calibration": ([I, I, _P, _P], I),
        "hs_noise_calibration_flags": ([I, I, I, _P, _P], I),
        "hs_plan_workspace_size": ([_P, I, ctypes.POINTER(SZ)], I),
        "hs_workspace_init": ([_P, _P, SZ, _P], I),
        "hs_sum_1d": ([_P, I, _P, I64, U32, ctypes.POINTER(Out), _P, SZ, _P], I),
        "hs_sum_batched": ([_P, I, _P, _P, I, U32, ctypes.POINTER(Out), _P, SZ, _P], I),
        "hs_sum_2d": ([_P, _P, I64, I64, U32, ctypes.POINTER(Out2d), _P, SZ, _P], I),
        "hs_sum_2d_variant": ([_P, I, _P, I64, I64, U32, ctypes.POINTER(Out2d), _P, SZ, _P], I),
        "hs_backward": ([_P, I, _P, _P, I, I64, _P, _P, _P, _P, _P], I),
        "hs_standardize_cast": ([_P, _P, I, I64, _P, _P, I, _P, _P], I),
        "hs_power_normalize": ([_P, _P, _P, I, I64, I, _P, I64, _P, _P, SZ, _P], I),
        "hs_sift_candidates": ([_P, _P, I64, ctypes.c_float, ctypes.c_float, I, _P, _P, _P, _P, SZ, _P], I),
        "hs_sort_candidates": ([_P, _P, I64, _P, _P, SZ, _P], I),
        "hs_graph_create_batched": ([_P, I, _P, _P, I, U32, _P, _P, SZ, _P, ctypes.POINTER(_P)], I),
        "hs_graph_launch": ([_P, _P], I),
        "hs_graph_destroy": ([_P], I),
        "hs_autotune": ([_P, I, I64, _P, SZ, _P, SZ, _P], I),
        "hs_sync_status": ([_P, _P, _P], I),
        "hs_sum_batched_host": ([_P, I, _P, _P, I, U32, _P, _P, _P, I, _P, SZ, _P], I),
        "hs_autotune_batched": ([_P, I, _P, _P, I, ctypes.POINTER(Out), _P, SZ, _P], I),
        "hs_plan_tile_bins": ([_P, I], I),
        "hs_plan_set_tile_bins": ([_P, I, I], I),
        "hs_plan_ctas_per_sm": ([_P, I], I),
        "hs_plan_set_ctas_per_sm": ([_P, I, I], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()
LIBRARY_PATH = _build.LIB


def hs_status_string(status: int) -> str:
    return _lib.hs_status_string(int(status)).decode()


def _check(status: int, where: str, allow=(OK,)):
    if status not in allow:
        raise HSError(status, where)
    return status


def _variant(v) -> int:
    return VARIANTS[v] if isinstance(v, str) else int(v)


def _dtype_code(t) -> int:
    import torch

    return {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}[t]


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# Storage type of each live plan, by handle.  The C calls take the spectra as a bare pointer and read
# them as the plan's type, so a tensor of another type would be read past its end.
_plan_dtype = {}


def _spectra(plan, x, rows=False):
    """Pointer to input spectra after checking them against the plan: the plan's storage type and
    contiguous elements (contiguous rows for a 2-D plane, whose row stride is passed separately);
    a mismatch is an error, not a read of the wrong bytes."""
    want = _plan_dtype.get(getattr(plan, "value", None))
    try:
        got = _dtype_code(x.dtype)
    except KeyError:
        got = None
    dense = x.stride(-1) == 1 if rows else x.is_contiguous()
    if (want is not None and got != want) or not dense:
        raise HSError(ERR_INVALID, "input spectra (%s%s) do not match the plan's storage type %s"
                      % (x.dtype, "" if dense else ", not contiguous", DTYPE_NAMES.get(want, want)))
    return _ptr(x)


def _offsets(offsets):
    """Pointer to a batch's int64 spectrum offsets (checked: another integer type would be misread)."""
    import torch

    if offsets is None:
        return None
    if offsets.dtype != torch.int64 or not offsets.is_contiguous():
        raise HSError(ERR_INVALID, "spectrum offsets must be a contiguous int64 tensor, got %s" % offsets.dtype)
    return _ptr(offsets)


def _stream(stream=None):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# ----------------------------------------------------------------------------------------------
# one-to-one wrappers of the C entry points
# ----------------------------------------------------------------------------------------------

def hs_plan_create(variants=0xF, hmax=32, dtype=F32, max_bins=1 << 22, nz=0, z_min=0, threshold=6.0,
                   cand_capacity=0, flags=0):
    d = PlanDesc(int(variants), int(hmax), int(dtype), int(max_bins), int(nz), int(z_min), float(threshold),
                 int(cand_capacity), int(flags))
    h = _P()
    _check(_lib.hs_plan_create(ctypes.byref(h), ctypes.byref(d)), "hs_plan_create")
    _plan_dtype[h.value] = int(dtype)
    return h, d


def hs_plan_destroy(plan):
    _plan_dtype.pop(getattr(plan, "value", None), None)
    return _lib.hs_plan_destroy(plan)


def hs_plan_set_calibration(plan, variant, mu=None, isig=None):
    mu = None if mu is None else np.ascontiguousarray(mu, np.float32)
    isig = None if isig is None else np.ascontiguousarray(isig, np.float32)
    _check(_lib.hs_plan_set_calibration(plan, _variant(variant), None if mu is None else mu.ctypes.data,
                                        None if isig is None else isig.ctypes.data), "hs_plan_set_calibration")


def hs_noise_calibration(variant, hmax=32, flags=0):
    mu = np.empty(hmax + 1, np.float32)
    isig = np.empty(hmax + 1, np.float32)
    if flags:
        _check(_lib.hs_noise_calibration_flags(_variant(variant), hmax, int(flags), mu.ctypes.data, isig.ctypes.data),
               "hs_noise_calibration_flags")
    else:
        _check(_lib.hs_noise_calibration(_variant(variant), hmax, mu.ctypes.data, isig.ctypes.data),
               "hs_noise_calibration")
    return mu, isig


def hs_plan_workspace_size(plan, n_spectra=1) -> int:
    b = ctypes.c_size_t()
    _check(_lib.hs_plan_workspace_size(plan, int(n_spectra), ctypes.byref(b)), "hs_plan_workspace_size")
    return b.value


def hs_workspace_init(plan, ws, stream=None):
    _check(_lib.hs_workspace_init(plan, _ptr(ws), ws.numel(), _stream(stream)), "hs_workspace_init")


def _out(best_snr, best_h, path=None, all_h=None, cand=None, cand_count=None):
    return Out(best_snr.data_ptr(), best_h.data_ptr(), None if path is None else path.data_ptr(),
               None if all_h is None else all_h.data_ptr(), None if cand is None else cand.data_ptr(),
               None if cand_count is None else cand_count.data_ptr())


def hs_sum_1d(plan, variant, x, out: Out, ws, spectrum_id=0, stream=None):
    return _check(_lib.hs_sum_1d(plan, _variant(variant), _spectra(plan, x), x.numel(), spectrum_id,
                                 ctypes.byref(out), _ptr(ws), ws.numel(), _stream(stream)), "hs_sum_1d")


def hs_sum_batched(plan, variant, x, offsets, out: Out, ws, first_id=0, stream=None):
    return _check(_lib.hs_sum_batched(plan, _variant(variant), _spectra(plan, x), _offsets(offsets),
                                      offsets.numel() - 1, first_id, ctypes.byref(out), _ptr(ws), ws.numel(),
                                      _stream(stream)), "hs_sum_batched")


def hs_sum_2d(plan, plane, out: Out2d, ws, plane_id=0, stream=None, variant="std"):
    """2-D sums over a (nz, n_bins) plane: Eq. 1 ("std") or its freq-bin form ("fbin")."""
    nz, nb = plane.shape
    p = _spectra(plan, plane, rows=True)
    if _variant(variant) == STD:
        return _check(_lib.hs_sum_2d(plan, p, nb, plane.stride(0), plane_id, ctypes.byref(out), _ptr(ws),
                                     ws.numel(), _stream(stream)), "hs_sum_2d")
    return _check(_lib.hs_sum_2d_variant(plan, _variant(variant), p, nb, plane.stride(0), plane_id,
                                         ctypes.byref(out), _ptr(ws), ws.numel(), _stream(stream)), "hs_sum_2d_variant")


def hs_backward(plan, variant, x, offsets, grad_snr, best_h, path, grad_x, stream=None):
    n_spec = 1 if offsets is None else offsets.numel() - 1
    return _check(_lib.hs_backward(plan, _variant(variant), _spectra(plan, x), _offsets(offsets), n_spec, x.numel(),
                                   _ptr(grad_snr), _ptr(best_h), _ptr(path), _ptr(grad_x), _stream(stream)),
                  "hs_backward")


def hs_standardize_cast(p, offsets, mu, sigma, dst_dtype, out, stream=None):
    n_spec = 1 if offsets is None else offsets.numel() - 1
    n_bins = p.numel() if offsets is None else 0
    if offsets is not None:
        n_bins = int(offsets.diff().max().item()) if n_spec > 0 else 0
    return _check(_lib.hs_standardize_cast(_ptr(p), _ptr(offsets), n_spec, n_bins, _ptr(mu), _ptr(sigma),
                                           int(dst_dtype), _ptr(out), _stream(stream)), "hs_standardize_cast")


def hs_sort_candidates(cand, cand_count, tmp, ws, stream=None):
    cap = cand.numel() // 16
    return _check(_lib.hs_sort_candidates(_ptr(cand), _ptr(cand_count), cap, _ptr(tmp), _ptr(ws), ws.numel(),
                                          _stream(stream)), "hs_sort_candidates")


def hs_power_normalize(plan, spec, offsets, n_bins, block, medians, out, ws, stream=None):
    """Power of complex spectra (``spec``: float32 pairs re, im, or complex64), dereddened by block
    medians and standardised into ``out`` (the plan's dtype).  ``offsets`` None: one spectrum of
    ``n_bins`` complex bins."""
    n_spectra = 1 if offsets is None else offsets.numel() - 1
    return _check(_lib.hs_power_normalize(plan, _ptr(spec), _ptr(offsets), n_spectra, int(n_bins), int(block),
                                          _ptr(medians), medians.numel(), _ptr(out), _ptr(ws), ws.numel(),
                                          _stream(stream)), "hs_power_normalize")


def hs_sift_candidates(cand, cand_count, out, out_count, tmp, ws, tol_bins=1.5, tol_z=1.5, kmax=8, stream=None):
    """Drop every candidate of a sorted list to which a stronger candidate of its (variant, spectrum)
    group is harmonically related or adjacent; the kept ones go to ``out`` (sorted), their number to
    ``out_count``."""
    cap = cand.numel() // 16
    return _check(_lib.hs_sift_candidates(_ptr(cand), _ptr(cand_count), cap, float(tol_bins), float(tol_z), int(kmax),
                                          _ptr(out), _ptr(out_count), _ptr(tmp), _ptr(ws), ws.numel(),
                                          _stream(stream)), "hs_sift_candidates")


def hs_graph_create_batched(plan, variant_mask, x, offsets, outs, ws, first_id=0, stream=None):
    arr = (Out * len(outs))(*outs)
    g = _P()
    _check(_lib.hs_graph_create_batched(plan, int(variant_mask), _spectra(plan, x), _offsets(offsets),
                                        offsets.numel() - 1, first_id, ctypes.cast(arr, _P), _ptr(ws), ws.numel(),
                                        _stream(stream), ctypes.byref(g)), "hs_graph_create_batched")
    return g


def hs_sum_batched_host(plan, variant_mask, x_host, offsets_host, x_dev, offsets_dev, outs, ws, n_chunks=8,
                        first_id=0, stream=None):
    """A pinned host batch streamed to the device in pieces, copies overlapping the sums.
    ``x_host`` is a pinned torch tensor, ``offsets_host`` a numpy int64 array (starting at 0)."""
    offs = np.ascontiguousarray(offsets_host, dtype=np.int64)
    arr = (Out * len(outs))(*outs)
    return _check(_lib.hs_sum_batched_host(plan, int(variant_mask), _spectra(plan, x_host),
                                           offs.ctypes.data, len(offs) - 1, first_id, _spectra(plan, x_dev),
                                           _offsets(offsets_dev),
                                           ctypes.cast(arr, _P), int(n_chunks), _ptr(ws), ws.numel(),
                                           _stream(stream)), "hs_sum_batched_host")


def hs_graph_launch(graph, stream=None):
    return _check(_lib.hs_graph_launch(graph, _stream(stream)), "hs_graph_launch")


def hs_graph_destroy(graph):
    return _lib.hs_graph_destroy(graph)


def hs_autotune(plan, variant, n_bins, scratch, ws, stream=None):
    return _check(_lib.hs_autotune(plan, _variant(variant), int(n_bins), _ptr(scratch), scratch.numel(), _ptr(ws),
                                   ws.numel(), _stream(stream)), "hs_autotune")


def hs_autotune_batched(plan, variant, x, offsets, out: Out, ws, stream=None):
    return _check(_lib.hs_autotune_batched(plan, _variant(variant), _spectra(plan, x), _offsets(offsets),
                                           offsets.numel() - 1, ctypes.byref(out), _ptr(ws), ws.numel(),
                                           _stream(stream)), "hs_autotune_batched")


def hs_plan_tile_bins(plan, variant) -> int:
    return _lib.hs_plan_tile_bins(plan, _variant(variant))


def hs_plan_set_tile_bins(plan, variant, tile_bins):
    return _check(_lib.hs_plan_set_tile_bins(plan, _variant(variant), int(tile_bins)), "hs_plan_set_tile_bins")


def hs_plan_ctas_per_sm(plan, variant) -> int:
    return _lib.hs_plan_ctas_per_sm(plan, _variant(variant))


def hs_plan_set_ctas_per_sm(plan, variant, ctas_per_sm):
    """Cap a variant's persistent batched launch at ctas_per_sm CTAs per SM (0: as many as fit), so
    that launches on other streams can run beside it."""
    return _check(_lib.hs_plan_set_ctas_per_sm(plan, _variant(variant), int(ctas_per_sm)),
                  "hs_plan_set_ctas_per_sm")


def hs_sync_status(plan, ws, stream=None) -> int:
    return _check(_lib.hs_sync_status(plan, _ptr(ws), _stream(stream)), "hs_sync_status",
                  allow=(OK, WARN_CAND_OVERFLOW))


def hs_version() -> int:
    return _lib.hs_version()


# ----------------------------------------------------------------------------------------------
# convenience layer
# ----------------------------------------------------------------------------------------------

class HarmonicSum:
    """A plan plus its workspace.  ``sum_1d`` / ``sum_batched`` / ``sum_2d`` allocate outputs as
    torch tensors on the input's device and return them in a dict."""

    def __init__(self, variants=0xF, hmax=32, dtype=F32, max_bins=1 << 22, nz=0, z_min=0, threshold=6.0,
                 cand_capacity=0, flags=0, max_spectra=1, calibration=None):
        import torch

        self.plan, self.desc = hs_plan_create(variants, hmax, dtype, max_bins, nz, z_min, threshold, cand_capacity,
                                              flags)
        self.hmax, self.nz, self.z_min, self.cand_capacity = hmax, nz, z_min, cand_capacity
        self.ws_bytes = hs_plan_workspace_size(self.plan, max_spectra)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        hs_workspace_init(self.plan, self.ws)
        if calibration:
            for v, (mu, isig) in calibration.items():
                hs_plan_set_calibration(self.plan, v, mu, isig)

    def __del__(self):
        try:
            hs_plan_destroy(self.plan)
        except Exception:
            pass

    def set_calibration(self, variant, mu=None, isig=None):
        hs_plan_set_calibration(self.plan, variant, mu, isig)

    def ensure_workspace(self, n_spectra):
        import torch

        need = hs_plan_workspace_size(self.plan, n_spectra)
        if need > self.ws.numel():
            self.ws = torch.empty(need, dtype=torch.uint8, device="cuda")
            hs_workspace_init(self.plan, self.ws)

    def new_outputs(self, n_bins, variant, device, path=True, all_h=False, candidates=True):
        import torch

        o = {"best_snr": torch.empty(n_bins, dtype=torch.float32, device=device),
             "best_h": torch.empty(n_bins, dtype=torch.uint8, device=device)}
        if path and _variant(variant) == GREEDY:
            o["path"] = torch.empty(n_bins, dtype=torch.int32, device=device)
        if all_h:
            o["all_h"] = torch.empty((self.hmax, n_bins), dtype=torch.float32, device=device)
        if candidates and self.cand_capacity > 0:
            o["cand"] = torch.empty(self.cand_capacity * 16, dtype=torch.uint8, device=device)
            o["cand_count"] = torch.zeros(1, dtype=torch.int64, device=device)
        return o

    @staticmethod
    def out_struct(o) -> Out:
        return _out(o["best_snr"], o["best_h"], o.get("path"), o.get("all_h"), o.get("cand"), o.get("cand_count"))

    def sum_1d(self, variant, x, spectrum_id=0, all_h=False, out=None, stream=None):
        o = out or self.new_outputs(x.numel(), variant, x.device, all_h=all_h)
        hs_sum_1d(self.plan, variant, x, self.out_struct(o), self.ws, spectrum_id, stream)
        return o

    def sum_batched(self, variant, x, offsets, first_id=0, out=None, stream=None):
        self.ensure_workspace(offsets.numel() - 1)
        o = out or self.new_outputs(x.numel(), variant, x.device)
        hs_sum_batched(self.plan, variant, x, offsets, self.out_struct(o), self.ws, first_id, stream)
        return o

    def sum_2d(self, plane, plane_id=0, out=None, stream=None, variant="std"):
        import torch

        nz, nb = plane.shape
        dev = plane.device
        o = out or {"best_snr": torch.empty((nz, nb), dtype=torch.float32, device=dev),
                    "best_h": torch.empty((nz, nb), dtype=torch.uint8, device=dev),
                    "best_snr_n": torch.empty(nb, dtype=torch.float32, device=dev),
                    "best_h_n": torch.empty(nb, dtype=torch.uint8, device=dev),
                    "best_z_n": torch.empty(nb, dtype=torch.int16, device=dev)}
        if out is None and self.cand_capacity > 0:
            o["cand"] = torch.empty(self.cand_capacity * 16, dtype=torch.uint8, device=dev)
            o["cand_count"] = torch.zeros(1, dtype=torch.int64, device=dev)
        s = Out2d(o["best_snr"].data_ptr(), o["best_h"].data_ptr(), o["best_snr_n"].data_ptr(),
                  o["best_h_n"].data_ptr(), o["best_z_n"].data_ptr(),
                  o["cand"].data_ptr() if "cand" in o else None,
                  o["cand_count"].data_ptr() if "cand_count" in o else None)
        hs_sum_2d(self.plan, plane, s, self.ws, plane_id, stream, variant=variant)
        return o

    def backward(self, variant, x, grad_snr, best_h, path=None, offsets=None, grad_x=None, stream=None):
        import torch

        g = torch.zeros(x.shape, dtype=torch.float32, device=x.device) if grad_x is None else grad_x
        hs_backward(self.plan, variant, x, offsets, grad_snr, best_h, path, g, stream)
        return g

    def sync_status(self, stream=None) -> int:
        return hs_sync_status(self.plan, self.ws, stream)


def read_candidates(o) -> np.ndarray:
    """Copy the stored candidates of an output dict to the host (unsorted, as appended)."""
    n = int(o["cand_count"].item())
    cap = o["cand"].numel() // 16
    raw = o["cand"][: min(n, cap) * 16].cpu().numpy()
    return raw.view(CANDIDATE_DTYPE)


class HarmonicSumFn:
    """``torch.autograd.Function`` over the best snr of every bin (the best H held fixed in backward)."""

    _fn = None

    @classmethod
    def apply(cls, x, hs: HarmonicSum, variant, offsets=None):
        if cls._fn is None:
            cls._fn = _make_autograd_fn()
        return cls._fn.apply(x, hs, variant, offsets)


def _make_autograd_fn():
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, hs, variant, offsets):
            if offsets is None:
                o = hs.sum_1d(variant, x)
            else:
                o = hs.sum_batched(variant, x, offsets)
            path = o.get("path")
            ctx.save_for_backward(x, o["best_h"], path if path is not None else o["best_h"], offsets
                                  if offsets is not None else o["best_h"])
            ctx.hs, ctx.variant, ctx.has_offsets, ctx.has_path = hs, variant, offsets is not None, path is not None
            ctx.mark_non_differentiable(o["best_h"])
            return o["best_snr"], o["best_h"]

        @staticmethod
        def backward(ctx, g_snr, g_h):
            x, best_h, path, offsets = ctx.saved_tensors
            g = ctx.hs.backward(ctx.variant, x, g_snr.contiguous(), best_h, path if ctx.has_path else None,
                                offsets if ctx.has_offsets else None)
            return g.to(x.dtype), None, None, None

    return _Fn


# ----------------------------------------------------------------------------------------------
# allocation-free batched entry point
# ----------------------------------------------------------------------------------------------
NOALLOC_MAX_SPECTRA = 16384
MAX_CTAS_PER_SM = 8

_lib.hs_sum_batched_noalloc.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(Out),
                                        _P]
_lib.hs_sum_batched_noalloc.restype = ctypes.c_int


def hs_sum_batched_noalloc(plan, variant, x, offsets, out: Out, first_id=0, stream=None):
    """hs_sum_batched without a workspace, for callers that may not allocate device memory while
    they run (the library's own fixed scratch array is used; see include/harmonic_sum.h)."""
    return _check(_lib.hs_sum_batched_noalloc(plan, _variant(variant), _spectra(plan, x), _offsets(offsets),
                                              offsets.numel() - 1, first_id, ctypes.byref(out), _stream(stream)),
                  "hs_sum_batched_noalloc")
