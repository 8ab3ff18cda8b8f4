"""CPU oracle for the incoherent harmonic sum (arXiv:1812.02647, Eq. 1-4) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` / reference legs
may import this package.  It is plain C (``hs_oracle.c``) behind ctypes, built with gcc
``-O2 -ffp-contract=off`` (no FMA contraction, no fast-math) so that its FP32 mode rounds every
operation in the order the definitions are written.  It shares no code with the GPU library.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py`` against closed
forms, brute force, special cases and hand-worked fixtures (``tests/golden``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

STD, MAX, FBIN, GREEDY, MAX0, GREEDY1 = 1, 2, 4, 8, 16, 32
POW2 = 64  # flag bit: search only H = 1, 2, 4, .. (pass pow2=True)
# "max0": Eq. 2 with the window j = 0..i (bins i*n .. i*n+i), a variant flag; "max" is the window as
# written, j = 1..i
# "greedy1": Eq. 4 with the first term fixed at x(n) and the first pair at 2n, a variant flag
VARIANTS = {"std": STD, "max": MAX, "fbin": FBIN, "greedy": GREEDY, "max0": MAX0, "greedy1": GREEDY1}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "hs_oracle.c"), os.path.join(_HERE, "hs_oracle_body.h")]
_LIB = os.path.join(_HERE, "libhs_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle in place with gcc (OpenMP when available)."""
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", _SRCS[0], "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRCS[0], "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.hs_oracle_hvalid.argtypes = [I, I64, I64, I]
        lib.hs_oracle_hvalid.restype = I
        for sfx in ("f32", "f64"):
            getattr(lib, "hs_oracle_1d_" + sfx).argtypes = [I, P, I64, I, P, P, P, P, P, P, I]
            getattr(lib, "hs_oracle_bins_" + sfx).argtypes = [I, P, I64, I, P, P, P, I64, P, P, P]
            getattr(lib, "hs_oracle_2d_cells_" + sfx).argtypes = [P, I, I, I64, I64, I, P, P, P, P, I64, P, P]
            getattr(lib, "hs_oracle_batched_" + sfx).argtypes = [I, P, P, I, I, P, P, P, P, P, I]
            getattr(lib, "hs_oracle_2d_" + sfx).argtypes = [P, I, I, I64, I64, I, P, P, P, P, P, P, P, P, I]
            getattr(lib, "hs_oracle_2d_fbin_" + sfx).argtypes = [P, I, I, I64, I64, I, P, P, P, P, P, P, P, P, I]
            getattr(lib, "hs_oracle_2d_rowwise_" + sfx).argtypes = [I, P, I, I, I64, I64, I, P, P, P, P, P, P, P, P,
                                                                    I]
        lib.hs_oracle_grad_f64.argtypes = [I, P, I64, I, P, P, P, P]
        lib.hs_oracle_standardize_cast.argtypes = [P, I64, ctypes.c_float, ctypes.c_float, I, P]
        lib.hs_oracle_noise_moments.argtypes = [I, I, P, P]
        lib.hs_oracle_power_normalize.argtypes = [P, I64, I, I, P, P]
        lib.hs_oracle_max_threads.restype = I
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _variant(v, pow2=False):
    return (VARIANTS[v] if isinstance(v, str) else int(v)) | (POW2 if pow2 else 0)


def _threads(n):
    return int(n) if n else 1


def max_threads() -> int:
    return _load().hs_oracle_max_threads()


def hvalid(variant, n: int, N: int, hmax: int) -> int:
    return _load().hs_oracle_hvalid(_variant(variant), n, N, hmax)


def _tables(mu, isig, hmax, dt):
    mu = None if mu is None else np.ascontiguousarray(mu, dtype=dt)
    isig = None if isig is None else np.ascontiguousarray(isig, dtype=dt)
    for t in (mu, isig):
        if t is not None and t.shape[0] < hmax + 1:
            raise ValueError("calibration tables need hmax+1 entries")
    return mu, isig


def hs_1d(variant, x, hmax: int = 32, mu=None, isig=None, fp64: bool = False, pow2: bool = False, all_h: bool = False,
          nthreads: int | None = None):
    """Per-bin best snr / H (and the greedy path, and optionally every H's snr) of one spectrum.

    FP32 mode takes float32 input; FP64 mode widens the input to float64 and computes in double.
    """
    v = _variant(variant, pow2)
    dt = np.float64 if fp64 else np.float32
    x = np.ascontiguousarray(x, dtype=dt)
    N = x.shape[0]
    mu, isig = _tables(mu, isig, hmax, dt)
    best = np.empty(N, dt)
    bh = np.empty(N, np.uint8)
    path = np.zeros(N, np.uint32) if v & ~POW2 in (GREEDY, GREEDY1) else None
    ah = np.empty((hmax, N), dt) if all_h else None
    fn = _load().hs_oracle_1d_f64 if fp64 else _load().hs_oracle_1d_f32
    fn(v, _ptr(x), N, hmax, _ptr(mu), _ptr(isig), _ptr(best), _ptr(bh), _ptr(path), _ptr(ah), _threads(nthreads))
    out = {"best_snr": best, "best_h": bh}
    if path is not None:
        out["path"] = path
    if ah is not None:
        out["all_h"] = ah
    return out


def hs_bins(variant, x, bins, hmax: int = 32, mu=None, isig=None, fp64: bool = False, pow2: bool = False):
    """Best snr / H / path of the listed output bins of one spectrum only."""
    v = _variant(variant, pow2)
    dt = np.float64 if fp64 else np.float32
    x = np.ascontiguousarray(x, dtype=dt)
    bins = np.ascontiguousarray(bins, dtype=np.int64)
    if bins.size and (bins.min() < 0 or bins.max() >= x.shape[0]):
        raise ValueError("bin out of range")
    mu, isig = _tables(mu, isig, hmax, dt)
    best = np.empty(bins.size, dt)
    bh = np.empty(bins.size, np.uint8)
    path = np.zeros(bins.size, np.uint32)
    fn = _load().hs_oracle_bins_f64 if fp64 else _load().hs_oracle_bins_f32
    fn(v, _ptr(x), x.shape[0], hmax, _ptr(mu), _ptr(isig), _ptr(bins), bins.size, _ptr(best), _ptr(bh), _ptr(path))
    return {"best_snr": best, "best_h": bh, "path": path}


def hs_batched(variant, x, offsets, hmax: int = 32, mu=None, isig=None, fp64: bool = False, pow2: bool = False,
               nthreads: int | None = None):
    v = _variant(variant, pow2)
    dt = np.float64 if fp64 else np.float32
    x = np.ascontiguousarray(x, dtype=dt)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    base = int(offsets[0])
    offs = offsets - base
    total = int(offs[-1])
    mu, isig = _tables(mu, isig, hmax, dt)
    best = np.empty(total, dt)
    bh = np.empty(total, np.uint8)
    path = np.zeros(total, np.uint32) if v & ~POW2 in (GREEDY, GREEDY1) else None
    fn = _load().hs_oracle_batched_f64 if fp64 else _load().hs_oracle_batched_f32
    fn(v, _ptr(x[base:base + total]), _ptr(offs), len(offs) - 1, hmax, _ptr(mu), _ptr(isig), _ptr(best), _ptr(bh),
       _ptr(path), _threads(nthreads))
    out = {"best_snr": best, "best_h": bh}
    if path is not None:
        out["path"] = path
    return out


def hs_2d(plane, z_min: int, hmax: int = 16, mu=None, isig=None, fp64: bool = False, all_h: bool = False,
          nthreads: int | None = None, variant: str = "std"):
    """2-D Eq. 1 (variant "std") or the row-wise 2-D forms of Eq. 2-4 ("fbin": harmonic i at
    (i n, i z); "max", "max0", "greedy", "greedy1": harmonic i taken on the row i z as the 1-D
    equation takes it) over a (nz, n_bins) plane whose row r holds z = z_min + r."""
    dt = np.float64 if fp64 else np.float32
    plane = np.ascontiguousarray(plane, dtype=dt)
    nz, nb = plane.shape
    mu, isig = _tables(mu, isig, hmax, dt)
    best = np.empty((nz, nb), dt)
    bh = np.empty((nz, nb), np.uint8)
    bn = np.empty(nb, dt)
    bhn = np.empty(nb, np.uint8)
    bzn = np.empty(nb, np.int32)
    ah = np.empty((hmax, nz, nb), dt) if all_h else None
    if variant == "std":
        fn = _load().hs_oracle_2d_f64 if fp64 else _load().hs_oracle_2d_f32
    elif variant == "fbin":
        fn = _load().hs_oracle_2d_fbin_f64 if fp64 else _load().hs_oracle_2d_fbin_f32
    elif variant in ("max", "max0", "greedy", "greedy1"):
        row = _load().hs_oracle_2d_rowwise_f64 if fp64 else _load().hs_oracle_2d_rowwise_f32
        v = _variant(variant)

        def fn(*a):
            return row(v, *a)
    else:
        raise ValueError("unknown 2-D variant %r" % variant)
    fn(_ptr(plane), nz, z_min, nb, nb, hmax, _ptr(mu), _ptr(isig), _ptr(best), _ptr(bh), _ptr(bn), _ptr(bhn),
       _ptr(bzn), _ptr(ah), _threads(nthreads))
    out = {"best_snr": best, "best_h": bh, "best_snr_n": bn, "best_h_n": bhn, "best_z_n": bzn}
    if ah is not None:
        out["all_h"] = ah
    return out


def hs_2d_cells(plane, z_min: int, rows, bins, hmax: int = 16, mu=None, isig=None, fp64: bool = False):
    """Best snr / H of the listed (row, bin) cells of a 2-D plane only."""
    dt = np.float64 if fp64 else np.float32
    plane = np.ascontiguousarray(plane, dtype=dt)
    nz, nb = plane.shape
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    bins = np.ascontiguousarray(bins, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= nz or bins.min() < 0 or bins.max() >= nb):
        raise ValueError("cell out of range")
    mu, isig = _tables(mu, isig, hmax, dt)
    best = np.empty(rows.size, dt)
    bh = np.empty(rows.size, np.uint8)
    fn = _load().hs_oracle_2d_cells_f64 if fp64 else _load().hs_oracle_2d_cells_f32
    fn(_ptr(plane), nz, z_min, nb, nb, hmax, _ptr(mu), _ptr(isig), _ptr(rows), _ptr(bins), rows.size, _ptr(best),
       _ptr(bh))
    return {"best_snr": best, "best_h": bh}


def grad_1d(variant, x, g, best_h, hmax: int = 32, isig=None):
    """FP64 adjoint: d/dx of sum_n g[n] * best_snr[n] with the best H of each bin held fixed."""
    v = _variant(variant)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    best_h = np.ascontiguousarray(best_h, dtype=np.uint8)
    isig = None if isig is None else np.ascontiguousarray(isig, dtype=np.float64)
    out = np.zeros_like(x)
    _load().hs_oracle_grad_f64(v, _ptr(x), x.shape[0], hmax, _ptr(isig), _ptr(g), _ptr(best_h), _ptr(out))
    return out


def standardize_cast(p, mu: float, sigma: float, dtype: str):
    """(p - mu) / sigma in FP32, rounded to nearest-even FP16 or BF16; returns the uint16 bit patterns."""
    p = np.ascontiguousarray(p, dtype=np.float32)
    out = np.empty(p.shape, np.uint16)
    code = {"f16": 1, "bf16": 2}[dtype]
    _load().hs_oracle_standardize_cast(_ptr(p), p.size, float(mu), float(sigma), code, _ptr(out))
    return out


def power_normalize(spec, block: int, dtype: str = "f32"):
    """Power of a complex spectrum (complex64, or float32 interleaved re/im), divided by the
    interpolated block-median estimate of its local mean and standardised; FP32 values, or the
    uint16 bit patterns of FP16/BF16.  Returns (x, block medians)."""
    s = np.ascontiguousarray(spec)
    if np.iscomplexobj(s):
        s = np.ascontiguousarray(s.astype(np.complex64)).view(np.float32)
    s = np.ascontiguousarray(s, dtype=np.float32)
    n = s.size // 2
    code = {"f32": 0, "f16": 1, "bf16": 2}[dtype]
    out = np.empty(n, np.float32 if code == 0 else np.uint16)
    med = np.empty(max(1, (n + block - 1) // block), np.float32)
    _load().hs_oracle_power_normalize(_ptr(s), n, int(block), code, _ptr(out), _ptr(med))
    return out, med[: (n + block - 1) // block]


def noise_moments(variant, hmax: int = 32):
    """Closed-form (mu_H, sigma_H) of h_H on standardised Exp(1) noise, H = 0..hmax (double)."""
    mu = np.empty(hmax + 1, np.float64)
    sd = np.empty(hmax + 1, np.float64)
    _load().hs_oracle_noise_moments(_variant(variant), hmax, _ptr(mu), _ptr(sd))
    return mu, sd


def noise_calibration(variant, hmax: int = 32):
    """The float32 (mu_H, 1/sigma_H) tables derived from ``noise_moments``, rounded once."""
    mu, sd = noise_moments(variant, hmax)
    return mu.astype(np.float32), (1.0 / sd).astype(np.float32)


CANDIDATE_DTYPE = np.dtype([("spectrum", "<u4"), ("bin", "<u4"), ("snr", "<f4"), ("z", "<i2"), ("h", "u1"),
                            ("variant", "u1")])


def _fundamentals32(cand):
    """(frequency, drift) of each candidate's fundamental in bins, FP32 arrays: Eq. 1 and its 2-D form
    report the H-th harmonic (bin / H, z / H); Eq. 2-4 report the fundamental's own bin."""
    h = np.maximum(cand["h"].astype(np.float32), np.float32(1))
    b = cand["bin"].astype(np.float32)
    z = cand["z"].astype(np.float32)
    is_std = cand["variant"].astype(np.int64) == STD
    f = np.where(is_std, (b / h).astype(np.float32), b).astype(np.float32)
    fz = np.where(is_std, (z / h).astype(np.float32), z).astype(np.float32)
    return f, fz


def sift_candidates(cand, tol: float = 1.5, tol_z: float = 1.5, kmax: int = 8):
    """Keep mask of a candidate list (structured CANDIDATE_DTYPE, in any order): a candidate is
    dropped when a stronger candidate of the same variant and spectrum is related to it (larger snr,
    or equal snr and earlier in the list).  Related: for some k = 1..kmax the higher fundamental lies
    within k*tol bins and k*tol_z rows of k times the lower one; every operation in FP32 (numpy
    float32 arrays, each elementwise operation rounded)."""
    n = len(cand)
    keep = np.ones(n, bool)
    f, fz = _fundamentals32(cand)
    snr = cand["snr"].astype(np.float32)
    group = cand["variant"].astype(np.int64) << 32 | cand["spectrum"].astype(np.int64)
    t, tz = np.float32(tol), np.float32(tol_z)
    for i in range(n):
        j = np.nonzero(group == group[i])[0]
        j = j[j != i]
        stronger = (snr[j] > snr[i]) | ((snr[j] == snr[i]) & (j < i))
        j = j[stronger]
        if j.size == 0:
            continue
        a_low = f[j] <= f[i]  # the other candidate is the lower one when its frequency is not higher
        fl = np.where(a_low, f[j], f[i]).astype(np.float32)
        zl = np.where(a_low, fz[j], fz[i]).astype(np.float32)
        fh = np.where(a_low, f[i], f[j]).astype(np.float32)
        zh = np.where(a_low, fz[i], fz[j]).astype(np.float32)
        rel = np.zeros(j.size, bool)
        for k in range(1, kmax + 1):
            kf = np.float32(k)
            rel |= (np.abs(fh - kf * fl) <= kf * t) & (np.abs(zh - kf * zl) <= kf * tz)
        keep[i] = not rel.any()
    return keep


def candidates(best_snr, best_h, threshold: float, spectrum: int = 0):
    """The thresholded candidate set: every bin whose best snr is strictly above the threshold,
    as (spectrum, bin, snr, H) rows in bin order."""
    idx = np.nonzero(best_snr > threshold)[0]
    return np.stack([np.full(idx.shape, spectrum, np.int64), idx.astype(np.int64)], 1), best_snr[idx], best_h[idx]
