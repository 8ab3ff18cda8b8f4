"""Seeded synthetic inputs for the harmonic sum (data only, no harmonic-sum arithmetic).

Shared by the CPU oracle's tests, the GPU parity tests and the benchmark.  The C core
(``synth.c``) makes every bin a pure function of (seed, noise stream, bin), so a sample
of a very large batch can be regenerated without building the whole batch.

Workloads (all seeded; seed = workload index * 1000 + trial):

* ``spectrum_1d``      one spectrum of 131072 bins, a pulsar at fundamental bin 1000.37 with 16
                       harmonics of amplitude 8/k, sinc^2 scalloping (the off-bin case of Section 3).
* ``batch_dm_trials``  2048 spectra, lengths uniform in {2^19..2^22}; 5% carry a pulsar with
                       f0 ~ U[50, 50000], K ~ U{8..32}, gaussian width ~ U[0.5, 2], A ~ U[4, 10].
* ``fdas_plane``       201 z rows (z = -100..100) x 2^21 bins; 4 drifting pulsars per plane,
                       f0 ~ U[1000, 100000], K ~ U{4..16}, |K z0| <= 80, width 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libhs_synth.so")
_lib = None


class Pulsar(ctypes.Structure):
    _fields_ = [
        ("shape", ctypes.c_int32),
        ("n_harm", ctypes.c_int32),
        ("f0", ctypes.c_double),
        ("amp", ctypes.c_double),
        ("width", ctypes.c_double),
        ("z0", ctypes.c_double),
    ]


NO_PULSAR = dict(shape=-1, n_harm=0, f0=0.0, amp=0.0, width=1.0, z0=0.0)


def build(force: bool = False) -> str:
    """Compile the generator core in place (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.hs_synth_uniform.restype = ctypes.c_double
        lib.hs_synth_uniform.argtypes = [ctypes.c_uint64] * 4
        lib.hs_synth_spectrum.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                          P, ctypes.c_int, P, ctypes.c_int]
        lib.hs_synth_batch.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, P, P, ctypes.c_int,
                                       P, ctypes.c_int]
        lib.hs_synth_plane.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int32, P, ctypes.c_int]
        _lib = lib
    return _lib


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def _pulsar(p):
    d = dict(NO_PULSAR)
    if p:
        d.update(p)
    return Pulsar(**d)


def uniform(seed: int, stream: int, a: int, b: int) -> float:
    return _load().hs_synth_uniform(seed, stream, a, b)


def spectrum(seed: int, row_id: int, n_bins: int, pulsar: dict | None = None, m0: int = 0,
             raw: bool = False, out=None, nthreads: int | None = None) -> np.ndarray:
    """Bins [m0, m0+n_bins) of one spectrum as float32 (standardised unless ``raw``)."""
    lib = _load()
    if out is None:
        out = np.empty(n_bins, dtype=np.float32)
    ptr = out.ctypes.data if isinstance(out, np.ndarray) else int(out)
    p = _pulsar(pulsar)
    lib.hs_synth_spectrum(seed, row_id, m0, n_bins, ctypes.addressof(p), int(raw), ptr, _threads(nthreads))
    return out


def batch(seed: int, offsets: np.ndarray, pulsars: list | None = None, first_id: int = 0,
          raw: bool = False, out=None, nthreads: int | None = None):
    """Fill a packed batch; ``out`` may be a numpy array or a raw host address."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    total = int(offsets[-1] - offsets[0])
    if out is None:
        out = np.empty(total, dtype=np.float32)
    ptr = out.ctypes.data if isinstance(out, np.ndarray) else int(out)
    arr = (Pulsar * max(n, 1))(*[_pulsar(p) for p in (pulsars or [None] * n)])
    lib.hs_synth_batch(seed, first_id, n, offsets.ctypes.data, ctypes.addressof(arr), int(raw), ptr,
                       _threads(nthreads))
    return out


def plane(seed: int, plane_id: int, nz: int, z_min: int, n_bins: int, pulsars: list | None = None,
          row_stride: int | None = None, out=None, nthreads: int | None = None):
    lib = _load()
    row_stride = n_bins if row_stride is None else row_stride
    if out is None:
        out = np.empty((nz, row_stride), dtype=np.float32)
    ptr = out.ctypes.data if isinstance(out, np.ndarray) else int(out)
    plist = pulsars or []
    arr = (Pulsar * max(len(plist), 1))(*[_pulsar(p) for p in plist])
    lib.hs_synth_plane(seed, plane_id, nz, z_min, n_bins, row_stride, ctypes.addressof(arr), len(plist), ptr,
                       _threads(nthreads))
    return out


# ----------------------------------------------------------------------------------------------
# Workload recipes
# ----------------------------------------------------------------------------------------------

def spectrum_1d_pulsar(trial: int = 0, n_bins: int = 131072):
    """One 131072-bin spectrum with a pulsar at 1000.37, 16 harmonics of amplitude 8/k (sinc^2)."""
    seed = 1 * 1000 + trial
    p = dict(shape=0, n_harm=16, f0=1000.37, amp=8.0, width=1.0)
    return spectrum(seed, 0, n_bins, p), p


def batch_dm_trials_layout(n_spectra: int = 2048, trial: int = 0, lengths=(1 << 19, 1 << 20, 1 << 21, 1 << 22),
                           pulsar_fraction: float = 0.05):
    """Lengths, offsets and pulsar list of the DM-trial batch (no bins generated)."""
    seed = 2 * 1000 + trial
    rng = np.random.default_rng(seed)
    lens = rng.choice(np.asarray(lengths, dtype=np.int64), size=n_spectra)
    offsets = np.zeros(n_spectra + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    n_psr = int(round(pulsar_fraction * n_spectra))
    with_psr = set(rng.choice(n_spectra, size=n_psr, replace=False).tolist()) if n_psr else set()
    pulsars = []
    for s in range(n_spectra):
        f0 = float(rng.uniform(50.0, 50000.0))
        k = int(rng.integers(8, 33))
        w = float(rng.uniform(0.5, 2.0))
        a = float(rng.uniform(4.0, 10.0))
        pulsars.append(dict(shape=1, n_harm=k, f0=f0, amp=a, width=w) if s in with_psr else None)
    return seed, offsets, pulsars


def batch_dm_trials(n_spectra: int = 2048, trial: int = 0, out=None, nthreads=None, **kw):
    seed, offsets, pulsars = batch_dm_trials_layout(n_spectra, trial, **kw)
    x = batch(seed, offsets, pulsars, out=out, nthreads=nthreads)
    return x, offsets, pulsars


def uniform_batch(n_spectra: int, n_bins: int, seed: int, pulsar_fraction: float = 0.05, out=None,
                  nthreads=None, raw: bool = False):
    """Equal-length batch (used by the differentiation and precision workloads)."""
    rng = np.random.default_rng(seed)
    offsets = np.arange(n_spectra + 1, dtype=np.int64) * n_bins
    n_psr = int(round(pulsar_fraction * n_spectra))
    with_psr = set(rng.choice(n_spectra, size=n_psr, replace=False).tolist()) if n_psr else set()
    pulsars = []
    for s in range(n_spectra):
        f0 = float(rng.uniform(50.0, n_bins / 40.0))
        k = int(rng.integers(8, 33))
        w = float(rng.uniform(0.5, 2.0))
        a = float(rng.uniform(4.0, 10.0))
        pulsars.append(dict(shape=1, n_harm=k, f0=f0, amp=a, width=w) if s in with_psr else None)
    x = batch(seed, offsets, pulsars, out=out, nthreads=nthreads, raw=raw)
    return x, offsets, pulsars


def fdas_plane_pulsars(plane_id: int, trial: int = 0, n_pulsars: int = 4, n_bins: int = 1 << 21):
    seed = 3 * 1000 + trial
    rng = np.random.default_rng([seed, plane_id])
    out = []
    for _ in range(n_pulsars):
        k = int(rng.integers(4, 17))
        hi = min(100000.0, (n_bins - 16) / k)
        f0 = float(rng.uniform(min(1000.0, hi / 2), hi))
        z0 = float(rng.uniform(-80.0 / k, 80.0 / k))
        out.append(dict(shape=1, n_harm=k, f0=f0, amp=float(rng.uniform(4.0, 10.0)), width=1.0, z0=z0))
    return seed, out


def fdas_plane(plane_id: int, trial: int = 0, nz: int = 201, z_min: int = -100, n_bins: int = 1 << 21,
               out=None, nthreads=None):
    seed, ps = fdas_plane_pulsars(plane_id, trial, n_bins=n_bins)
    return plane(seed, plane_id, nz, z_min, n_bins, ps, out=out, nthreads=nthreads), ps
