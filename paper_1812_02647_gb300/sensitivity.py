"""Sensitivity of the four harmonic sums to where a pulsar falls inside a Fourier bin.

The evaluation of Section 3 of arXiv:1812.02647, restated: a time series of 20 s sampled every 64 us
holds a pulse train with a von Mises pulse shape plus white Gaussian noise; its power spectrum
(bins 0.05 Hz wide) is standardised and harmonic-summed by every variant, and the SNR each variant
recovers for the pulsar is compared (a) as the pulsar frequency moves across one bin and (b)
averaged over many frequencies.  The paper states the outcome only in words (its figures have no
data): the standard sum (Eq. 1) recovers most at bin centres and declines between them, freq-bin
(Eq. 3) loses more than half off the bin centre, Max (Eq. 2) recovers less but evenly across the bin,
and averaged over frequencies greedy (Eq. 4) is close to the standard sum while freq-bin loses about
20% and Max about 40%.

Time series, FFT and standardisation run in PyTorch on the GPU (they precede the harmonic sum); the
harmonic sums run in this package's kernels through the C ABI.
"""
from __future__ import annotations

import math

import numpy as np

T_OBS = 20.0  # s
T_SAMP = 64e-6  # s
N_SAMPLES = int(round(T_OBS / T_SAMP))  # 312500
DF = 1.0 / T_OBS  # bin width, Hz
N_BINS = (N_SAMPLES // 2 + 1) // 8 * 8  # 156248: bins 0 .. N/2, trimmed to a 32-byte multiple
# "max0" is Eq. 2 with the window j = 0..i (plan flag HS_FLAG_MAX_WINDOW0), beside the window as written
VARIANTS = ("std", "max", "max0", "fbin", "greedy")


def pulse_spectra(torch, f0_hz, amp=0.1, kappa=50.0, seed=0, device="cuda"):
    """Standardised power spectra of pulse trains at frequencies ``f0_hz`` (one per row).

    Pulse shape exp(kappa (cos 2 pi phi - 1)) (a von Mises profile, peak 1, FWHM ~5% of the period
    for kappa = 50), amplitude ``amp`` in units of the noise sigma, random start phase; white
    N(0, 1) noise.  Power |X_k|^2 / N of the mean-subtracted series is Exp(1) for noise alone, so
    x = P - 1 has mean 0 and sigma 1.  Returns float32 [len(f0), N_BINS]."""
    f0 = torch.as_tensor(np.asarray(f0_hz, np.float64), device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    b = f0.numel()
    phi0 = torch.rand(b, 1, generator=g, device=device, dtype=torch.float64)
    t = torch.arange(N_SAMPLES, device=device, dtype=torch.float64) * T_SAMP
    phase = torch.remainder(f0[:, None] * t[None, :] + phi0, 1.0)
    series = (amp * torch.exp(kappa * (torch.cos(2.0 * math.pi * phase) - 1.0))).float()
    del phase
    series += torch.randn(b, N_SAMPLES, generator=g, device=device, dtype=torch.float32)
    series -= series.mean(dim=1, keepdim=True)
    spec = torch.fft.rfft(series, dim=1)
    del series
    p = (spec.real.square() + spec.imag.square()) / N_SAMPLES
    return (p[:, :N_BINS] - 1.0).contiguous()


def pulsar_bins(variant, f_bins, hmax=32, n_bins=N_BINS):
    """Output bins where a variant reports a pulsar whose fundamental sits at ``f_bins`` (fractional
    bin).  Eq. 1 reports harmonic H's bin, n ~ H f (its output index is the H-th harmonic); Eq. 2-4
    report the fundamental's bin (Eq. 2 reads x(n+1) .. for H = 1, so one bin lower is included; the
    same bins serve the j = 0..i window)."""
    if variant == "std":
        c = np.rint(np.arange(1, hmax + 1) * f_bins).astype(np.int64)
        cand = (c[:, None] + np.arange(-1, 2)[None, :]).ravel()
    else:
        c = int(np.rint(f_bins))
        cand = np.arange(c - 2, c + 2)
    return np.unique(cand[(cand >= 0) & (cand < n_bins)])


def recovered_snr(best_snr, variant, f_bins, hmax=32):
    """Largest best-H snr over the variant's pulsar bins (``best_snr``: one spectrum, numpy)."""
    return float(best_snr[pulsar_bins(variant, f_bins, hmax, best_snr.shape[0])].max())


def _sum_all(hs_mod, torch, x, variants, hmax):
    b = x.shape[0]
    flat = x.reshape(-1)
    offsets = torch.arange(b + 1, device=x.device, dtype=torch.int64) * N_BINS
    plans = {}
    out = {}
    for v in variants:
        flags = hs_mod.FLAG_MAX_WINDOW0 if v == "max0" else 0
        if flags not in plans:
            plans[flags] = hs_mod.HarmonicSum(variants=0xF, hmax=hmax, max_bins=N_BINS, threshold=6.0, max_spectra=b,
                                              flags=flags)
        h, lib_v = plans[flags], ("max" if v == "max0" else v)
        mu, isig = hs_mod.hs_noise_calibration(lib_v, hmax, flags=flags)
        h.set_calibration(lib_v, mu, isig)
        o = h.sum_batched(lib_v, flat, offsets)
        out[v] = o["best_snr"].reshape(b, N_BINS).cpu().numpy()
    return out


def run(base_bin=400, offsets=np.arange(20) / 20.0, trials=8, freqs_hz=None, freq_trials=4, freq_offsets=8,
        amp=0.1, kappa=50.0, hmax=32, seed=1, batch=64):
    """The two measurements: recovered snr against the fractional bin offset of a pulsar at
    ``base_bin + offset`` (mean over ``trials`` noise realisations), and against frequency (each
    frequency averaged over ``freq_offsets`` uniform offsets x ``freq_trials`` realisations)."""
    import torch

    import paper_1812_02647_gb300 as hs_mod

    if freqs_hz is None:
        freqs_hz = np.geomspace(2.0, 100.0, 16)

    def measure(f_bins_list, seed0):
        res = {v: [] for v in VARIANTS}
        for s0 in range(0, len(f_bins_list), batch):
            fb = np.asarray(f_bins_list[s0:s0 + batch], np.float64)
            x = pulse_spectra(torch, fb * DF, amp=amp, kappa=kappa, seed=seed0 + s0)
            snr = _sum_all(hs_mod, torch, x, VARIANTS, hmax)
            del x
            for v in VARIANTS:
                res[v].extend(recovered_snr(snr[v][k], v, fb[k], hmax) for k in range(fb.size))
        return {v: np.asarray(r) for v, r in res.items()}

    offsets = np.asarray(offsets, np.float64)
    fb1 = np.repeat(base_bin + offsets, trials)
    r1 = measure(fb1, seed * 1000)
    per_offset = {v: r1[v].reshape(offsets.size, trials).mean(axis=1) for v in VARIANTS}

    rng = np.random.default_rng(seed)
    fb2 = []
    for f in freqs_hz:
        for _ in range(freq_offsets * freq_trials):
            fb2.append(math.floor(f / DF) + rng.random())
    r2 = measure(fb2, seed * 1000 + 500)
    per_freq = {v: r2[v].reshape(len(freqs_hz), -1).mean(axis=1) for v in VARIANTS}
    averaged = {v: float(per_freq[v].mean()) for v in VARIANTS}
    return {
        "setup": {"t_obs_s": T_OBS, "t_samp_s": T_SAMP, "bin_width_hz": DF, "n_bins": N_BINS, "amp": amp,
                  "kappa": kappa, "hmax": hmax, "trials": trials, "base_bin": base_bin},
        "bin_offsets": offsets.tolist(),
        "per_offset": {v: per_offset[v].tolist() for v in VARIANTS},
        "frequencies_hz": [float(f) for f in freqs_hz],
        "per_frequency": {v: per_freq[v].tolist() for v in VARIANTS},
        "averaged": averaged,
        "averaged_relative_to_std": {v: averaged[v] / averaged["std"] for v in VARIANTS},
    }


if __name__ == "__main__":
    import json

    print(json.dumps(run(), indent=1))
