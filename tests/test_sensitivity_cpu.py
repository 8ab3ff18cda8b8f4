"""Plumbing of the sensitivity evaluation on the CPU: standardisation, where the pulse's harmonics
land, and which output bins each variant's pulsar is read from."""
import numpy as np
import pytest

from paper_1812_02647_gb300 import sensitivity as s


@pytest.fixture(scope="module")
def torch():
    import torch as t

    return t


def test_grid():
    assert s.N_SAMPLES == 312500 and s.DF == pytest.approx(0.05)  # 20 s at 64 us, 0.05 Hz bins
    assert s.N_BINS % 8 == 0 and s.N_BINS <= s.N_SAMPLES // 2 + 1


def test_noise_is_standardised(torch):
    x = s.pulse_spectra(torch, [10.0, 20.0], amp=0.0, seed=11, device="cpu").numpy()
    body = x[:, 1:]
    assert abs(body.mean()) < 0.01 and abs(body.std() - 1.0) < 0.01
    # Exp(1) - 1: the fraction above 3 is e^-4
    assert abs((body > 3.0).mean() - np.exp(-4.0)) < 0.002


def test_harmonics_land_on_multiples(torch):
    k0 = 200
    x = s.pulse_spectra(torch, [k0 * s.DF], amp=0.3, seed=5, device="cpu").numpy()[0]
    on = np.array([x[k * k0] for k in range(1, 6)])
    off = np.array([x[k * k0 + 37] for k in range(1, 6)])
    # expected power ~ N (amp c_k)^2 with c_k ~ 0.056 exp(-k^2 / 100) for kappa = 50: ~90 .. 60
    assert on.min() > 30.0 and off.max() < 10.0


def test_pulsar_bins():
    b = s.pulsar_bins("std", 100.4, hmax=4)
    assert set(b) == {99, 100, 101, 200, 201, 202, 300, 301, 302, 401, 402, 403}
    assert list(s.pulsar_bins("max", 100.6)) == [99, 100, 101, 102]
    assert list(s.pulsar_bins("fbin", 0.2)) == [0, 1]
    snr = np.zeros(1000)
    snr[402] = 7.0
    assert s.recovered_snr(snr, "std", 100.4, hmax=4) == 7.0
    assert s.recovered_snr(snr, "fbin", 100.4) == 0.0
