"""The paper's sensitivity evaluation (Section 3) run through the GPU path: the qualitative outcomes
its text states, checked on fresh synthetic pulse trains.  Not a parity test (the figures carry no
data); the oracle is not involved."""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def result():
    from paper_1812_02647_gb300 import sensitivity

    return sensitivity.run(offsets=[0.0, 0.5], trials=24, freqs_hz=np.geomspace(2.0, 100.0, 6), freq_trials=2,
                           freq_offsets=8, seed=7)


def test_standard_sum_peaks_at_bin_centre(result):
    s = result["per_offset"]["std"]
    assert s[0] > 1.1 * s[1]


def test_freq_bin_loses_over_half_off_centre(result):
    f = result["per_offset"]["fbin"]
    assert f[1] < 0.5 * f[0]


def test_max_recovers_less_than_standard_at_bin_centre(result):
    assert result["per_offset"]["max"][0] < result["per_offset"]["std"][0]


def test_averaged_ordering(result):
    rel = result["averaged_relative_to_std"]
    assert 0.75 < rel["greedy"] <= 1.05  # greedy close to the standard sum
    assert rel["fbin"] < 0.9 and rel["max"] < 0.9  # both lose sensitivity on average


def test_consistent_over_frequency(result):
    for v, per_f in result["per_frequency"].items():
        per_f = np.asarray(per_f)
        assert (np.abs(per_f / per_f.mean() - 1.0) < 0.25).all(), (v, per_f)
