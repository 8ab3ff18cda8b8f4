"""Eq. 2-4 run zone by zone (bins of equal valid-harmonic count, tiles sized by cost): every zone
boundary, the bins with no valid H at all, small hmax, the variant flags and the tile sizes must give
exactly the oracle's results, through the single-spectrum and the batched entry points."""
import numpy as np
import pytest

import hs_synth
import oracle

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

THR = 6.0
# (library variant, plan flag name or None, oracle variant)
FORMS = [("max", None, "max"), ("max", "FLAG_MAX_WINDOW0", "max0"), ("fbin", None, "fbin"),
         ("greedy", None, "greedy"), ("greedy", "FLAG_GREEDY_FIXED1", "greedy1")]


def _plan(hs_lib, v, flag, hmax, pow2, n_spectra, max_bins=1 << 22):
    flags = (getattr(hs_lib, flag) if flag else 0) | (hs_lib.FLAG_POW2_STAGES if pow2 else 0)
    h = hs_lib.HarmonicSum(variants=hs_lib.VARIANTS[v], hmax=hmax, max_bins=max_bins, threshold=THR,
                           cand_capacity=1 << 18, flags=flags, max_spectra=n_spectra)
    mu, isig = hs_lib.hs_noise_calibration(v, hmax, flags=flags & ~hs_lib.FLAG_POW2_STAGES)
    h.set_calibration(v, mu, isig)
    return h, mu, isig


def _check(hs_lib, o, r, v, a=0, b=None):
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy()[a:b], r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy()[a:b], r["best_h"])
    if v == "greedy":
        np.testing.assert_array_equal(o["path"].cpu().numpy().view(np.uint32)[a:b], r["path"])


@pytest.mark.parametrize("v,flag,ov", FORMS)
@pytest.mark.parametrize("hmax", [1, 3, 8, 9, 32])
@pytest.mark.parametrize("pow2", [False, True])
def test_zones_single_spectrum(hs_lib, v, flag, ov, hmax, pow2):
    import torch

    for n_bins in (1, 2, 3, 4, 5, 9, 17, 33, 65, 100, 257, 1000, 4097, 70001):
        x = hs_synth.spectrum(4400 + n_bins, 0, n_bins)
        h, mu, isig = _plan(hs_lib, v, flag, hmax, pow2, 1)
        for tile in (256, 16384):
            hs_lib.hs_plan_set_tile_bins(h.plan, v, tile)
            o = h.sum_1d(v, torch.from_numpy(x).cuda())
            assert h.sync_status() == hs_lib.OK
            r = oracle.hs_1d(ov, x, hmax=hmax, mu=mu, isig=isig, pow2=pow2)
            _check(hs_lib, o, r, v)
            assert int(o["cand_count"].item()) == int((r["best_snr"] > THR).sum())


@pytest.mark.parametrize("v,flag,ov", FORMS)
@pytest.mark.parametrize("hmax", [2, 8, 32])
def test_zones_batched(hs_lib, v, flag, ov, hmax):
    import torch

    lens = [4, 8, 0, 12, 36, 100, 260, 1000, 4096, 4100, 70004, 1 << 17, 8, 300000]
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = hs_synth.batch(4500 + hmax, offsets)
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    h, mu, isig = _plan(hs_lib, v, flag, hmax, False, len(lens))
    r = oracle.hs_batched(ov, x, offsets, hmax=hmax, mu=mu, isig=isig, nthreads=8)
    for tile in (256, 2048, 16384):
        hs_lib.hs_plan_set_tile_bins(h.plan, v, tile)
        o = h.sum_batched(v, xd, od, first_id=5)
        assert h.sync_status() == hs_lib.OK
        _check(hs_lib, o, r, v)
        got = hs_lib.read_candidates(o)
        assert got.size == int((r["best_snr"] > THR).sum())
        spec = np.searchsorted(offsets, np.arange(x.size), side="right") - 1
        want = np.nonzero(r["best_snr"] > THR)[0]
        np.testing.assert_array_equal(np.sort(got["spectrum"].astype(np.int64) * (1 << 32) + got["bin"]),
                                      np.sort((spec[want] + 5) * (1 << 32) + (want - offsets[spec[want]])))
