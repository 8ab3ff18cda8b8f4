"""The allocation-free batched entry point against the workspace one.

hs_sum_batched_noalloc serves callers that may not allocate device memory while they run (for
example a real-time pipeline whose GPU memory is all reserved at start-up): it uses a fixed scratch
array inside the library instead of a caller workspace.  Its results must equal hs_sum_batched's on
the same inputs, on two calls in a row (the array keeps the previous call's contents, so the second
call checks that everything that must start at zero is cleared).  This file is collected last.
"""
import numpy as np
import pytest

import hs_synth

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def test_noalloc_matches_workspace_entry_point(hs_lib):
    import torch

    lens = [4096, 100000, 0, 65536, 8, 250000, 12, 131072]
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = hs_synth.batch(303, offsets)
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    for v in ("std", "max", "fbin", "greedy"):
        hs = hs_lib.HarmonicSum(variants=hs_lib.VARIANTS[v], threshold=6.0, cand_capacity=1 << 16,
                                max_spectra=len(lens))
        mu, isig = hs_lib.hs_noise_calibration(v, 32)
        hs.set_calibration(v, mu, isig)
        ref = hs.sum_batched(v, xd, od, first_id=7)
        torch.cuda.synchronize()
        assert hs.sync_status() == hs_lib.OK
        for call in range(2):
            o = hs.new_outputs(x.size, v, "cuda")
            o["best_snr"].fill_(123.0)
            hs_lib.hs_sum_batched_noalloc(hs.plan, v, xd, od, hs.out_struct(o), first_id=7)
            torch.cuda.synchronize()
            assert torch.equal(o["best_snr"], ref["best_snr"]), (v, call)
            assert torch.equal(o["best_h"], ref["best_h"]), (v, call)
            if v == "greedy":
                assert torch.equal(o["path"], ref["path"]), call
            assert int(o["cand_count"].item()) == int(ref["cand_count"].item())
            a = np.sort(hs_lib.read_candidates(o), order=["spectrum", "bin"])
            b = np.sort(hs_lib.read_candidates(ref), order=["spectrum", "bin"])
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_noalloc_16bit_eq1_matches_the_fp32_groups(hs_lib, dtype):
    """For 16-bit storage the workspace entry point runs Eq. 1 through FP32 copies of 64-spectrum
    groups while the allocation-free one runs the 16-bit kernel directly: the two agree bit for bit."""
    import torch

    rng = np.random.default_rng(11)
    lens = [int(rng.integers(1, 3000)) * 8 for _ in range(90)]
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    xd = torch.from_numpy(hs_synth.batch(304, offsets)).to(tdt).cuda()
    od = torch.from_numpy(offsets).cuda()
    hs = hs_lib.HarmonicSum(variants=hs_lib.STD, dtype={"f16": hs_lib.F16, "bf16": hs_lib.BF16}[dtype],
                            max_bins=1 << 16, threshold=6.0, cand_capacity=1 << 16, max_spectra=len(lens))
    mu, isig = hs_lib.hs_noise_calibration("std", 32)
    hs.set_calibration("std", mu, isig)
    ref = hs.sum_batched("std", xd, od, first_id=2)
    torch.cuda.synchronize()
    assert hs.sync_status() == hs_lib.OK
    o = hs.new_outputs(xd.numel(), "std", "cuda")
    hs_lib.hs_sum_batched_noalloc(hs.plan, "std", xd, od, hs.out_struct(o), first_id=2)
    torch.cuda.synchronize()
    assert torch.equal(o["best_snr"], ref["best_snr"])
    assert torch.equal(o["best_h"], ref["best_h"])
    a = np.sort(hs_lib.read_candidates(o), order=["spectrum", "bin"])
    b = np.sort(hs_lib.read_candidates(ref), order=["spectrum", "bin"])
    np.testing.assert_array_equal(a, b)


def test_noalloc_staged_spans_matches_workspace_entry_point(hs_lib):
    """Eq. 1 through the staged-span kernel (HS_FLAG_STAGED_SPANS), the one path with bounded
    device waits and its own tile size over the same prefix array."""
    import torch

    lens = [4096, 100000, 0, 65536, 8, 250000, 16, 131072, 1 << 20]
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = hs_synth.batch(304, offsets)
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    hs = hs_lib.HarmonicSum(variants=hs_lib.STD, threshold=6.0, cand_capacity=1 << 16, max_spectra=len(lens),
                            flags=hs_lib.FLAG_STAGED_SPANS)
    mu, isig = hs_lib.hs_noise_calibration("std", 32)
    hs.set_calibration("std", mu, isig)
    for tile_bins in (1024, 8192):
        hs_lib.hs_plan_set_tile_bins(hs.plan, "std", tile_bins)
        ref = hs.sum_batched("std", xd, od, first_id=3)
        assert hs.sync_status() == hs_lib.OK
        for call in range(2):
            o = hs.new_outputs(x.size, "std", "cuda")
            o["best_snr"].fill_(-5.0)
            hs_lib.hs_sum_batched_noalloc(hs.plan, "std", xd, od, hs.out_struct(o), first_id=3)
            torch.cuda.synchronize()
            assert torch.equal(o["best_snr"], ref["best_snr"]), (tile_bins, call)
            assert torch.equal(o["best_h"], ref["best_h"]), (tile_bins, call)
            assert int(o["cand_count"].item()) == int(ref["cand_count"].item())


def test_noalloc_rejects_batches_beyond_its_scratch(hs_lib):
    import torch

    n = hs_lib.NOALLOC_MAX_SPECTRA + 1
    offsets = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    x = torch.zeros(16, device="cuda")
    hs = hs_lib.HarmonicSum(variants=hs_lib.FBIN, threshold=6.0)
    o = hs.new_outputs(16, "fbin", "cuda")
    with pytest.raises(hs_lib.HSError) as e:
        hs_lib.hs_sum_batched_noalloc(hs.plan, "fbin", x, offsets, hs.out_struct(o))
    assert e.value.status == hs_lib.ERR_INVALID
