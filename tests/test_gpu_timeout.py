"""The error path of the bounded device waits, exercised without any GPU fault.

The staged Eq. 1 kernel (HS_FLAG_STAGED_SPANS) is the library's only kernel that waits: its consumer
warps wait on shared-memory barriers for bulk copies, and its producer waits for slots to be
released, each wait giving up after about a second.  HS_FLAG_CHECK_TIMEOUT makes the work item
holding the batch's first tile arm one slot for more bytes than it copies, so that slot never fills:
a wait on a barrier that nothing completes.  The launch must still end on its own, the status word
must read HS_ERR_TIMEOUT, and the next ordinary call on the same workspace must be correct.
"""
import time

import numpy as np
import pytest

import hs_synth
import oracle

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def test_staged_wait_that_runs_out_reports_timeout(hs_lib):
    import torch

    lens = [1 << 16] * 40 + [4104, 8, 100000]
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = hs_synth.batch(911, offsets)
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    mu, isig = hs_lib.hs_noise_calibration("std", 32)
    bad = hs_lib.HarmonicSum(variants=hs_lib.STD, threshold=6.0, cand_capacity=1 << 16, max_spectra=len(lens),
                             flags=hs_lib.FLAG_STAGED_SPANS | hs_lib.FLAG_CHECK_TIMEOUT,
                             calibration={"std": (mu, isig)})
    hs_lib.hs_plan_set_tile_bins(bad.plan, "std", 1024)
    t0 = time.perf_counter()
    bad.sum_batched("std", xd, od)
    torch.cuda.synchronize()  # the launch ends by itself: every wait is bounded
    elapsed = time.perf_counter() - t0
    with pytest.raises(hs_lib.HSError) as e:
        bad.sync_status()
    assert e.value.status == hs_lib.ERR_TIMEOUT
    assert elapsed < 30.0, elapsed

    # the same workspace, cleared, serves an ordinary staged call that equals the oracle
    good = hs_lib.HarmonicSum(variants=hs_lib.STD, threshold=6.0, cand_capacity=1 << 16, max_spectra=len(lens),
                              flags=hs_lib.FLAG_STAGED_SPANS, calibration={"std": (mu, isig)})
    good.ws = bad.ws
    hs_lib.hs_workspace_init(good.plan, good.ws)
    hs_lib.hs_plan_set_tile_bins(good.plan, "std", 1024)
    o = good.sum_batched("std", xd, od)
    assert good.sync_status() == hs_lib.OK
    r = oracle.hs_batched("std", x, offsets, mu=mu, isig=isig, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    assert int(o["cand_count"].item()) == int((r["best_snr"] > 6.0).sum())
