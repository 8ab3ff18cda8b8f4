"""Full-size workloads on the GPU, checked against the oracle on sampled bins (evaluated one by one)
and by properties that hold at any size.

* DM-trial batch: 2048 spectra, lengths in {2^19..2^22} (4.02 G bins), all four variants, run
  through the graph-captured persistent launch the benchmark times.
* differentiation: 256 spectra x 2^20, Eq. 1 and Eq. 2, backward through hs_backward.
* precision: 4096 spectra x 2^20 stored FP16 and BF16 by the device cast.
"""
import numpy as np
import pytest

import hs_synth
import oracle

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

VARIANTS = ["std", "max", "fbin", "greedy"]
THR = 6.0


def _sample_bins(rng, n, tile=1024):
    """First and last bins, bins around tile and pair boundaries, and random bins of one spectrum."""
    b = [0, 1, 2, 3, n - 4, n - 3, n - 2, n - 1]
    for k in rng.integers(1, max(2, n // tile), 6):
        b += [int(k) * tile - 1, int(k) * tile, int(k) * tile + 1]
    b += rng.integers(0, n, 24).tolist()
    b += rng.integers(0, max(1, n // 32), 8).tolist()  # low bins, where every harmonic is valid
    return np.unique(np.clip(np.asarray(b, np.int64), 0, n - 1))


def _check_candidates_property(torch, o, capacity):
    """The stored candidates are exactly bins above threshold, carrying those bins' outputs."""
    cnt = int(o["cand_count"].item())
    assert cnt == int((o["best_snr"] > THR).sum().item())
    return min(cnt, capacity)


def test_dm_trial_batch_full_size(hs_lib):
    import torch

    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(2048)
    total = int(offsets[-1])
    xh = torch.empty(total, dtype=torch.float32, pin_memory=True)
    hs_synth.batch(seed, offsets, pulsars, out=xh.data_ptr())
    x_np = xh.numpy()
    xd = xh.cuda()
    od = torch.from_numpy(offsets).cuda()
    cap = 1 << 24
    h = hs_lib.HarmonicSum(variants=0xF, hmax=32, max_bins=1 << 22, threshold=THR, cand_capacity=cap,
                           max_spectra=2048)
    rng = np.random.default_rng(2)
    spectra = np.unique(np.concatenate([[0, 1, 2047], rng.integers(0, 2048, 40)]))
    for v in VARIANTS:
        mu, isig = oracle.noise_calibration(v, 32)
        h.set_calibration(v, mu, isig)
        o = h.new_outputs(total, v, "cuda")
        g = hs_lib.hs_graph_create_batched(h.plan, hs_lib.VARIANTS[v], xd, od, [h.out_struct(o)], h.ws)
        hs_lib.hs_graph_launch(g)
        torch.cuda.synchronize()
        assert h.sync_status() in (hs_lib.OK, hs_lib.WARN_CAND_OVERFLOW)
        n_c = _check_candidates_property(torch, o, cap)
        c = hs_lib.read_candidates(o)
        assert c.size == n_c
        glob = torch.from_numpy(offsets[c["spectrum"].astype(np.int64)] + c["bin"].astype(np.int64)).cuda()
        assert torch.equal(o["best_snr"][glob].cpu(), torch.from_numpy(c["snr"].copy()))
        bs = o["best_snr"].cpu().numpy()
        bh = o["best_h"].cpu().numpy()
        path = o["path"].cpu().numpy().view(np.uint32) if v == "greedy" else None
        for s in spectra:
            a, b = int(offsets[s]), int(offsets[s + 1])
            bins = _sample_bins(rng, b - a)
            r = oracle.hs_bins(v, x_np[a:b], bins, mu=mu, isig=isig)
            np.testing.assert_array_equal(bs[a + bins], r["best_snr"], err_msg="%s spectrum %d" % (v, s))
            np.testing.assert_array_equal(bh[a + bins], r["best_h"])
            if path is not None:
                np.testing.assert_array_equal(path[a + bins], r["path"])
        hs_lib.hs_graph_destroy(g)
        del o
        torch.cuda.empty_cache()


@pytest.mark.parametrize("variant", ["std", "max"])
def test_adjoint_full_size(hs_lib, variant):
    import torch

    n_s, n_b = 256, 1 << 20
    x, offsets, _ = hs_synth.uniform_batch(n_s, n_b, seed=4000, pulsar_fraction=0.0)
    mu, isig = oracle.noise_calibration(variant, 32)
    h = hs_lib.HarmonicSum(variants=hs_lib.VARIANTS[variant], max_bins=n_b, threshold=THR, max_spectra=n_s,
                           calibration={variant: (mu, isig)})
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    xr = xd.clone().requires_grad_(True)
    snr, bh = hs_lib.HarmonicSumFn.apply(xr, h, variant, od)
    torch.nn.functional.softplus(snr - 5.0).sum().backward()
    grad = xr.grad
    g = torch.sigmoid(snr.detach() - 5.0)
    # property: every bin scatters its weight g * c_H * isig_H to exactly H* bins
    c = torch.tensor([0.0] + [float(np.float32(1.0 / np.sqrt(k))) for k in range(1, 33)], device="cuda",
                     dtype=torch.float64)
    isg = torch.from_numpy(isig.astype(np.float64)).cuda()
    bhl = bh.long()
    expect_total = (g.double() * c[bhl] * isg[bhl] * bhl.double()).sum().item()
    assert grad.double().sum().item() == pytest.approx(expect_total, rel=1e-6)
    # sampled spectra: the whole FP64 oracle gradient, routed by the oracle's own FP32 best H
    for s in (0, 131, 255):
        a, b = int(offsets[s]), int(offsets[s + 1])
        r32 = oracle.hs_1d(variant, x[a:b], mu=mu, isig=isig, nthreads=8)
        np.testing.assert_array_equal(bh[a:b].cpu().numpy(), r32["best_h"])
        gn = g[a:b].double().cpu().numpy()
        exp = oracle.grad_1d(variant, x[a:b], gn, r32["best_h"], isig=isig.astype(np.float64))
        np.testing.assert_allclose(grad[a:b].double().cpu().numpy(), exp, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_precision_full_size(hs_lib, dtype):
    import torch

    n_s, n_b = 4096, 1 << 20
    code = {"f16": hs_lib.F16, "bf16": hs_lib.BF16}[dtype]
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    seed = 5000
    rng = np.random.default_rng(seed)
    offsets = np.arange(n_s + 1, dtype=np.int64) * n_b
    xh = torch.empty(n_s * n_b, dtype=torch.float32, pin_memory=True)
    hs_synth.batch(seed, offsets, None, out=xh.data_ptr())
    od = torch.from_numpy(offsets).cuda()
    xs = torch.empty(n_s * n_b, dtype=tdt, device="cuda")
    zeros = torch.zeros(n_s, device="cuda")
    ones = torch.ones(n_s, device="cuda")
    hs_lib.hs_standardize_cast(xh.cuda(), od, zeros, ones, code, xs)
    x_np = xh.numpy()
    h = hs_lib.HarmonicSum(variants=0xF, dtype=code, max_bins=n_b, threshold=THR, cand_capacity=1 << 24,
                           max_spectra=n_s)
    spectra = np.unique(np.concatenate([[0, n_s - 1], rng.integers(0, n_s, 10)]))
    stored = {}
    for s in spectra:
        a, b = int(offsets[s]), int(offsets[s + 1])
        bits = oracle.standardize_cast(x_np[a:b], 0.0, 1.0, dtype)
        got = xs[a:b].view(torch.int16).cpu().numpy().view(np.uint16)
        np.testing.assert_array_equal(got, bits)  # the device cast itself, bit for bit
        if dtype == "f16":
            wide = bits.view(np.float16).astype(np.float32)
        else:
            wide = (bits.astype(np.uint32) << 16).view(np.float32)
        stored[s] = wide
    for v in VARIANTS:
        mu, isig = oracle.noise_calibration(v, 32)
        h.set_calibration(v, mu, isig)
        o = h.new_outputs(n_s * n_b, v, "cuda")
        h.sum_batched(v, xs, od, out=o)
        torch.cuda.synchronize()
        _check_candidates_property(torch, o, 1 << 24)
        bs = o["best_snr"].cpu().numpy()
        bhh = o["best_h"].cpu().numpy()
        for s in spectra:
            a = int(offsets[s])
            bins = _sample_bins(rng, n_b)
            r = oracle.hs_bins(v, stored[s], bins, mu=mu, isig=isig)
            np.testing.assert_array_equal(bs[a + bins], r["best_snr"], err_msg="%s %s spectrum %d" % (dtype, v, s))
            np.testing.assert_array_equal(bhh[a + bins], r["best_h"])
        del o
        torch.cuda.empty_cache()


def test_precision_error_and_candidate_agreement(hs_lib):
    """Reduced-precision storage against FP64 on the original FP32 data.  Storing each bin with unit
    roundoff u (FP16 2^-11, BF16 2^-8) moves a term by at most u*max|x|, so an snr built from H
    terms moves by at most sqrt(H)*u*max|x|*isig_H (plus FP32 summation error, far smaller): that
    bound, at H = 32, is the tie margin.  Errors must stay inside it, and the candidate set must equal
    FP64's for every bin whose FP64 snr is further than the margin from the threshold.  Eq. 4 routes
    through comparisons, so rounding can flip a left/right choice and change the sum by a whole
    term: its bins whose path differs from FP64's are excluded (and must be few)."""
    import torch

    n_s, n_b = 8, 1 << 20
    x, offsets, _ = hs_synth.uniform_batch(n_s, n_b, seed=5100, pulsar_fraction=0.5)
    od = torch.from_numpy(offsets).cuda()
    xmax = float(np.abs(x).max())
    for dtype, code, tdt, u in (("f16", hs_lib.F16, torch.float16, 2.0 ** -11),
                                ("bf16", hs_lib.BF16, torch.bfloat16, 2.0 ** -8)):
        xs = torch.from_numpy(x).to(tdt).cuda()
        for v in VARIANTS:
            mu, isig = oracle.noise_calibration(v, 32)
            margin = np.sqrt(32) * u * xmax * float(isig[1:].max()) * 1.01 + 1e-4
            h = hs_lib.HarmonicSum(variants=hs_lib.VARIANTS[v], dtype=code, max_bins=n_b, threshold=THR,
                                   cand_capacity=1 << 20, max_spectra=n_s, calibration={v: (mu, isig)})
            o = h.sum_batched(v, xs, od)
            lo = o["best_snr"].cpu().numpy().astype(np.float64)
            r64 = oracle.hs_batched(v, x, offsets, mu=mu, isig=isig, fp64=True, nthreads=8)
            ok = np.isfinite(r64["best_snr"])
            if v == "greedy":
                same = o["path"].cpu().numpy().view(np.uint32) == r64["path"]
                assert (~same[ok]).mean() < 0.05, (dtype, (~same[ok]).mean())
                ok &= same
            err = np.abs(lo[ok] - r64["best_snr"][ok])
            assert err.max() < margin, (dtype, v, err.max(), margin)
            far = ok & (np.abs(r64["best_snr"] - THR) > margin)
            np.testing.assert_array_equal(lo[far] > THR, r64["best_snr"][far] > THR)
