"""GPU path against the CPU oracle, through the C ABI.

FP32 results (snr bits, best H, the Eq. 4 path, the every-H table, the candidate set) must equal
the oracle's FP32 mode bit for bit; FP16/BF16 storage must equal the FP32 oracle run on the widened
values bit for bit.  Sizes span several tiles and a ragged tail; full-size workloads are checked on
sampled bins the oracle evaluates one by one, plus properties that hold at any size.
"""
import numpy as np
import pytest

import hs_synth
import oracle

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

VARIANTS = ["std", "max", "fbin", "greedy"]
THR = 6.0


@pytest.fixture(scope="module")
def torch():
    import torch as t

    return t


def _calib(variant, calibrated):
    return oracle.noise_calibration(variant, 32) if calibrated else (None, None)


def _make(hs_mod, variant, calibrated, dtype=0, max_bins=1 << 22, cap=1 << 16, flags=1, max_spectra=1, hmax=32):
    hs = hs_mod.HarmonicSum(variants=hs_mod.VARIANTS[variant], hmax=hmax, dtype=dtype, max_bins=max_bins,
                            threshold=THR, cand_capacity=cap, flags=flags, max_spectra=max_spectra)
    mu, isig = _calib(variant, calibrated)
    if mu is not None:
        hs.set_calibration(variant, mu, isig)
    return hs, mu, isig


def _widen(torch, x_np, dtype):
    """Store as FP16/BF16 (round to nearest even) and return (device tensor, widened float32 copy)."""
    t = torch.from_numpy(x_np)
    if dtype == "f16":
        s = t.to(torch.float16)
    elif dtype == "bf16":
        s = t.to(torch.bfloat16)
    else:
        s = t
    return s.cuda(), s.float().numpy()


def _check_candidates(hs_mod, o, best_snr, best_h, spectrum_offsets=None, first_id=0):
    cands = hs_mod.read_candidates(o)
    exp = np.nonzero(best_snr > THR)[0]
    assert int(o["cand_count"].item()) == exp.size
    assert cands.size == exp.size
    if spectrum_offsets is None:
        got = np.sort(cands["bin"].astype(np.int64))
        np.testing.assert_array_equal(got, exp)
        order = np.argsort(cands["bin"])
        np.testing.assert_array_equal(cands["snr"][order], best_snr[exp])
        np.testing.assert_array_equal(cands["h"][order], best_h[exp])
    else:
        glob = spectrum_offsets[cands["spectrum"].astype(np.int64) - first_id] + cands["bin"].astype(np.int64)
        order = np.argsort(glob)
        np.testing.assert_array_equal(glob[order], exp)
        np.testing.assert_array_equal(cands["snr"][order], best_snr[exp])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("calibrated", [False, True])
def test_1d_pulsar_spectrum_bit_exact(hs_lib, torch, variant, calibrated):
    x, _ = hs_synth.spectrum_1d_pulsar()
    hs, mu, isig = _make(hs_lib, variant, calibrated)
    o = hs.sum_1d(variant, torch.from_numpy(x).cuda(), all_h=True)
    torch.cuda.synchronize()
    assert hs.sync_status() == hs_lib.OK
    r = oracle.hs_1d(variant, x, hmax=32, mu=mu, isig=isig, all_h=True, nthreads=8)
    np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    if variant == "greedy":
        np.testing.assert_array_equal(o["path"].cpu().numpy().view(np.uint32), r["path"])
    _check_candidates(hs_lib, o, r["best_snr"], r["best_h"])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n_bins", [1, 2, 3, 31, 33, 257, 1000, 4097, 65536 + 13, 300001])
def test_1d_ragged_sizes_bit_exact(hs_lib, torch, variant, n_bins):
    x = hs_synth.spectrum(77, n_bins, n_bins)
    hs, mu, isig = _make(hs_lib, variant, True)
    o = hs.sum_1d(variant, torch.from_numpy(x).cuda(), all_h=True)
    r = oracle.hs_1d(variant, x, hmax=32, mu=mu, isig=isig, all_h=True, nthreads=8)
    np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    if variant == "greedy":
        np.testing.assert_array_equal(o["path"].cpu().numpy().view(np.uint32), r["path"])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n_bins", [2, 31, 33, 100, 257, 1000, 4097, 8191, 65536 + 13, 300001, 1 << 20])
def test_1d_fast_paths_bit_exact(hs_lib, torch, variant, n_bins):
    """Without the every-H table the kernels take their fast paths (Eq. 1 output pairs, Eq. 2
    harmonics 1-4 by plain loads and longer windows by aligned 16-byte chunks); they must still
    equal the oracle bit for bit."""
    x = hs_synth.spectrum(79, n_bins, n_bins, pulsar=dict(shape=1, n_harm=20, f0=n_bins / 97.3, amp=9.0, width=1.5))
    hs, mu, isig = _make(hs_lib, variant, True, flags=0)
    o = hs.sum_1d(variant, torch.from_numpy(x).cuda())
    r = oracle.hs_1d(variant, x, hmax=32, mu=mu, isig=isig, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    if variant == "greedy":
        np.testing.assert_array_equal(o["path"].cpu().numpy().view(np.uint32), r["path"])
    _check_candidates(hs_lib, o, r["best_snr"], r["best_h"])


@pytest.mark.parametrize("variant", ["std", "max"])
@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_1d_fast_paths_reduced_precision(hs_lib, torch, variant, dtype):
    x = hs_synth.spectrum(80, 0, 200003)
    xd, xw = _widen(torch, x, dtype)
    hs, mu, isig = _make(hs_lib, variant, True, dtype={"f16": 1, "bf16": 2}[dtype], flags=0)
    o = hs.sum_1d(variant, xd)
    r = oracle.hs_1d(variant, xw, hmax=32, mu=mu, isig=isig, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("hmax", [1, 7, 16])
def test_1d_smaller_hmax(hs_lib, torch, variant, hmax):
    x = hs_synth.spectrum(78, 0, 20000)
    hs, _, _ = _make(hs_lib, variant, False, hmax=hmax)
    o = hs.sum_1d(variant, torch.from_numpy(x).cuda(), all_h=True)
    r = oracle.hs_1d(variant, x, hmax=hmax, all_h=True)
    np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_1d_reduced_precision_bit_exact(hs_lib, torch, variant, dtype):
    x, _ = hs_synth.spectrum_1d_pulsar()
    xd, xw = _widen(torch, x, dtype)
    hs, mu, isig = _make(hs_lib, variant, True, dtype={"f16": 1, "bf16": 2}[dtype])
    o = hs.sum_1d(variant, xd, all_h=True)
    r = oracle.hs_1d(variant, xw, hmax=32, mu=mu, isig=isig, all_h=True, nthreads=8)
    np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])


def test_special_inputs(hs_lib, torch):
    """Constant spectra (ties everywhere: smallest H, left bins), zeros, spikes."""
    for x in (np.zeros(5000, np.float32), np.full(5000, 1.5, np.float32), np.full(5000, -2.0, np.float32)):
        x = x.copy()
        x[1234] = 40.0
        for v in VARIANTS:
            hs, _, _ = _make(hs_lib, v, False)
            o = hs.sum_1d(v, torch.from_numpy(x).cuda(), all_h=True)
            r = oracle.hs_1d(v, x, all_h=True)
            np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
            np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
            if v == "greedy":
                np.testing.assert_array_equal(o["path"].cpu().numpy().view(np.uint32), r["path"])


@pytest.mark.parametrize("variant", VARIANTS)
def test_batched_uneven_bit_exact(hs_lib, torch, variant):
    lens = [0, 1, 5, 4096, 100003 - 3, 65536, 8, 0, 250000, 12]
    lens = [(l + 3) // 4 * 4 for l in lens]  # keep every spectrum 16-byte aligned
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = hs_synth.batch(91, offsets)
    hs, mu, isig = _make(hs_lib, variant, True, flags=0, max_spectra=len(lens))
    o = hs.sum_batched(variant, torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda(), first_id=100)
    assert hs.sync_status() == hs_lib.OK
    r = oracle.hs_batched(variant, x, offsets, mu=mu, isig=isig, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    if variant == "greedy":
        np.testing.assert_array_equal(o["path"].cpu().numpy().view(np.uint32), r["path"])
    _check_candidates(hs_lib, o, r["best_snr"], r["best_h"], offsets, first_id=100)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_batched_staged_spans_bit_exact(hs_lib, torch, dtype):
    """Eq. 1 with the input spans staged in shared memory (HS_FLAG_STAGED_SPANS): tiles of 1024
    bins, short spectra and ragged tails evaluated directly, several items per spectrum, candidates."""
    lens = [0, 8, 1024, 1024 + 8, 1032 + 8, 4096, 100003 - 3, 8200, 0, 250000, 1 << 18, 16]
    lens = [(l + 7) // 8 * 8 for l in lens]  # 16-byte aligned starts for every storage type
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x32 = hs_synth.batch(93, offsets)
    xd, xw = _widen(torch, x32, dtype)
    code = {"f32": 0, "f16": 1, "bf16": 2}[dtype]
    hs, mu, isig = _make(hs_lib, "std", True, dtype=code, flags=hs_lib.FLAG_STAGED_SPANS, max_spectra=len(lens))
    for tile_bins in (1024, 8192):  # one or eight 1024-bin tiles per work item
        hs_lib.hs_plan_set_tile_bins(hs.plan, "std", tile_bins)
        o = hs.sum_batched("std", xd, torch.from_numpy(offsets).cuda(), first_id=7)
        assert hs.sync_status() == hs_lib.OK
        r = oracle.hs_batched("std", xw, offsets, mu=mu, isig=isig, nthreads=8)
        np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
        np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
        _check_candidates(hs_lib, o, r["best_snr"], r["best_h"], offsets, first_id=7)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_eq1_16bit_batch_through_fp32_groups(hs_lib, torch, dtype):
    """Eq. 1 of a 16-bit batch runs groups of up to 64 spectra through an FP32 copy in the workspace:
    141 spectra (three groups, the last short), empty and ragged spectra, a batch slice with absolute
    offsets, equal to the FP32 oracle on the widened values."""
    rng = np.random.default_rng(5)
    lens = [int(rng.integers(0, 20000)) for _ in range(140)] + [12345]
    lens[3] = lens[40] = 0
    lens = [(l + 7) // 8 * 8 for l in lens[:-1]] + [lens[-1]]  # 16-byte aligned starts
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    offsets += 64  # the batch starts 64 elements into the buffer
    x32 = hs_synth.batch(41, np.concatenate([[0], offsets]))
    xd, xw = _widen(torch, x32, dtype)
    code = {"f16": 1, "bf16": 2}[dtype]
    hs, mu, isig = _make(hs_lib, "std", True, dtype=code, max_bins=1 << 16, flags=0, max_spectra=len(lens),
                         cap=1 << 18)
    o = hs.new_outputs(xd.numel(), "std", "cuda")
    o["best_snr"].fill_(-123.0)
    hs_lib.hs_sum_batched(hs.plan, "std", xd, torch.from_numpy(offsets).cuda(), hs.out_struct(o), hs.ws, 5)
    assert hs.sync_status() == hs_lib.OK
    r = oracle.hs_batched("std", xw, offsets, mu=mu, isig=isig, nthreads=8)
    got = o["best_snr"].cpu().numpy()  # the oracle's arrays start at the batch's first offset
    np.testing.assert_array_equal(got[64:], r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy()[64:], r["best_h"])
    assert np.all(got[:64] == -123.0)  # outside the batch: untouched
    _check_candidates(hs_lib, o, r["best_snr"], r["best_h"], offsets - 64, first_id=5)


def test_eq1_16bit_groups_refuse_spectra_outside_the_widened_range(hs_lib, torch):
    """Offsets that are not monotone: a spectrum of valid length that lies outside its group's
    widened range is skipped and reported (HS_ERR_INVALID from the status word), never read."""
    x32 = hs_synth.batch(42, np.array([0, 4096], np.int64))
    xd, _ = _widen(torch, x32, "f16")
    hs, _, _ = _make(hs_lib, "std", True, dtype=1, max_bins=4096, flags=0, max_spectra=3)
    offsets = np.array([1024, 2048, 0, 512], np.int64)  # [1024, 2048) valid, then negative, then [0, 512)
    o = hs.new_outputs(xd.numel(), "std", "cuda")
    o["best_snr"].fill_(-123.0)
    hs_lib.hs_sum_batched(hs.plan, "std", xd, torch.from_numpy(offsets).cuda(), hs.out_struct(o), hs.ws)
    with pytest.raises(hs_lib.HSError) as e:
        hs.sync_status()
    assert e.value.status == hs_lib.ERR_INVALID
    assert np.all(o["best_snr"].cpu().numpy() == -123.0)


def test_staged_spans_slice_and_graph(hs_lib, torch):
    """The staged path on a batch slice with absolute offsets, captured in a graph and replayed."""
    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(12, lengths=(1 << 15, 1 << 16, 1 << 17))
    x = hs_synth.batch(seed, offsets, pulsars)
    xd = torch.from_numpy(x).cuda()
    hs = hs_lib.HarmonicSum(variants=hs_lib.STD, threshold=THR, cand_capacity=1 << 16, max_spectra=12,
                            flags=hs_lib.FLAG_STAGED_SPANS)
    sl = torch.from_numpy(offsets[4:10].copy()).cuda()  # spectra 4..8, absolute offsets
    o = hs.new_outputs(x.size, "std", "cuda")
    g = hs_lib.hs_graph_create_batched(hs.plan, hs_lib.STD, xd, sl, [hs.out_struct(o)], hs.ws)
    r = oracle.hs_batched("std", x, offsets, nthreads=8)
    a, b = int(offsets[4]), int(offsets[9])
    for rep in range(2):
        o["cand_count"].zero_()
        hs_lib.hs_graph_launch(g)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o["best_snr"].cpu().numpy()[a:b], r["best_snr"][a:b])
        np.testing.assert_array_equal(o["best_h"].cpu().numpy()[a:b], r["best_h"][a:b])
        assert int(o["cand_count"].item()) == int((r["best_snr"][a:b] > THR).sum())
    hs_lib.hs_graph_destroy(g)


def test_batched_bad_layout_is_reported(hs_lib, torch):
    offsets = np.array([0, 1000, 999, 3000], np.int64)  # a negative length
    x = torch.zeros(4000, device="cuda")
    hs, _, _ = _make(hs_lib, "fbin", False, flags=0, max_spectra=3)
    hs.sum_batched("fbin", x, torch.from_numpy(offsets).cuda())
    with pytest.raises(hs_lib.HSError) as e:
        hs.sync_status()
    assert e.value.status == hs_lib.ERR_INVALID


def test_candidate_overflow_reports_true_count(hs_lib, torch):
    x = hs_synth.spectrum(5, 0, 200000)
    hs, _, _ = _make(hs_lib, "fbin", False, cap=8)
    o = hs.sum_1d("fbin", torch.from_numpy(x).cuda())
    assert hs.sync_status() == hs_lib.WARN_CAND_OVERFLOW
    r = oracle.hs_1d("fbin", x)
    assert int(o["cand_count"].item()) == int((r["best_snr"] > THR).sum())
    c = hs_lib.read_candidates(o)
    assert c.size == 8
    assert (r["best_snr"][c["bin"]] == c["snr"]).all()


def test_graph_replay_matches_direct(hs_lib, torch):
    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(24, lengths=(1 << 14, 1 << 15, 1 << 16))
    x = hs_synth.batch(seed, offsets, pulsars)
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    hs = hs_lib.HarmonicSum(variants=0xF, threshold=THR, cand_capacity=1 << 16, max_spectra=24)
    outs, structs = [], []
    for v in VARIANTS:
        o = hs.new_outputs(x.size, v, "cuda")
        outs.append(o)
        structs.append(hs.out_struct(o))
    g = hs_lib.hs_graph_create_batched(hs.plan, 0xF, xd, od, structs, hs.ws)
    for rep in range(2):
        for o in outs:
            o["cand_count"].zero_()
        hs_lib.hs_graph_launch(g)
        torch.cuda.synchronize()
        for v, o in zip(VARIANTS, outs):
            r = oracle.hs_batched(v, x, offsets, nthreads=8)
            np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
            np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
            assert int(o["cand_count"].item()) == int((r["best_snr"] > THR).sum())
    hs_lib.hs_graph_destroy(g)


def test_sort_candidates(hs_lib, torch):
    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(16, lengths=(1 << 16, 1 << 17))
    x = hs_synth.batch(seed, offsets, pulsars)
    hs = hs_lib.HarmonicSum(variants=0xF, threshold=3.0, cand_capacity=1 << 20, max_spectra=16)
    o = hs.new_outputs(x.size, "fbin", "cuda")
    hs.sum_batched("fbin", torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda(), out=o)
    hs.sum_batched("max", torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda(),
                   out={**hs.new_outputs(x.size, "max", "cuda", candidates=False), "cand": o["cand"],
                        "cand_count": o["cand_count"]})
    before = hs_lib.read_candidates(o).copy()
    assert before.size > 10000
    tmp = torch.empty_like(o["cand"])
    hs_lib.hs_sort_candidates(o["cand"], o["cand_count"], tmp, hs.ws)
    after = hs_lib.read_candidates(o)
    key = np.lexsort((before["bin"], before["z"], before["spectrum"], before["variant"]))
    np.testing.assert_array_equal(after, before[key])


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_standardize_cast_bit_exact(hs_lib, torch, dtype):
    offsets = np.array([0, 1000, 1000, 50000, 123456], np.int64)
    p = hs_synth.batch(12, offsets, raw=True)
    mu = np.array([1.0, 0.5, 1.1, 0.9], np.float32)
    sd = np.array([1.0, 2.0, 0.9, 1.3], np.float32)
    out = torch.empty(p.size, dtype=torch.int16, device="cuda")
    hs_lib.hs_standardize_cast(torch.from_numpy(p).cuda(), torch.from_numpy(offsets).cuda(),
                               torch.from_numpy(mu).cuda(), torch.from_numpy(sd).cuda(),
                               {"f16": 1, "bf16": 2}[dtype], out)
    got = out.cpu().numpy().view(np.uint16)
    for s in range(4):
        a, b = offsets[s], offsets[s + 1]
        np.testing.assert_array_equal(got[a:b], oracle.standardize_cast(p[a:b], mu[s], sd[s], dtype))


def test_2d_bit_exact(hs_lib, torch):
    nz, z_min, nb = 41, -20, 6000
    plane, _ = hs_synth.fdas_plane(0, nz=nz, z_min=z_min, n_bins=nb)
    hs = hs_lib.HarmonicSum(variants=1, hmax=16, nz=nz, z_min=z_min, max_bins=nb, threshold=THR,
                            cand_capacity=1 << 16)
    o = hs.sum_2d(torch.from_numpy(plane).cuda())
    r = oracle.hs_2d(plane, z_min, hmax=16, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    np.testing.assert_array_equal(o["best_snr_n"].cpu().numpy(), r["best_snr_n"])
    np.testing.assert_array_equal(o["best_h_n"].cpu().numpy(), r["best_h_n"])
    np.testing.assert_array_equal(o["best_z_n"].cpu().numpy().astype(np.int32), r["best_z_n"])
    c = hs_lib.read_candidates(o)
    exp = np.argwhere(r["best_snr"] > THR)
    assert c.size == exp.shape[0]
    got = np.sort((c["z"].astype(np.int64) - z_min) * nb + c["bin"])
    np.testing.assert_array_equal(got, np.sort(exp[:, 0] * nb + exp[:, 1]))


@pytest.mark.parametrize("nb,hmax", [(3001, 16), (4000, 9), (4000, 1), (2, 16)])
def test_2d_generic_and_edge_paths(hs_lib, torch, nb, hmax):
    """Odd row lengths and hmax < 16 take the generic kernel; tiny rows test the edges."""
    nz, z_min = 21, -10
    plane, _ = hs_synth.fdas_plane(5, nz=nz, z_min=z_min, n_bins=max(nb, 64))
    plane = np.ascontiguousarray(plane[:, :nb])
    stride = (nb + 3) // 4 * 4  # rows 16-byte aligned, as the ABI requires
    padded = torch.zeros((nz, stride), device="cuda")
    padded[:, :nb] = torch.from_numpy(plane).cuda()
    hs = hs_lib.HarmonicSum(variants=1, hmax=hmax, nz=nz, z_min=z_min, max_bins=nb, threshold=THR,
                            cand_capacity=1 << 16)
    o = hs.sum_2d(padded[:, :nb])
    r = oracle.hs_2d(plane, z_min, hmax=hmax, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    np.testing.assert_array_equal(o["best_snr_n"].cpu().numpy(), r["best_snr_n"])
    np.testing.assert_array_equal(o["best_z_n"].cpu().numpy().astype(np.int32), r["best_z_n"])


@pytest.mark.parametrize("variant", ["std", "fbin"])
@pytest.mark.parametrize("z_min,nz,nb", [(-32766, 32767, 64), (0, 32767, 64), (-300, 301, 130), (-32766, 32767, 63)])
def test_2d_extreme_drift_ranges(hs_lib, torch, variant, z_min, nz, nb):
    """Rows at the ends of the drift range the ABI accepts (|z| up to 32766), ranges on one side of
    z = 0 only, and rows padded to a longer stride: every output equal to the oracle's."""
    plane, _ = hs_synth.fdas_plane(7, nz=nz, z_min=z_min, n_bins=nb)
    stride = (nb + 3) // 4 * 4
    padded = torch.zeros((nz, stride), device="cuda")
    padded[:, :nb] = torch.from_numpy(plane).cuda()
    hs = hs_lib.HarmonicSum(variants=hs_lib.VARIANTS[variant], hmax=16, nz=nz, z_min=z_min, max_bins=nb,
                            threshold=THR, cand_capacity=1 << 20)
    o = hs.sum_2d(padded[:, :nb], variant=variant)
    assert hs.sync_status() == hs_lib.OK
    r = oracle.hs_2d(plane, z_min, hmax=16, variant=variant, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    np.testing.assert_array_equal(o["best_snr_n"].cpu().numpy(), r["best_snr_n"])
    np.testing.assert_array_equal(o["best_h_n"].cpu().numpy(), r["best_h_n"])
    np.testing.assert_array_equal(o["best_z_n"].cpu().numpy().astype(np.int32), r["best_z_n"])
    assert int(o["cand_count"].item()) == int((r["best_snr"] > THR).sum())


def test_2d_full_size_sampled(hs_lib, torch):
    nz, z_min, nb = 201, -100, 1 << 21
    plane, _ = hs_synth.fdas_plane(3, nz=nz, z_min=z_min, n_bins=nb)
    hs = hs_lib.HarmonicSum(variants=1, hmax=16, nz=nz, z_min=z_min, max_bins=nb, threshold=THR,
                            cand_capacity=1 << 22)
    o = hs.sum_2d(torch.from_numpy(plane).cuda())
    assert hs.sync_status() == hs_lib.OK
    rng = np.random.default_rng(1)
    rows = np.concatenate([rng.integers(0, nz, 3000), [0, nz - 1, 100, 100]])
    bins = np.concatenate([rng.integers(0, nb, 3000), [nb - 1, 0, 0, nb - 1]])
    r = oracle.hs_2d_cells(plane, z_min, rows, bins)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy()[rows, bins], r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy()[rows, bins], r["best_h"])
    for n in [0, 1, 777, nb - 1]:
        rr = oracle.hs_2d_cells(plane, z_min, np.arange(nz), np.full(nz, n))
        k = int(np.argmax(rr["best_snr"]))
        assert o["best_snr_n"][n].item() == rr["best_snr"][k]
        assert int(o["best_z_n"][n].item()) == z_min + k
    # candidates are exactly the cells above threshold
    assert int(o["cand_count"].item()) == int((o["best_snr"] > THR).sum().item())


@pytest.mark.parametrize("variant", VARIANTS)
def test_backward_matches_oracle_gradient(hs_lib, torch, variant):
    n_spec, N = 64, 4096
    offsets = np.arange(n_spec + 1, dtype=np.int64) * N
    x = hs_synth.batch(404, offsets)
    mu, isig = oracle.noise_calibration(variant, 32)
    hs = hs_lib.HarmonicSum(variants=hs_lib.VARIANTS[variant], max_bins=N, threshold=THR, max_spectra=n_spec,
                            calibration={variant: (mu, isig)})
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    o = hs.sum_batched(variant, xd, od)
    g = torch.sigmoid(o["best_snr"] - 5.0)
    grad = hs.backward(variant, xd, g, o["best_h"], o.get("path"), od).cpu().numpy().astype(np.float64)
    r32 = oracle.hs_batched(variant, x, offsets, mu=mu, isig=isig)
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r32["best_h"])
    gn = g.cpu().numpy().astype(np.float64)
    exp = np.zeros(x.size)
    for s in range(n_spec):
        a, b = offsets[s], offsets[s + 1]
        exp[a:b] = oracle.grad_1d(variant, x[a:b], gn[a:b], r32["best_h"][a:b], isig=isig.astype(np.float64))
    # FP32 atomics in any order against an FP64 sum: relative 1e-5 of the summed magnitudes
    np.testing.assert_allclose(grad, exp, rtol=1e-5, atol=1e-6)


# ---- power-of-two stages (HS_FLAG_POW2_STAGES), against the oracle's pow2 mode ----

@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_pow2_stages_bit_exact(hs_lib, torch, variant, dtype):
    x, _ = hs_synth.spectrum_1d_pulsar()
    xd, xw = _widen(torch, x, dtype)
    code = {"f32": 0, "bf16": 2}[dtype]
    hs, mu, isig = _make(hs_lib, variant, True, dtype=code, flags=hs_lib.FLAG_OUT_ALL_H | hs_lib.FLAG_POW2_STAGES)
    o = hs.sum_1d(variant, xd, all_h=True)
    r = oracle.hs_1d(variant, xw, hmax=32, mu=mu, isig=isig, all_h=True, pow2=True, nthreads=8)
    np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    # the fast paths (no every-H table): single spectrum and a batch
    hs2, _, _ = _make(hs_lib, variant, True, dtype=code, flags=hs_lib.FLAG_POW2_STAGES, max_spectra=3)
    o2 = hs2.sum_1d(variant, xd)
    np.testing.assert_array_equal(o2["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o2["best_h"].cpu().numpy(), r["best_h"])
    _check_candidates(hs_lib, o2, r["best_snr"], r["best_h"])
    n = x.size
    offsets = np.array([0, 4096, 4096 + 8, n // 8 * 8], np.int64)
    ob = hs2.sum_batched(variant, xd, torch.from_numpy(offsets).cuda())
    rb = oracle.hs_batched(variant, xw, offsets, mu=mu, isig=isig, pow2=True, nthreads=8)
    np.testing.assert_array_equal(ob["best_snr"].cpu().numpy()[: offsets[-1]], rb["best_snr"])
    np.testing.assert_array_equal(ob["best_h"].cpu().numpy()[: offsets[-1]], rb["best_h"])


# ---- Eq. 2 with the window j = 0..i (HS_FLAG_MAX_WINDOW0), against the oracle's "max0" ----

def _max0(hs_lib, dtype=0, max_spectra=1, flags=0):
    mu, isig = oracle.noise_calibration("max0", 32)
    hs = hs_lib.HarmonicSum(variants=hs_lib.MAX, dtype=dtype, max_bins=1 << 22, threshold=THR, cand_capacity=1 << 16,
                            flags=flags | hs_lib.FLAG_MAX_WINDOW0, max_spectra=max_spectra)
    hs.set_calibration("max", mu, isig)
    return hs, mu, isig


@pytest.mark.parametrize("n_bins", [2, 3, 33, 1000, 65536 + 13, 300001])
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_max_window0_bit_exact(hs_lib, torch, n_bins, dtype):
    x = hs_synth.spectrum(77, 0, n_bins)
    xd, xw = _widen(torch, x, dtype)
    hs, mu, isig = _max0(hs_lib, dtype={"f32": 0, "f16": 1, "bf16": 2}[dtype], flags=hs_lib.FLAG_OUT_ALL_H)
    o = hs.sum_1d("max", xd, all_h=True)
    r = oracle.hs_1d("max0", xw, hmax=32, mu=mu, isig=isig, all_h=True, nthreads=8)
    np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    _check_candidates(hs_lib, o, r["best_snr"], r["best_h"])


def test_max_window0_batched_and_adjoint(hs_lib, torch):
    lens = [0, 8, 4096, 100000, 12, 250000]
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = hs_synth.batch(95, offsets)
    hs, mu, isig = _max0(hs_lib, max_spectra=len(lens))
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    o = hs.sum_batched("max", xd, od, first_id=3)
    assert hs.sync_status() == hs_lib.OK
    r = oracle.hs_batched("max0", x, offsets, mu=mu, isig=isig, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    _check_candidates(hs_lib, o, r["best_snr"], r["best_h"], offsets, first_id=3)
    g = torch.sigmoid(o["best_snr"] - 5.0)
    grad = hs.backward("max", xd, g, o["best_h"], None, od).cpu().numpy().astype(np.float64)
    gn = g.cpu().numpy().astype(np.float64)
    exp = np.zeros(x.size)
    for s in range(len(lens)):
        a, b = offsets[s], offsets[s + 1]
        exp[a:b] = oracle.grad_1d("max0", x[a:b], gn[a:b], r["best_h"][a:b], isig=isig.astype(np.float64))
    np.testing.assert_allclose(grad, exp, rtol=1e-5, atol=1e-6)


def test_autograd_function(hs_lib, torch):
    N = 1 << 14
    x = torch.from_numpy(hs_synth.spectrum(8, 0, N)).cuda().requires_grad_(True)
    hs = hs_lib.HarmonicSum(variants=hs_lib.STD | hs_lib.MAX, max_bins=N, threshold=THR)
    snr, bh = hs_lib.HarmonicSumFn.apply(x, hs, "max")
    loss = torch.nn.functional.softplus(snr - 5).sum()
    loss.backward()
    g = torch.sigmoid(snr.detach() - 5)
    ref = hs.backward("max", x.detach(), g, bh)
    torch.testing.assert_close(x.grad, ref)


def test_autotune_batched_keeps_results(hs_lib, torch):
    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(12, lengths=(1 << 16, 1 << 18))
    x = hs_synth.batch(seed, offsets, pulsars)
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    hs = hs_lib.HarmonicSum(variants=0xF, threshold=THR, cand_capacity=1 << 16, max_spectra=12)
    for v in VARIANTS:
        o = hs.new_outputs(x.size, v, "cuda")
        hs_lib.hs_autotune_batched(hs.plan, v, xd, od, hs.out_struct(o), hs.ws)
        assert hs_lib.hs_plan_tile_bins(hs.plan, v) in (512, 1024, 2048, 4096, 8192, 16384)
        assert int(o["cand_count"].item()) == 0  # tuning leaves the candidate list alone
        hs.sum_batched(v, xd, od, out=o)
        r = oracle.hs_batched(v, x, offsets, nthreads=8)
        np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
        np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])


@pytest.mark.parametrize("caps", [(1, 1, 1, 1), (3, 1, 2, 1)])
def test_ctas_per_sm_cap_and_concurrent_streams_keep_results(hs_lib, torch, caps):
    """Persistent launches capped at k CTAs per SM, Eq. 1 on one stream and Eq. 2-4 on another at the
    same time (the caps leave room on every SM for both), equal the oracle bit for bit."""
    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(12, lengths=(1 << 16, 1 << 18))
    x = hs_synth.batch(seed, offsets, pulsars)
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    hs = hs_lib.HarmonicSum(variants=0xF, threshold=THR, cand_capacity=x.size, max_spectra=12)
    ws2 = torch.empty_like(hs.ws)
    hs_lib.hs_workspace_init(hs.plan, ws2)
    for v, k in zip(VARIANTS, caps):
        hs_lib.hs_plan_set_ctas_per_sm(hs.plan, v, k)
        assert hs_lib.hs_plan_ctas_per_sm(hs.plan, v) == k
    outs = {v: hs.new_outputs(x.size, v, "cuda") for v in VARIANTS}
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        hs_lib.hs_sum_batched(hs.plan, "std", xd, od, hs.out_struct(outs["std"]), hs.ws, stream=s1)
    with torch.cuda.stream(s2):
        for v in ("max", "fbin", "greedy"):
            hs_lib.hs_sum_batched(hs.plan, v, xd, od, hs.out_struct(outs[v]), ws2, stream=s2)
    torch.cuda.synchronize()
    assert hs_lib.hs_sync_status(hs.plan, hs.ws) == hs_lib.OK
    assert hs_lib.hs_sync_status(hs.plan, ws2) == hs_lib.OK
    for v in VARIANTS:
        r = oracle.hs_batched(v, x, offsets, nthreads=8)
        np.testing.assert_array_equal(outs[v]["best_snr"].cpu().numpy(), r["best_snr"])
        np.testing.assert_array_equal(outs[v]["best_h"].cpu().numpy(), r["best_h"])
    hs_lib.hs_plan_set_ctas_per_sm(hs.plan, "std", 0)
    assert hs_lib.hs_plan_ctas_per_sm(hs.plan, "std") == 0


def test_autotune_keeps_results(hs_lib, torch):
    N = 1 << 20
    x = hs_synth.spectrum(13, 0, N)
    hs = hs_lib.HarmonicSum(variants=0xF, max_bins=N, threshold=THR)
    scratch = torch.empty(8 * N * 13 + 8192, dtype=torch.uint8, device="cuda")
    hs.ensure_workspace(8)
    scratch[: N * 4].view(torch.float32).copy_(torch.from_numpy(x))
    for v in VARIANTS:
        hs_lib.hs_autotune(hs.plan, v, N, scratch, hs.ws)
        o = hs.sum_1d(v, torch.from_numpy(x).cuda())
        r = oracle.hs_1d(v, x, nthreads=8)
        np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])


@pytest.mark.parametrize("n_chunks", [1, 3, 8])
def test_host_batch_streamed_matches_device_batch(hs_lib, torch, n_chunks):
    """hs_sum_batched_host (copies of piece c+1 overlapping the sums of piece c) equals
    hs_sum_batched on the same batch, for every variant and piece count."""
    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(40, lengths=(1 << 14, 1 << 15, 1 << 17))
    total = int(offsets[-1])
    xh = torch.empty(total, dtype=torch.float32, pin_memory=True)
    hs_synth.batch(seed, offsets, pulsars, out=xh.data_ptr())
    hs = hs_lib.HarmonicSum(variants=0xF, threshold=THR, cand_capacity=1 << 16, max_spectra=40)
    for v in VARIANTS:
        mu, isig = oracle.noise_calibration(v, 32)
        hs.set_calibration(v, mu, isig)
    xd = torch.empty(total, device="cuda")
    od = torch.empty(41, dtype=torch.int64, device="cuda")
    outs = [hs.new_outputs(total, v, "cuda") for v in VARIANTS]
    hs_lib.hs_sum_batched_host(hs.plan, 0xF, xh, offsets, xd, od, [hs.out_struct(o) for o in outs], hs.ws,
                               n_chunks=n_chunks, first_id=3)
    torch.cuda.synchronize()
    assert hs.sync_status() == hs_lib.OK
    x_ref, od_ref = xh.cuda(), torch.from_numpy(offsets).cuda()
    for v, o in zip(VARIANTS, outs):
        ref = hs.sum_batched(v, x_ref, od_ref, first_id=3)
        assert torch.equal(o["best_snr"], ref["best_snr"])
        assert torch.equal(o["best_h"], ref["best_h"])
        if v == "greedy":
            assert torch.equal(o["path"], ref["path"])
        a = np.sort(hs_lib.read_candidates(o), order=["spectrum", "bin"])
        b = np.sort(hs_lib.read_candidates(ref), order=["spectrum", "bin"])
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_host_batch_streamed_16bit_eq1(hs_lib, torch, dtype):
    """A 16-bit host batch streamed in pieces: Eq. 1 of every piece runs through the FP32 groups of
    the workspace (sized for the whole batch, used per piece) and equals the oracle on the widened
    values."""
    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(70, lengths=(1 << 12, 1 << 13, 1 << 14))
    total = int(offsets[-1])
    x32 = hs_synth.batch(seed, offsets, pulsars)
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    xs = torch.from_numpy(x32).to(tdt)
    xh = torch.empty(total, dtype=tdt, pin_memory=True)
    xh.copy_(xs)
    xw = xs.float().numpy()
    hs, mu, isig = _make(hs_lib, "std", True, dtype={"f16": 1, "bf16": 2}[dtype], max_bins=1 << 14, flags=0,
                         max_spectra=70)
    xd = torch.empty(total, dtype=tdt, device="cuda")
    od = torch.empty(71, dtype=torch.int64, device="cuda")
    r = oracle.hs_batched("std", xw, offsets, mu=mu, isig=isig, nthreads=8)
    for n_chunks in (1, 3):
        o = hs.new_outputs(total, "std", "cuda")
        hs_lib.hs_sum_batched_host(hs.plan, hs_lib.STD, xh, offsets, xd, od, [hs.out_struct(o)], hs.ws,
                                   n_chunks=n_chunks)
        torch.cuda.synchronize()
        assert hs.sync_status() == hs_lib.OK
        np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
        np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])


def test_batch_slice_with_absolute_offsets(hs_lib, torch):
    """A batch may be a slice of a larger packed array: offsets are absolute indices."""
    lens = [4096, 8192, 12, 65536, 20000]
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = hs_synth.batch(17, offsets)
    hs = hs_lib.HarmonicSum(variants=hs_lib.MAX, threshold=THR, flags=0, max_spectra=5)
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    full = hs.sum_batched("max", xd, od)
    part = hs.new_outputs(x.size, "max", "cuda")
    part["best_snr"].fill_(7.0)
    hs.sum_batched("max", xd, od[2:], out=part)  # spectra 2..4 only
    a = int(offsets[2])
    assert torch.equal(part["best_snr"][a:], full["best_snr"][a:])
    assert bool((part["best_snr"][:a] == 7.0).all())
    assert hs.sync_status() == hs_lib.OK


# ---- the step before the sums: power, block-median dereddening, standardisation ----

def _complex_batch(lens, seed):
    rng = np.random.default_rng(seed)
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    k = np.arange(offsets[-1])
    trend = 1.0 + 50.0 / (1.0 + (k % 100000) / 30.0)
    z = (rng.standard_normal(offsets[-1]) + 1j * rng.standard_normal(offsets[-1])) * np.sqrt(trend / 2.0)
    return z.astype(np.complex64), offsets


@pytest.mark.parametrize("block", [32, 64, 128, 256])
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_power_normalize_bit_exact(hs_lib, torch, block, dtype):
    lens = [0, 2, 64, 1000, 4096 + 22, 100000, 256, 30, 1 << 17]
    z, offsets = _complex_batch(lens, 17 + block)
    code = {"f32": 0, "f16": 1, "bf16": 2}[dtype]
    hs = hs_lib.HarmonicSum(variants=hs_lib.STD, dtype=code, max_bins=1 << 18, max_spectra=len(lens))
    spec = torch.from_numpy(z.view(np.float32)).cuda()
    od = torch.from_numpy(offsets).cuda()
    nmed = sum((l + block - 1) // block for l in lens)
    med = torch.full((nmed,), -1.0, device="cuda")
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    out = torch.empty(offsets[-1], dtype=tdt, device="cuda")
    hs_lib.hs_power_normalize(hs.plan, spec, od, 0, block, med, out, hs.ws)
    assert hs.sync_status() == hs_lib.OK
    got = out.cpu().view(torch.int16 if dtype != "f32" else torch.float32).numpy()
    gm = med.cpu().numpy()
    moff = 0
    for s in range(len(lens)):
        a, b = offsets[s], offsets[s + 1]
        if b == a:
            continue
        x, m = oracle.power_normalize(z[a:b], block, dtype)
        np.testing.assert_array_equal(gm[moff:moff + m.size], m)
        if dtype == "f32":
            np.testing.assert_array_equal(got[a:b], x)
        else:
            np.testing.assert_array_equal(got[a:b].view(np.uint16), x)
        moff += m.size


def test_power_normalize_single_and_errors(hs_lib, torch):
    z, _ = _complex_batch([50000], 5)
    hs = hs_lib.HarmonicSum(variants=hs_lib.STD, max_bins=1 << 16)
    spec = torch.from_numpy(z.view(np.float32)).cuda()
    med = torch.empty(50000 // 128 + 1, device="cuda")
    out = torch.empty(50000, device="cuda")
    hs_lib.hs_power_normalize(hs.plan, spec, None, 50000, 128, med, out, hs.ws)
    assert hs.sync_status() == hs_lib.OK
    x, m = oracle.power_normalize(z, 128)
    np.testing.assert_array_equal(out.cpu().numpy(), x)
    np.testing.assert_array_equal(med.cpu().numpy(), m)
    # a median array one entry short: nothing written for that spectrum, reported by the status word
    hb = hs_lib.HarmonicSum(variants=hs_lib.STD, max_bins=1 << 16, max_spectra=1)
    od = torch.tensor([0, 50000], dtype=torch.int64, device="cuda")
    short = torch.empty(50000 // 128, device="cuda")
    hs_lib.hs_power_normalize(hb.plan, spec, od, 0, 128, short, out, hb.ws)
    with pytest.raises(hs_lib.HSError):
        hb.sync_status()
    with pytest.raises(hs_lib.HSError):
        hs_lib.hs_power_normalize(hs.plan, spec, None, 50000, 100, med, out, hs.ws)  # block not allowed


# ---- candidate sifting (the step after the sums) ----

def _synthetic_candidates(seed, n_groups=24):
    """A sorted candidate list with harmonic families, neighbouring bins, drifts and snr ties, drawn
    from a seeded generator (independent of any harmonic-sum output)."""
    rng = np.random.default_rng(seed)
    rows = {}
    for g in range(n_groups):
        v = [1, 2, 4, 8][g % 4]
        spec = 100 + g // 4
        for _ in range(rng.integers(1, 4)):  # pulsar families
            f0 = rng.uniform(40.0, 400.0)
            z0 = int(rng.integers(-6, 7)) if v == 1 and g % 8 == 0 else 0
            for k in range(1, int(rng.integers(2, 10))):
                for dn in (0, 1):
                    h = int(rng.integers(1, 33)) if v == 1 else int(rng.integers(1, 17))
                    b = int(round((h if v == 1 else 1) * k * f0 + dn + rng.normal(0, 0.4)))
                    z = (h * k * z0) if v == 1 else 0
                    rows[(v, spec, z, b)] = (round(float(rng.uniform(6, 30)) * 2) / 2, h)
        for _ in range(int(rng.integers(5, 30))):  # unrelated bins
            b = int(rng.integers(0, 20000))
            rows[(v, spec, 0, b)] = (round(float(rng.uniform(6, 12)) * 2) / 2, int(rng.integers(1, 33)))
    keys = sorted(rows, key=lambda k: (k[0], k[1], k[2] + 32768, k[3]))
    c = np.zeros(len(keys), oracle.CANDIDATE_DTYPE)
    for i, (v, spec, z, b) in enumerate(keys):
        snr, h = rows[(v, spec, z, b)]
        c[i] = (spec, b, snr, z, h, v)
    return c


@pytest.mark.parametrize("kmax,tol", [(8, 1.5), (3, 0.6), (1, 2.0)])
def test_sift_candidates_matches_oracle(hs_lib, torch, kmax, tol):
    c = _synthetic_candidates(11 + kmax)
    cap = c.size + 37
    hs = hs_lib.HarmonicSum(variants=0xF, cand_capacity=cap)
    cand = torch.zeros(cap * 16, dtype=torch.uint8, device="cuda")
    cand[: c.size * 16] = torch.from_numpy(c.view(np.uint8).copy()).cuda()
    count = torch.tensor([c.size], dtype=torch.int64, device="cuda")
    out = torch.empty_like(cand)
    out_count = torch.zeros(1, dtype=torch.int64, device="cuda")
    tmp = torch.empty_like(cand)
    hs_lib.hs_sift_candidates(cand, count, out, out_count, tmp, hs.ws, tol_bins=tol, tol_z=tol, kmax=kmax)
    torch.cuda.synchronize()
    keep = oracle.sift_candidates(c, tol=tol, tol_z=tol, kmax=kmax)
    n = int(out_count.item())
    got = out[: n * 16].cpu().numpy().view(oracle.CANDIDATE_DTYPE)
    assert n == int(keep.sum()) and 0 < n < c.size
    np.testing.assert_array_equal(got, c[keep])


def test_sift_candidates_dense_families(hs_lib, torch):
    """Many candidates per group with fundamentals spread over the whole k range, small ones near the
    tolerance, exact multiples and near-misses: the narrowed search of the kernel must agree with the
    oracle's loop over every k."""
    rng = np.random.default_rng(3)
    rows = {}
    for g in range(6):
        v = [4, 8, 2][g % 3]
        f = np.concatenate([rng.uniform(0.5, 3.0, 40), rng.uniform(3, 60, 150),
                            np.outer(rng.uniform(5, 40, 10), np.arange(1, 12)).ravel() + rng.normal(0, 0.8, 110)])
        for x in f:
            b = int(max(0, round(x)))
            rows[(v, 7 + g, 0, b)] = (round(float(rng.uniform(6, 20)) * 4) / 4, 1)
    keys = sorted(rows, key=lambda k: (k[0], k[1], k[2] + 32768, k[3]))
    c = np.zeros(len(keys), oracle.CANDIDATE_DTYPE)
    for i, (v, spec, z, b) in enumerate(keys):
        c[i] = (spec, b, rows[(v, spec, z, b)][0], z, 1, v)
    cap = c.size
    hs = hs_lib.HarmonicSum(variants=0xF, cand_capacity=cap)
    cand = torch.from_numpy(c.view(np.uint8).copy()).cuda()
    count = torch.tensor([c.size], dtype=torch.int64, device="cuda")
    out, tmp = torch.empty_like(cand), torch.empty_like(cand)
    out_count = torch.zeros(1, dtype=torch.int64, device="cuda")
    for kmax, tol in [(8, 1.5), (11, 0.7), (16, 2.5)]:
        hs_lib.hs_sift_candidates(cand, count, out, out_count, tmp, hs.ws, tol_bins=tol, tol_z=tol, kmax=kmax)
        keep = oracle.sift_candidates(c, tol=tol, tol_z=tol, kmax=kmax)
        n = int(out_count.item())
        np.testing.assert_array_equal(out[: n * 16].cpu().numpy().view(oracle.CANDIDATE_DTYPE), c[keep])


# ---- Eq. 4 with the first term fixed at x(n) (HS_FLAG_GREEDY_FIXED1), against the oracle's "greedy1" ----

def _greedy1(hs_lib, dtype=0, max_spectra=1, flags=0):
    mu, isig = oracle.noise_calibration("greedy1", 32)
    hs = hs_lib.HarmonicSum(variants=hs_lib.GREEDY, dtype=dtype, max_bins=1 << 22, threshold=THR,
                            cand_capacity=1 << 16, flags=flags | hs_lib.FLAG_GREEDY_FIXED1, max_spectra=max_spectra)
    hs.set_calibration("greedy", mu, isig)
    return hs, mu, isig


@pytest.mark.parametrize("n_bins", [1, 2, 3, 33, 1000, 65536 + 13, 300001])
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_greedy_fixed1_bit_exact(hs_lib, torch, n_bins, dtype):
    x = hs_synth.spectrum(78, 0, n_bins)
    xd, xw = _widen(torch, x, dtype)
    hs, mu, isig = _greedy1(hs_lib, dtype={"f32": 0, "f16": 1, "bf16": 2}[dtype], flags=hs_lib.FLAG_OUT_ALL_H)
    o = hs.sum_1d("greedy", xd, all_h=True)
    r = oracle.hs_1d("greedy1", xw, hmax=32, mu=mu, isig=isig, all_h=True, nthreads=8)
    np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    np.testing.assert_array_equal(o["path"].cpu().numpy().view(np.uint32), r["path"])
    _check_candidates(hs_lib, o, r["best_snr"], r["best_h"])


def test_greedy_fixed1_batched_and_adjoint(hs_lib, torch):
    lens = [0, 8, 4096, 100000, 12, 250000]
    offsets = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = hs_synth.batch(96, offsets)
    hs, mu, isig = _greedy1(hs_lib, max_spectra=len(lens))
    xd, od = torch.from_numpy(x).cuda(), torch.from_numpy(offsets).cuda()
    o = hs.sum_batched("greedy", xd, od, first_id=5)
    assert hs.sync_status() == hs_lib.OK
    r = oracle.hs_batched("greedy1", x, offsets, mu=mu, isig=isig, nthreads=8)
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    np.testing.assert_array_equal(o["path"].cpu().numpy().view(np.uint32), r["path"])
    _check_candidates(hs_lib, o, r["best_snr"], r["best_h"], offsets, first_id=5)
    g = torch.sigmoid(o["best_snr"] - 5.0)
    grad = hs.backward("greedy", xd, g, o["best_h"], o["path"], od).cpu().numpy().astype(np.float64)
    gn = g.cpu().numpy().astype(np.float64)
    exp = np.zeros(x.size)
    for s in range(len(lens)):
        a, b = offsets[s], offsets[s + 1]
        exp[a:b] = oracle.grad_1d("greedy1", x[a:b], gn[a:b], r["best_h"][a:b], isig=isig.astype(np.float64))
    np.testing.assert_allclose(grad, exp, rtol=1e-5, atol=1e-6)


# ---- 2-D freq-bin form ----

@pytest.mark.parametrize("nz,z_min,nb", [(11, -5, 3001), (7, -3, 4096), (1, 0, 1000)])
def test_2d_fbin_bit_exact(hs_lib, torch, nz, z_min, nb):
    stride = (nb + 3) // 4 * 4
    full = np.stack([hs_synth.spectrum(123, r, stride) for r in range(nz)]).astype(np.float32)
    plane = torch.from_numpy(full).cuda()[:, :nb]
    hs = hs_lib.HarmonicSum(variants=hs_lib.STD | hs_lib.FBIN, hmax=16, nz=nz, z_min=z_min, max_bins=stride,
                            threshold=THR, cand_capacity=1 << 16)
    o = hs.sum_2d(plane, plane_id=4, variant="fbin")
    r = oracle.hs_2d(full[:, :nb], z_min, hmax=16, variant="fbin", nthreads=8)
    for k in ("best_snr", "best_h", "best_snr_n", "best_h_n"):
        np.testing.assert_array_equal(o[k].cpu().numpy(), r[k], err_msg=k)
    np.testing.assert_array_equal(o["best_z_n"].cpu().numpy().astype(np.int32), r["best_z_n"])
    c = hs_lib.read_candidates(o)
    exp = np.nonzero(r["best_snr"].ravel() > THR)[0]
    assert c.size == exp.size and (c["variant"] == hs_lib.FBIN).all() and (c["spectrum"] == 4).all()
    got = np.sort((c["z"].astype(np.int64) - z_min) * nb + c["bin"].astype(np.int64))
    np.testing.assert_array_equal(got, exp)
    s = hs_lib.Out2d(o["best_snr"].data_ptr(), o["best_h"].data_ptr(), o["best_snr_n"].data_ptr(),
                     o["best_h_n"].data_ptr(), o["best_z_n"].data_ptr(), None, None)
    for v in ("max", "greedy"):  # not in this plan
        with pytest.raises(hs_lib.HSError) as e:
            hs_lib.hs_sum_2d(hs.plan, plane, s, hs.ws, variant=v)
        assert e.value.status == hs_lib.ERR_INVALID


@pytest.mark.parametrize("variant,flag,ovariant", [("max", None, "max"), ("max", "FLAG_MAX_WINDOW0", "max0"),
                                                   ("greedy", None, "greedy"),
                                                   ("greedy", "FLAG_GREEDY_FIXED1", "greedy1")])
@pytest.mark.parametrize("nz,z_min,nb,hmax", [(11, -5, 3001, 16), (7, -3, 4096, 16), (1, 0, 1000, 16),
                                              (9, -8, 257, 5), (31, -15, 64, 16)])
def test_2d_rowwise_max_greedy_bit_exact(hs_lib, torch, variant, flag, ovariant, nz, z_min, nb, hmax):
    """The row-wise 2-D forms of Eq. 2 and 4 (harmonic i on row i z) against the oracle, calibrated,
    with candidates, on planes whose drift range cuts the valid H at both ends."""
    stride = (nb + 3) // 4 * 4
    full = np.stack([hs_synth.spectrum(124, r, stride) for r in range(nz)]).astype(np.float32)
    plane = torch.from_numpy(full).cuda()[:, :nb]
    flags = getattr(hs_lib, flag) if flag else 0
    hs = hs_lib.HarmonicSum(variants=hs_lib.VARIANTS[variant], hmax=hmax, nz=nz, z_min=z_min, max_bins=stride,
                            threshold=THR, cand_capacity=1 << 16, flags=flags)
    mu, isig = hs_lib.hs_noise_calibration(variant, hmax, flags=flags)
    hs.set_calibration(variant, mu, isig)
    o = hs.sum_2d(plane, plane_id=9, variant=variant)
    assert hs.sync_status() == hs_lib.OK
    r = oracle.hs_2d(full[:, :nb], z_min, hmax=hmax, mu=mu, isig=isig, variant=ovariant, nthreads=8)
    for k in ("best_snr", "best_h", "best_snr_n", "best_h_n"):
        np.testing.assert_array_equal(o[k].cpu().numpy(), r[k], err_msg=k)
    np.testing.assert_array_equal(o["best_z_n"].cpu().numpy().astype(np.int32), r["best_z_n"])
    c = hs_lib.read_candidates(o)
    exp = np.nonzero(r["best_snr"].ravel() > THR)[0]
    assert c.size == exp.size and (c["variant"] == hs_lib.VARIANTS[variant]).all() and (c["spectrum"] == 9).all()
    got = np.sort((c["z"].astype(np.int64) - z_min) * nb + c["bin"].astype(np.int64))
    np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("variant,flag,ovariant", [("max", "FLAG_MAX_WINDOW0", "max0"),
                                                   ("greedy", "FLAG_GREEDY_FIXED1", "greedy1"),
                                                   ("std", None, "std")])
def test_flags_combined_with_pow2_stages(hs_lib, torch, variant, flag, ovariant):
    """A variant flag together with the power-of-two stage search, single spectrum and batch."""
    x = hs_synth.spectrum(79, 0, 70001)
    flags = hs_lib.FLAG_POW2_STAGES | (getattr(hs_lib, flag) if flag else 0)
    mu, isig = oracle.noise_calibration(ovariant, 32)
    hs = hs_lib.HarmonicSum(variants=hs_lib.VARIANTS[variant], threshold=THR, cand_capacity=1 << 16,
                            flags=flags | hs_lib.FLAG_OUT_ALL_H, max_spectra=2)
    hs.set_calibration(variant, mu, isig)
    xd = torch.from_numpy(x).cuda()
    o = hs.sum_1d(variant, xd, all_h=True)
    r = oracle.hs_1d(ovariant, x, hmax=32, mu=mu, isig=isig, all_h=True, pow2=True, nthreads=8)
    np.testing.assert_array_equal(o["all_h"].cpu().numpy(), r["all_h"])
    np.testing.assert_array_equal(o["best_snr"].cpu().numpy(), r["best_snr"])
    np.testing.assert_array_equal(o["best_h"].cpu().numpy(), r["best_h"])
    offsets = np.array([0, 30000, 70000], np.int64)
    ob = hs.sum_batched(variant, xd, torch.from_numpy(offsets).cuda())
    rb = oracle.hs_batched(ovariant, x, offsets, mu=mu, isig=isig, pow2=True, nthreads=8)
    np.testing.assert_array_equal(ob["best_snr"].cpu().numpy()[:70000], rb["best_snr"])
    np.testing.assert_array_equal(ob["best_h"].cpu().numpy()[:70000], rb["best_h"])
