"""Pins of the CPU oracle to what the definitions and the mathematics fix, independently of it.

Each check is chosen so that a plausible slip in the oracle (a dropped or doubled term, a wrong
rounding direction, an off-by-one window, a transposed plane index, a reversed tie rule) fails at
least one of them.  Sources: Eq. 1-4 of arXiv:1812.02647 Section 2, and the 2-D form of Eq. 1.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import hs_synth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
# max0: Eq. 2 with the window j = 0..i; greedy1: Eq. 4 with the first term fixed at x(n) (variant flags)
VARIANTS = ["std", "max", "fbin", "greedy", "max0", "greedy1"]
GREEDY = ("greedy", "greedy1")


def j0(variant):
    """First window offset of Eq. 2: j = 1 as written, j = 0 under the variant flag."""
    return 0 if variant == "max0" else 1


def half_up(fr: Fraction) -> int:
    """Round a rational half up (toward +infinity at exact halves), via exact rational arithmetic."""
    return math.floor(fr + Fraction(1, 2))


def rand_spectrum(n, seed):
    return hs_synth.spectrum(seed, 0, n)


# ---------------------------------------------------------------------------------------------
# hand-worked fixtures
# ---------------------------------------------------------------------------------------------

def test_golden_1d_hand_worked():
    g = json.load(open(os.path.join(GOLDEN, "hand_worked_1d.json")))
    x = np.array(g["x"], np.float64)
    for c in g["cases"]:
        r = oracle.hs_1d(c["variant"], x, hmax=8, fp64=True, all_h=True)
        assert sum(x[t] for t in c["terms"]) == c["S"]
        got = r["all_h"][c["H"] - 1, c["n"]]
        assert got == pytest.approx(c["S"] / math.sqrt(c["H"]), rel=1e-15), c
        if "path" in c:
            # the path bits up to H of the recursion; the oracle keeps extending the path to the last valid H
            assert int(r["path"][c["n"]]) & ((1 << c["H"]) - 1) == c["path"]


def test_golden_2d_hand_worked():
    g = json.load(open(os.path.join(GOLDEN, "hand_worked_2d.json")))
    zs = np.arange(g["z_min"], g["z_min"] + g["nz"])
    plane = np.array([[10 * (z + 1) + m for m in range(g["n_bins"])] for z in zs], np.float64)
    r = oracle.hs_2d(plane, g["z_min"], hmax=4, fp64=True, all_h=True)
    for c in g["cases"]:
        got = r["all_h"][c["H"] - 1, c["z"] - g["z_min"], c["n"]]
        assert got == pytest.approx(c["S"] / math.sqrt(c["H"]), rel=1e-15), c


# ---------------------------------------------------------------------------------------------
# special cases that reduce to something known
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", VARIANTS)
def test_h1_identity(variant):
    x = rand_spectrum(1000, 11)
    r = oracle.hs_1d(variant, x, hmax=4, all_h=True)
    row = r["all_h"][0]
    if variant in ("std", "fbin"):
        expect = x
    elif variant == "max":
        expect = np.append(x[1:], -np.inf)  # x(n+1); the last bin has no valid H
    elif variant == "max0":
        expect = np.append(np.maximum(x[:-1], x[1:]), -np.inf)  # max(x(n), x(n+1))
    elif variant == "greedy1":
        expect = x  # x(n) itself, valid at every bin
    else:
        expect = np.append(np.maximum(x[:-1], x[1:]), -np.inf)
    np.testing.assert_array_equal(row, expect.astype(np.float32))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("c", [1.0, -0.75, 3.5])
def test_constant_spectrum(variant, c):
    N, hmax = 300, 32
    x = np.full(N, c)
    r = oracle.hs_1d(variant, x, hmax=hmax, fp64=True, all_h=True)
    for n in range(N):
        hv = oracle.hvalid(variant, n, N, hmax)
        for H in range(1, hmax + 1):
            v = r["all_h"][H - 1, n]
            if H <= hv:
                assert v == pytest.approx(c * math.sqrt(H), rel=1e-14)
            else:
                assert v == -np.inf
        if hv:
            # positive c: the largest valid H wins; negative c: H = 1 wins
            assert r["best_h"][n] == (hv if c > 0 else 1)
    if variant in GREEDY:
        assert not r["path"].any()  # ties keep the left bin


@pytest.mark.parametrize("variant", VARIANTS)
def test_calibration_closed_form(variant):
    """A constant spectrum c has sum c*H, so the calibrated value is (c*sqrt(H) - mu_H) * isig_H for
    any per-H tables: pins both the order (subtract, then scale) and the per-H indexing."""
    N, hmax, c = 200, 32, 1.25
    rng = np.random.default_rng(4)
    mu = np.concatenate([[0.0], rng.uniform(-2, 2, hmax)])
    isig = np.concatenate([[1.0], rng.uniform(0.2, 3, hmax)])
    r = oracle.hs_1d(variant, np.full(N, c), hmax=hmax, mu=mu, isig=isig, fp64=True, all_h=True)
    for n in range(0, N, 7):
        for H in range(1, oracle.hvalid(variant, n, N, hmax) + 1):
            assert r["all_h"][H - 1, n] == pytest.approx((c * math.sqrt(H) - mu[H]) * isig[H], rel=1e-13)


def test_zero_spectrum_tie_break():
    x = np.zeros(100, np.float32)
    for v in VARIANTS:
        r = oracle.hs_1d(v, x, hmax=32)
        ok = r["best_h"] > 0
        assert (r["best_h"][ok] == 1).all()  # all snr equal -> smallest H
        assert (r["best_snr"][ok] == 0).all()


@pytest.mark.parametrize("variant", VARIANTS)
def test_range_limits(variant):
    N, hmax = 40, 32
    for n in range(N):
        hv = oracle.hvalid(variant, n, N, hmax)
        if variant == "std":
            assert hv == hmax
        elif variant == "fbin":
            assert hv == (hmax if n == 0 else min(hmax, (N - 1) // n))
            assert hv * n <= N - 1 and (hv == hmax or (hv + 1) * n > N - 1)
        elif variant == "greedy1":  # the furthest read is H n + H - 1
            assert hv * (n + 1) <= N and (hv == hmax or (hv + 1) * (n + 1) > N)
        else:
            assert hv * (n + 1) <= N - 1 and (hv == hmax or (hv + 1) * (n + 1) > N - 1)
    r = oracle.hs_1d(variant, rand_spectrum(N, 3), hmax=hmax)
    for n in range(N):
        if oracle.hvalid(variant, n, N, hmax) == 0:
            assert r["best_h"][n] == 0 and r["best_snr"][n] == -np.inf


# ---------------------------------------------------------------------------------------------
# delta spikes with counts derived by exact rational arithmetic
# ---------------------------------------------------------------------------------------------

def test_delta_spike_eq1():
    N, hmax, m0, A = 200, 12, 37, 2.5
    x = np.zeros(N)
    x[m0] = A
    r = oracle.hs_1d("std", x, hmax=hmax, fp64=True, all_h=True)
    for n in range(N):
        for H in range(1, hmax + 1):
            cnt = sum(1 for i in range(1, H + 1) if half_up(Fraction(n * i, H)) == m0)
            assert r["all_h"][H - 1, n] == pytest.approx(A * cnt / math.sqrt(H), abs=1e-15)


def test_delta_spike_fbin():
    N, hmax, m0, A = 300, 16, 72, -1.5
    x = np.zeros(N)
    x[m0] = A
    r = oracle.hs_1d("fbin", x, hmax=hmax, fp64=True, all_h=True)
    for n in range(1, N):
        for H in range(1, oracle.hvalid("fbin", n, N, hmax) + 1):
            hit = (m0 % n == 0) and (m0 // n <= H)
            assert r["all_h"][H - 1, n] == pytest.approx(A * hit / math.sqrt(H), abs=1e-15)


@pytest.mark.parametrize("variant", ["max", "max0"])
def test_delta_spike_max(variant):
    N, hmax, m0, A = 300, 16, 95, 3.0
    x = np.zeros(N)
    x[m0] = A
    r = oracle.hs_1d(variant, x, hmax=hmax, fp64=True, all_h=True)
    for n in range(N):
        for H in range(1, oracle.hvalid(variant, n, N, hmax) + 1):
            cnt = sum(1 for i in range(1, H + 1) if i * n + j0(variant) <= m0 <= i * n + i)
            assert r["all_h"][H - 1, n] == pytest.approx(A * cnt / math.sqrt(H), abs=1e-15)


def test_delta_spike_2d_negative_half_rounding():
    nz, z_min, nb, hmax = 11, -5, 40, 8
    for (m0, z0) in [(7, -2), (12, 0), (5, 3), (9, -3)]:
        plane = np.zeros((nz, nb))
        plane[z0 - z_min, m0] = 1.0
        r = oracle.hs_2d(plane, z_min, hmax=hmax, fp64=True, all_h=True)
        for z in range(z_min, z_min + nz):
            for n in range(nb):
                for H in range(1, hmax + 1):
                    cnt = sum(1 for i in range(1, H + 1)
                              if half_up(Fraction(n * i, H)) == m0 and half_up(Fraction(z * i, H)) == z0)
                    assert r["all_h"][H - 1, z - z_min, n] == pytest.approx(cnt / math.sqrt(H), abs=1e-15)


# ---------------------------------------------------------------------------------------------
# linearity of Eq. 1 and Eq. 3; 2-D reduces to 1-D on the z = 0 row
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["std", "fbin"])
def test_linearity(variant):
    x = rand_spectrum(2000, 21).astype(np.float64)
    y = rand_spectrum(2000, 22).astype(np.float64)
    a, b = 0.7, -1.3
    hx = oracle.hs_1d(variant, x, hmax=32, fp64=True, all_h=True)["all_h"]
    hy = oracle.hs_1d(variant, y, hmax=32, fp64=True, all_h=True)["all_h"]
    hz = oracle.hs_1d(variant, a * x + b * y, hmax=32, fp64=True, all_h=True)["all_h"]
    ok = np.isfinite(hz)
    np.testing.assert_allclose(hz[ok], a * hx[ok] + b * hy[ok], rtol=1e-11, atol=1e-11)


def test_2d_zero_row_is_1d_eq1():
    nz, z_min, nb = 9, -4, 3000
    plane = np.stack([rand_spectrum(nb, 100 + r) for r in range(nz)])
    r2 = oracle.hs_2d(plane, z_min, hmax=16, all_h=True)
    r1 = oracle.hs_1d("std", plane[-z_min], hmax=16, all_h=True)
    np.testing.assert_array_equal(r2["all_h"][:, -z_min, :], r1["all_h"])
    np.testing.assert_array_equal(r2["best_snr"][-z_min], r1["best_snr"])
    np.testing.assert_array_equal(r2["best_h"][-z_min], r1["best_h"])


def test_2d_constant_plane_and_row_tie():
    nz, z_min, nb = 7, -3, 50
    r = oracle.hs_2d(np.full((nz, nb), 2.0), z_min, hmax=16, fp64=True)
    np.testing.assert_allclose(r["best_snr"], 2.0 * 4.0, rtol=1e-14)
    assert (r["best_h"] == 16).all()
    assert (r["best_z_n"] == z_min).all()  # equal across rows -> lowest row


def test_2d_best_over_rows():
    nz, z_min, nb = 9, -4, 500
    plane = np.stack([rand_spectrum(nb, 300 + r) for r in range(nz)])
    r = oracle.hs_2d(plane, z_min, hmax=16)
    rows = np.argmax(r["best_snr"], axis=0)  # numpy argmax returns the first maximum
    np.testing.assert_array_equal(r["best_z_n"], rows + z_min)
    np.testing.assert_array_equal(r["best_snr_n"], r["best_snr"][rows, np.arange(nb)])
    np.testing.assert_array_equal(r["best_h_n"], r["best_h"][rows, np.arange(nb)])


# ---------------------------------------------------------------------------------------------
# brute force on tiny spectra
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["max", "max0"])
def test_max_bruteforce(variant):
    for seed in range(5):
        N = 64
        x = rand_spectrum(N, 500 + seed)
        r32 = oracle.hs_1d(variant, x, hmax=32, all_h=True)
        r64 = oracle.hs_1d(variant, x, hmax=32, fp64=True, all_h=True)
        for n in range(N):
            s32, s64 = np.float32(0), 0.0
            for H in range(1, oracle.hvalid(variant, n, N, 32) + 1):
                win = x[H * n + j0(variant): H * n + H + 1]
                assert len(win) == H + 1 - j0(variant)
                s32 = np.float32(s32 + win.max())
                s64 += float(win.max())
                assert r32["all_h"][H - 1, n] == np.float32(s32 * np.float32(1 / math.sqrt(H)))
                assert r64["all_h"][H - 1, n] == pytest.approx(s64 / math.sqrt(H), rel=1e-14, abs=1e-14)


@pytest.mark.parametrize("variant", GREEDY)
def test_greedy_bruteforce_paths(variant):
    """Enumerate every left/right choice sequence; exactly one obeys the step rule, and it is the
    oracle's path and sum (greedy1: the first term is x(n), its bit never set)."""
    first = 2 if variant == "greedy1" else 1
    for seed in range(6):
        N = 64
        x = rand_spectrum(N, 600 + seed).astype(np.float64)
        x[10] = x[11]  # plant a tie: the rule keeps the left bin
        r = oracle.hs_1d(variant, x, hmax=6, fp64=True, all_h=True)
        for n in range(N):
            hv = oracle.hvalid(variant, n, N, 6)
            for H in range(1, hv + 1):
                obeying = []
                for bits in range(1 << H):
                    if first == 2 and bits & 1:
                        continue
                    j, ok, s = 0, True, (x[n] if first == 2 else 0.0)
                    for i in range(first, H + 1):
                        right = (bits >> (i - 1)) & 1
                        l, rr = x[i * n + j], x[i * n + j + 1]
                        if right != (1 if rr > l else 0):
                            ok = False
                            break
                        s += rr if right else l
                        j += right
                    if ok:
                        obeying.append((bits, s))
                assert len(obeying) == 1
                bits, s = obeying[0]
                assert int(r["path"][n]) & ((1 << H) - 1) == bits
                assert r["all_h"][H - 1, n] == pytest.approx(s / math.sqrt(H), rel=1e-14, abs=1e-14)


def test_eq1_index_against_rationals():
    for n in list(range(0, 70)) + [1000003, 4194303]:
        for H in range(1, 33):
            r = oracle.hs_1d("std", np.arange(max(n + 1, 2), dtype=np.float64), hmax=H, fp64=True, all_h=True)
            s = sum(half_up(Fraction(n * i, H)) for i in range(1, H + 1))
            assert r["all_h"][H - 1, n] == pytest.approx(s / math.sqrt(H), rel=1e-15)
            if n > 100:
                break  # one H per large n keeps this quick


# ---------------------------------------------------------------------------------------------
# noise statistics against the closed forms
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", VARIANTS)
def test_noise_moments_monte_carlo(variant):
    """Mean and spread of h_H over noise-only spectra against the closed forms.  Bins of one
    spectrum share reads (e.g. Eq. 1 at n and n+1), so the standard error of the mean is taken
    from independent replicate spectra, not from the bin count."""
    R, N, hmax = 32, 1 << 17, 32
    mu, sd = oracle.noise_moments(variant, hmax)
    Hs = (1, 2, 3, 4, 8, 16, 32)
    means = {H: [] for H in Hs}
    stds = {H: [] for H in Hs}
    for rep in range(R):
        x = hs_synth.spectrum(4242, rep, N)
        r = oracle.hs_1d(variant, x, hmax=hmax, fp64=True, all_h=True, nthreads=oracle.max_threads())
        for H in Hs:
            v = r["all_h"][H - 1, H: N // 32 - 1]  # every H valid, all reads of a bin distinct
            means[H].append(v.mean())
            stds[H].append(v.std())
    for H in Hs:
        m = float(np.mean(means[H]))
        se = float(np.std(means[H], ddof=1)) / math.sqrt(R)
        assert abs(m - mu[H]) < 5 * se + 2e-3, (H, m, mu[H], se)
        assert abs(float(np.mean(stds[H])) - sd[H]) < 0.02 * sd[H], (H, np.mean(stds[H]), sd[H])


def test_noise_calibration_tables():
    for v in VARIANTS:
        mu, isig = oracle.noise_calibration(v, 32)
        assert mu.dtype == np.float32 and isig.dtype == np.float32
    mu, sd = oracle.noise_moments("max", 32)
    # values worked out by hand from the closed form (H = 2: (1 - 1 + 1.5 - 1)/sqrt 2; var (1 + 1.25)/2)
    assert mu[2] == pytest.approx(0.5 / math.sqrt(2), rel=1e-15)
    assert sd[2] == pytest.approx(math.sqrt(2.25 / 2), rel=1e-15)
    mu, sd = oracle.noise_moments("greedy", 32)
    assert mu[16] == pytest.approx(2.0) and sd[7] == pytest.approx(math.sqrt(1.25))
    # first term one standardised bin, then four maxima of two: mean 4/2, variance 1 + 4 x 5/4
    mu, sd = oracle.noise_moments("greedy1", 32)
    assert mu[1] == 0.0 and sd[1] == 1.0
    assert mu[5] == pytest.approx(2.0 / math.sqrt(5.0), rel=1e-15) and sd[5] == pytest.approx(math.sqrt(6.0 / 5.0))
    # windows of i + 1 bins: H = 1 is the max of two Exp(1) (mean 3/2, variance 5/4), H = 2 adds the
    # max of three (mean 11/6, variance 1 + 1/4 + 1/9)
    mu, sd = oracle.noise_moments("max0", 32)
    assert mu[1] == pytest.approx(0.5, rel=1e-15) and sd[1] == pytest.approx(math.sqrt(1.25), rel=1e-15)
    assert mu[2] == pytest.approx((0.5 + 5.0 / 6.0) / math.sqrt(2), rel=1e-15)
    assert sd[2] == pytest.approx(math.sqrt((1.25 + 1.25 + 1.0 / 9.0) / 2), rel=1e-15)


# ---------------------------------------------------------------------------------------------
# FP32 mode against FP64 within the sequential-summation bound
# ---------------------------------------------------------------------------------------------

def _abs_term_sum(variant, x64, hmax, r64):
    """sum_i |t_i| for every (H, n): the terms' absolute values, following the FP64 routing."""
    N = x64.shape[0]
    ax = np.abs(x64)
    if variant in ("std", "fbin"):
        return oracle.hs_1d(variant, ax, hmax=hmax, fp64=True, all_h=True)["all_h"] * np.sqrt(
            np.arange(1, hmax + 1))[:, None]
    out = np.full((hmax, N), np.nan)
    n = np.arange(N)
    acc = np.zeros(N)
    j = np.zeros(N, np.int64)
    for H in range(1, hmax + 1):
        ok = H * (n + 1) <= (N if variant == "greedy1" else N - 1)
        if variant in ("max", "max0"):
            w = np.stack([x64[np.minimum(H * n + k, N - 1)] for k in range(j0(variant), H + 1)])
            t = np.abs(w.max(axis=0))
        else:
            bit = (r64["path"].astype(np.int64) >> (H - 1)) & 1
            idx = np.minimum(H * n + j + bit, N - 1)
            t = ax[idx]
            j = j + bit
        acc = acc + np.where(ok, t, 0)
        out[H - 1] = np.where(ok, acc, np.nan)
    return out


@pytest.mark.parametrize("variant", VARIANTS)
def test_fp32_within_bound_of_fp64(variant):
    x, _ = hs_synth.spectrum_1d_pulsar(n_bins=1 << 14)
    hmax = 32
    mu, isig = oracle.noise_calibration(variant, hmax)
    r32 = oracle.hs_1d(variant, x, hmax=hmax, mu=mu, isig=isig, all_h=True)
    r64 = oracle.hs_1d(variant, x, hmax=hmax, mu=mu, isig=isig, fp64=True, all_h=True)
    a32, a64 = r32["all_h"].astype(np.float64), r64["all_h"]
    ok = np.isfinite(a64)
    assert (np.isfinite(a32) == ok).all()
    tsum = _abs_term_sum(variant, x.astype(np.float64), hmax, r64)
    H = np.arange(1, hmax + 1)[:, None]
    bound = 1e-5 * (np.abs(a64) + isig[1:hmax + 1, None].astype(np.float64) / np.sqrt(H) * tsum)
    err = np.abs(a32 - a64)
    assert (err[ok] <= bound[ok]).all()
    if variant in GREEDY:
        np.testing.assert_array_equal(r32["path"], r64["path"])  # compares only, same in both modes


# ---------------------------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["std", "fbin"])
def test_adjoint_is_transpose_of_linear_map(variant):
    N, hmax = 3000, 32
    x = rand_spectrum(N, 31).astype(np.float64)
    r = oracle.hs_1d(variant, x, hmax=hmax, fp64=True)
    bh = r["best_h"]
    g = np.random.default_rng(5).standard_normal(N)
    grad = oracle.grad_1d(variant, x, g, bh, hmax=hmax)
    for k in range(3):
        v = np.random.default_rng(100 + k).standard_normal(N)
        hv = oracle.hs_1d(variant, v, hmax=hmax, fp64=True, all_h=True)["all_h"]
        lin = sum(g[n] * hv[bh[n] - 1, n] for n in range(N) if bh[n] > 0)
        assert float(grad @ v) == pytest.approx(lin, rel=1e-10)


def test_adjoint_max_ties_route_to_first_maximum():
    """On an integer spectrum full of ties, the Max adjoint sends each term's weight to the first
    maximum of its window, the element numpy's argmax picks (brute force over every (n, i))."""
    N, hmax = 400, 32
    x = np.random.default_rng(8).integers(0, 3, N).astype(np.float64)
    r = oracle.hs_1d("max", x, hmax=hmax, fp64=True)
    g = np.random.default_rng(9).standard_normal(N)
    grad = oracle.grad_1d("max", x, g, r["best_h"], hmax=hmax)
    expect = np.zeros(N)
    for n in range(N):
        Hs = int(r["best_h"][n])
        for i in range(1, Hs + 1):
            expect[i * n + 1 + int(np.argmax(x[i * n + 1:i * n + i + 1]))] += g[n] / math.sqrt(Hs)
    np.testing.assert_allclose(grad, expect, rtol=1e-12, atol=1e-12)


def _routing(variant, x, hmax, mu=None, isig=None):
    """Everything that decides which bins a bin's best sum reads: the best H under the given
    calibration (the one the gradient is routed through), the Eq. 4 path, the Eq. 2 argmaxes."""
    r = oracle.hs_1d(variant, x, hmax=hmax, mu=mu, isig=isig, fp64=True, all_h=True)
    key = [r["best_h"].astype(np.int64)]
    if variant in GREEDY:
        key.append(r["path"].astype(np.int64))
    if variant in ("max", "max0"):
        N = x.shape[0]
        n = np.arange(N)
        for i in range(1, hmax + 1):
            ok = i * (n + 1) <= N - 1
            w = np.stack([x[np.minimum(i * n + k, N - 1)] for k in range(j0(variant), i + 1)])
            key.append(np.where(ok, np.argmax(w, axis=0), -1))
    return r, np.stack(key)


def _softplus(z):
    return np.logaddexp(0.0, z)


@pytest.mark.parametrize("variant", VARIANTS)
def test_adjoint_finite_differences(variant):
    """Directional central differences of L = sum_n softplus(snr_n - 5) in FP64, bins whose
    routing changes within +-eps excluded from both sides."""
    n_spec, N, hmax, eps = 4, 1024, 32, 1e-6
    mu, isig = oracle.noise_calibration(variant, hmax)
    mu64, isig64 = mu.astype(np.float64), isig.astype(np.float64)
    rng = np.random.default_rng(77)
    for s in range(n_spec):
        x = rand_spectrum(N, 700 + s).astype(np.float64)
        r0, k0 = _routing(variant, x, hmax, mu64, isig64)
        for d in range(2):
            v = rng.standard_normal(N)
            rp, kp = _routing(variant, x + eps * v, hmax, mu64, isig64)
            rm, km = _routing(variant, x - eps * v, hmax, mu64, isig64)
            keep = (k0 == kp).all(0) & (k0 == km).all(0) & (r0["best_h"] > 0)
            # snr with the same calibration as the analytic side
            def snr(rr):
                return rr["best_snr"]
            rp = oracle.hs_1d(variant, x + eps * v, hmax=hmax, mu=mu64, isig=isig64, fp64=True)
            rm = oracle.hs_1d(variant, x - eps * v, hmax=hmax, mu=mu64, isig=isig64, fp64=True)
            rc = oracle.hs_1d(variant, x, hmax=hmax, mu=mu64, isig=isig64, fp64=True)
            fd = (_softplus(snr(rp)[keep] - 5) - _softplus(snr(rm)[keep] - 5)).sum() / (2 * eps)
            g = np.where(keep, 1.0 / (1.0 + np.exp(-(rc["best_snr"] - 5))), 0.0)
            grad = oracle.grad_1d(variant, x, g, rc["best_h"], hmax=hmax, isig=isig64)
            assert float(grad @ v) == pytest.approx(fd, rel=1e-6, abs=1e-7)
            assert keep.mean() > 0.9


# ---------------------------------------------------------------------------------------------
# reduced-precision storage
# ---------------------------------------------------------------------------------------------

def test_standardize_cast_f16_matches_ieee_library():
    p = hs_synth.spectrum(9, 0, 50000, raw=True)
    special = np.array([0.0, 1e-8, 6e-8, 5.96e-8, 2.98e-8, 3e-5, 6.1e-5, 65504.0, 65519.0, 65520.0, 1e6,
                        -65520.0, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11], np.float32)
    p = np.concatenate([p, special, -special])
    for mu, sig in [(1.0, 1.0), (0.9, 1.1), (0.0, 1.0)]:
        got = oracle.standardize_cast(p, mu, sig, "f16")
        y = (p - np.float32(mu)) / np.float32(sig)
        assert y.dtype == np.float32
        np.testing.assert_array_equal(got, y.astype(np.float16).view(np.uint16))


def test_standardize_cast_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    p = hs_synth.spectrum(10, 0, 50000, raw=True)
    special = np.array([0.0, 1e-40, 3e38, 3.4e38, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8], np.float32)
    p = np.concatenate([p, special, -special])
    got = oracle.standardize_cast(p, 0.9, 1.1, "bf16")
    y = (p - np.float32(0.9)) / np.float32(1.1)
    ref = torch.from_numpy(y).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(got, ref)


# ---------------------------------------------------------------------------------------------
# batched = the 1-D definition applied to each spectrum
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", VARIANTS)
def test_batched_is_per_spectrum(variant):
    offsets = np.array([0, 1000, 1000, 1037, 5000, 5002], np.int64)  # includes an empty and a 2-bin spectrum
    x = hs_synth.batch(55, offsets)
    rb = oracle.hs_batched(variant, x, offsets, hmax=32, nthreads=4)
    for s in range(len(offsets) - 1):
        a, b = offsets[s], offsets[s + 1]
        if a == b:
            continue
        r1 = oracle.hs_1d(variant, x[a:b], hmax=32)
        np.testing.assert_array_equal(rb["best_snr"][a:b], r1["best_snr"])
        np.testing.assert_array_equal(rb["best_h"][a:b], r1["best_h"])


def test_sampled_entry_points_match_full():
    x = rand_spectrum(3000, 41)
    bins = np.array([0, 1, 2, 99, 1500, 2998, 2999])
    for v in VARIANTS:
        full = oracle.hs_1d(v, x)
        part = oracle.hs_bins(v, x, bins)
        np.testing.assert_array_equal(part["best_snr"], full["best_snr"][bins])
        np.testing.assert_array_equal(part["best_h"], full["best_h"][bins])
    plane = np.stack([rand_spectrum(700, 900 + r) for r in range(9)])
    full = oracle.hs_2d(plane, -4)
    rows = np.array([0, 4, 8, 3, 5])
    bins = np.array([0, 699, 350, 1, 17])
    part = oracle.hs_2d_cells(plane, -4, rows, bins)
    np.testing.assert_array_equal(part["best_snr"], full["best_snr"][rows, bins])
    np.testing.assert_array_equal(part["best_h"], full["best_h"][rows, bins])


# ---------------------------------------------------------------------------------------------
# power-of-two stages (variant flag): a restriction of the full search
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", VARIANTS)
def test_pow2_stages_restrict_the_full_search(variant):
    """With only H = 1, 2, 4, .. searched, every stage's snr is the full search's, the other H read
    -inf, and the best H is the first stage with the largest snr (numpy argmax over the stages)."""
    N, hmax = 3000, 32
    x = rand_spectrum(N, 41)
    mu, isig = oracle.noise_calibration(variant, hmax)
    full = oracle.hs_1d(variant, x, hmax=hmax, mu=mu, isig=isig, all_h=True)
    p2 = oracle.hs_1d(variant, x, hmax=hmax, mu=mu, isig=isig, all_h=True, pow2=True)
    stages = [1, 2, 4, 8, 16, 32]
    others = [h for h in range(1, hmax + 1) if h not in stages]
    np.testing.assert_array_equal(p2["all_h"][[h - 1 for h in stages]], full["all_h"][[h - 1 for h in stages]])
    assert np.isneginf(p2["all_h"][[h - 1 for h in others]]).all()
    sub = full["all_h"][[h - 1 for h in stages]]
    valid = np.isfinite(sub).any(axis=0)
    k = np.argmax(np.where(np.isfinite(sub), sub, -np.inf), axis=0)
    np.testing.assert_array_equal(p2["best_h"][valid], np.array(stages)[k[valid]])
    np.testing.assert_array_equal(p2["best_snr"][valid], sub[k[valid], np.nonzero(valid)[0]])
    assert (p2["best_h"][~valid] == 0).all()
    if variant in GREEDY:
        np.testing.assert_array_equal(p2["path"], full["path"])  # the recursion itself is unchanged


# ---------------------------------------------------------------------------------------------
# the step before the sums: power, block-median dereddening, standardisation
# ---------------------------------------------------------------------------------------------

def _cgauss(n, seed, scale=None):
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2.0)
    return (z * (1.0 if scale is None else np.sqrt(scale))).astype(np.complex64)


def _power32(z):
    f = z.view(np.float32).reshape(-1, 2)
    return f[:, 0] * f[:, 0] + f[:, 1] * f[:, 1]  # float32, each product and the sum rounded


@pytest.mark.parametrize("n,block", [(1000, 128), (4096, 64), (77, 128), (1, 32), (300, 256)])
def test_power_normalize_medians_are_lower_order_statistics(n, block):
    z = _cgauss(n, 3 + n)
    _, med = oracle.power_normalize(z, block)
    P = _power32(z)
    for j in range(med.size):
        b = P[j * block:(j + 1) * block]
        k = (b.size - 1) // 2
        assert med[j] == np.partition(b, k)[k]


def test_power_normalize_constant_and_zero():
    z = np.full(1000, 2.0 + 0.0j, np.complex64)  # power exactly 4 everywhere
    x, med = oracle.power_normalize(z, 128)
    assert (med == 4.0).all()
    assert (x == np.float32(0.693147180559945309417232) - np.float32(1.0)).all()
    x0, _ = oracle.power_normalize(np.zeros(500, np.complex64), 64)
    assert (x0 == 0.0).all()  # no power: no information


def test_power_normalize_interpolates_between_block_centres():
    """Blocks of constant power v_j: the baseline is the straight line through the points
    (block centre, v_j), held flat before the first and after the last centre (numpy interp)."""
    block, nblk = 64, 9
    n = block * nblk - 23  # a partial last block
    v = np.array([1.0, 3.0, 2.0, 8.0, 8.0, 0.5, 4.0, 2.5, 6.0])
    amp = np.repeat(np.sqrt(v), block)[:n]
    z = (amp + 0j).astype(np.complex64)
    x, med = oracle.power_normalize(z, block)
    P = _power32(z).astype(np.float64)
    np.testing.assert_array_equal(med, P[::block])
    sizes = np.minimum(block, n - np.arange(nblk) * block)
    centres = np.arange(nblk) * block + (sizes - 1) / 2.0
    base = np.interp(np.arange(n), centres, med.astype(np.float64))
    np.testing.assert_allclose(x, P * math.log(2.0) / base - 1.0, rtol=2e-6, atol=2e-6)


def test_power_normalize_whitens_red_noise():
    """White exponential power comes out with mean ~0 and sigma ~1 (the median of B exponentials
    estimates ln 2 of the mean), and the same noise times a smooth red trend comes out the same."""
    n, block = 1 << 16, 128
    k = np.arange(n)
    trend = 1.0 + 200.0 / (1.0 + k / 50.0)
    xw, _ = oracle.power_normalize(_cgauss(n, 12), block)
    xr, _ = oracle.power_normalize(_cgauss(n, 12, trend), block)
    for qw, qr in zip(np.array_split(xw[4 * block:], 4), np.array_split(xr[4 * block:], 4)):
        assert abs(qw.mean()) < 0.05 and abs(qw.std() - 1.0) < 0.1
        assert abs(qr.mean() - qw.mean()) < 0.01 and abs(qr.std() / qw.std() - 1.0) < 0.02


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_power_normalize_reduced_precision_is_the_rounded_fp32(dtype):
    z = _cgauss(5000, 21)
    x32, _ = oracle.power_normalize(z, 128)
    xr, _ = oracle.power_normalize(z, 128, dtype)
    if dtype == "f16":
        np.testing.assert_array_equal(xr, x32.astype(np.float16).view(np.uint16))
    else:
        import torch

        np.testing.assert_array_equal(xr, torch.from_numpy(x32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16))


# ---------------------------------------------------------------------------------------------
# candidate sifting: hand-built lists
# ---------------------------------------------------------------------------------------------

def _cands(rows):
    c = np.zeros(len(rows), oracle.CANDIDATE_DTYPE)
    for i, (spec, b, snr, z, h, v) in enumerate(rows):
        c[i] = (spec, b, snr, z, h, v)
    return c


def test_sift_drops_harmonics_and_neighbours_of_stronger_candidates():
    """Worked by hand (tol 1.5 bins, k <= 8): a candidate goes when any stronger one of its group is
    related to it, whether or not that stronger one is itself kept."""
    FB, STD = oracle.FBIN, oracle.STD
    c = _cands([
        (0, 100, 20.0, 0, 4, FB),   # 300 = 3 x 100 and 300 is stronger: dropped
        (0, 200, 10.0, 0, 4, FB),   # 200 = 2 x 100 (stronger): dropped
        (0, 101, 15.0, 0, 4, FB),   # |101 - 100| = 1 <= 1.5: dropped
        (0, 137, 12.0, 0, 4, FB),   # 137 - 100, 137 - 101, 300 - 2 x 137 = 26 > 3: kept
        (0, 300, 25.0, 0, 8, FB),   # the strongest of its group: kept
        (0, 1000, 9.0, 0, 4, FB),   # 1000 = 5 x 200 (snr 10 > 9): dropped
        (1, 200, 10.0, 0, 4, FB),   # another spectrum: kept
        (0, 400, 30.0, 0, 8, STD),  # Eq. 1 reports the H-th harmonic: fundamental 400/8 = 50; kept
        (0, 800, 29.0, 0, 16, STD), # fundamental 800/16 = 50 again, weaker: dropped
    ])
    keep = oracle.sift_candidates(c, tol=1.5, tol_z=1.5, kmax=8)
    np.testing.assert_array_equal(keep, [False, False, False, True, True, False, True, True, False])
    # with k <= 4 the fifth harmonic no longer counts
    assert oracle.sift_candidates(c, tol=1.5, tol_z=1.5, kmax=4)[5]


def test_sift_ties_keep_the_earlier_and_drift_counts():
    FB, STD = oracle.FBIN, oracle.STD
    c = _cands([(3, 500, 8.0, 0, 2, FB), (3, 501, 8.0, 0, 2, FB), (3, 1000, 8.0, 0, 2, FB)])
    np.testing.assert_array_equal(oracle.sift_candidates(c), [True, False, False])
    # 2-D candidates (Eq. 1 form): the same frequency but a different drift is not the same signal
    d = _cands([(0, 640, 12.0, 40, 4, STD), (0, 640, 11.0, -40, 4, STD), (0, 1280, 10.0, 80, 8, STD)])
    np.testing.assert_array_equal(oracle.sift_candidates(d, tol=1.5, tol_z=1.5), [True, True, False])


# ---------------------------------------------------------------------------------------------
# 2-D freq-bin form: harmonic i of the cell (n, z) at (i n, i z)
# ---------------------------------------------------------------------------------------------

def test_2d_fbin_zero_row_is_1d_fbin_and_ranges():
    nz, z_min, nb = 9, -4, 300
    plane = np.stack([rand_spectrum(nb, 70 + r) for r in range(nz)])
    r2 = oracle.hs_2d(plane, z_min, hmax=16, fp64=True, all_h=True, variant="fbin")
    r1 = oracle.hs_1d("fbin", plane[-z_min], hmax=16, fp64=True, all_h=True)
    np.testing.assert_array_equal(r2["all_h"][:, -z_min, :], r1["all_h"])
    # row z: valid H need H*z within [-4, 4] (and H*n <= nb - 1)
    for r in range(nz):
        z = z_min + r
        hz = 16 if z == 0 else (4 // abs(z))
        for n in (0, 1, 7, 150, 299):
            hn = 16 if n == 0 else min(16, (nb - 1) // n)
            hv = min(hz, hn)
            col = r2["all_h"][:, r, n]
            assert np.isfinite(col[:hv]).all() and np.isneginf(col[hv:]).all(), (z, n, hv)


def test_2d_fbin_delta_spike_and_constant():
    nz, z_min, nb, A = 13, -6, 200, 2.0
    n0, z0 = 120, -6
    plane = np.zeros((nz, nb))
    plane[z0 - z_min, n0] = A
    r = oracle.hs_2d(plane, z_min, hmax=16, fp64=True, all_h=True, variant="fbin")
    for rr in range(nz):
        z = z_min + rr
        for n in range(1, nb):
            for H in range(1, 17):
                v = r["all_h"][H - 1, rr, n]
                if not np.isfinite(v):
                    continue
                hit = any(i * n == n0 and i * z == z0 for i in range(1, H + 1))
                assert v == pytest.approx(A * hit / math.sqrt(H), abs=1e-15), (z, n, H)
    c = oracle.hs_2d(np.full((nz, nb), 1.5), z_min, hmax=16, fp64=True, all_h=True, variant="fbin")["all_h"]
    for H in range(1, 17):
        v = c[H - 1][np.isfinite(c[H - 1])]
        np.testing.assert_allclose(v, 1.5 * math.sqrt(H), rtol=1e-14)


# ---------------------------------------------------------------------------------------------
# 2-D forms of Eq. 2 and Eq. 4 (a reading: harmonic i of the cell (n, z) taken on the row i z as the
# 1-D equation takes it)
# ---------------------------------------------------------------------------------------------

ROWWISE = ["max", "max0", "greedy", "greedy1"]


@pytest.mark.parametrize("variant", ROWWISE)
def test_2d_rowwise_zero_row_is_1d_and_ranges(variant):
    """Every harmonic of a z = 0 cell lies on row 0, so that row's results are the 1-D sums of the
    row (including the Eq. 4 choices); row z keeps H while H z stays in the plane."""
    nz, z_min, nb = 9, -4, 300
    ties = np.random.default_rng(81).integers(0, 3, (nz, nb)).astype(np.float64)  # many equal neighbours
    for plane in (ties, np.stack([rand_spectrum(nb, 80 + r) for r in range(nz)])):
        for fp64 in (False, True):
            r2 = oracle.hs_2d(plane, z_min, hmax=16, fp64=fp64, all_h=True, variant=variant)
            r1 = oracle.hs_1d(variant, plane[-z_min], hmax=16, fp64=fp64, all_h=True)
            np.testing.assert_array_equal(r2["all_h"][:, -z_min, :], r1["all_h"])
            np.testing.assert_array_equal(r2["best_h"][-z_min], r1["best_h"])
    for r in range(nz):
        z = z_min + r
        hz = 16 if z == 0 else (4 // abs(z))
        for n in (0, 1, 7, 150, 298, 299):
            hv = min(hz, oracle.hvalid(variant, n, nb, 16))
            col = r2["all_h"][:, r, n]
            assert np.isfinite(col[:hv]).all() and np.isneginf(col[hv:]).all(), (z, n, hv)


@pytest.mark.parametrize("variant", ROWWISE)
def test_2d_rowwise_reads_only_rows_i_z(variant):
    """Changing every row that is not i z for some i <= H leaves the cell's sums up to H unchanged,
    and changing row i z changes them."""
    nz, z_min, nb = 15, -7, 160
    plane = np.stack([rand_spectrum(nb, 90 + r) for r in range(nz)])
    base = oracle.hs_2d(plane, z_min, hmax=16, fp64=True, all_h=True, variant=variant)["all_h"]
    for z in (-3, -2, 2, 3):
        used = {i * z for i in range(1, 17) if z_min <= i * z <= z_min + nz - 1}
        other = plane.copy()
        for rr in range(nz):
            if z_min + rr not in used:
                other[rr] = rand_spectrum(nb, 500 + rr)
        got = oracle.hs_2d(other, z_min, hmax=16, fp64=True, all_h=True, variant=variant)["all_h"]
        np.testing.assert_array_equal(got[:, z - z_min, :], base[:, z - z_min, :])
        bumped = plane.copy()
        bumped[2 * z - z_min] += 3.0  # row of harmonic 2
        got = oracle.hs_2d(bumped, z_min, hmax=16, fp64=True, all_h=True, variant=variant)["all_h"]
        ok = np.isfinite(base[1, z - z_min, :])
        assert (got[1, z - z_min, ok] != base[1, z - z_min, ok]).any()


@pytest.mark.parametrize("variant", ROWWISE)
def test_2d_rowwise_constant_plane(variant):
    """x = c everywhere: every window maximum and every choice (a tie keeps the left bin) is c, so
    h_H = c sqrt(H) for every valid H."""
    nz, z_min, nb = 11, -5, 120
    c = oracle.hs_2d(np.full((nz, nb), 1.5), z_min, hmax=16, fp64=True, all_h=True, variant=variant)["all_h"]
    for H in range(1, 17):
        v = c[H - 1][np.isfinite(c[H - 1])]
        assert v.size > 0
        np.testing.assert_allclose(v, 1.5 * math.sqrt(H), rtol=1e-14)


def test_2d_rowwise_max_delta_spike():
    """One spike A at (m0, z0) of an otherwise zero plane: harmonic i of the cell (n, z) takes A exactly
    when i z = z0 and m0 is in its window i n + 1 .. i n + i (i n .. i n + i for the window from 0)."""
    nz, z_min, nb, A = 13, -6, 150, 2.0
    m0, z0 = 97, -6
    plane = np.zeros((nz, nb))
    plane[z0 - z_min, m0] = A
    for variant, j0 in (("max", 1), ("max0", 0)):
        r = oracle.hs_2d(plane, z_min, hmax=16, fp64=True, all_h=True, variant=variant)["all_h"]
        for rr in range(nz):
            z = z_min + rr
            for n in range(nb):
                for H in range(1, 17):
                    v = r[H - 1, rr, n]
                    if not np.isfinite(v):
                        continue
                    hits = sum(1 for i in range(1, H + 1) if i * z == z0 and i * n + j0 <= m0 <= i * n + i)
                    assert v == pytest.approx(A * hits / math.sqrt(H), abs=1e-15), (variant, z, n, H)
