"""The C ABI without a GPU: the library loads, exports every entry point the header declares, and
its host-side validation rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

from conftest import gpu_available

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "harmonic_sum.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hs_plan_create", "hs_sum_1d", "hs_sum_2d", "hs_sum_batched", "hs_backward", "hs_plan_destroy",
              "hs_sync_status", "hs_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(hs_lib):
    lib = ctypes.CDLL(hs_lib.LIBRARY_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def header_defines():
    return {m.group(1): m.group(2) for m in re.finditer(r"#define\s+(HS_[A-Z0-9_]+)\s+(\S+)", open(HEADER).read())}


def test_binding_constants_match_the_header(hs_lib):
    """The Python binding restates some header constants; they must not drift apart."""
    d = header_defines()
    assert int(d["HS_NOALLOC_MAX_SPECTRA"]) == hs_lib.NOALLOC_MAX_SPECTRA
    assert int(d["HS_MAX_CTAS_PER_SM"]) == hs_lib.MAX_CTAS_PER_SM
    assert int(d["HS_HMAX_1D"]) == hs_lib.HMAX_1D and int(d["HS_HMAX_2D"]) == hs_lib.HMAX_2D
    for name in ("OUT_ALL_H", "STAGED_SPANS", "MAX_WINDOW0", "POW2_STAGES", "GREEDY_FIXED1", "CHECK_TIMEOUT"):
        assert int(d["HS_FLAG_" + name]) == getattr(hs_lib, "FLAG_" + name), name


def test_status_strings(hs_lib):
    for s in (0, 1, 2, 3, 4, 5, 6, 100):
        assert hs_lib.hs_status_string(s).startswith("HS_")
    assert hs_lib.hs_version() >= 100


@pytest.mark.parametrize("bad", [dict(variants=0), dict(variants=16), dict(hmax=0), dict(hmax=33),
                                 dict(dtype=3), dict(max_bins=-1), dict(max_bins=(1 << 26) + 1),
                                 dict(nz=5, z_min=1, hmax=16), dict(nz=5, z_min=-5, hmax=16),
                                 dict(nz=5, z_min=-2, hmax=17), dict(cand_capacity=-1), dict(flags=64),
                                 dict(nz=5, z_min=-2, hmax=16, flags=8),
                                 dict(threshold=float("nan"))])
def test_plan_create_rejects(hs_lib, bad):
    kw = dict(variants=0xF, hmax=32, dtype=0, max_bins=1 << 20, nz=0, z_min=0, threshold=6.0, cand_capacity=0,
              flags=0)
    kw.update(bad)
    with pytest.raises(hs_lib.HSError) as e:
        hs_lib.hs_plan_create(**kw)
    assert e.value.status == hs_lib.ERR_INVALID


def test_plan_accepts_and_sizes_workspace(hs_lib):
    p, _ = hs_lib.hs_plan_create(cand_capacity=1 << 20)
    a = hs_lib.hs_plan_workspace_size(p, 1)
    b = hs_lib.hs_plan_workspace_size(p, 100000)
    assert a % 256 == 0 and b % 256 == 0 and b >= 8 * 100000
    hs_lib.hs_plan_destroy(p)


def test_16bit_eq1_plans_reserve_the_fp32_staging_region(hs_lib):
    """Batched Eq. 1 over FP16/BF16 widens up to 64 spectra at a time into FP32 in the workspace, after
    the control words and prefix sums, so such plans ask for min(n_spectra, 64) * max_bins * 4 bytes
    there (the candidate sort, which runs after the sums, reuses the same space); other plans do not."""
    mb = 1 << 16
    sizes = {}
    for name, dtype, variants in (("f32", hs_lib.F32, hs_lib.STD), ("f16", hs_lib.F16, hs_lib.STD),
                                  ("bf16", hs_lib.BF16, hs_lib.STD), ("f16max", hs_lib.F16, hs_lib.MAX)):
        p, _ = hs_lib.hs_plan_create(variants=variants, dtype=dtype, max_bins=mb)
        sizes[name] = {n: hs_lib.hs_plan_workspace_size(p, n) for n in (1, 10, 64, 300)}
        hs_lib.hs_plan_destroy(p)
    for n in (1, 10, 64, 300):
        stage = min(n, 64) * mb * 4
        head = 256 + 8 * (n + 2)  # control words and tile prefix sums
        for name in ("f16", "bf16"):
            assert sizes[name][n] >= head + stage and sizes[name][n] >= sizes["f32"][n]
            assert sizes[name][n] <= max(sizes["f32"][n], head + stage + 512)
        assert sizes["f16max"][n] == sizes["f32"][n]


def test_calls_validate_before_device_work(hs_lib):
    lib = hs_lib._lib
    p, _ = hs_lib.hs_plan_create(variants=hs_lib.FBIN)
    out = hs_lib.Out()
    # null plan, variant not in plan, null input, misaligned input, null outputs, null workspace
    assert lib.hs_sum_1d(None, 4, 16, 10, 0, ctypes.byref(out), 256, 4096, None) == hs_lib.ERR_INVALID
    assert lib.hs_sum_1d(p, 2, 16, 10, 0, ctypes.byref(out), 256, 4096, None) == hs_lib.ERR_INVALID
    assert lib.hs_sum_1d(p, 4, None, 10, 0, ctypes.byref(out), 256, 4096, None) == hs_lib.ERR_INVALID
    assert lib.hs_sum_1d(p, 4, 18, 10, 0, ctypes.byref(out), 256, 4096, None) == hs_lib.ERR_ALIGN
    assert lib.hs_sum_1d(p, 4, 16, 10, 0, ctypes.byref(out), 256, 4096, None) == hs_lib.ERR_INVALID
    out2 = hs_lib.Out(256, 512, None, None, None, None)
    assert lib.hs_sum_1d(p, 4, 16, 10, 0, ctypes.byref(out2), None, 4096, None) == hs_lib.ERR_INVALID
    assert lib.hs_sum_1d(p, 4, 16, 10, 0, ctypes.byref(out2), 256, 16, None) == hs_lib.ERR_NOMEM
    assert lib.hs_sum_1d(p, 4, 16, -1, 0, ctypes.byref(out2), 256, 4096, None) == hs_lib.ERR_INVALID
    # all-H table needs the plan flag; candidates need a capacity
    out3 = hs_lib.Out(256, 512, None, 1024, None, None)
    assert lib.hs_sum_1d(p, 4, 16, 10, 0, ctypes.byref(out3), 256, 4096, None) == hs_lib.ERR_INVALID
    out4 = hs_lib.Out(256, 512, None, None, 2048, 4096)
    assert lib.hs_sum_1d(p, 4, 16, 10, 0, ctypes.byref(out4), 256, 4096, None) == hs_lib.ERR_INVALID
    # 2-D on a 1-D plan, greedy backward without a path
    assert lib.hs_sum_2d(p, 16, 10, 10, 0, None, 256, 4096, None) == hs_lib.ERR_INVALID
    pg, _ = hs_lib.hs_plan_create(variants=hs_lib.GREEDY)
    assert lib.hs_backward(pg, 8, 16, None, 1, 10, 256, 512, None, 1024, None) == hs_lib.ERR_INVALID
    hs_lib.hs_plan_destroy(p)
    hs_lib.hs_plan_destroy(pg)


def test_binding_checks_input_type_against_plan(hs_lib):
    """The C calls read the spectra as the plan's storage type through a bare pointer, so the binding
    refuses a tensor of another type, non-contiguous spectra and non-int64 offsets before any call."""
    torch = pytest.importorskip("torch")
    p, _ = hs_lib.hs_plan_create(variants=hs_lib.FBIN, dtype=hs_lib.F32)
    ph, _ = hs_lib.hs_plan_create(variants=hs_lib.FBIN, dtype=hs_lib.F16)
    offs = torch.tensor([0, 64, 128], dtype=torch.int64)
    out = hs_lib.Out()
    ws = torch.empty(16, dtype=torch.uint8)
    cases = [(p, torch.zeros(128, dtype=torch.float16), offs),
             (ph, torch.zeros(128, dtype=torch.float32), offs),
             (p, torch.zeros(128, dtype=torch.float64), offs),
             (p, torch.zeros(256, dtype=torch.float32)[::2], offs),
             (p, torch.zeros(128, dtype=torch.float32), offs.to(torch.int32))]
    for plan, x, o in cases:
        with pytest.raises(hs_lib.HSError) as e:
            hs_lib.hs_sum_batched(plan, "fbin", x, o, out, ws)
        assert e.value.status == hs_lib.ERR_INVALID
        with pytest.raises(hs_lib.HSError):
            hs_lib.hs_sum_batched_noalloc(plan, "fbin", x, o, out)
    with pytest.raises(hs_lib.HSError):
        hs_lib.hs_sum_1d(ph, "fbin", torch.zeros(64, dtype=torch.bfloat16), out, ws)
    hs_lib.hs_plan_destroy(p)
    hs_lib.hs_plan_destroy(ph)


def test_ctas_per_sm_cap_arguments(hs_lib):
    p, _ = hs_lib.hs_plan_create(variants=0xF)
    for v in ("std", "max", "fbin", "greedy"):
        assert hs_lib.hs_plan_ctas_per_sm(p, v) == 0  # default: as many as fit
    hs_lib.hs_plan_set_ctas_per_sm(p, "fbin", hs_lib.MAX_CTAS_PER_SM)
    assert hs_lib.hs_plan_ctas_per_sm(p, "fbin") == hs_lib.MAX_CTAS_PER_SM
    for bad in (-1, hs_lib.MAX_CTAS_PER_SM + 1):
        with pytest.raises(hs_lib.HSError) as e:
            hs_lib.hs_plan_set_ctas_per_sm(p, "std", bad)
        assert e.value.status == hs_lib.ERR_INVALID
    assert hs_lib._lib.hs_plan_set_ctas_per_sm(p, 3, 1) == hs_lib.ERR_INVALID  # not a single variant
    assert hs_lib._lib.hs_plan_ctas_per_sm(None, 1) == -1
    hs_lib.hs_plan_destroy(p)


def test_library_noise_calibration_matches_oracle(hs_lib):
    for v in ("std", "max", "fbin", "greedy"):
        mu, isig = hs_lib.hs_noise_calibration(v, 32)
        omu, oisig = oracle.noise_calibration(v, 32)
        np.testing.assert_array_equal(mu, omu)
        np.testing.assert_array_equal(isig, oisig)
    # Eq. 2 with the window j = 0..i
    mu, isig = hs_lib.hs_noise_calibration("max", 32, flags=hs_lib.FLAG_MAX_WINDOW0)
    omu, oisig = oracle.noise_calibration("max0", 32)
    np.testing.assert_array_equal(mu, omu)
    np.testing.assert_array_equal(isig, oisig)
    mu, isig = hs_lib.hs_noise_calibration("greedy", 32, flags=hs_lib.FLAG_GREEDY_FIXED1)
    omu, oisig = oracle.noise_calibration("greedy1", 32)
    np.testing.assert_array_equal(mu, omu)
    np.testing.assert_array_equal(isig, oisig)
    with pytest.raises(hs_lib.HSError):
        hs_lib.hs_noise_calibration("max", 32, flags=64)


def test_set_calibration_rejects_nonfinite(hs_lib):
    p, _ = hs_lib.hs_plan_create()
    mu = np.zeros(33, np.float32)
    isig = np.ones(33, np.float32)
    isig[5] = np.inf
    with pytest.raises(hs_lib.HSError):
        hs_lib.hs_plan_set_calibration(p, "max", mu, isig)
    hs_lib.hs_plan_set_calibration(p, "max", None, None)
    hs_lib.hs_plan_destroy(p)


@pytest.mark.skipif(gpu_available(), reason="the key names the device's SM count; with a GPU a miss would time "
                                             "kernels on the placeholder pointers")
def test_autotune_uses_cached_entry_without_timing(hs_lib, tmp_path, monkeypatch):
    """Without a device the cache key has SM count 0; an entry for it is taken as is, with no device
    work (the placeholder pointers are never used)."""
    cache = tmp_path / "tune.json"
    cache.write_text('{\n  "v1_d0_h32_b20_sm0": 8,\n  "v2_d0_h32_b20_sm0": 16\n}\n')
    monkeypatch.setenv("HS_AUTOTUNE_CACHE", str(cache))
    lib = hs_lib._lib
    p, _ = hs_lib.hs_plan_create(variants=0xF, max_bins=1 << 20)
    # fake device pointers: a cache hit returns before touching them
    st = lib.hs_autotune(p, 1, 1 << 20, ctypes.c_void_p(4096), 1 << 30, ctypes.c_void_p(8192), 1 << 20, None)
    assert st == hs_lib.OK
    assert lib.hs_autotune(p, 2, 1 << 20, ctypes.c_void_p(4096), 1 << 30, ctypes.c_void_p(8192), 1 << 20,
                           None) == hs_lib.OK
    assert lib.hs_autotune(p, 1, 0, ctypes.c_void_p(4096), 1 << 30, ctypes.c_void_p(8192), 1 << 20,
                           None) == hs_lib.ERR_INVALID
    hs_lib.hs_plan_destroy(p)


def test_tile_bins_round_trip(hs_lib):
    p, _ = hs_lib.hs_plan_create()
    hs_lib.hs_plan_set_tile_bins(p, "std", 8192)
    assert hs_lib.hs_plan_tile_bins(p, "std") == 8192
    for bad in (0, 100, 255, 257, 64 * 256 + 256):
        with pytest.raises(hs_lib.HSError):
            hs_lib.hs_plan_set_tile_bins(p, "max", bad)
    hs_lib.hs_plan_destroy(p)
