"""The pins must catch plausible mistakes in the oracle.

Each case copies the oracle's C source to a temporary directory, plants one mistake by a textual
edit (a dropped term, a wrong rounding, an off-by-one window, a reversed tie rule, ...), builds that
copy, points the oracle wrapper at it and runs the pins that should notice.  The real oracle source
is never modified.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.dirname(os.path.abspath(oracle.__file__))

# (name, file, text to replace, replacement, pins that must fail)
MUTANTS = [
    ("eq1 floor instead of round half up", "hs_oracle.c",
     "return (2 * n * (int64_t)i + H) / (2 * (int64_t)H);", "return (2 * n * (int64_t)i) / (2 * (int64_t)H);",
     ["test_golden_1d_hand_worked", "test_delta_spike_eq1"]),
    ("eq1 dropped last term", "hs_oracle_body.h",
     "for (int i = 1; i <= H; ++i) sum = sum + x[hs_oracle_eq1_index(n, i, H)];",
     "for (int i = 1; i < H; ++i) sum = sum + x[hs_oracle_eq1_index(n, i, H)];",
     ["test_h1_identity", "test_constant_spectrum"]),
    ("max window starts at j = 0", "hs_oracle_body.h", "int j0 = variant == HS_O_MAX0 ? 0 : 1;",
     "int j0 = variant == HS_O_MAX0 ? 0 : 0;", ["test_h1_identity", "test_max_bruteforce"]),
    ("max0 window starts at j = 1", "hs_oracle_body.h", "int j0 = variant == HS_O_MAX0 ? 0 : 1;",
     "int j0 = variant == HS_O_MAX0 ? 1 : 1;", ["test_h1_identity", "test_max_bruteforce"]),
    ("max window ends one bin early", "hs_oracle_body.h", "for (int jj = j0 + 1; jj <= H; ++jj) {",
     "for (int jj = j0 + 1; jj < H; ++jj) {", ["test_delta_spike_max", "test_max_bruteforce"]),
    ("max0 noise moments with the max window", "hs_oracle.c", "int w = variant == HS_O_MAX0 ? H + 1 : H;",
     "int w = H;", ["test_noise_calibration_tables"]),
    ("greedy takes the right bin on ties", "hs_oracle_body.h", "if (r > l) {", "if (r >= l) {",
     ["test_constant_spectrum", "test_greedy_bruteforce_paths"]),
    ("freq-bin reads the neighbour", "hs_oracle_body.h", "S = S + x[(int64_t)H * n];",
     "S = S + x[(int64_t)H * n + (H > 1)];", ["test_golden_1d_hand_worked", "test_delta_spike_fbin"]),
    ("largest H wins ties", "hs_oracle_body.h",
     "if (snr > best) {\n                    best = snr;\n                    best_h = H;",
     "if (snr >= best) {\n                    best = snr;\n                    best_h = H;", ["test_zero_spectrum_tie_break"]),
    ("max/greedy range off by one", "hs_oracle.c", "lim = (N - 1) / (n + 1); /* H*(n+1) <= N-1 */",
     "lim = N / (n + 1);", ["test_range_limits"]),
    ("2-D z rounded toward zero", "hs_oracle.c", "return (a % b != 0 && a < 0) ? q - 1 : q;", "return q;",
     ["test_golden_2d_hand_worked", "test_delta_spike_2d_negative_half_rounding"]),
    ("calibration applied in the wrong order", "hs_oracle_body.h",
     "REAL h = sum * cs[H];\n                snr = (h - mu[H]) * isig[H];",
     "REAL h = sum * cs[H];\n                snr = h * isig[H] - mu[H];", ["test_calibration_closed_form"]),
    ("2-D transposed plane index", "hs_oracle_body.h",
     "sum = sum + plane[(zi - z_min) * row_stride + ni];", "sum = sum + plane[ni * nz + (zi - z_min)];",
     ["test_2d_zero_row_is_1d_eq1", "test_golden_2d_hand_worked"]),
    ("adjoint scale without 1/sqrt(H)", "hs_oracle.c", "double w = g[n] * (1.0 / sqrt((double)Hs)) * isig;",
     "double w = g[n] * isig;", ["test_adjoint_is_transpose_of_linear_map"]),
    ("max adjoint routes to the last maximum", "hs_oracle.c", "if (x[base + jj] > x[m]) m = base + jj;",
     "if (x[base + jj] >= x[m]) m = base + jj;", ["test_adjoint_max_ties_route_to_first_maximum"]),
    ("every H is a power-of-two stage", "hs_oracle_body.h", "const int stage = !pow2 || (H & (H - 1)) == 0;",
     "const int stage = 1;", ["test_pow2_stages_restrict_the_full_search"]),
    ("odd H are stages", "hs_oracle_body.h", "const int stage = !pow2 || (H & (H - 1)) == 0;",
     "const int stage = !pow2 || (H & 1) == 0 || H == 1;", ["test_pow2_stages_restrict_the_full_search"]),
    ("upper median instead of lower", "hs_oracle.c", "m[j] = tmp[(size - 1) / 2];", "m[j] = tmp[size / 2];",
     ["test_power_normalize_medians_are_lower_order_statistics"]),
    ("interpolation against the wrong neighbour centre", "hs_oracle.c",
     "float t = (d - hj) / ((float)block - hj + hn);", "float t = (d - hj) / ((float)block);",
     ["test_power_normalize_interpolates_between_block_centres"]),
    ("dereddening by the median, not the mean estimate", "hs_oracle.c",
     "float x = base > 0.0f ? (P[k] * ln2) / base - 1.0f : 0.0f;", "float x = base > 0.0f ? P[k] / base - 1.0f : 0.0f;",
     ["test_power_normalize_constant_and_zero", "test_power_normalize_whitens_red_noise"]),
    ("greedy1 pairs from the first harmonic", "hs_oracle_body.h", "} else if (variant == HS_O_GREEDY1 && H == 1) {",
     "} else if (variant == HS_O_GREEDY1 && H == 0) {", ["test_h1_identity", "test_greedy_bruteforce_paths"]),
    ("greedy1 range as for greedy", "hs_oracle.c", "lim = N / (n + 1); /* H*(n+1) <= N */",
     "lim = (N - 1) / (n + 1);", ["test_range_limits"]),
    ("f16 ties round away from zero", "hs_oracle.c", "uint32_t h = (r + 0x0FFFu + ((r >> 13) & 1u)) >> 13;",
     "uint32_t h = (r + 0x1000u) >> 13;", ["test_standardize_cast_f16_matches_ieee_library"]),
    ("bf16 truncates", "hs_oracle.c", "return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);",
     "return (uint16_t)(u >> 16);", ["test_standardize_cast_bf16_matches_torch"]),
    ("f16 subnormal boundary one exponent off", "hs_oracle.c", "int shift = 126 - e;", "int shift = 125 - e;",
     ["test_standardize_cast_f16_matches_ieee_library"]),
    ("max noise mean drops the -1 of the standardised terms", "hs_oracle.c", "m_acc += harm - 1.0;",
     "m_acc += harm;", ["test_noise_calibration_tables"]),
    ("2-D row-wise forms read row z for every harmonic", "hs_oracle_body.h",
     "const REAL* row = plane + (H * z - z_min) * row_stride;", "const REAL* row = plane + (z - z_min) * row_stride;",
     ["test_2d_rowwise_reads_only_rows_i_z", "test_2d_rowwise_max_delta_spike"]),
    ("2-D row-wise greedy takes the right bin on ties", "hs_oracle_body.h", "if (rgt > lft) {", "if (rgt >= lft) {",
     ["test_2d_rowwise_zero_row_is_1d_and_ranges"]),
    ("2-D row-wise max window ends one bin early", "hs_oracle_body.h",
     "for (int jw = jfirst + 1; jw <= H; ++jw) {", "for (int jw = jfirst + 1; jw < H; ++jw) {",
     ["test_2d_rowwise_max_delta_spike", "test_2d_rowwise_zero_row_is_1d_and_ranges"]),
    ("2-D row-wise drift range one row short", "hs_oracle_body.h",
     "const int valid = H <= hv && H * z >= z_min && H * z <= z_max;",
     "const int valid = H <= hv && H * z > z_min && H * z <= z_max;", ["test_2d_rowwise_zero_row_is_1d_and_ranges"]),
]


def _build_mutant(tmp, fname, old, new):
    for f in ("hs_oracle.c", "hs_oracle_body.h"):
        shutil.copy(os.path.join(SRC, f), os.path.join(tmp, f))
    path = os.path.join(tmp, fname)
    text = open(path).read()
    assert text.count(old) == 1, "mutation anchor not found once: %r" % old
    open(path, "w").write(text.replace(old, new))
    lib = os.path.join(tmp, "libmutant.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    os.path.join(tmp, "hs_oracle.c"), "-o", lib, "-lm"], check=True, capture_output=True)
    return lib


def _run_pin(name):
    fn = getattr(pins, name)
    params = {"test_h1_identity": [(v,) for v in pins.VARIANTS],
              "test_max_bruteforce": [("max",), ("max0",)],
              "test_greedy_bruteforce_paths": [("greedy",), ("greedy1",)],
              "test_delta_spike_max": [("max",), ("max0",)],
              "test_constant_spectrum": [(v, c) for v in pins.VARIANTS for c in (1.0, 3.5)],
              "test_range_limits": [(v,) for v in pins.VARIANTS],
              "test_linearity": [("std",), ("fbin",)],
              "test_calibration_closed_form": [(v,) for v in pins.VARIANTS],
              "test_pow2_stages_restrict_the_full_search": [(v,) for v in pins.VARIANTS],
              "test_power_normalize_medians_are_lower_order_statistics": [(1000, 128), (77, 128), (300, 256)],
              "test_adjoint_is_transpose_of_linear_map": [("std",), ("fbin",)],
              "test_2d_rowwise_zero_row_is_1d_and_ranges": [(v,) for v in pins.ROWWISE],
              "test_2d_rowwise_reads_only_rows_i_z": [(v,) for v in pins.ROWWISE],
              "test_2d_rowwise_constant_plane": [(v,) for v in pins.ROWWISE]}
    for args in params.get(name, [()]):
        fn(*args)


@pytest.mark.parametrize("name,fname,old,new,expected", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, monkeypatch, name, fname, old, new, expected):
    lib = _build_mutant(str(tmp_path), fname, old, new)
    real = oracle._load()
    mutant = ctypes.CDLL(lib)
    for attr in dir(real):  # reuse the wrapper's argument declarations
        if attr.startswith("hs_oracle_"):
            f, g = getattr(real, attr), getattr(mutant, attr)
            g.argtypes, g.restype = f.argtypes, f.restype
    monkeypatch.setattr(oracle, "_lib", mutant)
    caught = []
    for pin in expected:
        try:
            _run_pin(pin)
        except AssertionError:
            caught.append(pin)
    assert caught, "no pin caught the planted mistake: %s" % name


def test_unmutated_copy_passes(tmp_path, monkeypatch):
    """Control: the same machinery with no edit passes the pins it would run."""
    lib = _build_mutant(str(tmp_path), "hs_oracle.c", "#define HS_O_STD 1", "#define HS_O_STD 1")
    real = oracle._load()
    mutant = ctypes.CDLL(lib)
    for attr in dir(real):
        if attr.startswith("hs_oracle_"):
            f, g = getattr(real, attr), getattr(mutant, attr)
            g.argtypes, g.restype = f.argtypes, f.restype
    monkeypatch.setattr(oracle, "_lib", mutant)
    for pin in ("test_golden_1d_hand_worked", "test_delta_spike_eq1", "test_max_bruteforce", "test_noise_calibration_tables",
                "test_greedy_bruteforce_paths", "test_zero_spectrum_tie_break", "test_golden_2d_hand_worked",
                "test_calibration_closed_form", "test_adjoint_max_ties_route_to_first_maximum"):
        _run_pin(pin)
