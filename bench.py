#!/usr/bin/env python3
"""Benchmark of the GB300 harmonic-sum library on the batched DM-trial workload.

Workload (one step): 2048 synthetic DM-trial spectra, lengths drawn uniformly from {2^19, 2^20,
2^21, 2^22} bins (4.02 G bins, 16.1 GB FP32), standardised exponential noise with pulsars injected
in 5% of them; all four harmonic-sum variants (Eq. 1-4), H = 1..32, per-bin best snr / H, the
Eq. 4 path, and candidates above 6.  Each variant is one persistent launch over a (spectrum, tile)
work queue, replayed from a CUDA graph.  The input is resident in HBM when the timed region starts
(it is larger than L2, so no flush is needed).

metric: harmonic-summed bins/s = (input bins x H_max) / step time, a step running all four
variants; under torchrun every rank processes its own batch (weak scaling) and the value counts
all ranks' bins over the slowest rank's time.

``--impl reference`` times the CPU oracle (the reference arm of this project: a plain C evaluation
of the paper's equations) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hs_synth  # noqa: E402

METRIC = "harmonic-summed bins/sec (input bins x H_max)"
UNIT = "bins*H/s"
HMAX = 32
VARIANTS = ("std", "max", "fbin", "greedy")
THR = 6.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--spectra", type=int, default=2048, help="spectra in the batch (2048 is the workload)")
    ap.add_argument("--variants", default=",".join(VARIANTS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default (or --tiles) tile sizes")
    ap.add_argument("--tiles", default="", help="variant=bins,... tile sizes to use instead of tuning")
    ap.add_argument("--cpu-sample-spectra", type=int, default=8)
    ap.add_argument("--staged-spans", action="store_true",
                    help="Eq. 1 with its input spans staged in shared memory by bulk copies (HS_FLAG_STAGED_SPANS)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the FP16/BF16, adjoint and 2-D measurements reported beside the main line")
    ap.add_argument("--section", default="", choices=("", "config1", "precision", "upstream", "adjoint", "fdas_2d"),
                    help="run only this secondary workload and print its JSON (for profiling one kernel)")
    ap.add_argument("--fdas-bins", type=int, default=1 << 21, help="bins per row of the 2-D planes")
    return ap.parse_args()


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]",) else 0.0,
                             parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        for r in rows:
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[3:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


def dist_setup():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def reduce_max(x, world):
    """Largest value over all ranks (the slowest rank's time decides a multi-GPU step)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(n_spectra, rank):
    """Weak scaling: every rank harmonic-sums its own batch of DM trials (trial index = rank), so
    ranks share no data and need no collective on the data path."""
    return hs_synth.batch_dm_trials_layout(n_spectra, trial=rank)


def cpu_oracle_sample(offsets, x_host, n_sample, variants, cores, reps=1):
    """Time the oracle's FP32 mode on the first n_sample spectra of the batch.  Each spectrum's bins
    are split across the given host cores (the oracle's single-spectrum path: chunks of 2048 bins
    handed out dynamically), so every core works however uneven the spectra are."""
    import oracle

    offs = offsets[: n_sample + 1].copy()
    xs = np.asarray(x_host[: int(offs[-1])])
    tables = {v: oracle.noise_calibration(v, HMAX) for v in variants}
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        for v in variants:
            mu, isig = tables[v]
            for s in range(n_sample):
                oracle.hs_1d(v, xs[int(offs[s]):int(offs[s + 1])], hmax=HMAX, mu=mu, isig=isig, nthreads=cores)
        times.append(time.perf_counter() - t0)
    bins = int(offs[-1])
    return bins, statistics.median(times)


def cpu_single_thread(offsets, x_host, variants, n_sample=2):
    """The oracle's FP32 mode on one host thread over the first n_sample spectra: the single-core
    figure reported beside the all-cores one."""
    bins, t = cpu_oracle_sample(offsets, x_host, n_sample, variants, 1)
    return {"value": bins * HMAX / t, "unit": UNIT, "cores": 1,
            "sample": "first %d spectra (%d bins), %s, FP32 oracle, one thread" % (n_sample, bins, "+".join(variants))}


def run_reference(args):
    """The reference arm: the CPU oracle on a bounded sample, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    variants = tuple(args.variants.split(","))
    seed, offsets, pulsars = hs_synth.batch_dm_trials_layout(args.spectra)
    n_sample = min(args.cpu_sample_spectra, args.spectra)  # the same sample as the main line's cpu_baseline
    x = hs_synth.batch(seed, offsets[: n_sample + 1], pulsars[:n_sample])
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_oracle_sample(offsets, x, n_sample, variants, cores)
    times = []
    for _ in range(args.steps):
        bins, t = cpu_oracle_sample(offsets, x, n_sample, variants, cores)
        times.append(t)
    step = statistics.mean(times)
    value = bins * HMAX / step
    sample = ("first %d of %d spectra (%d bins), %s, FP32 oracle, each spectrum's bins split across %d cores"
              % (n_sample, args.spectra, bins, "+".join(variants), cores))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, offsets, variants),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "single_thread": cpu_single_thread(offsets, x, variants)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def csrc_sha16():
    """Hash of the sources the batched 1-D kernels are built from, to tell whether a stored ncu
    traffic figure still belongs to the kernel being timed."""
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1812_02647_gb300", "csrc")
    for f in ("hs_1d.cu", "hs_common.cuh", "hs_farey.cuh", "hs_internal.cuh"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def workload_config(args, offsets, variants):
    return {"workload": "batched DM-trial spectra: %d spectra, lengths uniform in {2^19..2^22} bins, FP32, "
                        "H_max=32, variants %s, persistent graph-captured launch per variant" %
                        (args.spectra, "+".join(variants)),
            "n_spectra": args.spectra, "total_bins": int(offsets[-1]), "hmax": HMAX, "variants": list(variants),
            "threshold": THR, "l2": "inputs (%.1f GB) larger than L2; no flush" % (offsets[-1] * 4 / 1e9),
            "eq1_kernel": "staged spans" if args.staged_spans else "gather"}


def _noise(torch, shape, seed, dtype=None):
    """Standardised exponential noise generated on the device (secondary workloads only)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    u = torch.rand(shape, generator=g, device="cuda", dtype=torch.float32).clamp_(min=1e-30)
    return u.log_().neg_().sub_(1.0)


def _time_ms(torch, stream, fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    stream.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def secondary(torch, hs, stream, tiles=None, reps=2, only="", fdas_bins=1 << 21):
    """The single 131072-bin spectrum, the batched FP16/BF16 storage, the adjoint and the 2-D form on
    their own workloads, each next to the plain FP32 path on the same GPU.  Inputs are device-generated
    noise of the workload shapes (the single spectrum is the synthetic pulsar spectrum).  ``only``
    names one section to run alone."""
    out = {}
    for name, fn in (("config1", _sec_config1), ("precision", _sec_precision), ("upstream", _sec_upstream),
                     ("adjoint", _sec_adjoint), ("fdas_2d", _sec_fdas_2d)):
        if not only or only == name:
            out[name] = fn(torch, hs, stream, tiles, reps, fdas_bins)
            torch.cuda.empty_cache()
    return out


def fp64_sums(v, x, mu, isig, hmax=HMAX):
    """Eq. 1-4 over every bin of one spectrum in FP64 (numpy), for the accuracy report of the
    reduced-precision storage: best snr, best H, the snr of the runner-up H, and the Eq. 4 path.
    Same readings as the library: round-half-up Eq. 1 index, Eq. 2 window j = 1..i, Eq. 4 ties
    keep the left bin, harmonics truncated at the spectrum end, snr = (S/sqrt(H) - mu_H) isig_H."""
    x = np.asarray(x, dtype=np.float64)
    N = x.size
    n = np.arange(N, dtype=np.int64)
    mu64, is64 = np.asarray(mu, np.float64), np.asarray(isig, np.float64)
    best = np.full(N, -np.inf)
    second = np.full(N, -np.inf)
    bh = np.zeros(N, np.int64)
    path = np.zeros(N, np.uint32)

    def keep(H, snr, ok):
        snr = np.where(ok, snr, -np.inf)
        up = snr > best
        second[:] = np.where(up, best, np.maximum(second, snr))
        best[up] = snr[up]
        bh[up] = H

    if v == "std":
        for H in range(1, hmax + 1):
            S = np.zeros(N)
            for i in range(1, H + 1):
                S += x[(2 * n * i + H) // (2 * H)]
            keep(H, (S / np.sqrt(H) - mu64[H]) * is64[H], np.ones(N, bool))
        return best, bh, second, path
    S = np.zeros(N)
    j = np.zeros(N, np.int64)
    for i in range(1, hmax + 1):
        ok = (i * n <= N - 1) if v == "fbin" else (i * (n + 1) <= N - 1)
        m = n[ok]
        if v == "fbin":
            t = x[i * m]
        elif v == "max":
            t = x[i * m + 1]
            for k in range(2, i + 1):
                t = np.maximum(t, x[i * m + k])
        else:
            left, right = x[i * m + j[ok]], x[i * m + j[ok] + 1]
            r = right > left
            t = np.where(r, right, left)
            path[m[r]] |= np.uint32(1 << (i - 1))
            j[m[r]] += 1
        S[ok] += t
        keep(i, (S / np.sqrt(i) - mu64[i]) * is64[i], ok)
    return best, bh, second, path


def precision_accuracy(x32, got, mu, isig, tie=1e-3):
    """Error of one variant's GPU outputs (best snr, best H, path) against FP64 on the same FP32
    spectrum, and agreement beyond the tie margin."""
    v = got["variant"]
    b64, h64, s64, p64 = fp64_sums(v, x32, mu, isig)
    snr = got["best_snr"].astype(np.float64)
    ok = np.isfinite(b64)
    flips = 0
    if v == "greedy":
        same = got["path"] == p64
        flips = int((~same & ok).sum())
        ok &= same
    err = np.abs(snr[ok] - b64[ok])
    clear = ok & (np.abs(b64 - THR) > tie)
    cand = int(((snr > THR) != (b64 > THR))[clear].sum())
    with np.errstate(invalid="ignore"):  # bins with a single valid H have no runner-up (-inf - -inf)
        hclear = ok & (b64 - s64 > tie)
    hdis = int((got["best_h"].astype(np.int64) != h64)[hclear].sum())
    return {"max_abs_err_vs_fp64": float(err.max()) if err.size else 0.0,
            "max_rel_err_vs_fp64": float((err / np.maximum(np.abs(b64[ok]), 1.0)).max()) if err.size else 0.0,
            "candidates_disagreeing_beyond_tie": cand, "candidates_fp64": int((b64 > THR).sum()),
            "best_h_disagreeing_beyond_tie": hdis, "greedy_path_flips": flips, "bins": int(x32.size)}


def _sec_precision(torch, hs, stream, tiles, reps, fdas_bins):
    # 4096 spectra x 2^20 bins stored FP16 and BF16 after standardisation
    n_s, n_b = 4096, 1 << 20
    total = n_s * n_b
    od = (torch.arange(n_s + 1, device="cuda", dtype=torch.int64) * n_b)
    p = _noise(torch, (total,), 5000).add_(1.0)  # raw exponential power
    x32_first = p[:n_b].sub(1.0).cpu().numpy()  # spectrum 0 in FP32: the FP64 accuracy reference's input
    mu = torch.ones(n_s, device="cuda")
    sd = torch.ones(n_s, device="cuda")
    res = {}
    plans = {}
    for name, code, tdt in (("f32", hs.F32, torch.float32), ("f16", hs.F16, torch.float16),
                            ("bf16", hs.BF16, torch.bfloat16)):
        if name == "f32":
            x = p.sub(1.0)
            cast_ms = None
        else:
            x = torch.empty(total, dtype=tdt, device="cuda")
            cast_ms = _time_ms(torch, stream, lambda: hs.hs_standardize_cast(p, od, mu, sd, code, x, stream), reps)
        h = hs.HarmonicSum(variants=0xF, hmax=HMAX, dtype=code, max_bins=n_b, threshold=THR, cand_capacity=1 << 24,
                           max_spectra=n_s)
        for v, bins in (tiles or {}).items():
            hs.hs_plan_set_tile_bins(h.plan, v, bins)
        o = h.new_outputs(total, "greedy", "cuda")
        per = {}
        acc = {}
        for v in VARIANTS:
            mu_v, isig_v = hs.hs_noise_calibration(v, HMAX)
            h.set_calibration(v, mu_v, isig_v)

            def run(v=v):
                o["cand_count"].zero_()
                hs.hs_sum_batched(h.plan, v, x, od, h.out_struct(o), h.ws, 0, stream)

            per[v] = _time_ms(torch, stream, run, reps)
            stream.synchronize()
            got = {"variant": v, "best_snr": o["best_snr"][:n_b].cpu().numpy(),
                   "best_h": o["best_h"][:n_b].cpu().numpy(),
                   "path": o["path"][:n_b].cpu().numpy().view(np.uint32)}
            acc[v] = precision_accuracy(x32_first, got, mu_v, isig_v)
        step = sum(per.values())
        res[name] = {"ms_per_step": step, "per_variant_ms": per, "value": total * HMAX / (step / 1e3),
                     "input_bytes": total * x.element_size(), "cast_ms": cast_ms,
                     "cast_gbs": None if cast_ms is None else total * (4 + 2) / (cast_ms / 1e3) / 1e9,
                     "accuracy_spectrum0": acc}
        del x, o, h
        torch.cuda.empty_cache()
    for name in ("f16", "bf16"):
        res[name]["speedup_vs_f32"] = res["f32"]["ms_per_step"] / res[name]["ms_per_step"]
        res[name]["per_variant_speedup_vs_f32"] = {v: res["f32"]["per_variant_ms"][v] / res[name]["per_variant_ms"][v]
                                                   for v in VARIANTS}
    return {"workload": "4096 spectra x 2^20 bins, standardised Exp(1) noise, all four variants",
            "accuracy": "spectrum 0 (2^20 bins) of each storage type against an FP64 numpy evaluation of Eq. 1-4 on "
                        "its FP32 values; agreement counted where FP64 is more than 1e-3 from the threshold (candidates)"
                        " or from the runner-up H (best H); Eq. 4 bins whose path differs from FP64's are counted as "
                        "flips and left out of the error", **res}


def _sec_upstream(torch, hs, stream, tiles, reps, fdas_bins):
    # the step before the sums: power of complex spectra, block-median dereddening (128 bins),
    # standardisation, FP16 store; 1024 spectra x 2^20 complex bins (8 GiB in, 2 GiB out)
    n_s, n_b = 1024, 1 << 20
    g = torch.Generator(device="cuda")
    g.manual_seed(6000)
    spec = torch.randn(2 * n_s * n_b, generator=g, device="cuda").mul_(0.7071067811865476)
    od = torch.arange(n_s + 1, device="cuda", dtype=torch.int64) * n_b
    hu = hs.HarmonicSum(variants=hs.STD, dtype=hs.F16, max_bins=n_b, max_spectra=n_s)
    med = torch.empty(n_s * n_b // 128, device="cuda")
    out16 = torch.empty(n_s * n_b, dtype=torch.float16, device="cuda")
    ms = _time_ms(torch, stream, lambda: hs.hs_power_normalize(hu.plan, spec, od, 0, 128, med, out16, hu.ws, stream),
                  reps)
    compulsory = n_s * n_b * (8 + 2)  # complex in, FP16 out
    moved = n_s * n_b * (8 + 8 + 2)  # the median pass and the normalising pass each read the input
    peaks, _ = load_peaks()
    return {"workload": "1024 spectra x 2^20 complex bins -> FP16, blocks of 128 bins",
            "ms": ms, "gbs_compulsory": compulsory / (ms / 1e3) / 1e9,
            "gbs_moved": moved / (ms / 1e3) / 1e9,
            "frac_compulsory_of_hbm": compulsory / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}


def _sec_adjoint(torch, hs, stream, tiles, reps, fdas_bins):
    # differentiation: 256 spectra x 2^20, Eq. 1 and Max, loss = sum softplus(snr - 5)
    n_s, n_b = 256, 1 << 20
    total = n_s * n_b
    od = (torch.arange(n_s + 1, device="cuda", dtype=torch.int64) * n_b)
    x = _noise(torch, (total,), 4000)
    adj = {}
    for v in ("std", "max"):
        mu_v, isig_v = hs.hs_noise_calibration(v, HMAX)
        h = hs.HarmonicSum(variants=hs.VARIANTS[v], max_bins=n_b, threshold=THR, max_spectra=n_s,
                           calibration={v: (mu_v, isig_v)})
        if tiles and v in tiles:
            hs.hs_plan_set_tile_bins(h.plan, v, tiles[v])
        o = h.new_outputs(total, v, "cuda", candidates=False)
        g = torch.empty(total, device="cuda")
        gx = torch.empty(total, device="cuda")
        fwd = _time_ms(torch, stream, lambda: hs.hs_sum_batched(h.plan, v, x, od, h.out_struct(o), h.ws, 0, stream),
                       reps)
        torch.sigmoid(o["best_snr"] - 5.0, out=g)

        def bwd():
            gx.zero_()
            hs.hs_backward(h.plan, v, x, od, g, o["best_h"], o.get("path"), gx, stream)

        b = _time_ms(torch, stream, bwd, reps)
        # the backward scatters one FP32 atomic add per term of the chosen S_H*: H* per bin
        updates = int(o["best_h"].to(torch.int64).sum().item())
        adj[v] = {"forward_ms": fwd, "backward_ms": b, "backward_over_forward": b / fwd,
                  "value_fwd_bwd": total * HMAX / ((fwd + b) / 1e3),
                  "atomic_updates_per_bin": updates / total,
                  "atomic_updates_per_s": updates / (b / 1e3)}
        del h, o, g, gx
    return {"workload": "256 spectra x 2^20 bins FP32, loss = sum softplus(snr - 5)", **adj}


def _sec_fdas_2d(torch, hs, stream, tiles, reps, fdas_bins):
    # 2-D: 16 distinct FDAS planes of 201 z rows x 2^21 bins (27 GB), H = 1..16, each plane with its
    # own outputs; one pass over all 16 planes is timed
    nz, z_min, n_b, n_planes = 201, -100, fdas_bins, 16
    planes = [_noise(torch, (nz, n_b), 3000 + k) for k in range(n_planes)]
    h = hs.HarmonicSum(variants=hs.STD, hmax=16, nz=nz, z_min=z_min, max_bins=n_b, threshold=THR,
                       cand_capacity=1 << 24)
    outs = [h.sum_2d(planes[0], stream=stream)]
    outs += [{k: torch.empty_like(v) for k, v in outs[0].items()} for _ in range(n_planes - 1)]

    def all_planes():
        for k in range(n_planes):
            outs[k]["cand_count"].zero_()
            h.sum_2d(planes[k], plane_id=k, out=outs[k], stream=stream)

    t16 = _time_ms(torch, stream, all_planes, reps)
    cands = [int(o["cand_count"].item()) for o in outs]
    hf = hs.HarmonicSum(variants=hs.FBIN, hmax=16, nz=nz, z_min=z_min, max_bins=n_b, threshold=THR,
                        cand_capacity=1 << 24)

    def all_planes_fbin():
        for k in range(n_planes):
            outs[k]["cand_count"].zero_()
            hf.sum_2d(planes[k], plane_id=k, out=outs[k], stream=stream, variant="fbin")

    t16f = _time_ms(torch, stream, all_planes_fbin, reps)
    rowwise = {}
    for v in ("max", "greedy"):  # row-wise 2-D forms of Eq. 2 and 4 (harmonic i on row i z)
        hv = hs.HarmonicSum(variants=hs.VARIANTS[v], hmax=16, nz=nz, z_min=z_min, max_bins=n_b, threshold=THR,
                            cand_capacity=1 << 24)
        mu, isig = hs.hs_noise_calibration(v, 16)
        hv.set_calibration(v, mu, isig)

        def all_planes_v(v=v, hv=hv):
            for k in range(n_planes):
                outs[k]["cand_count"].zero_()
                hv.sum_2d(planes[k], plane_id=k, out=outs[k], stream=stream, variant=v)

        rowwise[v] = _time_ms(torch, stream, all_planes_v, reps)
    del planes, outs
    cells = n_planes * nz * n_b
    return {"workload": "16 distinct planes x 201 rows x %d bins FP32 (device noise), H = 1..16, one pass over all "
                        "planes timed" % n_b,
            "ms_per_16_planes": t16, "ms_per_plane": t16 / n_planes, "cells_per_s": cells / (t16 / 1e3),
            "harmonic_summed_cells_per_s": cells * 16 / (t16 / 1e3), "candidates_per_plane": cands,
            "fbin_ms_per_16_planes": t16f, "fbin_ms_per_plane": t16f / n_planes,
            "max_ms_per_16_planes": rowwise["max"], "greedy_ms_per_16_planes": rowwise["greedy"]}


def _sec_config1(torch, hs, stream, tiles, reps, fdas_bins):
    # one 131072-bin spectrum with the injected pulsar (f0 = 1000.37, 16 harmonics, 8/k), all four
    # variants through hs_sum_1d: per-variant device time of plain launches and of one CUDA graph
    # holding the whole step, and the host time to enqueue a call
    x, _ = hs_synth.spectrum_1d_pulsar(n_bins=131072)
    xd = torch.from_numpy(x).cuda()
    n_b = x.size
    hss, outs, tile = {}, {}, {}
    r = max(200, reps)
    for v in VARIANTS:
        mu, isig = hs.hs_noise_calibration(v, HMAX)
        h = hs.HarmonicSum(variants=hs.VARIANTS[v], hmax=HMAX, max_bins=n_b, threshold=THR, cand_capacity=1 << 16,
                           calibration={v: (mu, isig)})
        o = h.new_outputs(n_b, v, "cuda")
        best = None
        for tb in (256, 512, 1024, 2048, 4096):  # tile bins of the single-spectrum launch
            hs.hs_plan_set_tile_bins(h.plan, v, tb)
            t = _time_ms(torch, stream, lambda: hs.hs_sum_1d(h.plan, v, xd, h.out_struct(o), h.ws, 0, stream), r)
            if best is None or t < best[0]:
                best = (t, tb)
        hs.hs_plan_set_tile_bins(h.plan, v, best[1])
        hss[v], outs[v], tile[v] = h, o, best[1]
    per = {v: _time_ms(torch, stream, lambda v=v: hs.hs_sum_1d(hss[v].plan, v, xd, hss[v].out_struct(outs[v]),
                                                                  hss[v].ws, 0, stream), r) for v in VARIANTS}

    def step():
        for v in VARIANTS:
            outs[v]["cand_count"].zero_()
            hs.hs_sum_1d(hss[v].plan, v, xd, hss[v].out_struct(outs[v]), hss[v].ws, 0, stream)

    plain = _time_ms(torch, stream, step, r)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step()
    graph = _time_ms(torch, stream, g.replay, r)
    stream.synchronize()
    t0 = time.perf_counter()
    for _ in range(r):
        hs.hs_sum_1d(hss["std"].plan, "std", xd, hss["std"].out_struct(outs["std"]), hss["std"].ws, 0, stream)
    enqueue_us = (time.perf_counter() - t0) / r * 1e6
    stream.synchronize()
    step()
    stream.synchronize()
    found = {v: int(outs[v]["cand_count"].item()) for v in VARIANTS}
    return {"workload": "one spectrum of 131072 FP32 bins, pulsar at bin 1000.37 with 16 harmonics (8/k), "
                        "all four variants, H = 1..32, hs_sum_1d",
            "per_variant_us": {v: per[v] * 1e3 for v in VARIANTS}, "tile_bins": tile,
            "step_us_plain": plain * 1e3, "step_us_graph": graph * 1e3,
            "value_graph": n_b * HMAX / (graph / 1e3), "unit": UNIT,
            "host_enqueue_us_per_call": enqueue_us, "candidates": found}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    import paper_1812_02647_gb300 as hs

    if args.section:
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            print(json.dumps({"section": args.section,
                              **secondary(torch, hs, stream, reps=max(args.steps, 1), only=args.section,
                                          fdas_bins=args.fdas_bins)}))
        return 0
    rank, world, local = dist_setup()
    variants = tuple(args.variants.split(","))
    seed, offsets, pulsars = rank_workload(args.spectra, rank)
    total = int(offsets[-1])
    x_host = torch.empty(total, dtype=torch.float32, pin_memory=True)
    hs_synth.batch(seed, offsets, pulsars, out=x_host.data_ptr())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        xd = torch.empty(total, dtype=torch.float32, device="cuda")
        xd.copy_(x_host, non_blocking=True)
        od = torch.from_numpy(offsets).cuda()
        cap = 1 << 24
        h = hs.HarmonicSum(variants=0xF, hmax=HMAX, max_bins=1 << 22, threshold=THR, cand_capacity=cap,
                           max_spectra=args.spectra, flags=hs.FLAG_STAGED_SPANS if args.staged_spans else 0)
        for v in variants:
            mu, isig = hs.hs_noise_calibration(v, HMAX)
            h.set_calibration(v, mu, isig)
        outs = {v: h.new_outputs(total, v, "cuda") for v in variants}
        tuned = {}
        for kv in filter(None, args.tiles.split(",")):
            v, bins = kv.split("=")
            hs.hs_plan_set_tile_bins(h.plan, v, int(bins))
        if not args.no_autotune and not args.tiles:
            # tile sizes tuned on this very batch (outputs are rewritten by the timed steps)
            for v in variants:
                hs.hs_autotune_batched(h.plan, v, xd, od, h.out_struct(outs[v]), h.ws, stream)
        for v in variants:
            tuned[v] = hs.hs_plan_tile_bins(h.plan, v)
        cand_tmp = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
        graphs = {v: hs.hs_graph_create_batched(h.plan, hs.VARIANTS[v], xd, od, [h.out_struct(outs[v])], h.ws)
                  for v in variants}
        ev = {v: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for v in variants}
        per_variant = {v: [] for v in variants}

        ev_sort = {v: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for v in variants}
        sort_ms = {v: [] for v in variants}

        def step(record=False):
            for v in variants:
                outs[v]["cand_count"].zero_()
                if record:
                    ev[v][0].record(stream)
                hs.hs_graph_launch(graphs[v], stream)
                if record:
                    ev[v][1].record(stream)
                # the candidate list of the step, sorted by (variant, spectrum, z, bin) on the device
                hs.hs_sort_candidates(outs[v]["cand"], outs[v]["cand_count"], cand_tmp, h.ws, stream)
                if record:
                    ev_sort[v][1].record(stream)
            if record:
                stream.synchronize()
                for v in variants:
                    per_variant[v].append(ev[v][0].elapsed_time(ev[v][1]))
                    sort_ms[v].append(ev[v][1].elapsed_time(ev_sort[v][1]))

        for _ in range(max(args.warmup, 0)):
            step()
        torch.cuda.synchronize()
        assert h.sync_status(stream) in (hs.OK, hs.WARN_CAND_OVERFLOW)

        # per-variant launch durations, measured on the launching stream (separate pass, same work)
        for _ in range(max(2, min(args.steps, 5))):
            step(record=True)

        clocks = ClockSampler(local)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop()
        step_ms = reduce_max(e0.elapsed_time(e1) / args.steps, world)
        n_cands = {v: int(outs[v]["cand_count"].item()) for v in variants}

        # end to end through the public API: the pinned host batch streamed to the device in pieces
        # (each piece's copy overlapping the previous piece's sums), all variants, candidates back
        e2e = None
        if not args.no_e2e:
            cand_host = {v: torch.empty(cap * 16, dtype=torch.uint8, pin_memory=True) for v in variants}
            cnt_host = torch.empty(len(variants), dtype=torch.int64, pin_memory=True)
            od_stage = torch.empty(args.spectra + 1, dtype=torch.int64, device="cuda")
            structs = [h.out_struct(outs[v]) for v in variants]
            mask = sum(hs.VARIANTS[v] for v in variants)
            h2d_ms = _time_ms(torch, stream, lambda: xd.copy_(x_host, non_blocking=True), 1)
            k_e2e = max(1, min(args.steps, 3))
            d2h = 0
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(k_e2e):
                for v in variants:
                    outs[v]["cand_count"].zero_()
                hs.hs_sum_batched_host(h.plan, mask, x_host, offsets, xd, od_stage, structs, h.ws, n_chunks=8,
                                       stream=stream)
                for v in variants:
                    hs.hs_sort_candidates(outs[v]["cand"], outs[v]["cand_count"], cand_tmp, h.ws, stream)
                for i, v in enumerate(variants):
                    cnt_host[i : i + 1].copy_(outs[v]["cand_count"], non_blocking=True)
                stream.synchronize()
                d2h += 8 * len(variants)
                for i, v in enumerate(variants):
                    n = min(int(cnt_host[i]), cap)
                    cand_host[v][: n * 16].copy_(outs[v]["cand"][: n * 16], non_blocking=True)
                    d2h += n * 16
                stream.synchronize()
            t_e2e = reduce_max((time.perf_counter() - t0) / k_e2e, world)
            e2e = {"value": world * total * HMAX / t_e2e, "unit": UNIT, "h2d_bytes_per_step": total * 4,
                   "d2h_bytes_per_step": d2h // k_e2e, "ms_per_step": t_e2e * 1e3,
                   "api": "hs_sum_batched_host (8 pieces, copies overlapped with compute)",
                   "h2d_alone_ms": h2d_ms, "h2d_gbs": total * 4 / (h2d_ms / 1e3) / 1e9}

        # Eq. 1 with the input spans staged in shared memory by bulk copies (plan flag), on the same
        # batch after the timed region: its time next to the default gather path, and whether the
        # results agree bit for bit
        staged = None
        if "std" in variants and not args.no_secondary and not args.staged_spans:
            hst = hs.HarmonicSum(variants=hs.STD, hmax=HMAX, max_bins=1 << 22, threshold=THR, cand_capacity=cap,
                                 max_spectra=args.spectra, flags=hs.FLAG_STAGED_SPANS)
            mu, isig = hs.hs_noise_calibration("std", HMAX)
            hst.set_calibration("std", mu, isig)
            hs.hs_plan_set_tile_bins(hst.plan, "std", tuned["std"])
            ost = hst.new_outputs(total, "std", "cuda")

            def run_staged():
                ost["cand_count"].zero_()
                hs.hs_sum_batched(hst.plan, "std", xd, od, hst.out_struct(ost), hst.ws, 0, stream)

            st_ms = _time_ms(torch, stream, run_staged, 2)
            same = bool(torch.equal(ost["best_snr"], outs["std"]["best_snr"]) and
                        torch.equal(ost["best_h"], outs["std"]["best_h"]))
            staged = {"kernel": "hs::k_hs1d_eq1_staged (HS_FLAG_STAGED_SPANS)", "ms": st_ms,
                      "default_gather_ms": statistics.mean(per_variant["std"]), "bit_identical_to_default": same}
            del hst, ost
            torch.cuda.empty_cache()

        # the power-of-two stage search (H = 1, 2, 4, .., 32 only) on the same batch, after the timed
        # region: per-variant times next to the every-H search above
        pow2 = None
        if not args.no_secondary and not args.staged_spans:
            hp = hs.HarmonicSum(variants=0xF, hmax=HMAX, max_bins=1 << 22, threshold=THR, cand_capacity=cap,
                                max_spectra=args.spectra, flags=hs.FLAG_POW2_STAGES)
            op = hp.new_outputs(total, "greedy", "cuda")
            per_p2 = {}
            for v in variants:
                mu, isig = hs.hs_noise_calibration(v, HMAX)
                hp.set_calibration(v, mu, isig)
                hs.hs_plan_set_tile_bins(hp.plan, v, tuned[v])

                def run_p2(v=v):
                    op["cand_count"].zero_()
                    hs.hs_sum_batched(hp.plan, v, xd, od, hp.out_struct(op), hp.ws, 0, stream)

                per_p2[v] = _time_ms(torch, stream, run_p2, 2)
            pow2 = {"flag": "HS_FLAG_POW2_STAGES", "stages": [1, 2, 4, 8, 16, 32], "per_variant_ms": per_p2,
                    "ms_per_step": sum(per_p2.values()),
                    "speedup_vs_every_h": {v: statistics.mean(per_variant[v]) / per_p2[v] for v in variants}}
            del hp, op
            torch.cuda.empty_cache()

        # the step after the sums: sift the sorted Eq. 1 candidate list of the batch (harmonics and
        # neighbouring bins of stronger candidates dropped, k <= 8, 1.5 bins)
        sift = None
        if not args.no_secondary and "std" in variants:
            so = torch.empty(cap * 16, dtype=torch.uint8, device="cuda")
            so_count = torch.zeros(1, dtype=torch.int64, device="cuda")
            sift_ms = _time_ms(torch, stream, lambda: hs.hs_sift_candidates(outs["std"]["cand"], outs["std"]["cand_count"],
                                                                              so, so_count, cand_tmp, h.ws, stream=stream),
                               2)
            sift = {"variant": "std", "candidates_in": min(int(outs["std"]["cand_count"].item()), cap),
                    "kept": int(so_count.item()), "ms": sift_ms, "kmax": 8, "tol_bins": 1.5}
            del so, so_count

    value = world * total * HMAX / (step_ms / 1e3)
    peaks, peak_src = load_peaks()
    avg = {v: statistics.mean(per_variant[v]) for v in variants}
    dom = max(avg, key=avg.get)
    hbm_peak = peaks["hbm_gbs"]
    # FP32 add peak: 152 SMs x 128 FP32 lanes x the maximum SM clock (one add per lane per clock;
    # packed f32x2 adds do not raise it)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12

    def compulsory_bytes(v):
        return total * (4 + 4 + 1 + (4 if v == "greedy" else 0))

    # ncu figures per kernel (DRAM bytes and L2-to-L1 read bytes per bin, from a capture of the same
    # sources; null once a source file differs from the one captured)
    prof = {}
    try:
        tj = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        if tj.get("csrc_sha16") == csrc_sha16() and not args.staged_spans:
            prof = tj.get("kernels", {})
    except Exception:
        pass
    per_roof = {}
    for v in variants:
        gbs = compulsory_bytes(v) / (avg[v] / 1e3) / 1e9
        per_roof[v] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                       "kernel": prof.get(v, {}).get("kernel")}
        if v in prof:
            l2b = prof[v]["l2_read_bytes_per_bin"] * total
            # L2-to-L1 bytes of this launch (ncu bytes per bin x bins) over its time, and how busy ncu
            # found the L2 (lts__throughput, % of its peak) on a capture of the same sources
            pct = (prof[v].get("ncu_pct") or {}).get("l2_throughput_of_peak")
            per_roof[v]["l2"] = {"bytes_per_launch": l2b, "bytes_per_bin": prof[v]["l2_read_bytes_per_bin"],
                                 "achieved": l2b / (avg[v] / 1e3) / 1e9, "unit": "GB/s",
                                 "frac": None if pct is None else pct / 100.0,
                                 "peak_source": "ncu lts__throughput.avg.pct_of_peak_sustained_elapsed of the same "
                                                "kernel (32-spectrum capture of the same sources)"}
            per_roof[v]["traffic"] = prof[v]["dram_bytes_per_bin"] * total
            per_roof[v]["ncu_pct_of_peak"] = prof[v].get("ncu_pct")
    traffic = prof["std"]["dram_bytes_per_bin"] * total if "std" in prof else None
    binding = prof["std"].get("ncu_pct") if "std" in prof else None
    if dom == "std":
        # Eq. 1 performs 528 ordered FP32 adds per bin (sum_{H<=32} H); its HBM bytes are negligible
        tf = 528.0 * total / (avg[dom] / 1e3) / 1e12
        kname = "hs::k_hs1d_eq1_staged" if args.staged_spans else "hs::k_eq1_pairs_batched<float, false, false>"
        roof = {"bound": "alu", "kernel": kname, "achieved": tf, "peak": alu_peak,
                "peak_source": "derived: SMs x 128 FP32 lanes x max SM clock", "unit": "TFLOP/s",
                "frac": tf / alu_peak, "traffic": traffic, "algorithmic_flops_per_launch": 528.0 * total}
        if binding:  # what binds the kernel (ncu, same sources): L1 load wavefronts and issue
            roof["ncu_pct_of_peak"] = binding
    else:
        r = per_roof[dom]
        roof = {**r, "kernel": "hs::k_hs1d_zoned<%s>" % dom, "peak_source": peak_src,
                "traffic": r.get("traffic"), "algorithmic_bytes_per_launch": compulsory_bytes(dom)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, offsets, variants),
        "gpu_launches": args.steps * (2 + 36) * len(variants),
        "per_variant_ms": avg,
        "sort_ms": {v: statistics.mean(sort_ms[v]) for v in variants},
        "tile_bins": tuned,
        "per_variant_roofline": per_roof,
        "candidates": n_cands,
        "roofline": roof,
        "clocks": clk,
    }
    if e2e:
        line["e2e"] = e2e
    if staged:
        line["eq1_staged_spans"] = staged
    if pow2:
        line["pow2_stages"] = pow2
    if sift:
        line["sift"] = sift
    if not args.no_secondary:
        del graphs, outs, xd
        torch.cuda.empty_cache()
        with torch.cuda.stream(stream):
            line["secondary"] = secondary(torch, hs, stream, tiles=tuned, fdas_bins=args.fdas_bins)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        n_s = min(args.cpu_sample_spectra, args.spectra)
        bins, t = cpu_oracle_sample(offsets, x_host.numpy(), n_s, variants, cores)
        line["cpu_baseline"] = {"value": bins * HMAX / t, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "first %d spectra (%d bins), %s, FP32 oracle, each spectrum's bins split "
                                          "across %d cores" % (n_s, bins, "+".join(variants), cores),
                                "single_thread": cpu_single_thread(offsets, x_host.numpy(), variants)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
