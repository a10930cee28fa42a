"""Benchmark: fitted tracks/s of the GB300 Kalman-filter fitter on the barrel + endcap batch.

Workload (one "step" = one fit of the whole batch): 50 events of U{2000..20000} pions
(pT log-uniform 0.5-100 GeV, eta U(+-3), vertex z ~ N(0, 50 mm)) in a 10-layer barrel +
2 x 7-disk endcap silicon detector (0.3 mm modules), uniform 2 T along z, fitted under the
muon hypothesis in one launch; about 6.1e5 tracks and 7.0e6 measurements (synthetic data
standing in for the paper's ttbar events in the Open Data Detector). Inputs (~0.4 GB) are
larger than L2, so no flush is needed between steps.

Lines printed (rank 0): one JSON object. ``--impl reference`` times the CPU oracle instead.
"""

from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "fitted tracks/s on 1 GB300: mixed+learned vs plain FP64, at fixed pull error"
WORKLOAD = "barrel_endcap_50ev_uniform2T_pions"
WORKLOAD_MAP = "solenoid_map_100k_muons"

# Algorithmic FP64 flops per unit of the fit kernels, counted from the kernel source
# (add/sub/mul = 1, fma = 2, each div/sqrt/log/sin/cos = 1):
# (accepted RKN step, rejected step attempt, propagated measurement k >= 1, track).
# Two-filter: the step counters hold both passes; per measurement, the forward filter without
# the RTS terms (R = P J^T 180, smoother sums 210) plus the backward filter's prediction and
# update; per track, the backward start (update, reversal, direction) and the weighted mean
# with the seed (L D L^T 65, gain 225, parameters 52, covariance 800: 1,182).
# The barrel workload's field is uniform along z: the mixed path sets the theta row of the
# transport Jacobian to e_3 (theta is conserved) and copies instead of computing what it touches
# in R = P J^T (45 flops fewer per propagated measurement).
FLOPS = {
    "fp64": (493, 111, 1494, 330),
    # mixed: only the FP64 anchors, the Joseph update and the smoother count
    "mixed": (20, 8, 704, 330),
    "mixed_learned": (20, 8, 704, 330),
    # experimental FP32 covariance algebra: only the anchors and the smoothed sums stay FP64
    "mixed_fp32": (20, 8, 45, 30),
    "fp64_two_filter": (493, 111, 2209, 1837),
    "mixed_two_filter": (20, 8, 722, 1837),
}
# r-z field map: every attempt adds two stage positions and three bilinear lookups (FP64 in
# the plain path: 32 flops each incl. one square root and one division), every propagated
# measurement two more lookups; the mixed path looks up in FP32.
FLOPS_MAP = {
    "fp64": (619, 237, 1558, 330),
    "mixed": (20, 8, 749, 330),
    "mixed_learned": (20, 8, 749, 330),
    "mixed_fp32": (20, 8, 45, 30),
    "fp64_two_filter": (619, 237, 2337, 1837),
    "mixed_two_filter": (20, 8, 722, 1837),
}


# Hardware counts of one ncu capture of the fit kernel on a 20-event batch (279,450 tracks,
# 3,243,973 measurements; `--events 20 --shape ...`, one launch after three warm-ups): DRAM bytes
# (dram__bytes_read.sum + dram__bytes_write.sum), executed FP64 flops (2 dfma + dadd + dmul,
# thread-level) and executed FP32 flops (2 ffma + fadd + fmul + 4 ffma2 + 2 fadd2 + 2 fmul2), with
# the FLOPS model's count for the same launch. Traffic and FP32 flops grow with the tracks of a
# launch and are scaled by tracks to a full launch. Keyed by (workload, variant, register cap of
# the launched kernel); a kernel change voids the entries (profiles/ keeps the commands).
CAPTURES = {
    ("barrel", "mixed_learned", 64): {"tracks": 279450, "hits_after_first": 2964523, "attempts": 5100920,
        "rejected": 16960, "shape": "32,32,32,64", "dram_bytes": 8996654080,
        "fp64_exec": 2383301181, "fp64_model": 2281057572, "fp32_exec": 4787750993},
    ("barrel", "mixed", 64): {"tracks": 279450, "hits_after_first": 2964523, "attempts": 5014959,
        "rejected": 143605, "shape": "32,32,32,64", "dram_bytes": 9000243200,
        "fp64_exec": 2380095541, "fp64_model": 2277818612, "fp32_exec": 4703923835},
    ("barrel", "mixed_learned", 128): {"tracks": 279450, "hits_after_first": 2964523, "attempts": 5100793,
        "rejected": 18151, "shape": "128,4,32,128", "dram_bytes": 1410114048,
        "fp64_exec": 2377319935, "fp64_model": 2281040740, "fp32_exec": 4920394687},
    ("barrel", "mixed", 128): {"tracks": 279450, "hits_after_first": 2964523, "attempts": 5014959,
        "rejected": 143605, "shape": "64,8,32,128", "dram_bytes": 1368626432,
        "fp64_exec": 2374166495, "fp64_model": 2277818612, "fp32_exec": 4828531039},
    ("barrel", "fp64", 128): {"tracks": 279450, "hits_after_first": 2964523, "attempts": 5014958, "rejected": 143611,
                              "shape": "128,4,32,128", "dram_bytes": 2871720960,
                              "fp64_exec": 8183930686, "fp64_model": 6938730754, "fp32_exec": 71595040},
}


def fp32_peak_tflops(sm_mhz: float | None):
    """FP32 (CUDA-core) peak of GB300 from unit counts and clock: 152 SMs x 128 FP32 lanes x
    2 flop/clk (80.5 TFLOP/s at the 2070 MHz maximum clock)."""
    mhz = sm_mhz or 2070.0
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="auto", choices=["auto", "fp64", "mixed_fp32", "mixed", "mixed_learned",
                                                          "fp64_two_filter", "mixed_two_filter",
                                                          "mixed_fp32_two_filter", "fp64_all_states",
                                                          "mixed_all_states"])
    ap.add_argument("--events", type=int, default=50)
    ap.add_argument("--workload", default="barrel", choices=["barrel", "map"],
                    help="barrel: events in the barrel + endcap detector, uniform 2 T; map: 1e5 muons "
                         "in the solenoid field map")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch directly instead of replaying a CUDA graph")
    ap.add_argument("--no-autotune", action="store_true", help="the default launch shape instead of the tuned one")
    ap.add_argument("--shape", default=None,
                    help="fixed launch shape 'threads,blocks_per_sm,tracks_per_warp,registers[,lanes]' for every "
                         "variant (registers 128 or 64 apply to FP64 and mixed, 128 to mixed_fp32; lanes 1 or 4)")
    ap.add_argument("--proposer-quantile", type=float, default=0.05,
                    help="calibration quantile of the learned step proposer's output bias (0..1)")
    ap.add_argument("--tol", type=float, default=None,
                    help="RKN local error tolerance in mm for every variant (default: the library's 1e-4)")
    ap.add_argument("--tracks", type=int, default=0, help="fit only the first N tracks of the batch (default: all)")
    ap.add_argument("--muons", type=int, default=100_000, help="muons of the solenoid-map batch")
    ap.add_argument("--train-events", type=int, default=5,
                    help="barrel events of the step proposer's seed-disjoint training batch")
    ap.add_argument("--train-muons", type=int, default=100_000,
                    help="muons of the step proposer's training batch in the solenoid map")
    ap.add_argument("--max-records", type=int, default=0,
                    help="train the step proposer on at most N of its records (default: all)")
    ap.add_argument("--no-seeds", action="store_true",
                    help="skip the seed-estimation kernel, the chain from estimated seeds and track finding")
    ap.add_argument("--streams", action="store_true",
                    help="event-level concurrency: one launch per event on 1..16 CUDA streams against one "
                         "batched launch (one JSON line per configuration)")
    ap.add_argument("--sweep", action="store_true",
                    help="throughput sweep 1e3..1e7 tracks per launch in the solenoid map (one JSON line per point)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_seed(rank: int) -> int:
    # weak scaling: every rank fits its own batch of the same shape (seed offset by rank)
    return 2 + 1000 * rank


def make_workload(workload: str, events: int, rank: int, muons: int = 100_000, tracks: int = 0, **kw):
    """The timed batch: the barrel + endcap events in 2 T, or `muons` muons in the solenoid map;
    with `tracks`, its first `tracks` tracks."""
    if workload == "map":
        w = synth.solenoid_muon_workload(muons, seed=3 + shard_seed(rank), **kw)
    else:
        w = synth.barrel_workload(n_events=events, seed=shard_seed(rank), **kw)
    if tracks and tracks < w.tracks.n_tracks:
        w = synth.Workload(w.name, w.geometry, w.field, w.tracks.subset(np.arange(tracks)), w.mass)
    return w


def make_training_batch(args, rank: int):
    """Seed-disjoint tracks of the same kind for the step proposer's training records."""
    if args.workload == "map":
        return synth.solenoid_muon_workload(args.train_muons, seed=10_003 + shard_seed(rank)).tracks
    return synth.barrel_workload(n_events=args.train_events, seed=10_000 + shard_seed(rank)).tracks


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(tracks_per_rank: int, world_size: int, max_seconds: float) -> float:
    """Whole-job throughput: the tracks of all ranks over the slowest rank's time."""
    return world_size * tracks_per_rank / max_seconds


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def fp64_peak_tflops(sm_mhz: float | None):
    """FP64 (CUDA-core) peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM
    (4 flop/clk/SM; 1.26 TFLOP/s at the 2070 MHz maximum clock)."""
    mhz = sm_mhz or 2070.0
    return 152 * 4 * mhz * 1e6 / 1e12


def pull_stats(out, t):
    """Pulls of the fitted first-surface parameters against the simulated truth, and chi2/ndf."""
    par = out.par.cpu().numpy().T
    cov = out.cov.cpu().numpy().T
    status = out.status.cpu().numpy().view(np.uint32)
    ok = status == 0
    iu = np.triu_indices(5)
    diag = [int(np.where((iu[0] == k) & (iu[1] == k))[0][0]) for k in range(5)]
    sig = np.sqrt(cov[ok][:, diag])
    d = par[ok] - t.truth[ok]
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    pull = d / sig
    chi2 = out.chi2.cpu().numpy()[ok] / out.ndf.cpu().numpy()[ok]
    return {"sigma": [round(float(x), 4) for x in pull.std(0)], "mean": [round(float(x), 4) for x in pull.mean(0)],
            "chi2_ndf": round(float(chi2.mean()), 4)}


# Seed estimation, algorithmic bytes per track: its two offsets (4 bytes amortized), three
# measurements (loc0, loc1, v00, v01, v11, sid: 44 bytes each), 20 output doubles and a status.
SEED_BYTES_PER_TRACK = 4 + 3 * 44 + 20 * 8 + 4


def hbm_peak_gbs() -> tuple[float, str]:
    """The measured copy bandwidth of MEASURED_PEAKS.json, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def seed_stage(ctx, geo, fld, dev, t, opts, stream, steps: int, warmup: int, flush):
    """The seed-estimation kernel alone on the batch (HBM roofline), and the chain that starts
    from its seeds: estimated seeds -> fit -> refit with the fit's covariance inflated 100-fold,
    with the pulls of the refit against the truth."""
    import torch
    import paper_2505_22822_gb300 as tkf
    n = t.n_tracks
    device = dev.offsets.device
    out = tkf.SeedResult(torch.empty((5, n), dtype=torch.float64, device=device),
                         torch.empty((15, n), dtype=torch.float64, device=device),
                         torch.empty(n, dtype=torch.int32, device=device))

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            if flush is not None:
                flush.add_(1.0)
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)

    ms = timed(lambda: tkf.estimate_seeds(ctx, geo, fld, dev, out=out, stream=stream))
    status = out.status.cpu().numpy().view(np.uint32)
    par, cov = out.par.cpu().numpy().T, out.cov.cpu().numpy().T
    d = par - t.truth
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    iu = np.triu_indices(5)
    diag = [int(np.where((iu[0] == k) & (iu[1] == k))[0][0]) for k in range(5)]
    ok = status == 0
    seed_pulls = (d[ok] / np.sqrt(cov[ok][:, diag])).std(0)
    peak, peak_src = hbm_peak_gbs()
    achieved = SEED_BYTES_PER_TRACK * n / (ms * 1e-3) / 1e9
    seeds = {"kernel": "estimate_seeds_kernel", "ms": ms, "tracks_per_s": n / (ms * 1e-3),
             "status_ok": float(np.mean(ok)), "prior_pull_sigma": [round(float(x), 3) for x in seed_pulls],
             "median_rel_qop_error": float(np.median(np.abs(par[ok, 4] / t.truth[ok, 4] - 1.0))),
             "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                          "frac": achieved / peak, "peak_source": peak_src,
                          "algorithmic_bytes_per_track": SEED_BYTES_PER_TRACK}}
    # the chain, timed as one unit per step: estimate, fit, refit (direct launches)
    s1 = tkf.alloc_outputs(n, device, steps=False)
    s2 = tkf.alloc_outputs(n, device, steps=False)
    b1 = tkf.with_seeds(dev, out.par, out.cov)
    b2 = tkf.with_seeds(dev, s1.par, s1.cov)
    o1 = dataclasses.replace(opts, graph=False, kernel_events=None, step_mode=tkf.STEP_ADAPTIVE, mlp=None)
    o2 = dataclasses.replace(o1, seed_cov_scale=100.0)

    def chain():
        tkf.estimate_seeds(ctx, geo, fld, dev, out=out, stream=stream)
        tkf.fit(ctx, geo, fld, b1, o1, out=s1, stream=stream, steps=False)
        tkf.fit(ctx, geo, fld, b2, o2, out=s2, stream=stream, steps=False)

    cms = timed(chain)
    pulls = pull_stats(s2, t)
    chain_line = {"stages": "estimate_seeds -> fit -> refit (seed_cov_scale 100)",
                  "precision": {0: "fp64", 1: "mixed", 2: "mixed_fp32"}[opts.precision],
                  "ms_per_step": cms, "tracks_per_s": n / (cms * 1e-3),
                  "fit_status_ok": float(np.mean(s2.status.cpu().numpy() == 0)),
                  "pull_sigma": pulls["sigma"], "pull_mean": pulls["mean"], "chi2_ndf_mean": pulls["chi2_ndf"]}
    return seeds, chain_line


def ckf_stage(ctx, fld, w, stream, steps: int, warmup: int, events: int = 5, precision: int = 0):
    """Track finding on the first `events` events of the batch, all in one launch pair: seed
    estimation from triplets (the first measurements of each simulated track on three distinct
    layers, a stand-in for triplet seeding), then the combinatorial Kalman filter, each seed over
    its own event's measurements grouped by surface (FP64, or mixed: FP32 propagation and
    transport). Efficiency and purity against the simulation."""
    import torch
    import paper_2505_22822_gb300 as tkf
    g = w.geometry
    geo = tkf.Geometry.from_table(ctx, g.table).set_layers(g.layers, g.rings)
    dev = torch.device("cuda", torch.cuda.current_device())

    def T(x, dt=torch.float64):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dt).to(dev)

    t = w.tracks
    subs, mcs, offs, cols, bases, seed_ev = [], [], [], [[] for _ in range(5)], [], []
    base = 0
    for e in range(events):
        sub = t.subset(np.flatnonzero(t.event == e))
        mc = synth.measurement_container(sub, g.n)
        subs.append(sub)
        mcs.append(mc)
        offs.append(mc.offsets.astype(np.int64) + base)
        for k in range(5):
            cols[k].append(mc.meas[:, k])
        bases.append(base)
        seed_ev.append(np.full(sub.n_tracks, e))
        base += mc.meas.shape[0]
    # the same tracks, event by event in the order above
    allsub = t.subset(np.concatenate([np.flatnonzero(t.event == e) for e in range(events)]))
    s_off, s_meas, s_sid = synth.triplet_seed_hits(allsub, g)
    n_seeds = allsub.n_tracks
    seed_batch = tkf.Batch.from_arrays(s_off, s_meas, s_sid, np.zeros((n_seeds, 5)), np.zeros((n_seeds, 15))).to(dev)
    seed_sid = T(allsub.sid[allsub.offsets[:-1]].astype(np.int32), torch.int32)
    seed_event = T(np.concatenate(seed_ev).astype(np.int32), torch.int32)
    moff = T(np.stack(offs).astype(np.int32), torch.int32)
    mcols = [T(np.concatenate(c)) for c in cols]
    opts = tkf.Options(mass=w.mass, precision=precision)
    result = [None]

    def step():
        se = tkf.estimate_seeds(ctx, geo, fld, seed_batch, tkf.SEED_FIRST_THREE, stream=stream)
        result[0] = tkf.find_tracks(ctx, geo, fld, seed_sid, se.par, se.cov, moff, *mcols, opts, stream=stream,
                                    seed_event=seed_event)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    r = result[0]
    nm_all, em_all = r.n_entries.cpu().numpy(), r.entry_meas.cpu().numpy()
    eff, pur = [], []
    k = 0
    for sub, mc, b in zip(subs, mcs, bases):
        ntrue = np.diff(sub.offsets.astype(np.int64))
        for i in range(sub.n_tracks):
            ms_i = em_all[: nm_all[k], k]
            ms_i = ms_i[ms_i >= 0] - b
            good = int((mc.track[ms_i] == i).sum())
            eff.append(good / ntrue[i])
            pur.append(good / max(len(ms_i), 1))
            k += 1
    eff, pur = np.array(eff), np.array(pur)
    return {"events": events, "seeds": n_seeds, "ms_per_step": ms, "ms_per_event": ms / events,
            "seeds_per_s": n_seeds / (ms * 1e-3), "hit_efficiency": float(eff.mean()),
            "tracks_90pct_hits": float((eff >= 0.9).mean()), "purity": float(pur.mean()),
            "stages": "seed estimation (triplets) + combinatorial Kalman filter, beam 3, chi2 < 15, 2 holes; "
                      "all events in one launch each",
            "precision": {0: "fp64", 1: "mixed"}[precision], "launches_per_step": 2}


def cpu_baseline(w, max_seconds: float = 20.0):
    """The CPU oracle as it stands on this host's cores, on a bounded sample of the workload.
    Returns the baseline line, the sample's track indices and the oracle's results for them
    (which the accuracy table below compares the GPU variants with)."""
    import oracle
    t = w.tracks
    cores = os.cpu_count() or 1
    n_try = 4000
    rng = np.random.default_rng(0)
    while True:
        idx = np.sort(rng.choice(t.n_tracks, size=min(n_try, t.n_tracks), replace=False))
        sub = t.subset(idx)
        t0 = time.perf_counter()
        res = oracle.fit_tracks(w, tracks=sub, n_threads=cores)
        dt = time.perf_counter() - t0
        if dt > 0.25 * max_seconds or n_try >= t.n_tracks:
            break
        n_try = int(min(t.n_tracks, n_try * max(2.0, 0.3 * max_seconds / max(dt, 1e-3))))
    line = {"value": len(idx) / dt, "unit": "tracks/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(idx)} tracks drawn uniformly from the {t.n_tracks}-track batch, "
                      f"fit in {dt:.2f} s on {cores} threads"}
    # the same oracle on one thread, on the first sixteenth of the sample (on 16 cores about as
    # long as the threaded run)
    n1 = max(1, len(idx) // 16)
    t0 = time.perf_counter()
    oracle.fit_tracks(w, tracks=t.subset(idx[:n1]), n_threads=1)
    dt1 = time.perf_counter() - t0
    line["single_thread"] = {"value": n1 / dt1, "unit": "tracks/s",
                             "sample": f"{n1} tracks of the sample, {dt1:.2f} s on 1 thread"}
    # the oracle's two-filter smoother (backward filter and weighted mean) beside the GPU's
    # two-filter variants, on the first quarter of the sample
    n2 = max(1, len(idx) // 4)
    t0 = time.perf_counter()
    oracle.fit_tracks(w, opts=oracle.Options(mass=w.mass, smoother=1), tracks=t.subset(idx[:n2]), n_threads=cores)
    dt2 = time.perf_counter() - t0
    line["two_filter"] = {"value": n2 / dt2, "unit": "tracks/s", "cores": cores,
                          "sample": f"{n2} tracks of the sample, {dt2:.2f} s on {cores} threads"}
    return line, idx, res


def stage_oracles(w, max_seconds: float = 6.0, track_finding: bool = True):
    """The CPU oracle beside the seed-estimation and track-finding stages, each as it stands on
    that stage's own inputs: seed estimation (the oracle runs it on one thread) on the whole
    batch; track finding (FP64, all cores) on a sample of the
    first event's seeds over all of that event's measurements, with the stage's options (beam 3,
    chi2 < 15, 2 holes, 24 entries)."""
    import oracle
    t, g = w.tracks, w.geometry
    cores = os.cpu_count() or 1
    fo = oracle.field_from(w.field)
    rng = np.random.default_rng(1)
    t0 = time.perf_counter()
    oracle.estimate_seeds(g.table, fo, t.offsets, t.meas, t.sid)
    dt = time.perf_counter() - t0
    seeds = {"value": t.n_tracks / dt, "unit": "tracks/s", "cores": 1, "kind": "oracle",
             "sample": f"the whole batch, {t.n_tracks} tracks, {dt:.2f} s on 1 thread"}
    if not track_finding:
        return seeds, None
    ev = t.subset(np.flatnonzero(t.event == 0))
    mc = synth.measurement_container(ev, g.n)
    s_off, s_meas, s_sid = synth.triplet_seed_hits(ev, g)
    par, cov, _ = oracle.estimate_seeds(g.table, fo, s_off, s_meas, s_sid, first_three=True)
    seed_sid = ev.sid[ev.offsets[:-1]].astype(np.uint32)
    opts = oracle.Options(mass=w.mass)
    k = min(ev.n_tracks, 500)
    while True:
        sel = np.sort(rng.choice(ev.n_tracks, size=k, replace=False))
        t0 = time.perf_counter()
        oracle.find_tracks(g.table, fo, opts, g.layers, g.rings, mc.offsets, mc.meas, seed_sid[sel], par[sel],
                           cov[sel], n_threads=cores)
        dt = time.perf_counter() - t0
        if dt > 0.25 * max_seconds or k >= ev.n_tracks:
            break
        k = int(min(ev.n_tracks, k * max(2.0, 0.3 * max_seconds / max(dt, 1e-3))))
    ckf = {"value": k / dt, "unit": "seeds/s", "cores": cores, "kind": "oracle", "precision": "fp64",
           "sample": f"{k} of the first event's {ev.n_tracks} seeds over all its measurements, "
                     f"{dt:.2f} s on {cores} threads"}
    return seeds, ckf


PARAMS = ("l0", "l1", "phi", "theta", "qop")
MATCH_TOLS = (1e-4, 1e-3, 1e-2, 5e-2)


def accuracy_vs_oracle(g: dict, o, idx) -> dict:
    """One variant's fitted tracks (host arrays, track-major) against the FP64 oracle on the
    sample `idx`: for each parameter the largest and the 99th-percentile |dp_i| / sigma_i (sigma
    from the oracle's covariance; phi wrapped), the largest covariance error relative to
    sqrt(C_ii C_jj), the largest relative chi2 difference, and the paper's Table-1 matching
    ratios: the fraction of tracks with the oracle's status whose five parameters all lie within
    the relative tolerance |dp_i| <= r |p_i| (r = 0.01 %, 0.1 %, 1 %, 5 %)."""
    st_g, st_o = g["status"][idx], o.status
    same_status = st_g == st_o
    fitted = same_status & ((st_o & 0x39F) == 0)
    iu = np.triu_indices(5)
    C = np.zeros((len(idx), 5, 5))
    C[:, iu[0], iu[1]] = o.cov
    C[:, iu[1], iu[0]] = o.cov
    sig = np.sqrt(np.abs(np.einsum("nii->ni", C)))
    dp = g["par"][idx] - o.par
    dp[:, 2] = (dp[:, 2] + np.pi) % (2 * np.pi) - np.pi
    ds = np.abs(dp[fitted]) / sig[fitted]
    Cg = np.zeros_like(C)
    Cg[:, iu[0], iu[1]] = g["cov"][idx]
    Cg[:, iu[1], iu[0]] = g["cov"][idx]
    scale = np.einsum("ni,nj->nij", sig, sig)
    dc = (np.abs(Cg - C) / scale)[fitted].reshape(int(fitted.sum()), -1)
    dchi = np.abs(g["chi2"][idx] - o.chi2)[fitted] / np.maximum(np.abs(o.chi2[fitted]), 1.0)
    rel = np.abs(dp) / np.maximum(np.abs(o.par), 1e-300)
    out = {"tracks": int(len(idx)), "same_status": float(np.mean(same_status)),
           "dp_over_sigma_max": {k: float(ds[:, i].max(initial=0)) for i, k in enumerate(PARAMS)},
           "dp_over_sigma_p99": {k: float(np.quantile(ds[:, i], 0.99)) if len(ds) else 0.0
                                 for i, k in enumerate(PARAMS)},
           "cov_rel_max": float(dc.max(initial=0)), "chi2_rel_max": float(dchi.max(initial=0)),
           "match_ratio": {f"{100 * r:g}%": float(np.mean(fitted & np.all(rel <= r, axis=1)))
                           for r in MATCH_TOLS}}
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle  # noqa: F401
    w = make_workload(args.workload, args.events, 0)
    t = w.tracks
    cores = os.cpu_count() or 1
    # each step fits a bounded sample sized to keep the whole run within minutes
    per_step = min(t.n_tracks, 20000)
    rng = np.random.default_rng(1)
    subs = [t.subset(np.sort(rng.choice(t.n_tracks, per_step, replace=False)))
            for _ in range(min(args.steps, 4))]
    import oracle as orc
    for i in range(args.warmup):
        orc.fit_tracks(w, tracks=subs[i % len(subs)], n_threads=cores)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        orc.fit_tracks(w, tracks=subs[i % len(subs)], n_threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "tracks/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD_MAP if args.workload == "map" else WORKLOAD,
                                        "tracks_per_step": per_step,
                                        "sample": "bounded sample of the batch per step",
                                        "l2": "inputs on the host"},
        "cpu_baseline": {"value": value, "unit": "tracks/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} tracks per step from the {t.n_tracks}-track batch"},
        "e2e": {"value": value, "unit": "tracks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def setup_tune_cache() -> str:
    """Autotuner cache file (TKF_AUTOTUNE_CACHE, else a fresh temporary file); read back to
    report the tuned block shapes. Set before the first context is created."""
    path = os.environ.get("TKF_AUTOTUNE_CACHE")
    if not path:
        fd, path = tempfile.mkstemp(prefix="tkf_tune_", suffix=".json")
        os.close(fd)
        os.unlink(path)
        os.environ["TKF_AUTOTUNE_CACHE"] = path
    return path


def tuned_shape(path: str, variant: str, n_tracks: int, field: str, disabled: bool):
    """[threads, blocks per SM, tracks per warp, registers, lanes a track] the autotuner chose
    for this class."""
    two_filter = variant.endswith("_two_filter")
    all_states = variant.endswith("_all_states")
    base = variant.replace("_two_filter", "").replace("_all_states", "")
    if disabled:
        return ([128, 2, 32, 255, 1] if two_filter or all_states or base in ("fp64", "mixed_fp32")
                else [128, 4, 32, 128, 1])
    prec = base if base in ("fp64", "mixed_fp32") else "mixed"
    mode = "learned" if variant.endswith("learned") else ("states" if all_states else "adaptive")
    prefix = f"{prec}{'_two_filter' if two_filter else ''}.{mode}.{field}.n{int(n_tracks).bit_length() - 1}."
    try:
        with open(path) as fh:
            table = json.load(fh)
    except (OSError, ValueError):
        return None
    return next((v for k, v in table.items() if k.startswith(prefix)), None)


def _prefix_batch(b, n: int):
    """The first n tracks of a device batch (measurement arrays shared)."""
    import paper_2505_22822_gb300 as tkf
    return tkf.Batch(b.offsets[:n + 1].clone(), b.loc0, b.loc1, b.v00, b.v01, b.v11, b.sid,
                     b.seed_par[:, :n].contiguous(), b.seed_cov[:, :n].contiguous())


def _tile_batch(b, k: int):
    """k copies of a device batch back to back (offsets shifted)."""
    import torch
    import paper_2505_22822_gb300 as tkf
    m = b.n_meas
    off = b.offsets.to(torch.int64)
    offs = torch.cat([off[:-1] + j * m for j in range(k)] + [off[-1:] + (k - 1) * m]).to(torch.int32)
    rep = [getattr(b, f).repeat(k) for f in ("loc0", "loc1", "v00", "v01", "v11", "sid")]
    return tkf.Batch(offs, *rep, b.seed_par.repeat(1, k), b.seed_cov.repeat(1, k))


def run_sweep(args, local: int, rank: int, tune_file: str):
    """Tracks/s against tracks per launch (1e3..1e7) in the barrel + endcap detector and the
    solenoid field map, events of log-uniform 1e3..1e5 pions batched per launch, for plain
    FP64, mixed and mixed + learned, each replayed from a CUDA graph with the autotuned block
    shape (and, up to 1e5 tracks, also launched directly). 1e6 distinct tracks are simulated;
    the 1e7 point fits ten copies of them. One JSON line per point."""
    import torch
    import paper_2505_22822_gb300 as tkf
    from paper_2505_22822_gb300 import learn
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    g, f = synth.barrel_endcap_geometry(), synth.solenoid_map()
    pp = synth.barrel_params(step=5.0)
    t0 = time.perf_counter()
    counts = synth.event_counts_loguniform(500 + shard_seed(rank), 10 ** 6)
    t = synth.simulate(g, f, pp, 500 + shard_seed(rank), counts)
    tw = synth.simulate(g, f, pp, 20_000 + shard_seed(rank), synth.event_counts_loguniform(20_000, 200_000))
    gen_s = time.perf_counter() - t0
    ctx = tkf.Context(local)
    geo, fld = tkf.Geometry.from_table(ctx, g.table), tkf.Field.from_desc(ctx, f)
    full = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to(dev)
    tb = tkf.Batch.from_arrays(tw.offsets, tw.meas, tw.sid, tw.seed_par, tw.seed_cov).to(dev)
    proposer, info = learn.build_proposer(ctx, geo, fld, tb, tkf.MIXED, mass=synth.MUON_MASS)
    del tb
    print(json.dumps({"sweep": "setup", "workload": "barrel_endcap_solenoid_map_pions_loguniform_events",
                      "events": int(len(counts)), "tracks": int(t.n_tracks), "measurements": int(t.n_hits),
                      "generate_s": round(gen_s, 1), "proposer_records": info["records"]}), flush=True)
    sizes = [10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7]
    for n in sizes:
        k = -(-n // full.n_tracks)
        b = _prefix_batch(_tile_batch(full, k) if k > 1 else full, n)
        out = tkf.alloc_outputs(n, dev, steps=True)
        for variant in ("fp64", "mixed", "mixed_learned"):
            # (graph, autotune, lanes a track): tuned (the tuner also tries 4 lanes a track below
            # ~4e4 tracks), direct launches, the default shape, and 4 lanes a track forced
            policies = ([(True, True, 0), (False, True, 0), (True, False, 0), (True, False, 4)] if n <= 10 ** 5
                        else [(True, True, 0)])
            for graph, autotune, lanes in policies:
                opts = tkf.Options(precision=tkf.FP64 if variant == "fp64" else tkf.MIXED, mass=synth.MUON_MASS,
                                   graph=graph, autotune=autotune, lanes_per_track=lanes)
                if variant.endswith("learned"):
                    opts.step_mode, opts.mlp = tkf.STEP_LEARNED, proposer
                for _ in range(max(3, args.warmup)):
                    tkf.fit(ctx, geo, fld, b, opts, out=out, stream=stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tkf.fit(ctx, geo, fld, b, opts, out=out, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                reps = int(min(500, max(5, 0.5e3 / max(e0.elapsed_time(e1), 1e-3))))
                with ClockSampler(local) as clk:
                    e0.record(stream)
                    for _ in range(reps):
                        tkf.fit(ctx, geo, fld, b, opts, out=out, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                status = out.status.cpu().numpy().view(np.uint32)
                shape = tuned_shape(tune_file, variant, n, "grid", not autotune)
                if lanes == 4:
                    shape = [128, 2, 8, 255, 4]
                print(json.dumps({"sweep": "point", "tracks_per_launch": n, "variant": variant, "cuda_graph": graph,
                                  "autotune": autotune, "lanes_per_track": lanes, "tracks_per_s": n / (ms * 1e-3),
                                  "ms_per_launch": ms, "reps": reps, "launch_shape": shape,
                                  "fit_status_ok": float(np.mean(status == 0)),
                                  "clocks": clk.summary()}), flush=True)
        del b, out


def run_streams(args, local: int, rank: int):
    """Event-level concurrency against one batched launch: the bench batch's events fitted one
    launch per event on S CUDA streams (S = 1, 2, 4, 8, 16; one library context per stream,
    since a context's scratch serves one launch at a time; events dealt round-robin), and the
    whole batch in one launch. Mixed precision, autotuned shapes, direct launches. One JSON line
    per configuration."""
    import torch
    import paper_2505_22822_gb300 as tkf
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    w = make_workload("barrel", args.events, rank)
    t = w.tracks
    host = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov)
    full = host.to(dev)
    ev = t.event.astype(np.int64)
    starts = np.flatnonzero(np.r_[True, ev[1:] != ev[:-1]])
    bounds = list(zip(starts, np.r_[starts[1:], t.n_tracks]))
    opts = tkf.Options(precision=tkf.MIXED, mass=w.mass, autotune=True)

    def event_batch(t0, t1):
        return tkf.Batch(full.offsets[t0:t1 + 1].clone(), full.loc0, full.loc1, full.v00, full.v01, full.v11,
                         full.sid, full.seed_par[:, t0:t1].contiguous(), full.seed_cov[:, t0:t1].contiguous())

    events = [event_batch(t0, t1) for t0, t1 in bounds]
    outs = [tkf.alloc_outputs(t1 - t0, dev, steps=False) for t0, t1 in bounds]
    L2_BYTES = 129e6
    flush = torch.zeros(int(2 * L2_BYTES) // 4, dtype=torch.float32, device=dev)
    results = []
    for S in (1, 2, 4, 8, 16):
        ctxs = [tkf.Context(local) for _ in range(S)]
        hs = [(tkf.Geometry.from_table(c, w.geometry.table), tkf.Field.from_desc(c, w.field)) for c in ctxs]
        streams = [torch.cuda.Stream() for _ in range(S)]

        def step():
            for e, (b, o) in enumerate(zip(events, outs)):
                j = e % S
                tkf.fit(ctxs[j], hs[j][0], hs[j][1], b, opts, out=o, stream=streams[j])

        for _ in range(max(3, args.warmup)):  # the first tunes every size class per context
            step()
        torch.cuda.synchronize()
        main_s = torch.cuda.current_stream()
        times = []
        for _ in range(args.steps):
            flush.add_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main_s)
            for s in streams:
                s.wait_event(e0)
            step()
            for s in streams:
                done = torch.cuda.Event()
                done.record(s)
                main_s.wait_event(done)
            e1.record(main_s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.mean(times)
        line = {"streams_experiment": "per-event launches", "streams": S, "events": len(bounds),
                "tracks": int(t.n_tracks), "ms_per_step": ms, "tracks_per_s": t.n_tracks / (ms * 1e-3),
                "launches_per_step": 3 * len(bounds)}
        results.append(line)
        print(json.dumps(line), flush=True)
        del ctxs, hs
    # the whole batch in one launch (replayed from a CUDA graph, as the main bench)
    ctx = tkf.Context(local)
    geo, fld = tkf.Geometry.from_table(ctx, w.geometry.table), tkf.Field.from_desc(ctx, w.field)
    s = torch.cuda.Stream()
    out = tkf.alloc_outputs(t.n_tracks, dev, steps=False)
    gopts = dataclasses.replace(opts, graph=True)
    for _ in range(max(3, args.warmup)):
        tkf.fit(ctx, geo, fld, full, gopts, out=out, stream=s)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.add_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        tkf.fit(ctx, geo, fld, full, gopts, out=out, stream=s)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    print(json.dumps({"streams_experiment": "one batched launch", "streams": 1, "events": len(bounds),
                      "tracks": int(t.n_tracks), "ms_per_step": ms, "tracks_per_s": t.n_tracks / (ms * 1e-3),
                      "launches_per_step": 3}), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import paper_2505_22822_gb300 as tkf

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    tune_file = setup_tune_cache()
    if args.sweep:
        run_sweep(args, local, rank, tune_file)
        return
    if args.streams:
        run_streams(args, local, rank)
        return
    w = make_workload(args.workload, args.events, rank, muons=args.muons, tracks=args.tracks)
    t = w.tracks
    n_tracks, n_meas = t.n_tracks, t.n_hits
    ctx = tkf.Context(local)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    host = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov)
    dev = host.to(f"cuda:{local}")
    # the headline is the last: mixed + learned; mixed_fp32 is the experimental FP32 covariance algebra
    # *_two_filter: the optimal (two-filter) smoother instead of RTS
    # *_all_states: every entry's smoothed state too (backward RTS pass over stored states)
    variants = (["fp64", "fp64_two_filter", "fp64_all_states", "mixed_fp32", "mixed_two_filter", "mixed_all_states",
                 "mixed", "mixed_learned"]
                if args.variant == "auto" else [args.variant])
    # a side stream: CUDA graphs cannot be captured on the legacy default stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    hits_k1 = int((np.diff(t.offsets.astype(np.int64)) - 1).clip(min=0).sum())
    proposer, learn_info = None, None
    if any(v.endswith("learned") for v in variants):
        # the step proposer is trained before timing, on records of seed-disjoint tracks
        from paper_2505_22822_gb300 import learn
        tt = make_training_batch(args, rank)
        tb = tkf.Batch.from_arrays(tt.offsets, tt.meas, tt.sid, tt.seed_par, tt.seed_cov).to(f"cuda:{local}")
        t0 = time.perf_counter()
        proposer, info = learn.build_proposer(ctx, geo, fld, tb, tkf.MIXED, mass=w.mass, tol=args.tol,
                                              quantile=args.proposer_quantile,
                                              max_records=args.max_records or None)
        learn_info = {"records": info["records"], "final_loss": round(info["epoch_loss"][-1], 4),
                      "bias_shift": round(info["bias_shift"], 4), "train_s": round(time.perf_counter() - t0, 2),
                      "tracks": tt.n_tracks}
    results = {}
    L2_BYTES = 129e6
    flush = (torch.zeros(int(2 * L2_BYTES) // 4, dtype=torch.float32, device=f"cuda:{local}")
             if host.nbytes() < 2 * L2_BYTES else None)
    for variant in variants:
        two_filter = variant.endswith("_two_filter")
        all_states = variant.endswith("_all_states")
        base = variant.replace("_two_filter", "").replace("_all_states", "")
        opts = tkf.Options(precision={"fp64": tkf.FP64, "mixed_fp32": tkf.MIXED_FP32}.get(base, tkf.MIXED),
                           mass=w.mass, smoother=tkf.SMOOTHER_TWO_FILTER if two_filter else tkf.SMOOTHER_RTS,
                           graph=not args.no_graph, autotune=not args.no_autotune and args.shape is None)
        if args.shape:
            th, bps, tpw, regs, *lanes = (int(x) for x in args.shape.split(","))
            opts.block_threads, opts.blocks_per_sm, opts.tracks_per_warp = th, bps, tpw
            opts.max_registers = 255 if base == "mixed_fp32" and (two_filter or regs == 64) else regs
            opts.lanes_per_track = lanes[0] if lanes and base != "mixed_fp32" and not two_filter else 0
        if args.tol is not None:
            opts.tol = args.tol
        if variant.endswith("learned"):
            opts.step_mode, opts.mlp = tkf.STEP_LEARNED, proposer
        out = tkf.alloc_outputs(n_tracks, dev.offsets.device, steps=True, states_meas=n_meas if all_states else None)
        # warm-up: the first call tunes the block shape, the second captures the graph
        for _ in range(args.warmup):
            tkf.fit(ctx, geo, fld, dev, opts, out=out, stream=stream)
        torch.cuda.synchronize()
        # work counted from this batch's step counters (identical every step)
        st = out.steps.cpu().numpy().astype(np.int64)
        attempts, rejected = int(st[0].sum()), int(st[1].sum())
        status = out.status.cpu().numpy().view(np.uint32)
        barrier()
        torch.cuda.synchronize()
        if flush is None:
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with ClockSampler(local) as clk:
                ev0.record(stream)
                for _ in range(args.steps):
                    tkf.fit(ctx, geo, fld, dev, opts, out=out, stream=stream)
                ev1.record(stream)
                torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / args.steps
        else:
            # inputs smaller than L2: overwrite a buffer larger than L2 before every step, and
            # time each step alone
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            with ClockSampler(local) as clk:
                for e0, e1 in evs:
                    flush.add_(1.0)
                    e0.record(stream)
                    tkf.fit(ctx, geo, fld, dev, opts, out=out, stream=stream)
                    e1.record(stream)
                torch.cuda.synchronize()
            ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / args.steps
        barrier()
        # the fit kernel alone: the library records a pair of events around it (steps timed one
        # by one, after the timed region)
        kev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        for ev in kev:
            ev.record(stream)  # creates the events
        kopts = dataclasses.replace(opts, kernel_events=kev)
        kms = []
        for _ in range(args.steps):
            if flush is not None:
                flush.add_(1.0)
            tkf.fit(ctx, geo, fld, dev, kopts, out=out, stream=stream)
            kev[1].synchronize()
            kms.append(kev[0].elapsed_time(kev[1]))
        kernel_ms = statistics.mean(kms)
        ms_max = max_over_ranks(ms, dist, f"cuda:{local}")
        host_out = {"par": out.par.cpu().numpy().T.copy(), "cov": out.cov.cpu().numpy().T.copy(),
                    "chi2": out.chi2.cpu().numpy(), "status": out.status.cpu().numpy().view(np.uint32)}
        results[variant] = {"ms": ms, "ms_max": ms_max, "kernel_ms": kernel_ms, "clocks": clk.summary(), "opts": opts,
                            "host_out": host_out,
                            "shape": ([opts.block_threads, opts.blocks_per_sm, opts.tracks_per_warp, opts.max_registers,
                                       opts.lanes_per_track or 1]
                                      if args.shape else
                                      tuned_shape(tune_file, variant, n_tracks, "grid" if args.workload == "map" else "uz",
                                                  args.no_autotune)),
                            "attempts": attempts, "rejected": rejected, "status_ok": float(np.mean(status == 0)),
                            "pulls": pull_stats(out, t)}
    head = variants[-1]
    opts = results[head]["opts"]
    seeds = chain = ckf = ckf_mixed = None
    if not args.no_seeds:
        copts = results["mixed"]["opts"] if "mixed" in results else opts
        seeds, chain = seed_stage(ctx, geo, fld, dev, t, copts, stream, args.steps, args.warmup, flush)
        if args.workload == "barrel":
            ckf = ckf_stage(ctx, fld, w, stream, max(1, args.steps // 2), 1)
            ckf_mixed = ckf_stage(ctx, fld, w, stream, max(1, args.steps // 2), 1, precision=tkf.MIXED)
    ms, ms_max, clocks = results[head]["ms"], results[head]["ms_max"], results[head]["clocks"]
    for k, v in results.items():
        counts = (FLOPS_MAP if args.workload == "map" else FLOPS).get(k)  # no count for the two-filter form
        if counts is None:
            v["flops"] = None
            continue
        fa, fr, fh, ft = counts
        v["flops"] = fa * (v["attempts"] - v["rejected"]) + fr * v["rejected"] + fh * hits_k1 + ft * n_tracks

    # end to end through the host entry point: pinned host inputs -> fit -> host outputs
    e2e = None
    if not args.no_e2e:
        pinned = host.to("cpu", pin=True)
        hout = tkf.Result(torch.empty((5, n_tracks), dtype=torch.float64).pin_memory(),
                          torch.empty((15, n_tracks), dtype=torch.float64).pin_memory(),
                          torch.empty(n_tracks, dtype=torch.float64).pin_memory(),
                          torch.empty(n_tracks, dtype=torch.int32).pin_memory(),
                          torch.empty(n_tracks, dtype=torch.int32).pin_memory(), None)
        for _ in range(max(1, args.warmup)):
            tkf.fit_host(ctx, geo, fld, pinned, opts, out=hout, stream=stream)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tkf.fit_host(ctx, geo, fld, pinned, opts, out=hout, stream=stream)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, f"cuda:{local}")
        h2d = host.nbytes()
        d2h = n_tracks * (5 * 8 + 15 * 8 + 8 + 4 + 4)
        e2e = {"value": aggregate_throughput(n_tracks, ws, e2e_s), "unit": "tracks/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "variant": head}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak = fp64_peak_tflops(None)
    # the fit kernel's own duration, from the events the library records around it
    hv = results[head]
    head_shape = hv["shape"] or [None] * 5
    # the captured kernel: one lane a track (a group shape is another kernel)
    cap_key = (args.workload, head, head_shape[3]) if (head_shape[4:] or [1])[0] == 1 else None
    cap = CAPTURES.get(cap_key)
    # no FP64 flop count for the two-filter variants: their roofline stays null
    kernel_s = hv["kernel_ms"] * 1e-3
    achieved = hv["flops"] / kernel_s / 1e12 if hv["flops"] is not None else None
    algo_bytes = host.nbytes() + n_tracks * (5 * 8 + 15 * 8 + 8 + 4 + 4 + 8)
    roof = {"bound": "alu", "kernel": f"fit_persistent_kernel<{head}>", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if achieved is not None else None,
            "traffic": cap["dram_bytes"] / cap["tracks"] * n_tracks if cap else None,
            "traffic_note": ((f"ncu capture of {cap['tracks']} tracks (20 events, shape {cap['shape']}), scaled by "
                              "tracks" if cap else "no capture for this kernel variant") +
                             f"; algorithmic bytes (inputs + outputs) per launch: {algo_bytes}; above them: "
                             "local-memory spill traffic of the register-capped kernel"),
            "fp64_flop_per_launch": hv["flops"],
            "fp64_executed_over_algorithmic": cap["fp64_exec"] / cap["fp64_model"] if cap else None,
            "note": "FP64 CUDA-core pipe (the bound of both variants); peak derived from "
                    "152 SMs x 4 flop/clk x 2070 MHz; 1.20 TFLOP/s measured by an FMA probe"}
    if cap:
        f32 = cap["fp32_exec"] / cap["tracks"] * n_tracks
        p32 = fp32_peak_tflops(None)
        roof["fp32"] = {"achieved": f32 / kernel_s / 1e12, "peak": p32, "unit": "TFLOP/s",
                        "frac": f32 / kernel_s / 1e12 / p32, "flop_per_launch": f32,
                        "note": "executed FP32 flops of the ncu capture scaled by tracks; peak derived from "
                                "152 SMs x 128 lanes x 2 flop/clk x 2070 MHz"}
    line = {
        "metric": METRIC,
        "value": aggregate_throughput(n_tracks, ws, ms_max * 1e-3),
        "unit": "tracks/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32+f64 (+bf16 weights)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_MAP if args.workload == "map" else WORKLOAD, "variant": head,
                   "tracks_per_gpu": n_tracks, "measurements_per_gpu": n_meas,
                   "events_per_gpu": None if args.workload == "map" else args.events,
                   "field": ("solenoid r-z map, 241 x 1401 nodes, FP32" if args.workload == "map"
                             else "uniform 2 T along z"),
                   "l2": (f"inputs {host.nbytes() / 1e9:.2f} GB > L2, no flush" if flush is None else
                          f"inputs {host.nbytes() / 1e9:.3f} GB: L2 flushed (258 MB write) before every step, "
                          "steps timed one by one"),
                   "step_mode": "learned starting step + adaptive" if head.endswith("learned") else "adaptive",
                   "tol_mm": args.tol if args.tol is not None else 1e-4},
        # per step: key, scan and scatter kernels of the ordering, the proposal pre-pass
        # (learned), the persistent fit (plus one memset node)
        "gpu_launches": (5 if head.endswith("learned") else 4) * args.steps,
        "launch_policy": {"cuda_graph": not args.no_graph, "autotune": not args.no_autotune and args.shape is None,
                          "launch_shape": {k: v["shape"] for k, v in results.items()}},
        "roofline": roof,
        "clocks": clocks,
        "variants": {k: {"tracks_per_s": aggregate_throughput(n_tracks, ws, v["ms_max"] * 1e-3),
                         "ms_per_step": v["ms_max"],
                         "step_attempts": v["attempts"], "rejected": v["rejected"],
                         "fit_status_ok": v["status_ok"], "pull_sigma": v["pulls"]["sigma"],
                         "fit_kernel_ms": v["kernel_ms"], "fit_kernel_share": v["kernel_ms"] / v["ms"],
                         "fp64_tflops": (v["flops"] / (v["kernel_ms"] * 1e-3) / 1e12 if v["flops"] is not None
                                         else None),
                         "pull_mean": v["pulls"]["mean"], "chi2_ndf_mean": v["pulls"]["chi2_ndf"]}
                     for k, v in results.items()},
    }
    if "fp64" in results:
        line["speedup_vs_fp64"] = {k: results["fp64"]["ms_max"] / v["ms_max"] for k, v in results.items()
                                   if k != "fp64"}
    if learn_info:
        line["learned_proposer"] = learn_info
    if seeds:
        line["seed_estimation"] = seeds
        line["chain_from_estimated_seeds"] = chain
    if ckf:
        line["track_finding"] = ckf
        line["track_finding_mixed"] = ckf_mixed
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline:
        line["cpu_baseline"], idx, ores = cpu_baseline(w)
        if seeds:
            seeds["cpu_oracle"], ckf_oracle = stage_oracles(w, track_finding=ckf is not None)
            if ckf is not None:
                ckf["cpu_oracle"] = ckf_oracle
        # each variant's error against the FP64 oracle on the baseline's sample (the paper's
        # CPU-GPU agreement study, Sec. 3.1, Table 1); the two-filter variants against the
        # oracle's two-filter smoother
        ores2 = None
        if any(k.endswith("_two_filter") for k in results):
            import oracle
            ores2 = oracle.fit_tracks(w, oracle.Options(mass=w.mass, smoother=1), tracks=t.subset(idx),
                                      n_threads=os.cpu_count() or 1)
        line["accuracy_vs_oracle"] = {k: accuracy_vs_oracle(v["host_out"], ores2 if k.endswith("_two_filter") else ores,
                                                            idx)
                                      for k, v in results.items()}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
