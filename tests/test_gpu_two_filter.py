"""GPU parity of the two-filter smoother (tkf_fit_options.smoother = TKF_SMOOTHER_TWO_FILTER:
forward filter, backward filter of the reversed particle, weighted mean with the seed) against
the oracle's two-filter smoother: FP64 within 1e-10 in the parity metric, the mixed path within
1e-3 sigma and chi2 within 1e-3, every precision on edge tracks and holes; and the FP32
question (covariance algebra in FP32 end to end) measured against the FP64 oracle."""

import numpy as np
import pytest

import oracle
import paper_2505_22822_gb300 as tkf
import synth
from oracle import mlp
from tests import parity
from tests.test_gpu_parity import TOL64, _dp_over_sigma, _edge_tracks, check, check_mixed, run_gpu, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_TOL_SIGMA, MIXED_TOL_CHI2 = 1e-3, 1e-3


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return tkf.Context(0)


WORKLOADS = {
    "telescope": lambda: synth.telescope_workload(2000, seed=0),
    "barrel": lambda: synth.barrel_workload(n_events=2, lo=1500, hi=2500, seed=2),
    "map": lambda: synth.solenoid_muon_workload(3000, seed=3),
    "map_holes": lambda: synth.solenoid_muon_workload(2000, seed=11, p_hole=0.2),
}


def _opts(w, precision=tkf.FP64, **kw):
    return tkf.Options(precision=precision, mass=w.mass, smoother=tkf.SMOOTHER_TWO_FILTER, **kw)


def _oopts(w, **kw):
    return oracle.Options(mass=w.mass, smoother=1, **kw)


def _sensitivity(w, **kw):
    o = _oopts(w, **kw)
    return lambda idx: np.array([parity.self_sensitivity(w, int(k), opts=o) for k in idx])


@pytest.mark.parametrize("workload", list(WORKLOADS))
def test_two_filter_fp64_matches_the_oracle(ctx, workload):
    w = WORKLOADS[workload]()
    g = run_gpu(ctx, w, opts=_opts(w))
    o = run_oracle(w, opts=_oopts(w))
    check(g, o, TOL64, w=w, tracks=np.arange(w.tracks.n_tracks), sensitivity=_sensitivity(w))
    # the chi2 is the forward filter's: the same as with the RTS smoother
    r = run_gpu(ctx, w)
    np.testing.assert_array_equal(g["chi2"][g["status"] == 0], r["chi2"][g["status"] == 0])


@pytest.mark.parametrize("workload", ["telescope", "barrel", "map", "map_holes"])
def test_two_filter_mixed_within_1e3_sigma(ctx, workload):
    w = WORKLOADS[workload]()
    g = run_gpu(ctx, w, opts=_opts(w, tkf.MIXED))
    o = run_oracle(w, opts=_oopts(w))
    check_mixed(g, o)


@pytest.mark.parametrize("workload", ["barrel", "map"])
def test_two_filter_register_caps(ctx, workload):
    """The two-filter kernels capped at 128 and 64 registers (the tuner's candidates): mixed
    precision bit for bit the 255-register kernel's results; FP64 within the parity tolerance
    of the oracle (the FP64 instantiations may fuse a product of a two-term sum differently)."""
    w = WORKLOADS[workload]()
    ref = run_gpu(ctx, w, opts=_opts(w, tkf.MIXED))
    o = run_oracle(w, opts=_oopts(w))
    for regs in (128, 64):
        g = run_gpu(ctx, w, opts=_opts(w, tkf.MIXED, max_registers=regs))
        for k in ("par", "cov", "chi2", "ndf", "status"):
            np.testing.assert_array_equal(np.nan_to_num(g[k], nan=7.0), np.nan_to_num(ref[k], nan=7.0), err_msg=f"{regs} {k}")
        g64 = run_gpu(ctx, w, opts=_opts(w, max_registers=regs))
        check(g64, o, TOL64, w=w, tracks=np.arange(w.tracks.n_tracks), sensitivity=_sensitivity(w))


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED, tkf.MIXED_FP32])
def test_two_filter_edge_tracks(ctx, precision):
    w, tr = _edge_tracks()
    g = run_gpu(ctx, w, tr, opts=tkf.Options(precision=precision, smoother=tkf.SMOOTHER_TWO_FILTER))
    o = run_oracle(w, tr, opts=oracle.Options(smoother=1))
    np.testing.assert_array_equal(g["status"], o.status)
    np.testing.assert_array_equal(g["ndf"], o.ndf)
    if precision == tkf.FP64:
        wt = synth.Workload(w.name, w.geometry, w.field, tr, w.mass)
        check(g, o, TOL64, w=wt, tracks=np.arange(tr.n_tracks), sensitivity=_sensitivity(wt))


def test_two_filter_inflation_is_applied(ctx):
    """The backward filter's starting factor reaches the kernel: other factors give the oracle's
    other results (the covariance moves by ~1/inflation)."""
    w = WORKLOADS["barrel"]()
    for infl in (10.0, 1e5):
        g = run_gpu(ctx, w, opts=_opts(w, backward_inflation=infl))
        o = run_oracle(w, opts=_oopts(w, inflation=infl))
        check(g, o, TOL64, w=w, tracks=np.arange(w.tracks.n_tracks), sensitivity=_sensitivity(w, inflation=infl))


def test_two_filter_learned_mode(ctx):
    """The learned step proposer with the two-filter smoother: the network's proposals (the same
    BF16 weights on both sides) start the step-size control; the mixed path stays within the
    mixed tolerance of the oracle's result with the same proposals."""
    w = WORKLOADS["map"]()
    wbf = mlp.to_bf16(mlp.init(0))
    m = tkf.Mlp(ctx, wbf)
    g = run_gpu(ctx, w, opts=_opts(w, tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m))
    o = run_oracle(w, opts=_oopts(w, mlp=wbf))
    check_mixed(g, o)


def test_two_filter_fp32_end_to_end(ctx):
    """The FP32 question with the optimal smoother: TKF_MIXED_FP32 (forward and backward
    filters' covariance algebra and the weighted mean in FP32) against the FP64 oracle's
    two-filter result on the collider-like workloads."""
    for name in ("barrel", "map"):
        w = WORKLOADS[name]()
        g = run_gpu(ctx, w, opts=_opts(w, tkf.MIXED_FP32))
        o = run_oracle(w, opts=_oopts(w))
        assert np.mean(g["status"] != o.status) < 1e-3
        ds, dchi = _dp_over_sigma(g, o)
        stats = {"workload": name, "max_dp_over_sigma": float(ds.max()), "p99": float(np.quantile(ds, 0.99)),
                 "frac_within_1e-3": float(np.mean(ds <= MIXED_TOL_SIGMA)), "max_rel_chi2": float(dchi.max())}
        print(stats)
        assert np.mean(ds <= MIXED_TOL_SIGMA) >= 0.99 and dchi.max() <= MIXED_TOL_CHI2, stats


def test_two_filter_fp32_on_wide_priors(ctx):
    """Where the FP32 forward-evaluated RTS smoother loses part of the tolerance (telescope, wide
    1 mm / 10 mrad / 10 % priors: the smoother cancels most of the prior covariance), the FP32
    two-filter form: measured against the oracle's two-filter result."""
    w = WORKLOADS["telescope"]()
    g = run_gpu(ctx, w, opts=_opts(w, tkf.MIXED_FP32))
    o = run_oracle(w, opts=_oopts(w))
    assert np.array_equal(g["status"], o.status)
    ds, dchi = _dp_over_sigma(g, o)
    stats = {"max_dp_over_sigma": float(ds.max()), "p99": float(np.quantile(ds, 0.99)),
             "frac_within_1e-3": float(np.mean(ds <= MIXED_TOL_SIGMA)), "max_rel_chi2": float(dchi.max())}
    print(stats)
    assert np.mean(ds <= MIXED_TOL_SIGMA) >= 0.99 and dchi.max() <= MIXED_TOL_CHI2, stats


def test_two_filter_graph_key_and_options(ctx):
    """A replayed CUDA graph never serves one smoother's call with the other's launch; invalid
    combinations are refused."""
    w = WORKLOADS["telescope"]()
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    s = torch.cuda.Stream()
    outs = {}
    with torch.cuda.stream(s):
        for sm in (tkf.SMOOTHER_RTS, tkf.SMOOTHER_TWO_FILTER, tkf.SMOOTHER_RTS, tkf.SMOOTHER_TWO_FILTER):
            for _ in range(3):
                r = tkf.fit(ctx, geo, fld, b, tkf.Options(smoother=sm, graph=True), stream=s)
            torch.cuda.synchronize()
            outs.setdefault(sm, []).append(r.par.clone())
    for sm in outs:
        assert torch.equal(outs[sm][0], outs[sm][1])
    assert not torch.equal(outs[tkf.SMOOTHER_RTS][0], outs[tkf.SMOOTHER_TWO_FILTER][0])
    for bad in (dict(lanes_per_track=4), dict(max_registers=128, precision=tkf.MIXED_FP32),
                dict(backward_inflation=0.5), dict(backward_inflation=float("inf"))):
        with pytest.raises(tkf.TkfError, match="TWO_FILTER|backward_inflation"):
            tkf.fit(ctx, geo, fld, b, tkf.Options(smoother=tkf.SMOOTHER_TWO_FILTER, **bad))
    with pytest.raises(tkf.TkfError, match="smoother"):
        tkf.fit(ctx, geo, fld, b, tkf.Options(smoother=7))


def test_two_filter_host_and_noalloc_entry_points(ctx):
    """The host-buffer and the allocation-free entry points run the two-filter smoother too,
    with the device entry point's results bit for bit."""
    w = WORKLOADS["telescope"]()
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    host = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov)
    b = host.to("cuda:0")
    opts = tkf.Options(precision=tkf.MIXED, smoother=tkf.SMOOTHER_TWO_FILTER)
    r = tkf.fit(ctx, geo, fld, b, opts)
    out = tkf.alloc_outputs(t.n_tracks, b.offsets.device)
    tkf.fit_noalloc(ctx, geo, fld, b, out, opts)
    h = tkf.fit_host(ctx, geo, fld, host, opts)
    torch.cuda.synchronize()
    assert torch.equal(r.par, out.par) and torch.equal(r.cov, out.cov) and torch.equal(r.chi2, out.chi2)
    np.testing.assert_array_equal(r.par.cpu().numpy(), np.asarray(h.par))
    np.testing.assert_array_equal(r.cov.cpu().numpy(), np.asarray(h.cov))
