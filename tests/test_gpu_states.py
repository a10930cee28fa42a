"""GPU parity of the all-states output (tkf_fit_outputs.states_par / states_cov): every entry's
smoothed state from the backward RTS pass over the stored states, against the oracle's textbook
RTS pass, element by element (FP64: 1e-10 in the metric of tests/parity.py with each entry's
filtered covariance as the scale; mixed: 1e-3 sigma), plus the first-surface consistency,
unchanged default outputs, edge tracks and argument errors."""

import json

import numpy as np
import pytest

import oracle
import paper_2505_22822_gb300 as tkf
import synth
from tests import parity
from tests.test_gpu_parity import MIXED_TOL_CHI2, MIXED_TOL_SIGMA, TOL64, _edge_tracks, check, check_mixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return tkf.Context(0)


def _gpu(ctx, w, t, opts, states=True):
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    r = tkf.fit(ctx, geo, fld, b, opts, states=states)
    torch.cuda.synchronize()
    return r


def _oracle(w, t):
    return oracle.fit(w.geometry.table, oracle.field_from(w.field), oracle.Options(mass=w.mass), t.offsets, t.meas,
                      t.sid, t.seed_par, t.seed_cov, n_threads=8, states=True)


WORKLOADS = {
    "telescope": lambda: synth.telescope_workload(1000, seed=0),
    "barrel": lambda: synth.barrel_workload(n_events=2, lo=1500, hi=2500, seed=2),
    "solenoid_map": lambda: synth.solenoid_muon_workload(2000, seed=3),
    "map_holes": lambda: synth.solenoid_muon_workload(2000, seed=11, p_hole=0.2),
}


def _mixed_states_dev(sp, o, offsets):
    """Per-entry largest |dp_i| / sigma_i (oracle sigma at that entry) over entries of tracks
    that the oracle fits."""
    ok = ~np.isnan(o.states_par).any(1)
    C = oracle.unpack(o.states_cov[ok])
    sig = np.sqrt(np.einsum("nii->ni", C))
    dp = sp[ok] - o.states_par[ok]
    dp[:, 2] = (dp[:, 2] + np.pi) % (2 * np.pi) - np.pi
    return (np.abs(dp) / sig).max(1) if ok.any() else np.zeros(0)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_every_entry_fp64_matches_the_oracle(ctx, name):
    w = WORKLOADS[name]()
    t = w.tracks
    _check_fp64_states(w, t, _gpu(ctx, w, t, tkf.Options(mass=w.mass)), _oracle(w, t))


def _check_fp64_states(w, t, r, o):
    g = parity.gpu_to_track_major(r)
    # the first-surface outputs keep the parity of the default path
    check(g, o, TOL64, w=w, tracks=np.arange(t.n_tracks))
    sp, sc = parity.states_to_entry_major(r)
    dev, nan_same = parity.compare_states(sp, sc, o, t.offsets)
    assert nan_same
    same_steps = np.all(g["steps"] == o.steps, axis=1)
    bad = np.flatnonzero((dev > TOL64) & same_steps)
    stats = {"entries": int(len(sp)), "max_dev": float(dev[same_steps].max(initial=0)), "over_tol": int(len(bad))}
    if len(bad):  # the conditioning rule of `check`, on every entry
        sens = np.array([parity.states_self_sensitivity(w, int(k)) for k in bad])
        ratio = dev[bad] / np.maximum(sens, 1e-300)
        stats["worst_deviation_over_self_sensitivity"] = float(ratio.max())
        print(stats)
        assert ratio.max() <= 3.0, stats
    print(stats)
    other = ~same_steps
    if other.any():  # another valid step sequence: the mixed-path tolerance at every entry
        mask = np.repeat(other, np.diff(t.offsets.astype(np.int64)))
        ds = _mixed_states_dev(np.where(mask[:, None], sp, o.states_par), o, t.offsets)
        assert ds.max(initial=0) <= MIXED_TOL_SIGMA


@pytest.mark.parametrize("name", ["barrel", "solenoid_map", "map_holes"])
def test_every_entry_mixed_within_1e3_sigma(ctx, name):
    w = WORKLOADS[name]()
    t = w.tracks
    r = _gpu(ctx, w, t, tkf.Options(precision=tkf.MIXED, mass=w.mass))
    o = _oracle(w, t)
    check_mixed(parity.gpu_to_track_major(r), o)
    sp, _ = parity.states_to_entry_major(r)
    assert np.array_equal(np.isnan(sp).any(1), np.isnan(o.states_par).any(1))
    ds = _mixed_states_dev(sp, o, t.offsets)
    print({"entries": int(len(ds)), "max_dp_over_sigma": float(ds.max()), "p99": float(np.quantile(ds, 0.99))})
    assert ds.max() <= MIXED_TOL_SIGMA


def test_register_caps_and_autotune(ctx, tmp_path, monkeypatch):
    """The all-states kernels capped at 128 and 64 registers, and the autotuned call: in mixed
    precision every output, every entry's state included, bit for bit the 255-register result;
    in FP64 every entry within the parity tolerance of the oracle (the FP64 instantiations may
    fuse a product of a two-term sum differently); the tuned shape is cached under the
    all-states class."""
    w = WORKLOADS["barrel"]()
    t = w.tracks
    keys = ("par", "cov", "chi2", "ndf", "status", "steps", "states_par", "states_cov")
    ref = _gpu(ctx, w, t, tkf.Options(precision=tkf.MIXED, mass=w.mass))
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("TKF_AUTOTUNE_CACHE", str(cache))
    ctx2 = tkf.Context(0)
    runs = [(regs, _gpu(ctx, w, t, tkf.Options(precision=tkf.MIXED, mass=w.mass, max_registers=regs)))
            for regs in (128, 64)]
    runs.append(("tuned", _gpu(ctx2, w, t, tkf.Options(precision=tkf.MIXED, mass=w.mass, autotune=True))))
    for label, r in runs:
        for k in keys:
            a, b = getattr(r, k), getattr(ref, k)
            assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0)), (label, k)
    (key,) = json.loads(cache.read_text())
    assert key.startswith("mixed.states.uz.")
    o = _oracle(w, t)
    for regs in (128, 64):
        _check_fp64_states(w, t, _gpu(ctx, w, t, tkf.Options(mass=w.mass, max_registers=regs)), o)


def test_first_entry_is_the_first_surface_result_and_defaults_are_unchanged(ctx):
    """The backward pass's state at entry 0 equals the forward-evaluated first-surface result
    (1e-10); the first-surface outputs, chi2, ndf, status and step counters are bit-identical to a
    fit without the all-states output."""
    w = WORKLOADS["barrel"]()
    t = w.tracks
    opts = tkf.Options(mass=w.mass)
    r = _gpu(ctx, w, t, opts)
    d = _gpu(ctx, w, t, opts, states=False)
    for k in ("par", "cov", "chi2", "ndf", "status", "steps"):
        np.testing.assert_array_equal(getattr(r, k).cpu().numpy(), getattr(d, k).cpu().numpy(), err_msg=k)
    sp, sc = parity.states_to_entry_major(r)
    first = t.offsets[:-1].astype(np.int64)
    g = parity.gpu_to_track_major(r)
    o = _oracle(w, t)  # for the covariance scale (filtered covariance at the first surface)
    ok, _, st = parity.compare({"par": sp[first], "cov": sc[first], "chi2": g["chi2"], "ndf": g["ndf"],
                                "status": g["status"], "steps": None}, parity_result(g, o), TOL64)
    st.pop("dev")
    print(st)
    assert ok.all(), st


def parity_result(g, o):
    """The GPU's own first-surface result in the oracle's result layout (with the oracle's
    filtered covariance as the scale), to compare another GPU output against it."""
    return oracle.FitResult(g["par"], g["cov"], g["chi2"], g["ndf"], g["status"], g["steps"], o.cov_filt0)


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED])
def test_edge_tracks_rows(ctx, precision):
    """0-3 measurements, a bad surface id, a NaN seed: statuses equal the oracle's; rows of
    failed tracks and of the track without measurements are NaN on both sides; the rest match."""
    w, tr = _edge_tracks()
    r = _gpu(ctx, w, tr, tkf.Options(precision=precision))
    o = _oracle(w, tr)
    np.testing.assert_array_equal(r.status.cpu().numpy().view(np.uint32), o.status)
    sp, sc = parity.states_to_entry_major(r)
    dev, nan_same = parity.compare_states(sp, sc, o, tr.offsets)
    assert nan_same
    tol = TOL64 if precision == tkf.FP64 else 1e-3
    print(dev)
    ok = (o.status & 0x39F) == 0
    if precision == tkf.FP64:
        assert dev[ok].max() <= TOL64
    else:
        ds = _mixed_states_dev(sp, o, tr.offsets)
        assert ds.max() <= tol


def test_states_argument_errors(ctx):
    w = synth.telescope_workload(8, seed=1)
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    out = tkf.alloc_outputs(t.n_tracks, b.offsets.device, states_meas=b.n_meas)
    with pytest.raises(tkf.TkfError, match="all-states"):
        tkf.fit(ctx, geo, fld, b, tkf.Options(smoother=tkf.SMOOTHER_TWO_FILTER), out=out)
    half = tkf.alloc_outputs(t.n_tracks, b.offsets.device)
    half.states_par = out.states_par
    with pytest.raises(tkf.TkfError, match="both"):
        tkf.fit(ctx, geo, fld, b, tkf.Options(), out=half)
    hb = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov)
    hout = tkf.Result(np.empty((5, t.n_tracks)), np.empty((15, t.n_tracks)), np.empty(t.n_tracks),
                      np.empty(t.n_tracks, np.int32), np.empty(t.n_tracks, np.uint32), None,
                      np.empty((5, t.n_hits)), np.empty((15, t.n_hits)))
    with pytest.raises(tkf.TkfError, match="all-states"):
        tkf.fit_host(ctx, geo, fld, hb, out=hout)
