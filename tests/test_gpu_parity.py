"""GPU parity: the CUDA fitter through the C interface against the CPU oracle, element by
element on the same seeded inputs (FP64 path: tolerance 1e-10 in the metric of
tests/parity.py), plus edge cases and the host-buffer entry point."""

import numpy as np
import pytest

import oracle
import paper_2505_22822_gb300 as tkf
import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
MIXED_TOL_SIGMA = 1e-3   # |dp_i| <= 1e-3 sigma_i
MIXED_TOL_CHI2 = 1e-3    # relative


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return tkf.Context(0)


def run_gpu(ctx, w, tracks=None, opts=None):
    t = tracks if tracks is not None else w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    res = tkf.fit(ctx, geo, fld, b, opts or tkf.Options(mass=w.mass))
    torch.cuda.synchronize()
    return parity.gpu_to_track_major(res)


def run_oracle(w, tracks=None, opts=None):
    t = tracks if tracks is not None else w.tracks
    o = opts or oracle.Options(mass=w.mass)
    return oracle.fit(w.geometry.table, oracle.field_from(w.field), o, t.offsets, t.meas, t.sid, t.seed_par,
                      t.seed_cov, n_threads=8)


def mixed_deviation(g, o, mask):
    """Per-track largest |dp_i| / sigma_i (sigma from the oracle's covariance; phi wrapped) and
    relative chi2 difference |dchi2| / max(chi2, 1), over the tracks in `mask`."""
    C = oracle.unpack(o.cov[mask])
    sig = np.sqrt(np.einsum("nii->ni", C))
    dp = g["par"][mask] - o.par[mask]
    dp[:, 2] = (dp[:, 2] + np.pi) % (2 * np.pi) - np.pi
    ds = (np.abs(dp) / sig).max(1) if mask.any() else np.zeros(0)
    dchi = np.abs(g["chi2"][mask] - o.chi2[mask]) / np.maximum(o.chi2[mask], 1.0)
    return ds, dchi


def check(g, o, tol=TOL64, min_same_steps=0.999, w=None, tracks=None, sensitivity=None):
    """FP64 parity, every track compared.
    * Statuses and ndf are identical for every track.
    * A track with the oracle's adaptive step sequence is within `tol` in the metric of
      tests/parity.py, or, if it misses `tol`, it is ill-conditioned: its deviation is within
      3x the oracle's own movement under one-ulp input changes (`sensitivity(track_indices) ->
      array`, by default `parity.self_sensitivity` of the workload `w`; `tracks` are the compared
      tracks' indices in it), which for a well-conditioned track is ~1e-13.
    * A track whose step sequence differs (an accept/reject at eps ~ tol flipped by rounding;
      at most 0.1 % of the tracks) took another valid path through the same field; it is held
      to the mixed-path tolerance: every parameter within 1e-3 sigma, chi2 within 1e-3."""
    ok, same, stats = parity.compare(g, o, tol)
    dev = stats.pop("dev")
    n = stats["n"]
    assert stats["status_mismatch"] == 0, stats
    if same is None:
        same = np.ones(n, bool)
    other_steps = ~same
    stats["other_step_sequence"] = int(other_steps.sum())
    assert other_steps.sum() <= (1 - min_same_steps) * n + 1e-9, stats
    if other_steps.any():
        assert len(g["par"]) == len(o.status)
        cmp = other_steps & ((o.status & 0x39F) == 0)
        ds, dchi = mixed_deviation(g, o, cmp)
        stats["other_steps_max_dp_over_sigma"] = float(ds.max(initial=0))
        stats["other_steps_max_rel_chi2"] = float(dchi.max(initial=0))
        assert ds.max(initial=0) <= MIXED_TOL_SIGMA and dchi.max(initial=0) <= MIXED_TOL_CHI2, stats
    print(stats)
    bad = ~ok & same
    if bad.any():
        if sensitivity is None and w is not None:
            def sensitivity(idx):
                return np.array([parity.self_sensitivity(w, int(k)) for k in idx])
        assert sensitivity is not None, ("a track with the oracle's step sequence differs", stats)
        js = np.where(bad)[0]
        trk = np.asarray(tracks) if tracks is not None else np.arange(n)
        sens = np.asarray(sensitivity(trk[js]))
        ratio = dev[js] / np.maximum(sens, 1e-300)
        stats["ill_conditioned"] = int(len(js))
        stats["worst_deviation_over_self_sensitivity"] = float(ratio.max())
        print(stats)
        k = int(np.argmax(ratio))
        assert ratio[k] <= 3.0, ("a well-conditioned track differs", int(trk[js[k]]), float(dev[js[k]]),
                                 float(sens[k]))
    return stats


def test_telescope_fp64(ctx):
    w = synth.telescope_workload(1000, seed=0)
    g = run_gpu(ctx, w)
    o = run_oracle(w)
    assert np.all(g["status"] == 0)
    check(g, o)


def test_barrel_uniform_fp64_pions(ctx):
    w = synth.barrel_workload(n_events=2, lo=1500, hi=2500, seed=2)
    g = run_gpu(ctx, w)
    o = run_oracle(w)
    check(g, o)


def test_solenoid_map_fp64(ctx):
    w = synth.solenoid_muon_workload(3000, seed=3)
    g = run_gpu(ctx, w)
    o = run_oracle(w)
    check(g, o)


def test_general_uniform_field_direction(ctx):
    # a uniform field with x and y components takes the general (non-axial) kernel
    g0 = synth.telescope_geometry()
    f = synth.Field(kind=0, B=(0.3, -0.5, 1.8))
    t = synth.simulate(g0, f, synth.telescope_params(), 9, [500])
    w = synth.Workload("telescope_tilted_field", g0, f, t)
    check(run_gpu(ctx, w), run_oracle(w))


def _edge_tracks():
    """Telescope tracks edited into edge cases: 0, 1, 2 measurements, a bad surface id,
    decreasing offsets, a NaN seed, and a very long track (a 60-plane telescope)."""
    w = synth.telescope_workload(12, seed=4)
    t = w.tracks
    offs, meas, sid = [0], [], []
    seeds, covs = [], []
    nhits = [9, 0, 1, 2, 9, 9, 9, 9, 3, 9, 9, 9]
    for i, nh in enumerate(nhits):
        a = t.offsets[i]
        meas.append(t.meas[a:a + nh])
        s = t.sid[a:a + nh].copy()
        if i == 4:
            s[3] = 10_000  # out of range
        sid.append(s)
        offs.append(offs[-1] + nh)
        sp = t.seed_par[i].copy()
        if i == 5:
            sp[2] = np.nan
        seeds.append(sp)
        covs.append(t.seed_cov[i])
    offs = np.array(offs, np.uint32)
    tr = synth.Tracks(offs, np.concatenate(sid).astype(np.uint32), np.concatenate(meas), np.zeros((offs[-1], 2)),
                      np.array(seeds), np.array(seeds), np.array(covs), np.array(seeds),
                      np.zeros(len(nhits), np.uint32))
    return w, tr


def test_edge_cases_match_oracle_status_and_values(ctx):
    w, tr = _edge_tracks()
    g = run_gpu(ctx, w, tr)
    o = run_oracle(w, tr)
    np.testing.assert_array_equal(g["status"], o.status)
    np.testing.assert_array_equal(g["ndf"], o.ndf)
    assert g["status"][1] == tkf.TRACK_STATUS["TOO_FEW_HITS"]
    np.testing.assert_array_equal(g["par"][1], tr.seed_par[1])  # N = 0 returns the seed
    assert g["status"][4] & tkf.TRACK_STATUS["BAD_INPUT"]
    assert g["status"][5] & tkf.TRACK_STATUS["NON_FINITE"]
    assert np.all(np.isnan(g["par"][4])) and np.all(np.isnan(g["par"][5]))
    check(g, o, min_same_steps=1.0)


def test_decreasing_offsets_flag_bad_input(ctx):
    w = synth.telescope_workload(4, seed=6)
    t = w.tracks
    offs = t.offsets.copy()
    offs[2] = offs[1] - 1  # track 1 ends before it starts; track 2 starts one hit early
    tr = synth.Tracks(offs, t.sid, t.meas, t.hit_truth, t.truth, t.seed_par, t.seed_cov, t.truth_last, t.event)
    g = run_gpu(ctx, w, tr)
    o = run_oracle(w, tr)
    np.testing.assert_array_equal(g["status"], o.status)
    assert g["status"][1] == tkf.TRACK_STATUS["BAD_INPUT"]


def test_long_tracks_and_step_limits(ctx):
    g0 = synth.telescope_geometry(n_planes=60, spacing=20.0)
    f = synth.uniform_field(2.0)
    t = synth.simulate(g0, f, synth.telescope_params(min_hits=60, max_hits=60, pmin=0.5, pmax=1.0), 5, [200])
    w = synth.Workload("telescope60", g0, f, t)
    check(run_gpu(ctx, w), run_oracle(w))
    # max_steps = 1 forces TKF_TRACK_MAX_STEPS on both sides
    g = run_gpu(ctx, w, opts=tkf.Options(max_steps=1, tol=1e-9))
    o = run_oracle(w, opts=oracle.Options(max_steps=1, tol=1e-9))
    np.testing.assert_array_equal(g["status"], o.status)
    assert np.all(g["status"] & tkf.TRACK_STATUS["MAX_STEPS"])


def test_surface_behind_is_missed(ctx):
    w = synth.telescope_workload(50, seed=8)
    t = w.tracks
    sid = t.sid.copy()
    for i in range(t.n_tracks):  # swap the 3rd and 5th planes: plane 4 is then 100 mm behind
        a = t.offsets[i]
        sid[a + 2], sid[a + 4] = sid[a + 4], sid[a + 2]
    tr = synth.Tracks(t.offsets, sid, t.meas, t.hit_truth, t.truth, t.seed_par, t.seed_cov, t.truth_last, t.event)
    g = run_gpu(ctx, w, tr)
    o = run_oracle(w, tr)
    np.testing.assert_array_equal(g["status"], o.status)
    assert np.all(g["status"] & tkf.TRACK_STATUS["SURFACE_MISSED"])


def test_empty_batch_is_a_no_op(ctx):
    w = synth.telescope_workload(3, seed=1)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    t = w.tracks
    b = tkf.Batch.from_arrays(np.zeros(1, np.uint32), t.meas[:0], t.sid[:0], t.seed_par[:0], t.seed_cov[:0])
    out = tkf.fit(ctx, geo, fld, b.to("cuda:0"))
    torch.cuda.synchronize()
    assert out.par.shape == (5, 0)


def test_host_entry_point_equals_device_entry_point(ctx):
    w = synth.barrel_workload(n_events=1, lo=4000, hi=4000, seed=12)
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    hb = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov)
    h = tkf.fit_host(ctx, geo, fld, hb)
    d = tkf.fit(ctx, geo, fld, hb.to("cuda:0"))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(h.par, d.par.cpu().numpy())
    np.testing.assert_array_equal(h.cov, d.cov.cpu().numpy())
    np.testing.assert_array_equal(h.status, d.status.cpu().numpy().view(np.uint32))


def test_invalid_arguments_enqueue_nothing(ctx):
    w = synth.telescope_workload(3, seed=1)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    t = w.tracks
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    with pytest.raises(tkf.TkfError):
        tkf.fit(ctx, geo, fld, b, tkf.Options(tol=-1.0))
    with pytest.raises(tkf.TkfError):
        tkf.fit(ctx, geo, fld, b, tkf.Options(step_mode=tkf.STEP_LEARNED))
    bad = np.tile(np.eye(3).reshape(1, 9), (2, 1))
    bad[1, 0] = 2.0
    with pytest.raises(tkf.TkfError):
        tkf.Geometry(ctx, bad, np.zeros((2, 3)), 0.3, 93.7)


# ---------------------------------------------------------------- mixed precision


def check_mixed(g, o):
    """Mixed path vs the FP64 oracle, every track: identical statuses and ndf; every track the
    oracle fits (no fatal status bit) within 1e-3 sigma in each parameter and chi2 within 1e-3
    relative."""
    np.testing.assert_array_equal(g["status"], o.status)
    np.testing.assert_array_equal(g["ndf"], o.ndf)
    good = (o.status & 0x39F) == 0
    ds, dchi = mixed_deviation(g, o, good)
    bad = (ds > MIXED_TOL_SIGMA) | (dchi > MIXED_TOL_CHI2)
    stats = {"n": int(good.sum()), "max_dp_over_sigma": float(ds.max(initial=0)),
             "p99_dp_over_sigma": float(np.quantile(ds, 0.99)) if len(ds) else 0.0,
             "max_rel_chi2": float(dchi.max(initial=0)), "bad": int(bad.sum())}
    print(stats)
    assert bad.sum() == 0, stats
    return stats


MIXED = tkf.Options(precision=tkf.MIXED)


@pytest.mark.parametrize("name", ["telescope", "barrel", "solenoid_map"])
def test_mixed_precision_within_1e3_sigma(ctx, name):
    if name == "telescope":
        w = synth.telescope_workload(2000, seed=0)
    elif name == "barrel":
        w = synth.barrel_workload(n_events=2, lo=1500, hi=2500, seed=2)
    else:
        w = synth.solenoid_muon_workload(3000, seed=3)
    g = run_gpu(ctx, w, opts=tkf.Options(precision=tkf.MIXED, mass=w.mass))
    o = run_oracle(w)
    check_mixed(g, o)


def test_mixed_edge_cases_status(ctx):
    w, tr = _edge_tracks()
    g = run_gpu(ctx, w, tr, opts=MIXED)
    o = run_oracle(w, tr)
    np.testing.assert_array_equal(g["status"], o.status)
    np.testing.assert_array_equal(g["ndf"], o.ndf)


# ---------------------------------------------------------------- FP32 covariance algebra
def _dp_over_sigma(g, o):
    good = ((o.status & 0x39F) == 0) & (g["status"] == o.status)
    C = oracle.unpack(o.cov[good])
    sig = np.sqrt(np.einsum("nii->ni", C))
    dp = g["par"][good] - o.par[good]
    dp[:, 2] = (dp[:, 2] + np.pi) % (2 * np.pi) - np.pi
    dchi = np.abs(g["chi2"][good] - o.chi2[good]) / np.maximum(o.chi2[good], 1.0)
    return (np.abs(dp) / sig).max(1), dchi


@pytest.mark.parametrize("name", ["barrel", "solenoid_map"])
def test_fp32_covariance_algebra_meets_the_mixed_tolerance(ctx, name):
    """The experimental TKF_MIXED_FP32 (Joseph update and smoother in FP32 too, no C^-1 in the
    forward-accumulated smoother): on the barrel and field-map workloads every track stays
    within 1e-3 sigma of the FP64 oracle and chi2 within 1e-3 relative."""
    w = (synth.barrel_workload(n_events=2, lo=1500, hi=2500, seed=2) if name == "barrel"
         else synth.solenoid_muon_workload(5000, seed=3))
    g = run_gpu(ctx, w, opts=tkf.Options(precision=tkf.MIXED_FP32, mass=w.mass))
    o = run_oracle(w)
    assert np.array_equal(g["status"], o.status)
    ds, dchi = _dp_over_sigma(g, o)
    print({"max_dp_over_sigma": float(ds.max()), "max_rel_chi2": float(dchi.max())})
    assert ds.max() <= MIXED_TOL_SIGMA and dchi.max() <= MIXED_TOL_CHI2


def test_fp32_covariance_algebra_misses_on_wide_priors(ctx):
    """Where the seed prior is wide (telescope: 1 mm, 10 mrad, 10 % in q/p) the smoother cancels
    more of the prior covariance, and FP32 covariance algebra loses part of the tolerance: a
    fraction of a percent of tracks land between 1e-3 and 3e-3 sigma (the mixed path, with its
    FP64 update and smoother, stays below 1e-3 sigma on the same tracks)."""
    w = synth.telescope_workload(2000, seed=0)
    o = run_oracle(w)
    ds32, _ = _dp_over_sigma(run_gpu(ctx, w, opts=tkf.Options(precision=tkf.MIXED_FP32)), o)
    ds, _ = _dp_over_sigma(run_gpu(ctx, w, opts=tkf.Options(precision=tkf.MIXED)), o)
    print({"fp32_frac_within": float(np.mean(ds32 <= 1e-3)), "fp32_max": float(ds32.max()), "mixed_max": float(ds.max())})
    assert ds.max() <= MIXED_TOL_SIGMA
    assert 0.98 < np.mean(ds32 <= MIXED_TOL_SIGMA) < 1.0
    assert ds32.max() < 3e-3
