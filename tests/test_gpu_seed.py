"""GPU parity of the seed parameter estimation (tkf_estimate_seeds, the helix through three
measurements of each track) against the oracle's, and of the chain it starts: estimated seeds
-> fit -> refit from the fit's result with its covariance inflated 100-fold
(tkf_fit_options.seed_cov_scale), which replaces the smeared-truth seeds of the other tests."""

import dataclasses

import numpy as np
import pytest

import oracle
import paper_2505_22822_gb300 as tkf
import synth
from tests import parity
from tests.test_gpu_parity import TOL64, check, check_mixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA = 2.99792458e-4
EPS = np.finfo(float).eps
WHICH = {False: tkf.SEED_FIRST_MIDDLE_LAST, True: tkf.SEED_FIRST_THREE}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return tkf.Context(0)


def _handles(ctx, w):
    return tkf.Geometry.from_table(ctx, w.geometry.table), tkf.Field.from_desc(ctx, w.field)


def _device_batch(t, offsets=None, sid=None):
    offsets = t.offsets if offsets is None else offsets
    sid = t.sid if sid is None else sid
    n = len(offsets) - 1
    return tkf.Batch.from_arrays(offsets, t.meas, sid, np.zeros((n, 5)), np.zeros((n, 15))).to("cuda:0")


def seeds_gpu(ctx, w, first_three, offsets=None, sid=None, stream=None):
    geo, fld = _handles(ctx, w)
    b = _device_batch(w.tracks, offsets, sid)
    r = tkf.estimate_seeds(ctx, geo, fld, b, WHICH[first_three], stream=stream)
    torch.cuda.synchronize()
    return (r.par.cpu().numpy().T.copy(), r.cov.cpu().numpy().T.copy(),
            r.status.cpu().numpy().view(np.uint32).copy())


def seeds_oracle(w, first_three, offsets=None, sid=None):
    t = w.tracks
    return oracle.estimate_seeds(w.geometry.table, oracle.field_from(w.field),
                                 t.offsets if offsets is None else offsets, t.meas,
                                 t.sid if sid is None else sid, first_three=first_three)


def qop_rtol(w, par, st, first_three):
    """Relative q/p agreement that a different rounding order allows: the curvature comes from
    the sagitta of the three points, so one ulp of their coordinates moves q/p by eps |r| /
    sagitta (hits of overlapping modules are millimetres apart: sagittas far below a micron)."""
    t, g = w.tracks, w.geometry
    k = np.zeros((t.n_tracks, 3), dtype=np.int64)
    for i in range(t.n_tracks):  # the measured entries the seed is made of
        e = t.offsets[i] + np.flatnonzero((t.sid[t.offsets[i]:t.offsets[i + 1]] & 0x80000000) == 0)
        if len(e) >= 3:
            k[i] = e[[0, 1, 2]] if first_three else e[[0, (len(e) - 1) // 2, len(e) - 1]]
    s = t.sid[k] & 0x7FFFFFFF
    r = g.table[s, 9:12] + t.meas[k, 0, None] * g.table[s, 0:3] + t.meas[k, 1, None] * g.table[s, 3:6]
    lt = np.hypot(*(r[:, 2, :2] - r[:, 0, :2]).T)
    with np.errstate(divide="ignore", invalid="ignore"):
        fld = oracle.field_from(w.field)
        bz = np.abs(np.mean([oracle.field_at(fld, r[:, j])[0][:, 2] for j in range(3)], axis=0))
        R = np.sin(par[:, 3]) / np.abs(par[:, 4]) / (KAPPA * bz)
        sag = lt * lt / (8 * R)
        tol = 1e-10 + 1e3 * EPS * np.abs(r).max(axis=(1, 2)) / sag
    return np.where((st == 0) & np.isfinite(tol), tol, 1e-10)


def compare_seeds(g, o, rtol_qop):
    gp, gc, gs = g
    op, oc, os_ = o
    np.testing.assert_array_equal(gs, os_)
    bad = (os_ & (tkf.SEED_STATUS["TOO_FEW_HITS"] | tkf.SEED_STATUS["BAD_INPUT"])) != 0
    assert np.all(np.isnan(gp[bad])) and np.all(gc[bad] == 0)
    ok = ~bad
    # the local position and its covariance are the first measurement's, bit for bit
    np.testing.assert_array_equal(gp[ok, :2], op[ok, :2])
    for j in (0, 1, 5):
        np.testing.assert_array_equal(gc[ok, j], oc[ok, j])
    dphi = np.abs((gp[ok, 2] - op[ok, 2] + np.pi) % (2 * np.pi) - np.pi)
    assert dphi.max(initial=0) < 1e-10, dphi.max()
    assert np.abs(gp[ok, 3] - op[ok, 3]).max(initial=0) < 1e-10
    straight = ok & (os_ == tkf.SEED_STATUS["NO_CURVATURE"])
    assert np.all(gp[straight, 4] == 0)
    cur = ok & (os_ == 0)
    rel = np.abs(gp[cur, 4] / op[cur, 4] - 1.0)
    assert np.all(rel <= rtol_qop[cur]), np.max(rel / rtol_qop[cur])
    # the prior's diagonal depends on q/p (scattering at the estimated momentum, the radius)
    off = [j for j in range(15) if j not in (0, 1, 5, 9, 12, 14)]
    assert np.all(gc[ok][:, off] == 0)
    for j in (9, 12, 14):
        relc = np.abs(gc[ok, j] / oc[ok, j] - 1.0)
        assert np.all(relc <= 1e-9 + 4 * rtol_qop[ok]), (j, np.max(relc))
    return {"n": int(len(gs)), "ok": int(ok.sum()), "max_qop_rel": float(rel.max(initial=0))}


@pytest.mark.parametrize("first_three", [False, True])
@pytest.mark.parametrize("workload", ["telescope", "barrel", "map"])
def test_seed_parity(ctx, workload, first_three):
    w = {"telescope": lambda: synth.telescope_workload(2000, seed=4),
         "barrel": lambda: synth.barrel_workload(n_events=1, lo=6000, hi=6000, seed=21),
         "map": lambda: synth.solenoid_muon_workload(20_000, seed=7)}[workload]()
    g = seeds_gpu(ctx, w, first_three)
    o = seeds_oracle(w, first_three)
    print(compare_seeds(g, o, qop_rtol(w, o[0], o[2], first_three)))
    assert np.all(o[2] == 0)


def test_seed_edge_cases(ctx):
    """0, 1, 2 and 3 measurements, a bad surface id on the first and on another measurement,
    decreasing offsets, an offset beyond the measurements, and a ragged count of tracks that
    ends inside a block (1077)."""
    w = synth.telescope_workload(1077, seed=8)
    t = w.tracks
    offsets = t.offsets.astype(np.uint32).copy()
    sid = t.sid.astype(np.uint32).copy()
    offsets[1] = offsets[0]          # track 0: none
    offsets[2] = offsets[1] + 1      # track 1: one
    offsets[3] = offsets[2] + 2      # track 2: two
    offsets[4] = offsets[3] + 3      # track 3: three
    sid[offsets[10]] = 9999          # track 10: first measurement on a missing surface
    sid[offsets[11] + 1] = 9999      # track 11: another measurement on a missing surface
    offsets[21] = offsets[22] + 1    # track 20 ends after track 21 starts, track 21 decreasing
    offsets[-1] = offsets[-1] + 5    # last track beyond n_meas
    for first_three in (False, True):
        g = seeds_gpu(ctx, w, first_three, offsets, sid)
        o = seeds_oracle(w, first_three, offsets, sid)
        compare_seeds(g, o, np.full(len(offsets) - 1, 1e-10))
        st = g[2]
        assert list(st[:4]) == [1, 1, 1, 0]
        assert st[10] == 4 and st[11] == 4
        assert st[21] == 4 and st[-1] == 4


def test_seed_straight_tracks_without_field(ctx):
    g0 = synth.telescope_geometry()
    f = synth.Field(kind=0, B=(0.0, 0.0, 0.0))
    t = synth.simulate(g0, f, synth.telescope_params(), 5, [300])
    w = synth.Workload("telescope_no_field", g0, f, t)
    g = seeds_gpu(ctx, w, False)
    o = seeds_oracle(w, False)
    compare_seeds(g, o, np.full(300, 1e-10))
    assert np.all(g[2] == tkf.SEED_STATUS["NO_CURVATURE"]) and np.all(g[1][:, 14] == 1.0)


def test_seed_errors(ctx):
    w = synth.telescope_workload(10, seed=1)
    geo, fld = _handles(ctx, w)
    b = _device_batch(w.tracks)
    with pytest.raises(tkf.TkfError, match="unknown measurement selection"):
        tkf.estimate_seeds(ctx, geo, fld, b, 7)
    other = tkf.Context(0)
    with pytest.raises(tkf.TkfError, match="another context"):
        tkf.estimate_seeds(other, geo, fld, b)
    # no tracks: nothing to do, no launch
    e = tkf.Batch.from_arrays(np.zeros(1, np.uint32), np.zeros((0, 5)), np.zeros(0, np.uint32), np.zeros((0, 5)),
                              np.zeros((0, 15))).to("cuda:0")
    r = tkf.estimate_seeds(ctx, geo, fld, e)
    assert r.par.shape == (5, 0)
    with pytest.raises(tkf.TkfError, match="seed_cov_scale"):
        tkf.fit(ctx, geo, fld, b, tkf.Options(seed_cov_scale=0.0))


def test_seed_cov_scale_is_the_scaled_covariance(ctx):
    """A fit with seed_cov_scale = 100 is bit for bit the fit of the covariance multiplied by
    100 beforehand (one IEEE product either way), on the GPU and in the oracle."""
    w = synth.barrel_workload(n_events=1, lo=2000, hi=2000, seed=5)
    t = w.tracks
    geo, fld = _handles(ctx, w)
    b1 = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    b2 = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov * 100.0).to("cuda:0")
    for prec in (tkf.FP64, tkf.MIXED):
        r1 = tkf.fit(ctx, geo, fld, b1, tkf.Options(precision=prec, mass=w.mass, seed_cov_scale=100.0))
        r2 = tkf.fit(ctx, geo, fld, b2, tkf.Options(precision=prec, mass=w.mass))
        torch.cuda.synchronize()
        for k in ("par", "cov", "chi2"):
            assert torch.equal(getattr(r1, k), getattr(r2, k)), (prec, k)
    o = oracle.fit(w.geometry.table, oracle.field_from(w.field), oracle.Options(mass=w.mass), t.offsets, t.meas,
                   t.sid, t.seed_par, t.seed_cov * 100.0, n_threads=8)
    r = tkf.fit(ctx, geo, fld, b1, tkf.Options(mass=w.mass, seed_cov_scale=100.0))
    torch.cuda.synchronize()
    check(parity.gpu_to_track_major(r), o)


def _oracle_chain(w, idx, opts, first_three=False):
    sub = w.tracks.subset(idx)
    fld = oracle.field_from(w.field)
    sp, sc, st = oracle.estimate_seeds(w.geometry.table, fld, sub.offsets, sub.meas, sub.sid, first_three)
    r1 = oracle.fit(w.geometry.table, fld, opts, sub.offsets, sub.meas, sub.sid, sp, sc, n_threads=8)
    r2 = oracle.fit(w.geometry.table, fld, opts, sub.offsets, sub.meas, sub.sid, r1.par, r1.cov * 100.0,
                    n_threads=8)
    return r2


def gpu_chain(ctx, geo, fld, batch, opts, stream=None):
    """Estimated seeds -> fit -> refit from the fit's smoothed state at the first surface with
    its covariance inflated 100-fold; all on the device, three library calls."""
    s = tkf.estimate_seeds(ctx, geo, fld, batch, stream=stream)
    r1 = tkf.fit(ctx, geo, fld, tkf.with_seeds(batch, s.par, s.cov), opts, stream=stream)
    opts2 = dataclasses.replace(opts, seed_cov_scale=100.0)
    r2 = tkf.fit(ctx, geo, fld, tkf.with_seeds(batch, r1.par, r1.cov), opts2, stream=stream)
    return s, r1, r2


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED])
def test_chain_from_estimated_seeds(ctx, precision):
    """Muons in the solenoid map from estimated seeds: the GPU chain matches the oracle's chain,
    and the refit's pulls against the truth are unit normal (the first pass alone, whose prior
    is built from the same measurements and linearized at the rough seed, is not)."""
    w = synth.solenoid_muon_workload(4000, seed=7)
    t = w.tracks
    geo, fld = _handles(ctx, w)
    b = _device_batch(t)
    opts = tkf.Options(precision=precision, mass=w.mass)
    s, r1, r2 = gpu_chain(ctx, geo, fld, b, opts)
    torch.cuda.synchronize()
    assert torch.all(s.status == 0)
    g = parity.gpu_to_track_major(r2)
    assert np.mean(g["status"] == 0) > 0.999
    idx = np.arange(t.n_tracks)
    o = _oracle_chain(w, idx, oracle.Options(mass=w.mass))
    if precision == tkf.FP64:
        # the chain is less well conditioned than a fit from fixed seeds: the first fit's
        # linearization point moves with the measurements (parity.chain_self_sensitivity)
        check(g, o, TOL64, tracks=idx, sensitivity=lambda js: parity.chain_self_sensitivity(w, js))
    else:
        check_mixed(g, o)
    ok = g["status"] == 0
    sig = np.sqrt(np.einsum("nii->ni", oracle.unpack(g["cov"][ok])))
    d = g["par"][ok] - t.truth[ok]
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    pulls = d / sig
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.05), pulls.std(0)
    assert np.all(np.abs(pulls.mean(0)) < 0.06), pulls.mean(0)


def test_full_batch_seeds(ctx):
    """The 605,172-track barrel batch in bench configuration (a side stream): a seeded sample of
    3000 tracks against the oracle; every track gets curvature, and the priors cover the seeds'
    deviations from the truth."""
    w = synth.barrel_workload(n_events=50, seed=2)
    t = w.tracks
    assert t.n_tracks == 605172
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = seeds_gpu(ctx, w, False, stream=s)
    assert np.all(g[2] == 0)
    idx = np.sort(np.random.default_rng(13).choice(t.n_tracks, 3000, replace=False))
    sub = w.tracks.subset(idx)
    ws = synth.Workload(w.name, w.geometry, w.field, sub)
    o = seeds_oracle(ws, False)
    compare_seeds(tuple(x[idx] for x in g), o, qop_rtol(ws, o[0], o[2], False))
    d = g[0] - t.truth
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    pulls = d / np.sqrt(np.einsum("nii->ni", oracle.unpack(g[1])))
    assert np.all(pulls.std(0) < 1.1), pulls.std(0)
