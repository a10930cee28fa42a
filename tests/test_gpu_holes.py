"""GPU parity for track entries without a measurement (holes in sensitive modules, passive
surfaces; surface ids carrying TKF_SID_NO_MEASUREMENT): the fit propagates through them and
applies their material without an update, in FP64 (1e-10) and mixed (1e-3 sigma) against the
oracle; seed estimation skips them."""

import numpy as np
import pytest

import oracle
import paper_2505_22822_gb300 as tkf
import synth
from tests import parity
from tests.test_gpu_parity import TOL64, check, check_mixed
from tests.test_gpu_seed import compare_seeds, qop_rtol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HOLE = np.uint32(tkf.SID_NO_MEASUREMENT)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return tkf.Context(0)


def _gpu(ctx, w, t, opts):
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    r = tkf.fit(ctx, geo, fld, b, opts)
    torch.cuda.synchronize()
    return parity.gpu_to_track_major(r)


def _oracle(w, t):
    return oracle.fit(w.geometry.table, oracle.field_from(w.field), oracle.Options(mass=w.mass), t.offsets, t.meas,
                      t.sid, t.seed_par, t.seed_cov, n_threads=8)


def _passive_telescope():
    """A 9-plane telescope whose planes 3 and 6 are passive (material, no readout): their
    entries carry the flag and NaN measurement fields."""
    w = synth.telescope_workload(2000, seed=12)
    t = w.tracks
    a = t.offsets[:-1].astype(np.int64)
    for j in (3, 6):
        t.sid[a + j] |= HOLE
        t.meas[a + j] = np.nan
    return w


WORKLOADS = {
    "map_holes": lambda: synth.solenoid_muon_workload(4000, seed=11, p_hole=0.2),
    "barrel_holes": lambda: synth.barrel_workload(n_events=1, lo=4000, hi=4000, seed=23, p_hole=0.15),
    "telescope_passive": _passive_telescope,
}


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED])
@pytest.mark.parametrize("workload", list(WORKLOADS))
def test_parity_with_holes(ctx, workload, precision):
    w = WORKLOADS[workload]()
    t = w.tracks
    assert np.mean((t.sid & HOLE) != 0) > 0.1
    g = _gpu(ctx, w, t, tkf.Options(precision=precision, mass=w.mass))
    o = _oracle(w, t)
    np.testing.assert_array_equal(g["ndf"], o.ndf)
    if precision == tkf.FP64:
        check(g, o, TOL64, w=w, tracks=np.arange(t.n_tracks))
    else:
        check_mixed(g, o)


def test_edge_entries_without_measurement(ctx):
    """Two measurements left, none left (the seed is returned), a hole as the first entry, one
    hole in the middle, and a flagged surface id out of range."""
    w = synth.telescope_workload(7, seed=3)
    t = w.tracks
    a = t.offsets.astype(np.int64)

    def hole(e):
        t.sid[e] |= HOLE
        t.meas[e] = np.nan

    for e in range(a[1] + 1, a[1] + 8):
        hole(e)
    for e in range(a[2], a[3]):
        hole(e)
    hole(a[3])
    hole(a[4] + 4)
    t.sid[a[5] + 2] = HOLE | np.uint32(5000)
    g = _gpu(ctx, w, t, tkf.Options(mass=w.mass))
    o = _oracle(w, t)
    np.testing.assert_array_equal(g["ndf"], o.ndf)
    np.testing.assert_array_equal(g["status"], o.status)
    assert list(g["ndf"][:5]) == [18, 4, 0, 16, 16]
    np.testing.assert_array_equal(g["par"][2], t.seed_par[2])
    # track 1 keeps two measurements for five parameters: its result rests on the prior and
    # moves by ~1e-9 under one-ulp input changes (the conditioning-aware reading applies)
    check(g, o, TOL64, w=w, tracks=np.arange(t.n_tracks))


def test_pulls_with_holes_on_the_gpu(ctx):
    """20,000 muons in the solenoid map with 20 % holes, mixed precision: unit pulls."""
    w = synth.solenoid_muon_workload(20_000, seed=11, p_hole=0.2)
    t = w.tracks
    g = _gpu(ctx, w, t, tkf.Options(precision=tkf.MIXED, mass=w.mass))
    ok = g["status"] == 0
    assert ok.mean() > 0.999
    sig = np.sqrt(np.einsum("nii->ni", oracle.unpack(g["cov"][ok])))
    d = g["par"][ok] - t.truth[ok]
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    pulls = d / sig
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.02), pulls.std(0)


@pytest.mark.parametrize("first_three", [False, True])
def test_seeds_with_holes(ctx, first_three):
    w = synth.barrel_workload(n_events=1, lo=4000, hi=4000, seed=23, p_hole=0.15)
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    sid = t.sid.astype(np.uint32).copy()
    sid[t.offsets[7]] |= HOLE  # track 7: a first entry without a measurement
    n = t.n_tracks
    b = tkf.Batch.from_arrays(t.offsets, t.meas, sid, np.zeros((n, 5)), np.zeros((n, 15))).to("cuda:0")
    r = tkf.estimate_seeds(ctx, geo, fld, b, tkf.SEED_FIRST_THREE if first_three else tkf.SEED_FIRST_MIDDLE_LAST)
    torch.cuda.synchronize()
    g = (r.par.cpu().numpy().T.copy(), r.cov.cpu().numpy().T.copy(), r.status.cpu().numpy().view(np.uint32).copy())
    o = oracle.estimate_seeds(w.geometry.table, oracle.field_from(w.field), t.offsets, t.meas, sid,
                              first_three=first_three)
    assert g[2][7] == tkf.SEED_STATUS["BAD_INPUT"]
    compare_seeds(g, o, np.maximum(qop_rtol(w, o[0], o[2], first_three), 1e-9))
