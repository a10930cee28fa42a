"""Group-per-track mapping (tkf_fit_options.lanes_per_track = 4): four lanes share a track, each
transporting one derivative column and one row of the covariance transport. Every element is
computed by the same operations in the same order as with one lane a track, so the results
are bit-identical to that mapping, and within the parity tolerances of the oracle."""

import numpy as np
import pytest

import oracle
import paper_2505_22822_gb300 as tkf
import synth
from tests import parity
from tests.test_gpu_parity import TOL64, check, check_mixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return tkf.Context(0)


WORKLOADS = {
    "telescope": lambda: synth.telescope_workload(1000, seed=0),
    "barrel": lambda: synth.barrel_workload(n_events=1, lo=3000, hi=3000, seed=2),
    "map": lambda: synth.solenoid_muon_workload(3000, seed=3),
    "map_holes": lambda: synth.solenoid_muon_workload(2000, seed=11, p_hole=0.2),
}


def _fit(ctx, w, opts):
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    r = tkf.fit(ctx, geo, fld, b, opts)
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED])
@pytest.mark.parametrize("workload", list(WORKLOADS))
def test_group_is_bit_identical_and_matches_the_oracle(ctx, workload, precision):
    w = WORKLOADS[workload]()
    one = _fit(ctx, w, tkf.Options(precision=precision, mass=w.mass, lanes_per_track=1))
    four = _fit(ctx, w, tkf.Options(precision=precision, mass=w.mass, lanes_per_track=4))
    for k in ("par", "cov", "chi2", "ndf", "status", "steps"):
        a, b = getattr(one, k), getattr(four, k)
        assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0)), k
    g = parity.gpu_to_track_major(four)
    t = w.tracks
    o = oracle.fit(w.geometry.table, oracle.field_from(w.field), oracle.Options(mass=w.mass), t.offsets, t.meas,
                   t.sid, t.seed_par, t.seed_cov, n_threads=8)
    if precision == tkf.FP64:
        check(g, o, TOL64, w=w, tracks=np.arange(t.n_tracks))
    else:
        check_mixed(g, o)


@pytest.mark.parametrize("tpw", [1, 2, 8])
def test_group_tracks_per_warp_and_block_shapes(ctx, tpw):
    """Any tracks-per-warp count up to 8 and any block shape give the same results."""
    w = synth.barrel_workload(n_events=1, lo=1500, hi=1500, seed=5)
    ref = _fit(ctx, w, tkf.Options(precision=tkf.MIXED, mass=w.mass, lanes_per_track=1))
    for threads, bps in ((32, 8), (128, 2), (256, 1)):
        r = _fit(ctx, w, tkf.Options(precision=tkf.MIXED, mass=w.mass, lanes_per_track=4, tracks_per_warp=tpw,
                                     block_threads=threads, blocks_per_sm=bps))
        assert torch.equal(r.par, ref.par) and torch.equal(r.cov, ref.cov)


def test_group_edge_tracks(ctx):
    """Tracks with 0, 1, 2 and 3 measurements, holes and a bad surface id, and a ragged count
    (1,001 tracks: the last warp is part full) under the group mapping."""
    w = synth.telescope_workload(1001, seed=4)
    t = w.tracks
    a = t.offsets.astype(np.int64)
    t.sid[a[5] + 3] |= np.uint32(tkf.SID_NO_MEASUREMENT)
    t.meas[a[5] + 3] = np.nan
    t.sid[a[6] + 2] = 10_000
    offsets = t.offsets.copy()
    offsets[1:4] = offsets[0] + np.array([0, 1, 3])  # tracks 0, 1, 2: 0, 1, 2 measurements
    t2 = synth.Tracks(offsets, t.sid, t.meas, t.hit_truth, t.truth, t.seed_par, t.seed_cov, t.truth_last, t.event)
    w2 = synth.Workload(w.name, w.geometry, w.field, t2)
    one = _fit(ctx, w2, tkf.Options(mass=w.mass, lanes_per_track=1))
    four = _fit(ctx, w2, tkf.Options(mass=w.mass, lanes_per_track=4))
    for k in ("par", "cov", "chi2"):
        assert torch.equal(torch.nan_to_num(getattr(one, k), nan=7.0), torch.nan_to_num(getattr(four, k), nan=7.0)), k
    assert torch.equal(one.status, four.status) and torch.equal(one.ndf, four.ndf)


def test_group_option_errors(ctx):
    w = synth.telescope_workload(10, seed=1)
    for bad in (dict(lanes_per_track=2), dict(lanes_per_track=4, precision=tkf.MIXED_FP32),
                dict(lanes_per_track=4, precision=tkf.MIXED, max_registers=64),
                dict(lanes_per_track=4, tracks_per_warp=16)):
        with pytest.raises(tkf.TkfError, match="lanes_per_track"):
            _fit(ctx, w, tkf.Options(mass=w.mass, **bad))
