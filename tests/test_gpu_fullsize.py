"""GPU parity at the full benchmark sizes, in the launch configuration bench.py times (side
stream, tuned launch shape, CUDA-graph replay): the 50-event barrel + endcap batch
(605,172 pion tracks, uniform 2 T) and the 10^5-muon solenoid-map batch, fitted whole on the
GPU by every variant; a seeded sample of tracks is fitted by the CPU oracle and compared track
by track, and properties that hold at any size are checked on the whole batch."""

import numpy as np
import pytest

import oracle
import paper_2505_22822_gb300 as tkf
import synth
from tests import parity, proposer
from tests.test_gpu_parity import TOL64, check, check_mixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLE = 3000


def _bench_like_fit(ctx, geo, fld, batch, opts, calls=3):
    """Calls as bench.py makes them: a side stream, autotune on the first call, graph capture on
    the second, replay on the third; returns the third call's results."""
    s = torch.cuda.Stream()
    opts.autotune, opts.graph = True, True
    out = tkf.alloc_outputs(batch.n_tracks, "cuda:0")
    for _ in range(calls):
        with torch.cuda.stream(s):
            tkf.fit(ctx, geo, fld, batch, opts, out=out, stream=s)
    s.synchronize()
    return parity.gpu_to_track_major(out)


@pytest.fixture(scope="module")
def barrel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = tkf.Context(0)
    w = synth.barrel_workload(n_events=50, seed=2)  # the bench batch
    t = w.tracks
    assert t.n_tracks == 605172
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    idx = np.sort(np.random.default_rng(11).choice(t.n_tracks, SAMPLE, replace=False))
    return ctx, w, geo, fld, b, idx


def _oracle_sample(w, idx, opts):
    sub = w.tracks.subset(idx)
    return oracle.fit(w.geometry.table, oracle.field_from(w.field), opts, sub.offsets, sub.meas, sub.sid,
                      sub.seed_par, sub.seed_cov, n_threads=8)


def _whole_batch_properties(g, w):
    """All tracks fitted, chi2 / ndf near 1 on average (muon hypothesis on pions: within 1 %)."""
    assert np.all(g["status"] == 0)
    assert np.all(g["ndf"] == 2 * np.diff(w.tracks.offsets.astype(np.int64)))
    assert abs(np.mean(g["chi2"] / g["ndf"]) - 1.0) < 0.01


def test_fp64_full_batch(barrel):
    ctx, w, geo, fld, b, idx = barrel
    g = _bench_like_fit(ctx, geo, fld, b, tkf.Options(precision=tkf.FP64, mass=w.mass))
    _whole_batch_properties(g, w)
    o = _oracle_sample(w, idx, oracle.Options(mass=w.mass))
    gs = {k: (v[idx] if v is not None else None) for k, v in g.items()}
    check(gs, o, TOL64, w=w, tracks=idx)


def test_mixed_full_batch(barrel):
    ctx, w, geo, fld, b, idx = barrel
    g = _bench_like_fit(ctx, geo, fld, b, tkf.Options(precision=tkf.MIXED, mass=w.mass))
    _whole_batch_properties(g, w)
    o = _oracle_sample(w, idx, oracle.Options(mass=w.mass))
    check_mixed({k: (v[idx] if v is not None else None) for k, v in g.items()}, o)


def test_mixed_learned_full_batch(barrel):
    """Learned mode on the whole bench batch with a network trained without the CUDA path
    (oracle records of a seed-disjoint event, numpy training): sampled tracks against the
    oracle running the same network."""
    ctx, w, geo, fld, b, idx = barrel
    wbf, info = proposer.barrel_proposer()
    m = tkf.Mlp(ctx, wbf)
    g = _bench_like_fit(ctx, geo, fld, b, tkf.Options(precision=tkf.MIXED, mass=w.mass, step_mode=tkf.STEP_LEARNED,
                                                      mlp=m))
    _whole_batch_properties(g, w)
    o = _oracle_sample(w, idx, oracle.Options(mass=w.mass, mlp=wbf))
    check_mixed({k: (v[idx] if v is not None else None) for k, v in g.items()}, o)
    # the proposals cut the plain control's rejected attempts on the whole batch
    plain = _bench_like_fit(ctx, geo, fld, b, tkf.Options(precision=tkf.MIXED, mass=w.mass))
    assert g["steps"][:, 1].sum() < 0.2 * plain["steps"][:, 1].sum()


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED])
def test_solenoid_map_full_batch(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = tkf.Context(0)
    w = synth.solenoid_muon_workload(100_000, seed=3)  # the map bench batch
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    g = _bench_like_fit(ctx, geo, fld, b, tkf.Options(precision=precision, mass=w.mass))
    assert np.mean(g["status"] == 0) > 0.999
    idx = np.sort(np.random.default_rng(12).choice(t.n_tracks, SAMPLE, replace=False))
    o = _oracle_sample(w, idx, oracle.Options(mass=w.mass))
    gs = {k: (v[idx] if v is not None else None) for k, v in g.items()}
    if precision == tkf.FP64:
        check(gs, o, TOL64, w=w, tracks=idx)
    else:
        check_mixed(gs, o)
    # muons, the fit's own hypothesis: pulls against the truth are unit normal on the batch
    ok = g["status"] == 0
    C = oracle.unpack(g["cov"][ok])
    sig = np.sqrt(np.einsum("nii->ni", C))
    d = g["par"][ok] - t.truth[ok]
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    pulls = d / sig
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.02), pulls.std(0)
    assert np.all(np.abs(pulls.mean(0)) < 0.02), pulls.mean(0)


def _host_vs_device(ctx, geo, fld, hb, opts):
    h = tkf.fit_host(ctx, geo, fld, hb, opts)
    d = tkf.fit(ctx, geo, fld, hb.to("cuda:0"), opts)
    torch.cuda.synchronize()
    for k in ("par", "cov", "chi2"):
        np.testing.assert_array_equal(getattr(h, k), getattr(d, k).cpu().numpy(), err_msg=k)
    np.testing.assert_array_equal(h.ndf, d.ndf.cpu().numpy())
    np.testing.assert_array_equal(h.status, d.status.cpu().numpy().view(np.uint32))
    np.testing.assert_array_equal(h.steps, d.steps.cpu().numpy().view(np.uint32))
    return h


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED])
def test_host_entry_point_pipelines_chunks_with_identical_results(barrel, precision):
    """605,172 tracks through tkf_fit_host: five chunks (a small first one, then four) whose copies
    overlap the fits, results
    bit for bit those of the device entry point."""
    ctx, w, geo, fld, _, _ = barrel
    t = w.tracks
    hb = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov)
    _host_vs_device(ctx, geo, fld, hb, tkf.Options(precision=precision, mass=w.mass))


def test_host_entry_point_learned_mode_with_identical_results(barrel):
    """Learned mode through tkf_fit_host on the whole batch: the proposals of every track come
    from one pre-pass over the batch's offsets, surface ids and seeds (copied first), then the
    chunks are fitted; results bit for bit those of the device entry point, whose fit runs the
    pre-pass itself."""
    ctx, w, geo, fld, _, _ = barrel
    t = w.tracks
    wbf, _ = proposer.barrel_proposer()
    m = tkf.Mlp(ctx, wbf)
    hb = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov)
    _host_vs_device(ctx, geo, fld, hb, tkf.Options(precision=tkf.MIXED, mass=w.mass, step_mode=tkf.STEP_LEARNED,
                                                   mlp=m))


def test_host_entry_point_with_decreasing_offsets_matches_the_device_entry_point(barrel):
    """Offsets that decrease somewhere: each chunk copies the measurements between the least and
    the greatest of its tracks' offsets, and the copied range grows as one interval (below and
    above what earlier chunks copied) with no byte copied twice; the results still match the
    device entry point, and the reversed ranges are flagged BAD_INPUT."""
    ctx, w, geo, fld, _, _ = barrel
    sub = w.tracks.subset(np.arange(200_000))  # three chunks
    offsets = sub.offsets.astype(np.uint32).copy()
    assert offsets[1] >= 5
    offsets[0] = 5                              # the first chunk's range starts at 5
    offsets[70_000] = offsets[70_001] + 3       # track 69,999 ends after track 70,000 starts
    offsets[-1] = 2                             # the last track's range is reversed, below 5
    hb = tkf.Batch.from_arrays(offsets, sub.meas, sub.sid, sub.seed_par, sub.seed_cov)
    h = _host_vs_device(ctx, geo, fld, hb, tkf.Options(precision=tkf.MIXED, mass=w.mass))
    assert h.status[70_000] & tkf.TRACK_STATUS["BAD_INPUT"]
    assert h.status[-1] & tkf.TRACK_STATUS["BAD_INPUT"]
