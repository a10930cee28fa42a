"""GPU tests of the launch policy: every block shape, the autotuner and CUDA-graph replay give
bit-identical fits (each track's arithmetic does not depend on how tracks are spread over
warps and blocks), the tuner's cache file round-trips, graph replay reads the current input
contents, and bad shapes or flags are rejected before anything is enqueued."""

import json

import numpy as np
import pytest

import paper_2505_22822_gb300 as tkf
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (threads, blocks per SM, tracks per warp, registers); 0 = default
SHAPES = [(32, 8, 0, 0), (64, 4, 0, 0), (128, 2, 0, 0), (256, 1, 0, 0), (64, 2, 0, 0), (128, 1, 0, 0), (256, 3, 0, 0),
          (128, 2, 16, 0), (64, 4, 8, 0), (32, 8, 4, 0), (0, 0, 1, 0), (0, 0, 7, 0),
          (128, 4, 0, 128), (32, 16, 0, 128), (128, 8, 0, 64), (64, 16, 5, 64), (0, 0, 0, 64), (0, 0, 0, 255)]
SHAPES_255 = [(t, b, w) for t, b in [(32, 8), (64, 4), (128, 2), (256, 1), (64, 2), (128, 1)] for w in (32, 16, 8, 4)]
# [threads, blocks per SM, tracks per warp, registers, lanes a track]
CANDIDATES = ({(t, b, w, 255, 1) for t, b, w in SHAPES_255}
              | {(t, b, w, r, 1) for t, b, r in [(128, 4, 128), (64, 8, 128), (32, 16, 128), (128, 8, 64), (64, 16, 64),
                                                 (32, 32, 64)] for w in (32, 16, 8, 4)}
              | {(t, b, w, 255, 4) for t, b in [(32, 8), (64, 4), (128, 2), (256, 1), (64, 2), (128, 1)]
                 for w in (8, 4, 2, 1)})


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = tkf.Context(0)
    w = synth.barrel_workload(n_events=1, lo=3000, hi=3001, seed=21)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    t = w.tracks
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    return ctx, geo, fld, b, w


def _handles(ctx, w):
    return tkf.Geometry.from_table(ctx, w.geometry.table), tkf.Field.from_desc(ctx, w.field)


def _host(r):
    return {k: getattr(r, k).cpu().numpy().copy() for k in ("par", "cov", "chi2", "ndf", "status", "steps")}


def _same(x, y):
    for k in x:
        assert np.array_equal(x[k], y[k], equal_nan=True), k


def _run(ctx, geo, fld, b, stream=None, **kw):
    r = tkf.fit(ctx, geo, fld, b, tkf.Options(**kw), stream=stream)
    torch.cuda.synchronize()
    return _host(r)


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED])
def test_every_block_shape_gives_identical_results(setup, precision):
    ctx, geo, fld, b, _ = setup
    ref = _run(ctx, geo, fld, b, precision=precision)
    for t, bps, tpw, regs in SHAPES:
        if precision == tkf.FP64 and regs not in (0, 255):
            continue
        _same(_run(ctx, geo, fld, b, precision=precision, block_threads=t, blocks_per_sm=bps, tracks_per_warp=tpw,
                   max_registers=regs), ref)


def test_autotune_picks_a_candidate_and_writes_the_cache(setup, tmp_path, monkeypatch):
    _, _, _, b, w = setup
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("TKF_AUTOTUNE_CACHE", str(cache))
    ctx = tkf.Context(0)
    geo, fld = _handles(ctx, w)
    ref = _run(ctx, geo, fld, b, precision=tkf.MIXED)
    _same(_run(ctx, geo, fld, b, precision=tkf.MIXED, autotune=True), ref)
    entries = json.loads(cache.read_text())
    assert len(entries) == 1
    (key, shape), = entries.items()
    assert key.startswith("mixed.adaptive.uz.n11.")
    assert tuple(shape) in CANDIDATES
    # a second call of the same class takes the tuned shape without timing again
    before = cache.stat().st_mtime_ns
    _same(_run(ctx, geo, fld, b, precision=tkf.MIXED, autotune=True), ref)
    assert cache.stat().st_mtime_ns == before
    # a new context reads the file: with a planted entry (the older four-number form, one lane a
    # track) it tunes nothing for that class
    cache.write_text(json.dumps({key: [64, 8, 8, 128]}))
    before = cache.stat().st_mtime_ns
    ctx2 = tkf.Context(0)
    geo2, fld2 = _handles(ctx2, w)
    _same(_run(ctx2, geo2, fld2, b, precision=tkf.MIXED, autotune=True), ref)
    assert cache.stat().st_mtime_ns == before
    # another class (FP64) is tuned and added
    _run(ctx2, geo2, fld2, b, precision=tkf.FP64, autotune=True)
    entries = json.loads(cache.read_text())
    assert set(entries) == {key, key.replace("mixed.", "fp64.", 1)}
    assert entries[key] == [64, 8, 8, 128, 1]


def test_graph_replay_matches_direct_launches_and_reads_current_inputs(setup):
    ctx, geo, fld, b, _ = setup
    s = torch.cuda.Stream()
    ref = _run(ctx, geo, fld, b, precision=tkf.MIXED)
    out = tkf.alloc_outputs(b.n_tracks, "cuda:0")
    opts = tkf.Options(precision=tkf.MIXED, graph=True)
    for _ in range(4):  # direct, capture + launch, replay, replay
        for v in vars(out).values():
            if v is not None:
                v.fill_(0)
        with torch.cuda.stream(s):
            tkf.fit(ctx, geo, fld, b, opts, out=out, stream=s)
        s.synchronize()
        _same(_host(out), ref)
    # the graph reads the buffers at replay time: change the seeds in place
    saved = b.seed_par.clone()
    b.seed_par[4].mul_(1.01)
    ref2 = _run(ctx, geo, fld, b, precision=tkf.MIXED)
    with torch.cuda.stream(s):
        tkf.fit(ctx, geo, fld, b, opts, out=out, stream=s)
    s.synchronize()
    _same(_host(out), ref2)
    assert not np.array_equal(ref2["par"], ref["par"])
    b.seed_par.copy_(saved)
    # different output buffers are a different launch: direct again, then a new capture
    out2 = tkf.alloc_outputs(b.n_tracks, "cuda:0")
    for _ in range(3):
        with torch.cuda.stream(s):
            tkf.fit(ctx, geo, fld, b, opts, out=out2, stream=s)
        s.synchronize()
        _same(_host(out2), ref)


def test_graph_flag_on_the_legacy_stream_launches_directly(setup):
    ctx, geo, fld, b, _ = setup
    ref = _run(ctx, geo, fld, b, precision=tkf.FP64)
    for _ in range(3):
        _same(_run(ctx, geo, fld, b, precision=tkf.FP64, graph=True), ref)


def test_graph_and_autotune_with_learned_proposals(setup):
    ctx, geo, fld, b, _ = setup
    rng = np.random.default_rng(5)
    from oracle import mlp
    w = mlp.to_bf16(mlp.init(3) + 0.01 * rng.normal(size=tkf.MLP_PARAMS))
    m = tkf.Mlp(ctx, w)
    ref = _run(ctx, geo, fld, b, precision=tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m)
    s = torch.cuda.Stream()
    out = tkf.alloc_outputs(b.n_tracks, "cuda:0")
    opts = tkf.Options(precision=tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m, graph=True, autotune=True)
    for _ in range(3):
        with torch.cuda.stream(s):
            tkf.fit(ctx, geo, fld, b, opts, out=out, stream=s)
        s.synchronize()
        _same(_host(out), ref)


@pytest.mark.parametrize("kw", [dict(block_threads=96, blocks_per_sm=1), dict(block_threads=128, blocks_per_sm=0),
                                dict(block_threads=0, blocks_per_sm=2), dict(block_threads=512, blocks_per_sm=1),
                                dict(block_threads=64, blocks_per_sm=33), dict(tracks_per_warp=33),
                                dict(max_registers=100, precision=tkf.MIXED), dict(max_registers=64, precision=tkf.MIXED_FP32),
                                dict(max_registers=128, precision=tkf.MIXED, block_threads=256, blocks_per_sm=1)])
def test_bad_block_shapes_are_rejected(setup, kw):
    ctx, geo, fld, b, _ = setup
    with pytest.raises(tkf.TkfError, match="block shape"):
        tkf.fit(ctx, geo, fld, b, tkf.Options(**kw))


def test_unknown_flags_are_rejected(setup):
    ctx, geo, fld, b, _ = setup
    o = tkf.Options().c()
    o.flags = 8
    import ctypes
    from paper_2505_22822_gb300 import _inputs_struct, _outputs_struct, lib
    out = tkf.alloc_outputs(b.n_tracks, "cuda:0")
    st = lib().tkf_fit(ctx.handle, geo.handle, fld.handle, ctypes.byref(o), ctypes.byref(_inputs_struct(b)),
                       ctypes.byref(_outputs_struct(out)), None)
    assert st != 0
    assert "unknown flag" in lib().tkf_last_error(ctx.handle).decode()


def test_kernel_events_time_the_fit_kernel_alone(setup):
    ctx, geo, fld, b, _ = setup
    ref = _run(ctx, geo, fld, b, precision=tkf.MIXED)
    s = torch.cuda.Stream()
    kev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    outer = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for ev in kev:
        ev.record(s)
    out = tkf.alloc_outputs(b.n_tracks, "cuda:0")
    for _ in range(3):
        with torch.cuda.stream(s):
            outer[0].record(s)
            tkf.fit(ctx, geo, fld, b, tkf.Options(precision=tkf.MIXED, graph=True, kernel_events=kev), out=out,
                    stream=s)
            outer[1].record(s)
        s.synchronize()
        _same(_host(out), ref)
        k, o = kev[0].elapsed_time(kev[1]), outer[0].elapsed_time(outer[1])
        assert 0.0 < k <= o
