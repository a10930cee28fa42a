"""GPU test of tkf_fit_noalloc, the entry point for callers that may not allocate device
memory while running (an online trigger process that reserves its GPU memory at start-up, or a
framework whose pool allocator owns the device): through the C interface, two calls in a row on
different batches must give the results of tkf_fit, bit for bit, in every precision, with the
two-filter smoother and with record capture; learned mode and oversized batches are rejected. This file is collected last so that a run
stopping at the first failure has already run every other test."""

import ctypes

import numpy as np
import pytest

import paper_2505_22822_gb300 as tkf
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

def _same(a, b, what):
    np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy(), err_msg=what)


CASES = {
    "fp64": dict(precision=tkf.FP64),
    "mixed": dict(precision=tkf.MIXED),
    "mixed_fp32": dict(precision=tkf.MIXED_FP32),
    "fp64_two_filter": dict(precision=tkf.FP64, smoother=tkf.SMOOTHER_TWO_FILTER),
    "mixed_record": dict(precision=tkf.MIXED, record=True),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_fit_on_two_calls(case):
    """Two calls in a row on different batches: every output equals tkf_fit's bit for bit (the
    same kernel, launch shape and per-track arithmetic; only the scratch differs). Record
    capture writes the same number of step records."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kw = dict(CASES[case])
    record = kw.pop("record", False)
    ctx = tkf.Context(0)
    w = synth.barrel_workload(n_events=2, lo=1000, hi=3000, seed=31)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    t = w.tracks
    half = t.n_tracks // 2
    for idx in (np.arange(half), np.arange(half, t.n_tracks)):  # two calls in a row
        sub = t.subset(idx)
        b = tkf.Batch.from_arrays(sub.offsets, sub.meas, sub.sid, sub.seed_par, sub.seed_cov).to("cuda:0")
        recs = []
        for _ in range(2):
            o = tkf.Options(mass=w.mass, **kw)
            if record:
                o.records = torch.zeros((200_000, 13), dtype=torch.float32, device="cuda:0")
                o.record_count = torch.zeros(1, dtype=torch.int32, device="cuda:0")
            recs.append(o)
        ref = tkf.fit(ctx, geo, fld, b, recs[0])
        out = tkf.alloc_outputs(sub.n_tracks, b.offsets.device)
        tkf.fit_noalloc(ctx, geo, fld, b, out, recs[1])
        torch.cuda.synchronize()
        for k in ("status", "ndf", "steps", "par", "cov", "chi2"):
            _same(getattr(out, k), getattr(ref, k), k)
        if record:
            assert int(recs[0].record_count.item()) > 0
            assert int(recs[1].record_count.item()) == int(recs[0].record_count.item())


def test_noalloc_rejects_learned_mode():
    """Learned step mode needs a per-track starting step, for which the static scratch has no
    room: rejected with TKF_ERR_UNSUPPORTED and a message that says so."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = tkf.Context(0)
    w = synth.telescope_workload(4, seed=1)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    t = w.tracks
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    out = tkf.alloc_outputs(t.n_tracks, b.offsets.device)
    m = tkf.Mlp(ctx, np.zeros(tkf.MLP_PARAMS, np.uint16))
    o = tkf.Options(step_mode=tkf.STEP_LEARNED, mlp=m).c()
    code = tkf.lib().tkf_fit_noalloc(ctx.handle, geo.handle, fld.handle, ctypes.byref(o),
                                     ctypes.byref(tkf._inputs_struct(b)), ctypes.byref(tkf._outputs_struct(out)), None)
    assert code == 5  # TKF_ERR_UNSUPPORTED
    assert b"no room" in tkf.lib().tkf_last_error(ctx.handle)


def test_noalloc_rejects_batches_above_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = tkf.Context(0)
    w = synth.telescope_workload(4, seed=1)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    t = w.tracks
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    out = tkf.alloc_outputs(t.n_tracks, b.offsets.device)
    s = tkf._inputs_struct(b)
    s.n_tracks = tkf.NOALLOC_MAX_TRACKS + 1  # rejected before anything is read or enqueued
    o = tkf.Options().c()
    code = tkf.lib().tkf_fit_noalloc(ctx.handle, geo.handle, fld.handle, ctypes.byref(o), ctypes.byref(s),
                                     ctypes.byref(tkf._outputs_struct(out)), None)
    assert code == 1  # TKF_ERR_INVALID_ARG
    assert b"exceeds the maximum" in tkf.lib().tkf_last_error(ctx.handle)
