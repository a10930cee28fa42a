"""GPU test of tkf_fit_noalloc, the entry point for callers that may not allocate device
memory while running (an online trigger process that reserves its GPU memory at start-up, or a
framework whose pool allocator owns the device): through the C interface, two calls in a row on
different batches must give the results of tkf_fit. This file is collected last so that a run
stopping at the first failure has already run every other test."""

import ctypes

import numpy as np
import pytest

import paper_2505_22822_gb300 as tkf
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


def _relmax(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    both_nan = np.isnan(a) & np.isnan(b)
    d = np.where(both_nan, 0.0, np.abs(a - b) / np.maximum(np.abs(b), 1e-300))
    return float(np.max(d)) if d.size else 0.0


@pytest.mark.parametrize("precision", [tkf.FP64, tkf.MIXED])
def test_noalloc_matches_fit_on_two_calls(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = tkf.Context(0)
    w = synth.barrel_workload(n_events=2, lo=1000, hi=3000, seed=31)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    t = w.tracks
    half = t.n_tracks // 2
    opts = tkf.Options(precision=precision, mass=w.mass)
    for idx in (np.arange(half), np.arange(half, t.n_tracks)):  # two calls in a row
        sub = t.subset(idx)
        b = tkf.Batch.from_arrays(sub.offsets, sub.meas, sub.sid, sub.seed_par, sub.seed_cov).to("cuda:0")
        ref = tkf.fit(ctx, geo, fld, b, opts)
        out = tkf.alloc_outputs(sub.n_tracks, b.offsets.device)
        tkf.fit_noalloc(ctx, geo, fld, b, out, opts)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.status.cpu().numpy(), ref.status.cpu().numpy())
        np.testing.assert_array_equal(out.ndf.cpu().numpy(), ref.ndf.cpu().numpy())
        np.testing.assert_array_equal(out.steps.cpu().numpy(), ref.steps.cpu().numpy())
        assert _relmax(out.par.cpu().numpy(), ref.par.cpu().numpy()) <= TOL
        assert _relmax(out.cov.cpu().numpy(), ref.cov.cpu().numpy()) <= TOL
        assert _relmax(out.chi2.cpu().numpy(), ref.chi2.cpu().numpy()) <= TOL


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
