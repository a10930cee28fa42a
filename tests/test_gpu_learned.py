"""GPU tests of the learned step proposer: the library's training kernels against the FP64
numpy reference (gradients, a short training run), record capture, and fits with learned
proposals against the oracle running the same proposals, plus the gain over plain control."""

import numpy as np
import pytest

import oracle
import paper_2505_22822_gb300 as tkf
import synth
from oracle import mlp
from tests import parity, proposer
from tests.test_gpu_parity import MIXED_TOL_CHI2, MIXED_TOL_SIGMA, TOL64, check, check_mixed, mixed_deviation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return tkf.Context(0)


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dtype)


def test_loss_and_gradient_match_the_fp64_reference(ctx):
    rng = np.random.default_rng(0)
    theta = mlp.init(1) + 0.05 * rng.normal(size=mlp.N_PARAMS)
    X = rng.normal(size=(777, 12))
    y = rng.normal(size=777)
    loss, g = tkf.mlp_loss_grad(ctx, _cuda(theta), _cuda(X), _cuda(y))
    torch.cuda.synchronize()
    # the library's contractions take BF16 operands: the reference rounds the same operands
    ref_loss, ref_g = mlp.loss_and_grad(theta.astype(np.float32).astype(np.float64), X.astype(np.float32),
                                        y.astype(np.float32), bf16_operands=True)
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    g = g.cpu().numpy().astype(np.float64)
    # per element: the FP32 accumulation, plus one BF16 unit on the operands where an FP32 value
    # and its FP64 reference round to neighbouring BF16 values
    th = theta.astype(np.float32).astype(np.float64)
    scale = mlp.grad_term_scale(th, X.astype(np.float32), y.astype(np.float32))
    tol = 1e-4 * np.abs(ref_g) + 2.0 ** -7 * scale + 1e-6 * scale
    err = np.abs(g - ref_g)
    print({"max_rel": float(np.max(err / np.maximum(np.abs(ref_g), 1e-30))), "worst_over_tol": float(np.max(err / tol)),
           "over_1e-3_rel": int(np.sum(err > 1e-3 * np.abs(ref_g) + 1e-5 * np.abs(ref_g).max()))})
    assert np.all(err <= tol)
    # a rounding flip moves a few elements; a dropped term or a wrong index moves most of them
    assert np.sum(err > 1e-3 * np.abs(ref_g) + 1e-5 * np.abs(ref_g).max()) <= 0.005 * g.size


def test_forward_matches_the_oracle(ctx):
    rng = np.random.default_rng(2)
    theta = mlp.init(3) + 0.1 * rng.normal(size=mlp.N_PARAMS)
    w = mlp.to_bf16(theta)
    X = rng.normal(size=(500, 12)).astype(np.float32)
    out = tkf.mlp_forward(ctx, _cuda(mlp.from_bf16(w)), _cuda(X)).cpu().numpy()
    np.testing.assert_allclose(out, oracle.mlp_forward(w, X), rtol=1e-5, atol=1e-5)


def test_training_steps_follow_the_fp64_adam_reference(ctx):
    rng = np.random.default_rng(4)
    X = rng.normal(size=(2048, 12))
    y = np.sin(X[:, 0]) + 0.5 * X[:, 6] ** 2 - 0.3 * X[:, 10]
    theta0 = mlp.init(5)
    rec = np.concatenate([X, y[:, None]], axis=1)
    p = _cuda(theta0)
    mom = torch.zeros((2, mlp.N_PARAMS), dtype=torch.float32, device="cuda:0")
    loss, t = tkf.mlp_train(ctx, _cuda(rec), p, mom, 0, batch=256, epochs=2, lr=1e-3)
    torch.cuda.synchronize()
    ref, ref_losses = mlp.train(theta0.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64),
                                y.astype(np.float32).astype(np.float64), batch=256, epochs=2, lr=1e-3,
                                bf16_operands=True)
    assert t == 16
    got = p.cpu().numpy().astype(np.float64)
    # 16 Adam steps of 1e-3: FP32 vs FP64 agree to a small fraction of the total move
    assert np.max(np.abs(got - ref)) < 2e-4
    np.testing.assert_allclose(loss.cpu().numpy(), ref_losses, rtol=1e-3)


def _fit(ctx, w, opts, tracks=None):
    t = tracks if tracks is not None else w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    fld = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    res = tkf.fit(ctx, geo, fld, b, opts)
    torch.cuda.synchronize()
    return res


def train_proposer(ctx, fld, n_tracks=20000, epochs=8, seed=1000):
    """The library's own pipeline: records from the plain stepper on seed-disjoint tracks,
    initialisation, training and calibration on the GPU, BF16 rounding on loading."""
    from paper_2505_22822_gb300 import learn
    w = synth.solenoid_muon_workload(n_tracks, seed=seed, fld=fld)
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    f = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    rec = learn.record_steps(ctx, geo, f, b, tkf.MIXED)
    assert rec.shape[0] > 5000
    params, losses = learn.train(ctx, rec, epochs=epochs)
    q = learn.calibrate(ctx, params, rec)
    losses = losses.cpu().numpy()
    print({"records": int(rec.shape[0]), "losses": [round(float(x), 4) for x in losses], "bias_shift": q})
    return rec, params, losses


@pytest.fixture(scope="module")
def trained(ctx):
    """GPU-trained network (for the gain and timeout tests)."""
    fld = synth.solenoid_map()
    rec, params, losses = train_proposer(ctx, fld)
    return fld, rec, params, losses


@pytest.fixture(scope="module")
def reference_weights():
    """BF16 weights trained without the CUDA path (oracle records, numpy training): the network
    both sides run in the parity tests."""
    fld = synth.solenoid_map()
    w, info = proposer.map_proposer(fld)
    print(info)
    return fld, w


def test_records_are_sane_and_training_converges(trained):
    fld, rec, params, losses = trained
    r = rec.cpu().numpy()
    assert np.all(np.isfinite(r))
    assert np.all(np.abs(r[:, 3:6]) <= 1.0 + 1e-3)           # direction components
    assert np.all((r[:, 12] > np.log(1e-4)) & (r[:, 12] < 12))  # ln(step / mm)
    assert losses[-1] < 0.3 * losses[0]
    assert torch.all(torch.isfinite(params))


def test_initialisation_is_seeded_and_bounded(ctx):
    a = tkf.mlp_init(ctx, torch.empty(tkf.MLP_PARAMS, dtype=torch.float32, device="cuda:0"), 3).cpu().numpy()
    b = tkf.mlp_init(ctx, torch.empty(tkf.MLP_PARAMS, dtype=torch.float32, device="cuda:0"), 3).cpu().numpy()
    c = tkf.mlp_init(ctx, torch.empty(tkf.MLP_PARAMS, dtype=torch.float32, device="cuda:0"), 4).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    p = mlp.unpack(a.astype(np.float64))
    for name, fan_in in (("W1", 12), ("W2", 64), ("w3", 64)):
        x = p[name].ravel()
        assert np.all(np.abs(x) <= 1 / np.sqrt(fan_in))
        # uniform on (-1/sqrt(fan_in), 1/sqrt(fan_in)): mean ~ 0, variance ~ 1 / (3 fan_in)
        assert abs(x.mean()) < 4 * np.sqrt(1 / (3 * fan_in) / x.size)
        assert abs(x.var() * 3 * fan_in - 1.0) < 0.2
    for name in ("b1", "b2", "b3"):
        assert np.all(p[name] == 0.0)


def test_calibration_shifts_the_bias_by_the_residual_quantile(ctx, reference_weights):
    """tkf_mlp_calibrate against the numpy reference: the shift is the 5 % quantile of
    label - output over the records (FP64 reference forward; the library's is FP32, so the two
    agree to ~1e-5), added to the output bias only."""
    fld, _ = reference_weights
    w = synth.solenoid_muon_workload(1500, seed=1001, fld=fld)
    t = w.tracks
    rec = oracle.record_steps(w.geometry.table, oracle.field_from(w.field), oracle.Options(), t.offsets, t.meas,
                              t.sid, t.seed_par, t.seed_cov)
    rng = np.random.default_rng(9)
    theta = (mlp.init(5) + 0.05 * rng.normal(size=mlp.N_PARAMS)).astype(np.float32)
    p = _cuda(theta)
    shift = tkf.mlp_calibrate(ctx, p, _cuda(rec), 0.05)
    ref_theta, ref_q = mlp.calibrate(theta.astype(np.float64), rec[:, :12], rec[:, 12], 0.05)
    print({"records": len(rec), "shift": shift, "reference": ref_q})
    assert abs(shift - ref_q) < 1e-5
    got = p.cpu().numpy()
    np.testing.assert_array_equal(got[:-1], theta[:-1])
    assert got[-1] == np.float32(np.float64(theta[-1]) + shift)
    # the quantile is an order statistic: a fraction 0.05 of the residuals lies below it
    out = tkf.mlp_forward(ctx, _cuda(theta), _cuda(rec[:, :12])).cpu().numpy()
    frac = np.mean(rec[:, 12] - out < shift)
    assert abs(frac - 0.05) < 2.0 / len(rec)


def test_loading_fp32_parameters_rounds_them_to_bf16(ctx, reference_weights):
    """tkf_mlp_load_f32 (the library rounds on the device) gives the network of tkf_mlp_load with
    the reference's BF16 rounding: identical proposals on 5000 tracks; a non-finite parameter
    is rejected."""
    fld, _ = reference_weights
    rng = np.random.default_rng(11)
    theta = (mlp.init(6) + 0.05 * rng.normal(size=mlp.N_PARAMS)).astype(np.float32)
    m32 = tkf.Mlp.from_params(ctx, _cuda(theta))
    m16 = tkf.Mlp(ctx, mlp.to_bf16(theta))
    w = synth.solenoid_muon_workload(5000, seed=1002, fld=fld)
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    f = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    h32 = tkf.propose_start(ctx, geo, f, b, tkf.Options(precision=tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m32))
    h16 = tkf.propose_start(ctx, geo, f, b, tkf.Options(precision=tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m16))
    assert torch.equal(h32, h16)
    bad = theta.copy()
    bad[100] = np.nan
    with pytest.raises(tkf.TkfError, match="non-finite"):
        tkf.Mlp.from_params(ctx, _cuda(bad))
    with pytest.raises(tkf.TkfError, match="expected"):
        tkf.Mlp(ctx, mlp.to_bf16(theta)[:-1])


def _subset(o, idx):
    return oracle.FitResult(*(getattr(o, f)[idx] for f in ("par", "cov", "chi2", "ndf", "status", "steps", "cov_filt0")))


@pytest.mark.parametrize("precision", [tkf.MIXED, tkf.FP64])
def test_learned_fit_matches_the_oracle_with_the_same_proposals(ctx, reference_weights, precision):
    """Every track against the oracle running the same network. The proposals are integers on a
    1/32 grid of ln h decided in FP32 on both sides; the tensor cores' accumulation order may put
    an output that lies within rounding of a grid boundary on the other side of it (both
    proposals are then valid, one grid step apart). Tracks whose proposal equals the oracle's are
    held to the plain parity rule of their precision (FP64: 1e-10 with the step-sequence and
    conditioning rules of `check`; mixed: 1e-3 sigma); a track whose proposal differs starts from
    another valid step and is held to the mixed-path tolerance."""
    fld, wbf = reference_weights
    m = tkf.Mlp(ctx, wbf)
    w = synth.solenoid_muon_workload(3000, seed=3, fld=fld)
    t = w.tracks
    opts = tkf.Options(precision=precision, step_mode=tkf.STEP_LEARNED, mlp=m)
    res = _fit(ctx, w, opts)
    g = parity.gpu_to_track_major(res)
    oopts = oracle.Options(mlp=wbf)
    o = oracle.fit(w.geometry.table, oracle.field_from(w.field), oopts, t.offsets,
                   t.meas, t.sid, t.seed_par, t.seed_cov, n_threads=8)
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    f = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    h_gpu = tkf.propose_start(ctx, geo, f, b, opts).cpu().numpy().astype(np.float64)
    h_orc = oracle.propose_start(w.geometry.table, oracle.field_from(w.field), oopts, t.offsets, t.sid,
                                 t.seed_par, t.n_hits)
    same_prop = np.abs(np.log(h_gpu / h_orc)) * 32.0 < 1e-3
    print({"tracks": t.n_tracks, "other_proposal": int((~same_prop).sum())})
    assert np.mean(~same_prop) <= 1e-3
    np.testing.assert_array_equal(g["status"], o.status)
    idx = np.flatnonzero(same_prop)
    gs = {k: (v[idx] if v is not None else None) for k, v in g.items()}
    os_ = _subset(o, idx)
    if precision == tkf.FP64:
        check(gs, os_, TOL64, w=w, tracks=idx,
              sensitivity=lambda js: np.array([parity.self_sensitivity(w, int(k), opts=oopts) for k in js]))
    else:
        check_mixed(gs, os_)
    other = ~same_prop & ((o.status & 0x39F) == 0)
    ds, dchi = mixed_deviation(g, o, other)
    assert ds.max(initial=0) <= MIXED_TOL_SIGMA and dchi.max(initial=0) <= MIXED_TOL_CHI2


@pytest.mark.parametrize("precision", [tkf.MIXED, tkf.FP64])
def test_learned_fit_with_four_lanes_a_track_is_bit_identical(ctx, trained, precision):
    """The learned mode under the group-per-track mapping: the same proposals (one pre-pass per
    track) and the same results as one lane a track."""
    fld, _, params, _ = trained
    m = tkf.Mlp.from_params(ctx, params)
    w = synth.solenoid_muon_workload(2000, seed=3, fld=fld)
    one = _fit(ctx, w, tkf.Options(precision=precision, step_mode=tkf.STEP_LEARNED, mlp=m, lanes_per_track=1))
    four = _fit(ctx, w, tkf.Options(precision=precision, step_mode=tkf.STEP_LEARNED, mlp=m, lanes_per_track=4))
    for k in ("par", "cov", "chi2", "steps"):
        assert torch.equal(getattr(one, k), getattr(four, k)), k


def test_learned_proposals_save_step_attempts_at_equal_tolerance(ctx, trained):
    fld, _, params, _ = trained
    m = tkf.Mlp.from_params(ctx, params)
    w = synth.solenoid_muon_workload(20000, seed=3, fld=fld)
    plain = _fit(ctx, w, tkf.Options(precision=tkf.MIXED))
    learn = _fit(ctx, w, tkf.Options(precision=tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m))
    sp = plain.steps.cpu().numpy().astype(np.int64).sum(1)
    sl = learn.steps.cpu().numpy().astype(np.int64).sum(1)
    print({"plain_attempts": int(sp[0]), "plain_rejected": int(sp[1]),
           "learned_attempts": int(sl[0]), "learned_rejected": int(sl[1])})
    # same physics: the fits agree to a small fraction of sigma (different, valid step sequences)
    gp, gl = parity.gpu_to_track_major(plain), parity.gpu_to_track_major(learn)
    ok = (gp["status"] == 0) & (gl["status"] == 0)
    C = oracle.unpack(gp["cov"][ok])
    sig = np.sqrt(np.einsum("nii->ni", C))
    d = gl["par"][ok] - gp["par"][ok]
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    assert np.quantile(np.abs(d) / sig, 0.999) < 0.05
    # the proposals avoid the plain control's rejected attempts without costing extra steps
    assert sl[1] < sp[1]
    assert sl[0] <= sp[0]


def test_tensor_core_proposals_match_the_oracle(ctx, reference_weights):
    """The pre-pass's two dense layers run on the tensor cores (BF16 operands, FP32 accumulate);
    its proposals sit on a 1/32 grid of ln h, so they equal the oracle's except where an
    accumulation-order difference flips a rounding (then by one grid step)."""
    fld, wbf = reference_weights
    m = tkf.Mlp(ctx, wbf)
    w = synth.solenoid_muon_workload(20000, seed=33, fld=fld)
    t = w.tracks
    geo = tkf.Geometry.from_table(ctx, w.geometry.table)
    f = tkf.Field.from_desc(ctx, w.field)
    b = tkf.Batch.from_arrays(t.offsets, t.meas, t.sid, t.seed_par, t.seed_cov).to("cuda:0")
    opts = tkf.Options(precision=tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m)
    h_gpu = tkf.propose_start(ctx, geo, f, b, opts).cpu().numpy().astype(np.float64)
    o = oracle.Options(mlp=wbf)
    h_orc = oracle.propose_start(w.geometry.table, oracle.field_from(w.field), o, t.offsets, t.sid, t.seed_par,
                                 t.n_hits)
    assert np.all(h_gpu > 0)
    ratio = np.log(h_gpu / h_orc) * 32.0
    same = np.abs(ratio) < 1e-3
    assert np.mean(same) > 0.999, np.mean(same)
    # the rest differ by exactly one grid step (or meet a clamp)
    k = np.abs(ratio[~same])
    assert np.all((np.abs(k - 1.0) < 1e-3) | (h_gpu[~same] == np.float32(o.h_max)) |
                  (h_gpu[~same] == np.float32(o.h_min)))
    # a spread of proposals, not a constant
    assert np.unique(np.round(np.log(h_gpu[same]) * 32)).size > 10


def test_pre_pass_timeout_falls_back_to_the_plain_start(ctx, trained):
    """Failure path without a GPU fault: with the test flag the pre-pass issues no tensor-core
    work, so nothing ever arrives on its mbarrier; its bounded waits run out, it frees its tensor
    memory and returns, and the fit starts every track from h_max with PROPOSAL_FALLBACK, which
    gives the plain adaptive fit's results. The context stays usable."""
    fld, _, params, _ = trained
    m = tkf.Mlp.from_params(ctx, params)
    w = synth.solenoid_muon_workload(2000, seed=34, fld=fld)
    stalled = _fit(ctx, w, tkf.Options(precision=tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m,
                                       test_proposal_timeout=True))
    plain = _fit(ctx, w, tkf.Options(precision=tkf.MIXED))
    fb = tkf.TRACK_STATUS["PROPOSAL_FALLBACK"]
    st = stalled.status.cpu().numpy().view(np.uint32)
    assert np.all(st & fb)
    np.testing.assert_array_equal(st & ~np.uint32(fb), plain.status.cpu().numpy().view(np.uint32))
    for k in ("par", "cov", "chi2", "steps"):
        np.testing.assert_array_equal(getattr(stalled, k).cpu().numpy(), getattr(plain, k).cpu().numpy(), err_msg=k)
    # the context still works: a normal learned fit afterwards has no fallback
    again = _fit(ctx, w, tkf.Options(precision=tkf.MIXED, step_mode=tkf.STEP_LEARNED, mlp=m))
    assert not np.any(again.status.cpu().numpy().view(np.uint32) & fb)
