"""Pins of the step-proposer network references (no GPU): the FP64 numpy backward pass vs
central finite differences, SiLU's derivative, Adam's first step (-lr sign(g)), BF16 rounding
on known bit patterns, the oracle's C++ FP32 forward vs the FP64 numpy forward, and the
learned step control in the oracle fit (same pulls, proposals judged by the error estimate)."""

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp


def _data(seed, n=64):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.N_IN))
    y = rng.normal(size=n)
    return X, y


def test_backward_matches_finite_differences():
    theta = mlp.init(1) + 0.05 * np.random.default_rng(2).normal(size=mlp.N_PARAMS)
    X, y = _data(3)
    loss, g = mlp.loss_and_grad(theta, X, y)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 120, replace=False), [mlp.N_PARAMS - 1]])
    h = 1e-6
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = h
        fd = (mlp.loss_and_grad(theta + e, X, y)[0] - mlp.loss_and_grad(theta - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_silu_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.dsilu(z), fd, atol=1e-8)


def test_adam_first_step_is_lr_times_sign():
    theta = mlp.init(5)
    g = np.random.default_rng(6).normal(size=mlp.N_PARAMS)
    new, m, v = mlp.adam_step(theta, g, np.zeros_like(theta), np.zeros_like(theta), 1, lr=1e-3)
    np.testing.assert_allclose(new - theta, -1e-3 * np.sign(g), rtol=1e-4)


def test_bf16_rounding_bit_patterns():
    vals = np.array([1.0, -2.0, 0.5, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 65504.0, 0.0])
    bits = mlp.to_bf16(vals)
    assert list(bits) == [0x3F80, 0xC000, 0x3F00, 0x3F80, 0x3F82, 0x4780, 0x0000]
    x = np.random.default_rng(7).normal(size=1000)
    r = mlp.from_bf16(mlp.to_bf16(x))
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2 ** -8


def test_oracle_cpp_forward_matches_numpy_forward():
    theta = mlp.init(8) + 0.1 * np.random.default_rng(9).normal(size=mlp.N_PARAMS)
    w = mlp.to_bf16(theta)
    X = np.random.default_rng(10).normal(size=(200, mlp.N_IN)).astype(np.float32)
    got = oracle.mlp_forward(w, X)
    ref, _ = mlp.forward(mlp.from_bf16(w).astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5)


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(11)
    X = rng.normal(size=(4096, mlp.N_IN))
    y = np.sin(X[:, 0]) + 0.5 * X[:, 6] ** 2 - 0.3 * X[:, 10]
    theta, losses = mlp.train(mlp.init(12), X, y, batch=256, epochs=8, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0]


def test_learned_control_in_the_oracle_keeps_the_fit(n_threads):
    # a network that proposes a constant 20 mm step (weights zero, output bias ln(20/0.9))
    theta = np.zeros(mlp.N_PARAMS)
    theta[-1] = np.log(20.0 / 0.9)
    w = mlp.to_bf16(theta)
    wl = synth.solenoid_muon_workload(3000, seed=44)
    plain = oracle.fit_tracks(wl, n_threads=n_threads)
    learned = oracle.fit_tracks(wl, oracle.Options(mlp=w), n_threads=n_threads)
    assert np.all(plain.status == 0) and np.all(learned.status == 0)
    # different step sequences, both within tolerance: the fits agree to a small fraction of sigma
    C = oracle.unpack(plain.cov)
    sig = np.sqrt(np.einsum("nii->ni", C))
    d = learned.par - plain.par
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    assert np.max(np.abs(d) / sig) < 0.05
    assert not np.array_equal(plain.steps, learned.steps)


def test_proposal_grid_ties_and_clamps_in_closed_form():
    """With every weight zero the hidden layers are silu(0) = 0, so the output is b3 and the
    proposal is 0.9 exp(k / 32), k = b3 * 32 rounded to nearest (ties to even), clamped to
    [h_min, h_max]; a track with fewer than two measurements gets h_max."""
    w = synth.telescope_workload(4, seed=5)
    t = w.tracks
    offsets = t.offsets.astype(np.uint32).copy()
    offsets[1] = offsets[0] + 1  # track 0: one measurement
    for b3, k in ((2.265625, 72), (2.28125, 73), (-1.015625, -32), (10.0, None), (-12.0, None)):
        theta = np.zeros(mlp.N_PARAMS)
        theta[-1] = b3
        wbf = mlp.to_bf16(theta)
        assert float(mlp.from_bf16(wbf)[-1]) == b3  # exactly representable in BF16
        o = oracle.Options(mlp=wbf)
        h = oracle.propose_start(w.geometry.table, oracle.field_from(w.field), o, offsets, t.sid, t.seed_par,
                                 t.n_hits)
        assert h[0] == o.h_max
        if k is None:
            expect = o.h_max if b3 > 0 else o.h_min
        else:
            expect = float(np.float32(0.9) * np.exp(np.float32(k / 32.0), dtype=np.float32))
        np.testing.assert_allclose(h[1:], expect, rtol=2e-7)


def test_oracle_training_records_are_consistent():
    """The oracle's record capture: finite inputs, a unit direction in the target frame, the
    clamped straight-line path, labels above ln(h_min); the same records on a second run; and
    a network trained on them by the reference explains part of the labels' variance."""
    import oracle
    import synth
    w = synth.solenoid_muon_workload(600, seed=1003)
    t = w.tracks
    args = (w.geometry.table, oracle.field_from(w.field), oracle.Options(), t.offsets, t.meas, t.sid, t.seed_par,
            t.seed_cov)
    rec = oracle.record_steps(*args)
    assert len(rec) > 1000 and np.all(np.isfinite(rec))
    np.testing.assert_array_equal(rec, oracle.record_steps(*args))
    d2 = (rec[:, 3:6].astype(np.float64) ** 2).sum(1)
    assert np.all(np.abs(d2 - 1.0) < 1e-5)
    assert np.all(np.abs(rec[:, 11]) <= 2.0) and np.all(rec[:, 12] > np.log(1e-4))
    X, y = rec[:, :12].astype(np.float64), rec[:, 12].astype(np.float64)
    theta, losses = mlp.train(mlp.init(1), X, y, batch=128, epochs=8, lr=2e-3)
    print({"records": len(y), "label_var": float(np.var(y)), "losses": losses})
    assert losses[-1] < 0.75 * np.var(y) and losses[-1] < losses[1]


def test_bf16_operand_gradient_stays_close_to_the_exact_one():
    """The BF16-operand reference (the tensor-core training's arithmetic) against the exact FP64
    gradient: rounding every contraction operand to 8 significant bits moves the loss by well
    under 1 % and the gradient by a few per mille of its scale, and it rounds exactly the
    values that BF16 cannot represent (BF16 values themselves pass through unchanged)."""
    rng = np.random.default_rng(3)
    theta = mlp.init(2) + 0.05 * rng.normal(size=mlp.N_PARAMS)
    X = rng.normal(size=(512, 12))
    y = np.sin(X[:, 0]) + 0.3 * X[:, 5]
    l0, g0 = mlp.loss_and_grad(theta, X, y)
    l1, g1 = mlp.loss_and_grad(theta, X, y, bf16_operands=True)
    assert abs(l1 / l0 - 1.0) < 1e-2
    assert np.max(np.abs(g1 - g0)) < 2e-2 * np.max(np.abs(g0))
    assert np.corrcoef(g0, g1)[0, 1] > 0.999
    b = mlp.bf16_round(X)
    np.testing.assert_array_equal(mlp.bf16_round(b), b)
    assert np.max(np.abs(b / X - 1.0)) <= 2.0 ** -8  # half a unit of the 7 stored bits
