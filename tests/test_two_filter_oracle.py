"""Pins of the oracle's two-filter smoother (the optimal smoother: weighted mean of a forward
and a backward filter) against what mathematics and the simulation fix, independently of the
oracle's own code:

* on a linear-Gaussian chain the weighted mean at step 0 is the batch posterior: its mean
  exactly (the backward filter's start, centred on the forward filter's last state, which is the
  posterior mean there, moves no minimiser), its covariance up to the start's residual
  information, which falls as 1/inflation;
* noise-free tracks with energy loss fit back to the truth (a wrong reversal of the angles or of
  the energy loss in the backward filter misses it by orders of magnitude);
* pulls are unit normal, the chi2 is the forward filter's, and the estimator is as accurate as
  the RTS smoother's."""

import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import _batch_posterior


def _chain(seed, rank, N=7, holes=()):
    rng = np.random.default_rng(seed)
    J = np.array([np.eye(5) + 0.2 * rng.normal(size=(5, 5)) for _ in range(N)])
    L = 0.05 * rng.normal(size=(N, 5, rank))
    Q = np.einsum("kij,klj->kil", L, L)
    p0 = 0.1 * rng.normal(size=5)
    X = rng.normal(size=(5, 5))
    C0 = X @ X.T * 0.05 + 0.01 * np.eye(5)
    m = 0.1 * rng.normal(size=(N, 2))
    m[list(holes)] = np.nan
    V = []
    for _ in range(N):
        Y = rng.normal(size=(2, 2))
        V.append(Y @ Y.T * 0.01 + 0.002 * np.eye(2))
    return J, L, Q, p0, C0, m, np.array(V)


@pytest.mark.parametrize("seed,rank,holes", [(0, 2, ()), (1, 5, ()), (2, 1, ()), (3, 2, (1, 4)), (4, 5, (0, 6))])
def test_linear_two_filter_is_the_batch_posterior(seed, rank, holes):
    J, L, Q, p0, C0, m, V = _chain(seed, rank, holes=holes)
    means, covs, _ = _batch_posterior(J, L, p0, C0, m, V)
    sig = np.sqrt(np.diag(covs[0]))
    errs = []
    for infl in (1e2, 1e3, 1e4):
        ps, Cs, st = oracle.linear_chain_two_filter(J, Q, p0, C0, m, V, infl)
        assert st == 0
        assert np.abs((ps - means[0]) / sig).max() < 1e-10
        e = np.abs(Cs - covs[0]).max() / np.abs(covs[0]).max()
        assert e < 2.0 / infl, (infl, e)
        errs.append(e)
    # the start's residual information: the covariance error falls as 1/inflation
    assert 7.0 < errs[1] / errs[2] < 13.0 and 7.0 < errs[0] / errs[1] < 13.0, errs


def test_linear_two_filter_planted_mistakes_fail():
    """The pin above separates the method from plausible slips: the backward noise of the
    wrong step, or none at all, moves the mean by far more than its tolerance."""
    J, L, Q, p0, C0, m, V = _chain(7, 2)
    means, covs, _ = _batch_posterior(J, L, p0, C0, m, V)
    sig = np.sqrt(np.diag(covs[0]))
    for bad in (np.zeros_like(Q), np.roll(Q, 1, axis=0)):
        ps, _, _ = oracle.linear_chain_two_filter(J, bad, p0, C0, m, V, 1e3)
        assert np.abs((ps - means[0]) / sig).max() > 1e-3


def test_noise_free_tracks_fit_back_to_truth_two_filter(n_threads):
    w = synth.barrel_workload(n_events=1, lo=500, hi=500, seed=21, mass=synth.MUON_MASS, ms=0,
                              sigma_hit=0.0, seed_smear=0)
    r = oracle.fit_tracks(w, oracle.Options(tol=1e-9, smoother=1), n_threads=n_threads)
    assert np.all(r.status == 0)
    d = r.par - w.tracks.truth
    assert np.max(np.abs(d[:, :2])) < 1e-7      # mm
    assert np.max(np.abs(d[:, 2:4])) < 1e-8     # rad
    # energy loss given back in the backward filter (taken away instead: ~5e-3)
    assert np.max(np.abs(d[:, 4] / w.tracks.truth[:, 4])) < 2e-7
    assert np.max(r.chi2) < 1e-6


def test_noise_free_with_holes_two_filter(n_threads):
    w = synth.barrel_workload(n_events=1, lo=300, hi=300, seed=12, mass=synth.MUON_MASS, p_hole=0.25, ms=0,
                              sigma_hit=0.0, seed_smear=0)
    r = oracle.fit_tracks(w, oracle.Options(tol=1e-9, smoother=1), n_threads=n_threads)
    assert np.all(r.status == 0)
    d = r.par - w.tracks.truth
    assert np.max(np.abs(d[:, :2])) < 1e-7
    assert np.max(np.abs(d[:, 2:4])) < 1e-8
    assert np.max(np.abs(d[:, 4] / w.tracks.truth[:, 4])) < 2e-7


def _errors(w, r, sigma_from=None):
    ok = r.status == 0
    d = r.par[ok] - w.tracks.truth[ok]
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    src = r if sigma_from is None else sigma_from
    sig = np.sqrt(np.einsum("nii->ni", oracle.unpack(src.cov[ok])))
    return d / sig


@pytest.mark.parametrize("workload", ["telescope", "barrel"])
def test_two_filter_pulls_chi2_and_accuracy(workload, n_threads):
    w = (synth.telescope_workload(20000, seed=5, pmin=1.0, pmax=2.0) if workload == "telescope"
         else synth.barrel_workload(n_events=1, lo=8000, hi=8000, seed=2))
    rts = oracle.fit_tracks(w, oracle.Options(mass=w.mass), n_threads=n_threads)
    tf = oracle.fit_tracks(w, oracle.Options(mass=w.mass, smoother=1), n_threads=n_threads)
    assert np.array_equal(rts.status, tf.status)
    np.testing.assert_array_equal(rts.chi2, tf.chi2)  # the forward filter's chi2
    pull = _errors(w, tf)
    assert np.all(np.abs(pull.mean(0)) < 0.04)
    assert np.all(np.abs(pull.std(0) - 1.0) < 0.03), pull.std(0)
    # as accurate as RTS: the r.m.s. error in units of the RTS sigma within 1 %
    e_rts = np.sqrt((_errors(w, rts) ** 2).mean(0))
    e_tf = np.sqrt((_errors(w, tf, sigma_from=rts) ** 2).mean(0))
    assert np.all(np.abs(e_tf / e_rts - 1.0) < 0.01), (e_rts, e_tf)
    # the same weights up to the start's residual information and the linearisation
    ok = rts.status == 0
    sr = np.sqrt(np.einsum("nii->ni", oracle.unpack(rts.cov[ok])))
    st = np.sqrt(np.einsum("nii->ni", oracle.unpack(tf.cov[ok])))
    assert np.all(np.abs(np.median(st / sr, 0) - 1.0) < 5e-3)
