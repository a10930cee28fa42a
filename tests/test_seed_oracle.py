"""Pins of the oracle's seed parameter estimation (the helix through a track's first three
measurements, Sec. 2): analytic helices written from the Lorentz force, the sagitta formula,
straight lines, noise-free simulated tracks whose truth is known, and the degenerate inputs."""

import numpy as np
import pytest

import oracle
import synth

KAPPA = 2.99792458e-4  # GeV / (T mm) per unit charge


def _helix_points(q, p, theta, phi0, bz, s_list, r0=(0.0, 0.0, 0.0)):
    """Points at 3D path lengths s of the solution of dT/ds = (q/p) kappa T x B for B = (0, 0, bz):
    the transverse direction angle turns at omega = -kappa (q/p) bz per unit path. The
    differences of sines and cosines are taken as products (no cancellation at large radius)."""
    w = -KAPPA * (q / p) * bz
    st, ct = np.sin(theta), np.cos(theta)
    out = []
    for s in s_list:
        half = 0.5 * w * s
        chord = 2.0 * st / w * np.sin(half)  # transverse chord length
        x = r0[0] + chord * np.cos(phi0 + half)
        y = r0[1] + chord * np.sin(phi0 + half)
        out.append(np.array([x, y, r0[2] + s * ct]))
    return out


def test_analytic_helices_are_recovered_exactly():
    rng = np.random.default_rng(5)
    for _ in range(400):
        q = rng.choice([-1.0, 1.0])
        bz = rng.choice([-2.0, -0.5, 0.5, 2.0, 4.0])
        theta = rng.uniform(0.05, np.pi - 0.05)
        phi0 = rng.uniform(-np.pi, np.pi)
        p = np.exp(rng.uniform(np.log(0.3), np.log(200.0)))
        R = p * np.sin(theta) / (KAPPA * abs(bz))
        # hit 3 within 0.95 of a full turn of the transverse circle, hit 2 between
        s_turn = 2 * np.pi * R / np.sin(theta)
        s3 = min(rng.uniform(50.0, 1500.0), rng.uniform(0.02, 0.95) * s_turn)
        s2 = rng.uniform(0.1, 0.9) * s3
        r = _helix_points(q, p, theta, phi0, bz, [0.0, s2, s3], r0=rng.normal(0, 100, 3))
        out, st = oracle.helix_seed(r[0], r[1], r[2], bz)
        assert st == 0
        dphi = (out[0] - phi0 + np.pi) % (2 * np.pi) - np.pi
        assert abs(dphi) < 1e-9, (dphi, p, theta)
        assert abs(out[1] - theta) < 1e-9, (out[1], theta, p)
        # the curvature comes from the sagitta of hits 1-3: rounding of the coordinates (one ulp
        # of their magnitude) moves it by that much, which bounds the relative error of q/p
        chord = np.hypot(*(r[2] - r[0])[:2])
        sagitta = chord * chord / (R + np.sqrt(max(R * R - 0.25 * chord * chord, 0.0))) / 2
        scale = max(np.abs(np.concatenate(r)).max(), 1.0)
        tol = 1e-10 + 16 * np.finfo(float).eps * scale / sagitta
        assert abs(out[2] * p / q - 1.0) < tol, (out[2], q / p, tol)


def test_sagitta_formula_and_charge_sign():
    """Chord 2L along +x with the middle hit raised by the sagitta s: R = (L^2 + s^2) / (2 s).
    The track turns clockwise seen from +z, which in B_z > 0 is a positive charge (F = q v x B
    points to -y for v along +x)."""
    L, s, bz = 400.0, 3.0, 2.0
    R = (L * L + s * s) / (2 * s)
    out, st = oracle.helix_seed([0, 0, 0], [L, s, 0], [2 * L, 0, 0], bz)
    assert st == 0
    pt = KAPPA * bz * R
    np.testing.assert_allclose(out[2], 1.0 / pt, rtol=1e-12)  # theta = pi/2: p = pT, q = +1
    np.testing.assert_allclose(out[1], np.pi / 2, atol=1e-15)
    np.testing.assert_allclose(out[0], np.arctan2(L, R - s), rtol=1e-12)  # tangent at hit 1
    out_neg, _ = oracle.helix_seed([0, 0, 0], [L, s, 0], [2 * L, 0, 0], -bz)
    assert out_neg[2] == -out[2]
    out_mirror, _ = oracle.helix_seed([0, 0, 0], [L, -s, 0], [2 * L, 0, 0], bz)
    assert out_mirror[2] == pytest.approx(-out[2], rel=1e-12)
    # with a longitudinal slope: p = pT / sin(theta)
    dz = 150.0
    arc = 2 * R * np.arcsin(L / R)
    out_z, _ = oracle.helix_seed([0, 0, 0], [L, s, 0.5 * dz], [2 * L, 0, dz], bz)
    th = np.arctan2(arc, dz)
    np.testing.assert_allclose(out_z[1], th, rtol=1e-12)
    np.testing.assert_allclose(out_z[2], np.sin(th) / pt, rtol=1e-12)


def test_straight_lines_and_zero_field_have_no_curvature():
    out, st = oracle.helix_seed([1, 2, 3], [101, 52, 23], [301, 152, 63], 2.0)
    assert st == 2 and out[2] == 0.0
    np.testing.assert_allclose(out[0], np.arctan2(150, 300), rtol=1e-14)
    np.testing.assert_allclose(out[1], np.arctan2(np.hypot(300, 150), 60), rtol=1e-14)
    out, st = oracle.helix_seed([0, 0, 0], [400, 3, 0], [800, 0, 0], 0.0)
    assert st == 2 and out[2] == 0.0
    np.testing.assert_allclose(out[0], 0.0, atol=0)


def _noise_free(workload_fn, **kw):
    return workload_fn(sigma_hit=0.0, ms=0, eloss=0, seed_smear=0, **kw)


def _seed_points(w, first_three):
    """Global positions [n, 3, 3] (r = c + l0 u + l1 v) of the measurements a seed is made of: the
    first, middle and last of every track, or its first three."""
    t, g = w.tracks, w.geometry
    a = t.offsets[:-1].astype(np.int64)
    n = np.diff(t.offsets.astype(np.int64))
    k = a[:, None] + (np.arange(3) if first_three else np.stack([0 * n, (n - 1) // 2, n - 1], 1))
    s = t.sid[k]
    return (g.table[s, 9:12] + t.meas[k, 0, None] * g.table[s, 0:3] + t.meas[k, 1, None] * g.table[s, 3:6])


def _qop_tolerance(w, bz, first_three):
    """Relative q/p error that rounding of the simulated hit positions can cause, over the sagitta
    of hits 1-3 (hits in overlapping modules of one layer are millimetres apart, and their
    sagitta is far below a micron): one ulp of the coordinates, plus the generator's helix steps
    (40 mm each from the vertex), whose (1 - cos(a s)) / a term is rounded by eps R at radius R."""
    t = w.tracks
    r = _seed_points(w, first_three)
    R = np.sin(t.truth[:, 3]) / np.abs(t.truth[:, 4]) / (KAPPA * abs(bz))
    chord = np.hypot(*(r[:, 2, :2] - r[:, 0, :2]).T)
    sagitta = chord * chord / (R + np.sqrt(R * R - 0.25 * chord * chord)) / 2
    scale = np.abs(r).max(axis=(1, 2))
    return 1e-9 + 64 * np.finfo(float).eps * (scale + R * (1.0 + scale / 40.0)) / sagitta


@pytest.mark.parametrize("first_three", [False, True])
def test_noise_free_barrel_tracks_give_their_truth(first_three):
    """Exact helices in the uniform 2 T field, no material, no hit noise: the seeds equal the
    simulated truth at the first measurement, whichever three measurements they are made of."""
    w = _noise_free(lambda **k: synth.barrel_workload(n_events=1, lo=3000, hi=3000, seed=21, **k))
    t = w.tracks
    par, cov, st = oracle.estimate_seeds(w.geometry.table, oracle.field_from(w.field), t.offsets, t.meas, t.sid,
                                         first_three=first_three)
    assert np.all(st == 0)
    d = par - t.truth
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    assert np.max(np.abs(d[:, :4])) < 1e-8, np.max(np.abs(d[:, :4]), 0)
    rel = np.abs(d[:, 4] / t.truth[:, 4])
    assert np.median(rel) < 1e-9
    tol = _qop_tolerance(w, 2.0, first_three)
    assert np.all(rel < tol), np.max(rel / tol)
    # the covariance is a positive diagonal prior
    C = oracle.unpack(cov)
    assert np.all(np.linalg.eigvalsh(C) > 0)


def test_noise_free_telescope_tracks_give_their_truth():
    """Planes normal to x at 50 mm spacing, B along z: the helix axis is across the planes' normals."""
    w = synth.telescope_workload(500, seed=4, sigma_hit=0.0, ms=0, eloss=0, seed_smear=0)
    t = w.tracks
    par, _, st = oracle.estimate_seeds(w.geometry.table, oracle.field_from(w.field), t.offsets, t.meas, t.sid)
    assert np.all(st == 0)
    d = par - t.truth
    assert np.max(np.abs(d[:, :4])) < 1e-9
    assert np.all(np.abs(d[:, 4] / t.truth[:, 4]) < _qop_tolerance(w, 2.0, False))


def test_degenerate_inputs():
    w = synth.telescope_workload(4, seed=4)
    t = w.tracks
    offsets = t.offsets.astype(np.uint32).copy()
    sid = t.sid.astype(np.uint32).copy()
    offsets[1] = 2  # track 0 keeps two hits
    sid[offsets[2]] = 10_000  # track 2: first hit on a surface that does not exist
    offsets = np.concatenate([offsets, [offsets[-1] - 1]]).astype(np.uint32)  # track 4: decreasing
    par, cov, st = oracle.estimate_seeds(w.geometry.table, oracle.field_from(w.field), offsets, t.meas, sid)
    assert list(st) == [1, 0, 4, 0, 4]
    assert np.all(np.isnan(par[[0, 2, 4]])) and np.all(cov[[0, 2, 4]] == 0)
    assert np.all(np.isfinite(par[[1, 3]]))


@pytest.mark.parametrize("workload", ["map", "barrel", "telescope"])
def test_smeared_seeds_are_covered_by_their_covariance(workload):
    """With hit noise, multiple scattering and energy loss (and the solenoid map's varying field)
    the seeds scatter about the truth within the prior they carry, which is meant to be wide
    rather than narrow: every pull's spread is below 1.1 and almost no pull exceeds 4."""
    w = {"map": lambda: synth.solenoid_muon_workload(4000, seed=7),
         "barrel": lambda: synth.barrel_workload(n_events=1, lo=4000, hi=4000, seed=21),
         "telescope": lambda: synth.telescope_workload(2000, seed=4)}[workload]()
    t = w.tracks
    par, cov, st = oracle.estimate_seeds(w.geometry.table, oracle.field_from(w.field), t.offsets, t.meas, t.sid)
    assert np.all(st == 0)
    d = par - t.truth
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    sig = np.sqrt(np.einsum("nii->ni", oracle.unpack(cov)))
    pulls = d / sig
    assert np.all(pulls.std(0) < 1.1), pulls.std(0)
    assert np.mean(np.abs(pulls) > 4) < 2e-3, np.mean(np.abs(pulls) > 4, 0)


def test_first_middle_last_beats_first_three():
    """The longer lever arm of the first, middle and last measurements: on the barrel batch the
    median relative q/p error of the seeds drops from above 10 % to below 1 %."""
    w = synth.barrel_workload(n_events=1, lo=4000, hi=4000, seed=21)
    t = w.tracks
    f = oracle.field_from(w.field)
    med = {}
    for ft in (False, True):
        par, _, _ = oracle.estimate_seeds(w.geometry.table, f, t.offsets, t.meas, t.sid, first_three=ft)
        med[ft] = np.median(np.abs(par[:, 4] / t.truth[:, 4] - 1.0))
    assert med[False] < 0.01 < 0.1 < med[True], med
