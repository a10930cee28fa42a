"""Checks of the seeded input generator (geometry, solenoid field map, simulation).

The field-map pins use the closed forms of an ideal finite solenoid: on the axis
B_z(0, z) = (mu0 n I / 2) [(z + b)/sqrt((z + b)^2 + a^2) - (z - b)/sqrt((z - b)^2 + a^2)], and
off the axis the field is divergence- and curl-free inside the coil.
"""

import numpy as np
import pytest

import synth

A, HALF = 1200.0, 2900.0


def test_cel_matches_quadrature_of_its_definition():
    integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(0)
    for _ in range(40):
        kc = rng.uniform(0.05, 1.5)
        p = rng.choice([rng.uniform(0.05, 2.0), rng.uniform(-0.9, -0.05)])
        c, s = rng.normal(size=2)

        def f(t):
            ct, st = np.cos(t) ** 2, np.sin(t) ** 2
            return (c * ct + s * st) / ((ct + p * st) * np.sqrt(ct + kc * kc * st))

        if p < 0:  # principal value; compare only where the integrand has no pole
            continue
        ref = integrate.quad(f, 0, np.pi / 2, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
        assert abs(synth.cel(kc, p, c, s) - ref) < 1e-11 * max(1.0, abs(ref))


def test_solenoid_on_axis_closed_form():
    zs = np.linspace(-3500, 3500, 57)
    raw = np.array([synth.solenoid_raw(A, HALF, 0.0, z) for z in zs])
    # raw unit is mu0 n I / pi, so the closed form is (pi/2) [...]
    ref = 0.5 * np.pi * ((zs + HALF) / np.hypot(zs + HALF, A) - (zs - HALF) / np.hypot(zs - HALF, A))
    np.testing.assert_allclose(raw[:, 1], ref, rtol=1e-12, atol=1e-14)
    assert np.all(np.abs(raw[:, 0]) < 1e-14)


def test_solenoid_field_is_divergence_and_curl_free_inside():
    rng = np.random.default_rng(1)
    d = 1e-3
    for _ in range(30):
        r, z = rng.uniform(50, 1100), rng.uniform(-2800, 2800)
        br = lambda rr, zz: synth.solenoid_raw(A, HALF, rr, zz)[0]
        bz = lambda rr, zz: synth.solenoid_raw(A, HALF, rr, zz)[1]
        div = ((r + d) * br(r + d, z) - (r - d) * br(r - d, z)) / (2 * d * r) + \
              (bz(r, z + d) - bz(r, z - d)) / (2 * d)
        curl = (br(r, z + d) - br(r, z - d)) / (2 * d) - (bz(r + d, z) - bz(r - d, z)) / (2 * d)
        scale = abs(bz(r, z)) / 1000.0
        assert abs(div) < 1e-6 * scale + 1e-12
        assert abs(curl) < 1e-6 * scale + 1e-12


def test_solenoid_map_grid_and_scale():
    f = synth.solenoid_map()
    assert (f.nr, f.nz) == (241, 1401)
    j0 = (f.nz - 1) // 2
    assert abs(f.Bz[j0, 0] - 2.0) < 1e-6
    assert np.all(np.isfinite(f.Br)) and np.all(np.isfinite(f.Bz))
    # uniform to a few per cent inside the tracker volume near the centre
    assert np.all(np.abs(f.Bz[j0 - 100:j0 + 100, :150] - 2.0) < 0.05)


def test_geometry_frames_are_proper_rotations():
    for g in (synth.telescope_geometry(), synth.barrel_endcap_geometry()):
        R = g.rotation().reshape(-1, 3, 3)
        np.testing.assert_allclose(np.einsum("nji,njk->nik", R, R), np.broadcast_to(np.eye(3), R.shape),
                                   atol=1e-14)
        np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)
    g = synth.barrel_endcap_geometry()
    assert 30000 < g.n < 45000


def test_simulation_is_seeded_and_respects_hit_limits():
    g = synth.barrel_endcap_geometry()
    f = synth.uniform_field(2.0)
    counts = synth.event_counts(2, 50, 2000, 20000)
    assert counts.min() >= 2000 and counts.max() <= 20000
    a = synth.simulate(g, f, synth.barrel_params(), 2, [300, 200], n_threads=3)
    b = synth.simulate(g, f, synth.barrel_params(), 2, [300, 200], n_threads=1)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.meas, b.meas)
    n = a.hits_per_track()
    assert n.min() >= 6 and n.max() <= 18
    assert a.sid.max() < g.n
    # hits lie inside their modules
    half = g.table[a.sid, 14:16]
    assert np.all(np.abs(a.hit_truth) <= half + 1e-9)
