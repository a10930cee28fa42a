"""Pins of the oracle's entries without a measurement (holes in sensitive modules, passive
surfaces: Sec. 2's navigation through every crossed surface). Such an entry carries the surface
id with bit 31 set; the fit propagates to it and applies its material, and makes no update.
The simulation marks a crossing as a hole with a given probability (its material still acts)
and writes NaN into the entry's measurement fields, so any read of them would show."""

import numpy as np
import pytest

import oracle
import synth

HOLE = np.uint32(0x80000000)
TOO_FEW_HITS = 1 << 5


def drop_holes(t):
    """The same tracks with their hole entries removed (what a fit without navigation sees)."""
    keep = (t.sid & HOLE) == 0
    counts = np.array([keep[a:b].sum() for a, b in zip(t.offsets[:-1], t.offsets[1:])], dtype=np.int64)
    offs = np.zeros(t.n_tracks + 1, np.uint32)
    offs[1:] = np.cumsum(counts)
    return synth.Tracks(offs, t.sid[keep], t.meas[keep], t.hit_truth[keep], t.truth, t.seed_par, t.seed_cov,
                        t.truth_last, t.event)


def _fit(w, t, **kw):
    return oracle.fit(w.geometry.table, oracle.field_from(w.field), oracle.Options(mass=w.mass, **kw), t.offsets,
                      t.meas, t.sid, t.seed_par, t.seed_cov, n_threads=8)


def _pulls(w, r):
    ok = r.status == 0
    sig = np.sqrt(np.einsum("nii->ni", oracle.unpack(r.cov[ok])))
    d = r.par[ok] - w.tracks.truth[ok]
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    return d / sig, r.chi2[ok] / r.ndf[ok]


def test_simulated_holes():
    w = synth.solenoid_muon_workload(2000, seed=11, p_hole=0.2)
    t = w.tracks
    hole = (t.sid & HOLE) != 0
    assert 0.15 < hole.mean() < 0.22
    assert np.all(np.isnan(t.meas[hole])) and np.all(np.isfinite(t.meas[~hole]))
    assert not np.any(hole[t.offsets[:-1]])  # the first entry is always measured
    # without holes asked for, nothing changes (no extra random draws)
    a = synth.solenoid_muon_workload(500, seed=11).tracks
    b = synth.solenoid_muon_workload(500, seed=11, p_hole=0.0).tracks
    np.testing.assert_array_equal(a.meas, b.meas)


def test_holes_keep_unit_pulls_and_dropping_them_does_not():
    """Muons in the solenoid map, 20 % of the crossings after the first without a measurement:
    with the holes' material the pulls are unit normal and chi2/ndf is 1; a fit that never sees
    the holes misses their scattering (q/p pull width 1.10, chi2/ndf 1.06)."""
    w = synth.solenoid_muon_workload(20_000, seed=11, p_hole=0.2)
    r = _fit(w, w.tracks)
    assert np.all(r.status == 0)
    pulls, chi2ndf = _pulls(w, r)
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.02), pulls.std(0)
    assert np.all(np.abs(pulls.mean(0)) < 0.03), pulls.mean(0)
    assert abs(chi2ndf.mean() - 1.0) < 0.01
    nd = 2 * np.array([((w.tracks.sid[a:b] & HOLE) == 0).sum()
                       for a, b in zip(w.tracks.offsets[:-1], w.tracks.offsets[1:])])
    np.testing.assert_array_equal(r.ndf, nd)
    rd = _fit(w, drop_holes(w.tracks))
    pd, cd = _pulls(w, rd)
    assert pd.std(0)[4] > 1.05 and cd.mean() > 1.03, (pd.std(0), cd.mean())


def test_noise_free_tracks_with_holes_fit_back_to_truth():
    """No scattering and no hit noise, but energy loss in every crossed module: the fit with the
    holes' material returns the truth; without them q/p misses the holes' energy loss."""
    w = synth.barrel_workload(n_events=1, lo=500, hi=500, seed=21, mass=synth.MUON_MASS, ms=0, sigma_hit=0.0,
                              seed_smear=0, p_hole=0.3)
    t = w.tracks
    assert np.mean((t.sid & HOLE) != 0) > 0.2
    r = _fit(w, t, tol=1e-9)
    assert np.all(r.status == 0)
    d = r.par - t.truth
    assert np.max(np.abs(d[:, :2])) < 1e-7
    assert np.max(np.abs(d[:, 2:4])) < 1e-8
    assert np.max(np.abs(d[:, 4] / t.truth[:, 4])) < 1e-7
    rd = _fit(w, drop_holes(t), tol=1e-9)
    assert np.max(np.abs(rd.par[:, 4] / t.truth[:, 4] - 1.0)) > 1e-5


def test_entry_counts_status_and_seed_only_tracks():
    """ndf counts measurements only; fewer than 3 measurements flag TOO_FEW_HITS; a track whose
    entries are all holes returns its seed; a hole as the first entry carries the seed."""
    w = synth.telescope_workload(6, seed=3)
    t = w.tracks
    sid = t.sid.astype(np.uint32).copy()
    meas = t.meas.copy()
    a = t.offsets.astype(np.int64)

    def hole(e):
        sid[e] |= HOLE
        meas[e] = np.nan

    for e in range(a[1] + 1, a[1] + 8):  # track 1: 2 measurements of 9
        hole(e)
    for e in range(a[2], a[3]):          # track 2: no measurement
        hole(e)
    hole(a[3])                           # track 3: the first entry is a hole
    hole(a[4] + 4)                       # track 4: one hole in the middle
    r = oracle.fit(w.geometry.table, oracle.field_from(w.field), oracle.Options(mass=w.mass), t.offsets, meas, sid,
                   t.seed_par, t.seed_cov)
    np.testing.assert_array_equal(r.ndf, [18, 4, 0, 16, 16, 18])
    assert list(r.status) == [0, TOO_FEW_HITS, TOO_FEW_HITS, 0, 0, 0]
    np.testing.assert_array_equal(r.par[2], t.seed_par[2])
    np.testing.assert_array_equal(r.cov[2], t.seed_cov[2])
    assert r.chi2[2] == 0.0
    assert np.all(np.isfinite(r.par[[0, 1, 3, 4, 5]]))
    # a surface id out of range is bad input with or without the bit
    sid2 = t.sid.astype(np.uint32).copy()
    sid2[a[5] + 2] = HOLE | np.uint32(5000)
    r2 = oracle.fit(w.geometry.table, oracle.field_from(w.field), oracle.Options(mass=w.mass), t.offsets, t.meas, sid2,
                    t.seed_par, t.seed_cov)
    assert r2.status[5] == 1 << 7


@pytest.mark.parametrize("first_three", [False, True])
def test_seeds_skip_holes(first_three):
    """Seed estimation takes its three space points from measured entries only: noise-free
    helices with holes give the truth; a first entry without a measurement is bad input."""
    w = synth.barrel_workload(n_events=1, lo=1000, hi=1000, seed=21, sigma_hit=0.0, ms=0, eloss=0, seed_smear=0,
                              p_hole=0.3)
    t = w.tracks
    fld = oracle.field_from(w.field)
    par, _, st = oracle.estimate_seeds(w.geometry.table, fld, t.offsets, t.meas, t.sid, first_three=first_three)
    ok = st == 0
    assert ok.mean() > 0.99 and np.all(st[~ok] == 1)  # a few tracks keep fewer than 3 measurements
    d = par[ok] - t.truth[ok]
    d[:, 2] = (d[:, 2] + np.pi) % (2 * np.pi) - np.pi
    assert np.median(np.abs(d[:, 4] / t.truth[ok, 4])) < 1e-9
    assert np.max(np.abs(d[:, 2:4])) < 1e-7
    sid = t.sid.astype(np.uint32).copy()
    sid[t.offsets[0]] |= HOLE
    _, _, st2 = oracle.estimate_seeds(w.geometry.table, fld, t.offsets, t.meas, sid, first_three=first_three)
    assert st2[0] == 4
