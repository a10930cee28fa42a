"""Element-wise comparison of a GPU fit with the CPU oracle (test infrastructure).

Metric (the first-surface smoothed state is a difference of terms of the size of the
filtered covariance C_0|0, so that is the scale of rounding differences between two correct
FP64 evaluations):
  parameters   |dp_i|   <= tol * max(|p_i|, sigma_i)      (phi difference wrapped)
  covariance   |dC_ij|  <= tol * sqrt(C0_ii C0_jj)         (C0 = filtered cov at surface 0)
  chi2         |dchi2|  <= tol * max(chi2, 1)
  status, ndf  identical
"""

import numpy as np

import oracle


def gpu_to_track_major(res):
    """paper_2505_22822_gb300.Result (torch or numpy, SoA) -> dict of numpy track-major arrays."""
    def host(x):
        if x is None:
            return None
        if hasattr(x, "detach"):
            x = x.detach().cpu().numpy()
        return np.asarray(x)
    out = {"par": host(res.par).T.copy(), "cov": host(res.cov).T.copy(), "chi2": host(res.chi2),
           "ndf": host(res.ndf).astype(np.int64), "status": host(res.status).astype(np.uint32)}
    st = host(res.steps)
    out["steps"] = st.T.astype(np.uint32) if st is not None else None
    return out


def compare(g: dict, o: "oracle.FitResult", tol: float, idx=None):
    """Returns (ok mask over compared tracks, same-step-sequence mask, stats dict); stats["dev"]
    is each track's largest deviation in the metric above."""
    if idx is None:
        idx = np.arange(o.par.shape[0])
    gp, gc, gx = g["par"][idx], g["cov"][idx], g["chi2"][idx]
    op, oc, ox = o.par, o.cov, o.chi2
    if op.shape[0] != len(idx):
        op, oc, ox = op[idx], oc[idx], ox[idx]
        ocf, ost, ondf = o.cov_filt0[idx], o.status[idx], o.ndf[idx]
        osteps = o.steps[idx]
    else:
        ocf, ost, ondf, osteps = o.cov_filt0, o.status, o.ndf, o.steps
    status_eq = g["status"][idx] == ost
    ndf_eq = g["ndf"][idx] == ondf
    good = status_eq & ((ost & 0x39F) == 0)  # fatal bits clear on both
    C = oracle.unpack(oc)
    sig = np.sqrt(np.abs(np.einsum("nii->ni", C)))
    dp = gp - op
    dp[:, 2] = (dp[:, 2] + np.pi) % (2 * np.pi) - np.pi
    rel_p = np.abs(dp) / np.maximum(np.abs(op), sig)
    C0 = oracle.unpack(ocf)
    C0 = np.where(np.isfinite(C0), C0, C)  # no filtered state (N = 0): the seed covariance
    d0 = np.sqrt(np.abs(np.einsum("nii->ni", C0)))
    scale = np.einsum("ni,nj->nij", d0, d0)
    rel_c = np.abs(oracle.unpack(gc) - C) / scale
    rel_x = np.abs(gx - ox) / np.maximum(np.abs(ox), 1.0)
    rp = np.where(good[:, None], rel_p, 0).max(1)
    rc = np.where(good[:, None, None], rel_c, 0).reshape(len(idx), -1).max(1)
    rx = np.where(good, rel_x, 0)
    # a track that failed on both sides must be NaN on the GPU too
    nan_ok = good | ~status_eq | ((ost & 0x39F) == 0) | np.all(np.isnan(gp), axis=1)
    ok = status_eq & ndf_eq & (rp <= tol) & (rc <= tol) & (rx <= tol) & nan_ok
    dev = np.maximum(np.maximum(rp, rc), rx)
    same_steps = None
    if g.get("steps") is not None:
        same_steps = np.all(g["steps"][idx] == osteps, axis=1)
    stats = {
        "n": int(len(idx)), "ok": int(ok.sum()), "status_mismatch": int((~status_eq).sum()),
        "dev": dev,
        "max_rel_par": float(rp.max()) if len(rp) else 0.0,
        "max_rel_cov": float(rc.max()) if len(rc) else 0.0,
        "max_rel_chi2": float(rx.max()) if len(rx) else 0.0,
        "same_steps": int(same_steps.sum()) if same_steps is not None else None,
        "dp_over_sigma_max": float(np.where(good[:, None], np.abs(dp) / np.maximum(sig, 1e-300), 0).max())
        if len(idx) else 0.0,
    }
    return ok, same_steps, stats


def self_sensitivity(w, track: int, trials: int = 8, seed: int = 0, opts=None) -> float:
    """How far the oracle's own result for one track moves, in the metric above, when its seed
    parameters and measured positions change by one unit in the last place (random signs): the
    resolution to which the track's FP64 result is determined at all. Two correct FP64
    evaluations in different orders cannot be expected to agree more closely than this."""
    t = w.tracks
    sub = t.subset(np.array([track]))
    fo = oracle.field_from(w.field)
    opts = opts or oracle.Options(mass=w.mass)
    base = oracle.fit(w.geometry.table, fo, opts, sub.offsets, sub.meas, sub.sid, sub.seed_par, sub.seed_cov)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(trials):
        sp = sub.seed_par * (1 + rng.choice([-1.0, 1.0], size=sub.seed_par.shape) * 2.0 ** -52)
        m = sub.meas.copy()
        m[:, :2] *= 1 + rng.choice([-1.0, 1.0], size=m[:, :2].shape) * 2.0 ** -52
        o = oracle.fit(w.geometry.table, fo, opts, sub.offsets, m, sub.sid, sp, sub.seed_cov)
        g = {"par": o.par, "cov": o.cov, "chi2": o.chi2, "ndf": o.ndf.astype(np.int64), "status": o.status,
             "steps": o.steps}
        if not np.array_equal(o.steps, base.steps):
            continue  # a different step sequence is another comparison
        _, _, st = compare(g, base, np.inf)
        worst = max(worst, float(st["dev"][0]))
    return worst


def chain_self_sensitivity(w, tracks, scale: float = 100.0, trials: int = 32, seed: int = 0,
                           n_threads: int = 8) -> np.ndarray:
    """The same for the chain estimated seeds -> fit -> refit (covariance multiplied by
    `scale`), for each of the `tracks` (indices into the workload): how far the oracle's chain
    result moves when the measured positions, the estimated seeds and the first fit's result
    each change by one unit in the last place (every hand-off between the stages is a place
    where another correct FP64 evaluation order rounds differently). The tracks are perturbed
    together, `trials` times; a trial that changes a track's step sequence does not count for
    that track."""
    t = w.tracks
    sub = t.subset(np.asarray(tracks, dtype=np.int64))
    fo = oracle.field_from(w.field)
    opts = oracle.Options(mass=w.mass)
    table = w.geometry.table

    def ulp(x, rng):
        return x * (1 + rng.choice([-1.0, 1.0], size=x.shape) * 2.0 ** -52) if rng is not None else x

    def run(rng=None):
        meas = sub.meas.copy()
        meas[:, :2] = ulp(meas[:, :2], rng)
        sp, sc, _ = oracle.estimate_seeds(table, fo, sub.offsets, meas, sub.sid)
        r1 = oracle.fit(table, fo, opts, sub.offsets, meas, sub.sid, ulp(sp, rng), ulp(sc, rng), n_threads=n_threads)
        return oracle.fit(table, fo, opts, sub.offsets, meas, sub.sid, ulp(r1.par, rng), ulp(r1.cov, rng) * scale,
                          n_threads=n_threads)

    base = run()
    rng = np.random.default_rng(seed)
    worst = np.zeros(sub.n_tracks)
    for _ in range(trials):
        o = run(rng)
        same = np.all(o.steps == base.steps, axis=1)
        g = {"par": o.par, "cov": o.cov, "chi2": o.chi2, "ndf": o.ndf.astype(np.int64), "status": o.status,
             "steps": o.steps}
        _, _, st = compare(g, base, np.inf)
        worst = np.where(same, np.maximum(worst, st["dev"]), worst)
    return worst


def states_to_entry_major(res):
    """The all-states output of a GPU result (SoA [5][n_meas], [15][n_meas]) -> entry-major numpy."""
    def host(x):
        return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    return host(res.states_par).T.copy(), host(res.states_cov).T.copy()


def compare_states(sp, sc, o: "oracle.FitResult", offsets):
    """Every entry's smoothed state against the oracle's (`o` from oracle.fit(..., states=True)),
    in the metric above with the entry's own filtered covariance as the covariance scale (the
    backward pass at entry k subtracts terms of that size). Returns each track's largest
    deviation (0 for tracks whose rows are NaN on both sides) and whether NaN rows agree."""
    offsets = np.asarray(offsets, dtype=np.int64)
    op, oc, ocf = o.states_par, o.states_cov, o.states_cov_filt
    with np.errstate(invalid="ignore", divide="ignore"):
        return _compare_states(sp, sc, op, oc, ocf, offsets)


def _compare_states(sp, sc, op, oc, ocf, offsets):
    nan_g = np.isnan(sp).any(1)
    nan_o = np.isnan(op).any(1)
    C = unpack_safe(oc)
    sig = np.sqrt(np.abs(np.einsum("nii->ni", C)))
    dp = sp - op
    dp[:, 2] = (dp[:, 2] + np.pi) % (2 * np.pi) - np.pi
    rel_p = np.abs(dp) / np.maximum(np.abs(op), sig)
    Cf = unpack_safe(ocf)
    d0 = np.sqrt(np.abs(np.einsum("nii->ni", Cf)))
    rel_c = np.abs(unpack_safe(sc) - C) / np.einsum("ni,nj->nij", d0, d0)
    dev_e = np.maximum(rel_p.max(1), rel_c.reshape(len(sp), -1).max(1))
    dev_e = np.where(nan_g & nan_o, 0.0, dev_e)
    dev_e = np.where(nan_g != nan_o, np.inf, dev_e)
    n = len(offsets) - 1
    dev_t = np.zeros(n)
    if len(dev_e):
        idx = np.repeat(np.arange(n), np.diff(offsets))
        np.maximum.at(dev_t, idx, np.nan_to_num(dev_e, nan=np.inf))
    return dev_t, bool(np.array_equal(nan_g, nan_o))


def unpack_safe(cov15):
    return oracle.unpack(np.nan_to_num(cov15, nan=0.0)) if len(cov15) else np.zeros((0, 5, 5))


def states_self_sensitivity(w, track: int, trials: int = 8, seed: int = 0, opts=None) -> float:
    """`self_sensitivity` for every entry's smoothed state: how far the oracle's all-states
    result of one track moves under one-ulp changes of its seed and measured positions."""
    t = w.tracks
    sub = t.subset(np.array([track]))
    fo = oracle.field_from(w.field)
    opts = opts or oracle.Options(mass=w.mass)
    base = oracle.fit(w.geometry.table, fo, opts, sub.offsets, sub.meas, sub.sid, sub.seed_par, sub.seed_cov,
                      states=True)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(trials):
        sp = sub.seed_par * (1 + rng.choice([-1.0, 1.0], size=sub.seed_par.shape) * 2.0 ** -52)
        m = sub.meas.copy()
        m[:, :2] *= 1 + rng.choice([-1.0, 1.0], size=m[:, :2].shape) * 2.0 ** -52
        o = oracle.fit(w.geometry.table, fo, opts, sub.offsets, m, sub.sid, sp, sub.seed_cov, states=True)
        if not np.array_equal(o.steps, base.steps):
            continue
        dev, _ = compare_states(o.states_par, o.states_cov, base, sub.offsets)
        worst = max(worst, float(dev[0]))
    return worst
