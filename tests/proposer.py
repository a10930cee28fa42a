"""Step-proposer weights made without the CUDA path, for the parity tests of the learned mode:
training records from the oracle's own plain adaptive fit of seed-disjoint tracks, FP64 Adam
training and calibration by the numpy reference (oracle/mlp.py), rounding to BF16 there. The
library's GPU training is checked separately against the same reference."""

import numpy as np

import oracle
import synth
from oracle import mlp


def oracle_trained_bf16(w, epochs: int = 8, seed: int = 7, quantile: float = 0.05,
                        max_records: int = 150_000) -> tuple[np.ndarray, dict]:
    """BF16 weights of a proposer trained on records of workload `w` (its own tracks, which the
    caller draws with a seed disjoint from every compared batch)."""
    t = w.tracks
    rec = oracle.record_steps(w.geometry.table, oracle.field_from(w.field), oracle.Options(mass=w.mass), t.offsets,
                              t.meas, t.sid, t.seed_par, t.seed_cov)
    rng = np.random.default_rng(seed)
    rec = rec[rng.permutation(len(rec))[:max_records]]
    X, y = rec[:, :12].astype(np.float64), rec[:, 12].astype(np.float64)
    theta, losses = mlp.train(mlp.init(seed), X, y, batch=256, epochs=epochs, lr=2e-3)
    theta, q = mlp.calibrate(theta, X, y, quantile)
    return mlp.to_bf16(theta), {"records": int(len(rec)), "losses": [float(x) for x in losses], "bias_shift": q}


def map_proposer(fld=None):
    """Trained on 4000 seed-disjoint muons in the solenoid map."""
    return oracle_trained_bf16(synth.solenoid_muon_workload(4000, seed=1000, fld=fld))


def barrel_proposer():
    """Trained on one seed-disjoint event of the barrel batch's kind."""
    return oracle_trained_bf16(synth.barrel_workload(n_events=1, seed=10_002))
