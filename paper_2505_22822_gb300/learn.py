"""Training harness of the learned step proposer: argument marshalling around the library's
record-capture, initialisation, training, calibration and BF16-loading calls (every step's
arithmetic runs in the library's kernels).

1. ``record_steps``: fit a batch with the plain adaptive stepper and capture, for every accepted
   RKN step that the step-size control limited, the network inputs and the label
   ln(|h| (tol/eps)^(1/4)) (the largest step within tolerance at the step's error constant).
2. ``train``: seeded initialisation (tkf_mlp_init), then mean-squared-error regression of the
   label with Adam (tkf_mlp_train) on the shuffled records.
3. ``calibrate``: shift the output bias to a low quantile of the training residuals
   (tkf_mlp_calibrate), so that a proposal (0.9 exp(output)) rarely exceeds the largest step
   within tolerance: a rejected proposal costs a step attempt, a short one only a little length.
4. ``build_proposer``: the three above, then the BF16 handle (tkf_mlp_load_f32 rounds on the
   device).
"""

from __future__ import annotations

from . import MLP_PARAMS, MLP_RECORD, Mlp, Options, STEP_ADAPTIVE, fit, mlp_calibrate, mlp_init, mlp_train


def record_steps(ctx, geo, field, batch, precision: int, capacity: int = 2_000_000, mass=None, tol=None):
    """Training records [n, 13] (CUDA float32) from the plain stepper on ``batch``."""
    import torch
    dev = batch.offsets.device
    rec = torch.zeros((capacity, MLP_RECORD), dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    opts = Options(precision=precision, step_mode=STEP_ADAPTIVE, records=rec, record_count=cnt)
    if mass is not None:
        opts.mass = mass
    if tol is not None:
        opts.tol = tol
    fit(ctx, geo, field, batch, opts)
    torch.cuda.synchronize()
    n = min(int(cnt.item()), capacity)
    return rec[:n].contiguous()


def train(ctx, records, epochs: int = 8, batch: int = 1024, lr: float = 2e-3, seed: int = 7):
    """Shuffled records, seeded initial parameters, then ``epochs`` passes of Adam; returns the
    FP32 parameters (CUDA tensor) and the epoch losses (CUDA tensor)."""
    import torch
    g = torch.Generator(device=records.device)
    g.manual_seed(seed)
    rec = records[torch.randperm(records.shape[0], device=records.device, generator=g)].contiguous()
    p = torch.empty(MLP_PARAMS, dtype=torch.float32, device=records.device)
    mlp_init(ctx, p, seed)
    mom = torch.zeros((2, MLP_PARAMS), dtype=torch.float32, device=records.device)
    losses, _ = mlp_train(ctx, rec, p, mom, 0, batch=batch, epochs=epochs, lr=lr)
    torch.cuda.synchronize()
    return p, losses


def calibrate(ctx, params, records, quantile: float = 0.05) -> float:
    """Shifts the output bias of ``params`` (in place) by the ``quantile`` of (label - output)
    over the records; returns the shift."""
    return mlp_calibrate(ctx, params, records, quantile)


def build_proposer(ctx, geo, field, batch, precision: int, epochs: int = 8, quantile: float = 0.05,
                   mass=None, tol=None, max_records: int | None = None) -> tuple[Mlp, dict]:
    """Records (at the RKN tolerance `tol`, default the library's; at most ``max_records``) ->
    training -> calibration -> BF16 handle, with a summary of the run."""
    rec = record_steps(ctx, geo, field, batch, precision, mass=mass, tol=tol)
    if max_records is not None:
        rec = rec[:max_records]
    params, losses = train(ctx, rec, epochs=epochs)
    q = calibrate(ctx, params, rec, quantile)
    return Mlp.from_params(ctx, params), {"records": int(rec.shape[0]),
                                          "epoch_loss": [float(x) for x in losses.cpu()], "bias_shift": q}
