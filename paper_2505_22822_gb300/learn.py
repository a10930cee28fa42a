"""Training harness of the learned step proposer (argument marshalling around the library's
record-capture, training and forward kernels).

1. ``record_steps``: fit a batch with the plain adaptive stepper and capture, for every accepted
   RKN step, the network inputs and the label ln(|h| (tol/eps)^(1/4)) (the largest step within
   tolerance at the step's error constant).
2. ``train``: mean-squared-error regression of the label with Adam on the GPU.
3. ``calibrate``: shift the output bias to a low quantile of the training residuals, so that a
   proposal (0.9 exp(output)) rarely exceeds the largest step within tolerance: a rejected
   proposal costs a step attempt, while a short one costs only a little length.
4. ``to_bf16``: round to the BF16 weights that ``Mlp`` loads.
"""

from __future__ import annotations

import numpy as np

from . import MLP_PARAMS, Mlp, Options, STEP_ADAPTIVE, fit, mlp_forward, mlp_train

N_IN, N_HID = 12, 64


def init_params(seed: int) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights and zero biases, packed W1, b1, W2, b2, w3, b3."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-1, 1, N_HID * N_IN) / np.sqrt(N_IN), np.zeros(N_HID),
             rng.uniform(-1, 1, N_HID * N_HID) / np.sqrt(N_HID), np.zeros(N_HID),
             rng.uniform(-1, 1, N_HID) / np.sqrt(N_HID), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def record_steps(ctx, geo, field, batch, precision: int, capacity: int = 2_000_000, mass=None):
    """Training records [n, 13] (CUDA float32) from the plain stepper on ``batch``."""
    import torch
    dev = batch.offsets.device
    rec = torch.zeros((capacity, 13), dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    opts = Options(precision=precision, step_mode=STEP_ADAPTIVE, records=rec, record_count=cnt)
    if mass is not None:
        opts.mass = mass
    fit(ctx, geo, field, batch, opts)
    torch.cuda.synchronize()
    n = min(int(cnt.item()), capacity)
    return rec[:n].contiguous()


def train(ctx, records, epochs: int = 8, batch: int = 1024, lr: float = 2e-3, seed: int = 7):
    """Shuffled records, then ``epochs`` passes of Adam; returns (FP32 params, epoch losses)."""
    import torch
    g = torch.Generator(device=records.device)
    g.manual_seed(seed)
    rec = records[torch.randperm(records.shape[0], device=records.device, generator=g)].contiguous()
    p = torch.from_numpy(init_params(seed)).to(records.device)
    mom = torch.zeros((2, MLP_PARAMS), dtype=torch.float32, device=records.device)
    losses, _ = mlp_train(ctx, rec, p, mom, 0, batch=batch, epochs=epochs, lr=lr)
    torch.cuda.synchronize()
    return p.cpu().numpy(), losses.cpu().numpy()


def calibrate(ctx, params: np.ndarray, records, quantile: float = 0.05) -> tuple[np.ndarray, float]:
    """Shifts the output bias by the ``quantile`` of (label - output) over the records."""
    import torch
    p = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).to(records.device)
    x = records[:, :12].contiguous()
    out = mlp_forward(ctx, p, x)
    torch.cuda.synchronize()
    resid = (records[:, 12] - out).cpu().numpy()
    q = float(np.quantile(resid, quantile))
    cal = np.array(params, dtype=np.float32)
    cal[-1] += q
    return cal, q


def to_bf16(params: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even BF16 bit patterns of FP32 params."""
    u = np.ascontiguousarray(params, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def build_proposer(ctx, geo, field, batch, precision: int, epochs: int = 8, quantile: float = 0.05,
                   mass=None) -> tuple[Mlp, dict]:
    """Records -> training -> calibration -> BF16 handle, with a summary of the run."""
    rec = record_steps(ctx, geo, field, batch, precision, mass=mass)
    params, losses = train(ctx, rec, epochs=epochs)
    cal, q = calibrate(ctx, params, rec, quantile)
    w = to_bf16(cal)
    return Mlp(ctx, w), {"records": int(rec.shape[0]), "epoch_loss": [float(x) for x in losses],
                         "bias_shift": q, "weights_bf16": w}
