"""Training mode of the cost model (Sec. 3: fit the model to runtimes measured
on the target; Sec. 5 Exp. 3: z-score standardised features, MLP, RMSE/NRMSE
on a held-out 20 % split).

The loop runs advisor_train_step (forward, MSE on ln runtime, hand-written
backward, Adam on the FP32 master weights) on device-resident features and
labels; checkpoints hold the whole parameter block (master weights, Adam
moments, packed copies) and the Adam step, so a resumed run continues
bit-identically.
"""
from __future__ import annotations

import os

import numpy as np
import torch

from . import advisor, metrics


def evaluate(model: advisor.Model, feat: torch.Tensor, labels: torch.Tensor, precision="fp32") -> dict:
    """RMSE and NRMSE (Eq. rmse, Eq. nrmse) of the predictions on a split."""
    y = model.score(feat, None, precision).double().cpu().numpy()
    t = labels.double().cpu().numpy()
    return {"rmse": metrics.rmse(y, t), "nrmse": metrics.nrmse(y, t)}


def train(model: advisor.Model, feat: torch.Tensor, labels: torch.Tensor, steps: int, batch: int,
          lr: float = 1e-3, seed: int = 0, losses: list | None = None, precision: str = "fp32"):
    """`steps` Adam steps on mini-batches of `batch` rows drawn without
    replacement per epoch (a fixed permutation per epoch from `seed`);
    precision "fp32" (SIMT) or "bf16" / "fp16" (tensor-core GEMMs)."""
    n = feat.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    perm = None
    pos = n
    for _ in range(steps):
        if pos + batch > n:
            perm = torch.randperm(n, generator=g).to(feat.device)
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        if batch == n:
            fb, lb = feat, labels
        else:
            fb, lb = feat.index_select(0, idx).contiguous(), labels.index_select(0, idx).contiguous()
        model.train_step(fb, lb, precision, lr=lr, loss=loss)
        if losses is not None:
            losses.append(loss.clone())
    return model


def train_paper_recipe(model: advisor.Model, feat: torch.Tensor, labels: torch.Tensor, epochs: int = 150,
                       batch: int = 16, lr: float = 0.01, step_epochs: int = 30, gamma: float = 0.1,
                       weight_decay: float = 1e-4, seed: int = 0, precision: str = "fp32",
                       epoch_losses: list | None = None):
    """The training recipe of Sec. 5 Exp. 3: RMSprop with an initial learning
    rate of 0.01 multiplied by 0.1 every 30 epochs, weight decay 1e-4, the
    RMSE loss, mini-batches of 16 rows (a fresh permutation per epoch; the
    last partial batch of an epoch is dropped), 150 epochs.  `epoch_losses`
    (optional) receives the mean batch RMSE of every epoch."""
    n = feat.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    steps_per_epoch = n // batch
    for ep in range(epochs):
        rate = lr * gamma ** (ep // step_epochs)
        perm = torch.randperm(n, generator=g).to(feat.device)
        acc = torch.zeros(1, dtype=torch.float32, device=feat.device)
        for i in range(steps_per_epoch):
            idx = perm[i * batch:(i + 1) * batch]
            model.train_step_ex(feat.index_select(0, idx).contiguous(), labels.index_select(0, idx).contiguous(),
                                precision, optimizer="rmsprop", loss_fn="rmse", lr=rate,
                                weight_decay=weight_decay, loss=loss)
            acc += loss
        if epoch_losses is not None:
            epoch_losses.append(float(acc.item()) / max(steps_per_epoch, 1))
    return model


def save_checkpoint(model: advisor.Model, path: str):
    torch.cuda.synchronize()
    blob = {"widths": model.widths, "param_block": model.param_block.cpu(), "adam_step": model.adam_step}
    tmp = path + ".tmp"
    torch.save(blob, tmp)
    os.replace(tmp, path)


def load_checkpoint(model: advisor.Model, path: str):
    blob = torch.load(path, map_location="cpu")
    assert tuple(blob["widths"]) == model.widths, "checkpoint of another network shape"
    model.param_block.copy_(blob["param_block"].to(model.device))
    model.adam_step = blob["adam_step"]
    torch.cuda.synchronize()
    return model


def labels_for(desc: np.ndarray, seed: int) -> np.ndarray:
    from . import workloads
    return workloads.make_labels(desc, seed)
