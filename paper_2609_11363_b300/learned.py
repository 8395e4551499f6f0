"""The learned correction from NInv towards SelInv, driven through the C ABI.

Every arithmetic step runs in the library's kernels: SelInv and the NInv
truncation stack (``sinv_selinv``, ``sinv_ninv_stack``), the features
(``sinv_mlp_features``), the targets, the BF16 forward/backward and Adam
(``sinv_mlp_train_step``) and the prediction (``sinv_mlp_predict``).  This
module only orders the calls: it concatenates training sets, draws the
mini-batch order with ``torch.randperm`` and reports errors.

SelInv is the reference: ``evaluate`` measures ||N - G||_F / ||G||_F on S for plain
NInv and for the corrected NInv, and ``choose`` keeps the corrected values only
when they beat NInv by the requested margin on held-out matrices (otherwise the
caller uses SelInv, the method the network imitates).
"""
from __future__ import annotations

import time

import torch

from .binding import Handle, Mlp


class LearnedCorrection:
    def __init__(self, m: int = 3, seed: int = 0, device: int = 0, batch: int = 8192):
        self.m = int(m)
        self.batch = int(batch)
        self.mlp = Mlp(seed=seed, max_batch=self.batch, device=device)
        self.device = self.mlp.device
        self.history = []

    def prepare(self, h: Handle, L_val, D_val, prec: str = "fp64", with_target: bool = True) -> dict:
        """SelInv (the target), the NInv stack and the features of one matrix."""
        Nst = h.ninv_stack(L_val, D_val, self.m, prec)
        X, scale = h.mlp_features(Nst, self.m, L_val, D_val)
        d = {"X": X, "scale": scale, "N": Nst[self.m].contiguous()}
        if with_target:
            d["G"] = h.selinv(L_val, D_val, prec)
            d["y"] = self.mlp.targets(d["G"], d["N"], scale)
        h.sync_status()
        return d

    def fit(self, sets, epochs: int = 4, lr: float = 2e-3, seed: int = 0, log_every: int = 0):
        """Mini-batch Adam over the union of the prepared training sets."""
        X = torch.cat([s["X"] for s in sets])
        y = torch.cat([s["y"] for s in sets])
        total = X.shape[0]
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        t0 = time.time()
        step = 0
        for ep in range(epochs):
            perm = torch.randperm(total, device=self.device, generator=gen)
            for b0 in range(0, total - self.batch + 1, self.batch):
                loss = self.mlp.train_step(X, y, perm[b0:b0 + self.batch], lr)
                step += 1
                if log_every and step % log_every == 0:
                    self.history.append((ep, step, float(loss.item())))
        torch.cuda.synchronize()
        return {"steps": step, "seconds": time.time() - t0, "entries": total}

    def save(self, path):
        """Checkpoint the network's training state (weights, Adam moments, steps)."""
        self.mlp.save(path)

    def load(self, path):
        """Resume from a checkpoint written by save()."""
        self.mlp.load(path)

    def predict(self, d) -> torch.Tensor:
        return self.mlp.predict(d["X"], d["scale"], d["N"])

    def evaluate(self, d) -> dict:
        """Relative Frobenius errors on S of NInv and of the corrected NInv against SelInv."""
        G, N = d["G"], d["N"]
        Nh = self.predict(d)
        g = torch.linalg.norm(G)
        return {"err_ninv": float(torch.linalg.norm(N - G) / g), "err_learned": float(torch.linalg.norm(Nh - G) / g)}

    @staticmethod
    def choose(evals, margin: float = 0.9) -> bool:
        """Keep the correction only if it beats NInv by `margin` on every held-out set."""
        return all(e["err_learned"] < margin * e["err_ninv"] for e in evals)
