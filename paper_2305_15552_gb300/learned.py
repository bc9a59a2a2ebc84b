"""Training of the learned per-row preconditioner on the GPU.

The preconditioner K of Eq. (wblock) only has to approximate H (Sec. 2.3); this one scales each
residual entry by m = J (1 + MLP(6 features)), J the Jacobi scale (the features, the network and
the training target are documented in include/eig.h beside eig_lp_sample).  Everything numeric runs in the library's
kernels: samples (eig_lp_sample: residuals, H r, features, targets), loss and gradient
(eig_lp_grad: fused forward + backward), and the Adam step (eig_lp_adam).  This module only
orders the calls: it runs the solver to get Ritz pairs, collects samples, and loops over them.

Typical use on a family of matrices H(g):
    samples = []
    for H in training_matrices:
        S = Solver(H, n_ev, block)
        samples += collect_samples(S, X0, iters=(0, 1, 2, 3))
    params = init_params(*feature_stats(samples))      # starts as the Jacobi K
    params, hist = train(samples, params, epochs=...)
    S.solve("hybrid", precond=2, rmm_precond=2, lp_params=params, ...)
"""
from __future__ import annotations

import numpy as np

from . import binding as B

N_PARAMS = B.N_LP_PARAMS
OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = 12, 204, 236, 1260, 1292, 1324


def init_params(mu, sigma, seed=0):
    """He-normal hidden layers, zero biases and a zero output layer (o = 0: the network starts as
    the Jacobi K); mu, sigma are the feature statistics (fixed, not trained)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(N_PARAMS, dtype=np.float64)
    p[0:6] = mu
    p[6:12] = sigma
    p[OFF_W1:OFF_B1] = rng.standard_normal(32 * 6) * np.sqrt(2.0 / 6)
    p[OFF_W2:OFF_B2] = rng.standard_normal(32 * 32) * np.sqrt(2.0 / 32)
    return p.astype(np.float32)


def converged_space(S, X0, tol=1e-9, maxiter=400):
    """X* of the correction targets: the wanted eigenvectors to tol, LOBPCG with FP64 vectors
    (device FP64 n x n_ev)."""
    rc, st = S.solve("lobpcg", X0=X0, vec_type="f64", tol=tol, maxiter=maxiter, certify=0)
    _, X, _ = S.ritz(X_on_device=True)
    return X, rc, st


def collect_samples(S, X0, iters=(0, 1, 2, 3), Xstar=None, floor=2.0, vec_type="f32", min_relres=1e-5):
    """Samples (eig_lp_sample, correction target) at the Ritz pairs LOBPCG with the Jacobi K
    reaches after each of `iters` iterations from X0; iterates already below min_relres are
    skipped (their target is dominated by the error of X*)."""
    if Xstar is None:
        Xstar, _, _ = converged_space(S, X0)
    out = []
    for k in iters:
        S.solve("lobpcg", X0=X0, vec_type=vec_type, maxiter=int(k), certify=1, precond=1)
        th, X, rel = S.ritz(X_on_device=True)
        if np.max(rel) < min_relres:
            break
        out.append(S.lp_sample(X, th, Xstar, target=0, floor=floor))
    return out


def feature_stats(samples):
    """Mean and standard deviation (floored at 1e-6) of the six features over the samples."""
    import torch
    s1 = torch.zeros(6, dtype=torch.float64, device="cuda")
    s2 = torch.zeros(6, dtype=torch.float64, device="cuda")
    cnt = 0
    for smp in samples:
        F = smp["F"].double()
        s1 += F.sum(0)
        s2 += (F * F).sum(0)
        cnt += F.shape[0]
    mu = (s1 / cnt).cpu().numpy()
    var = (s2 / cnt).cpu().numpy() - mu * mu
    return mu, np.sqrt(np.maximum(var, 1e-12))


class Trainer:
    """Adam on the device: params, moments, gradient and workspace stay in HBM."""

    def __init__(self, params):
        import torch
        lib = B.load()
        self.p = torch.tensor(np.asarray(params, dtype=np.float32), device="cuda")
        self.m1 = torch.zeros_like(self.p)
        self.m2 = torch.zeros_like(self.p)
        self.grad = torch.empty(B.N_LP_TRAINED + 1, dtype=torch.float64, device="cuda")
        self.ws = torch.empty(lib.eig_lp_grad_workspace_bytes(), dtype=torch.uint8, device="cuda")
        self.t = 0

    def step(self, sample, lr):
        B.lp_grad(self.p, sample, self.grad, self.ws)
        self.t += 1
        B.lp_adam(self.p, self.grad, self.m1, self.m2, self.t, lr)
        return self.grad

    def loss(self, sample):
        return float(B.lp_grad(self.p, sample, self.grad, self.ws)[-1].item())

    def params(self):
        return self.p.cpu().numpy().copy()


def train(samples, params, epochs=40, lr=3e-3, seed=0, lr_decay=0.97):
    """Adam over the samples (one step per sample, shuffled each epoch); returns the trained
    parameters and the mean training loss of each epoch."""
    tr = Trainer(params)
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        acc = 0.0
        for i in order:
            acc += float(tr.step(samples[i], lr * lr_decay ** ep)[-1].item())
        hist.append(acc / max(len(samples), 1))
    return tr.params(), hist


def mean_loss(samples, params):
    tr = Trainer(params)
    return float(np.mean([tr.loss(s) for s in samples])) if samples else float("nan")


def jacobi_loss(sample, floor=2.0):
    """The loss of the Jacobi K on a sample (m = 1 / floor(H_ii - theta_j)), for comparison."""
    import torch
    F, r, z, colw, m = sample["F"], sample["r"], sample["z"], sample["colw"], sample["m"]
    den = F[:, 2].double()
    mag = torch.clamp(den.abs(), min=floor)
    den = torch.where(den < 0, -mag, mag)
    err = r.double() / den - z.double()
    w = colw.repeat(F.shape[0] // m)
    return float((w * err * err).sum().item())


def time_forward(rows=8_000_000, reps=20, seed=0):
    """Mean device time (ms) of the network kernel (eig_lp_forward) on `rows` random feature rows,
    after three warm-up launches: a quick check of its throughput (2516 FLOP per row)."""
    import torch
    rng = np.random.default_rng(seed)
    F = torch.tensor(rng.standard_normal((rows, 6)).astype(np.float32), device="cuda")
    p = init_params(np.zeros(6), np.ones(6), seed=seed + 1)
    p[OFF_W3:OFF_B3 + 1] = (rng.standard_normal(33) * 0.1).astype(np.float32)
    for _ in range(3):
        B.lp_forward(p, F)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        B.lp_forward(p, F)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="time the learned preconditioner's network kernel")
    ap.add_argument("--rows", type=int, default=8_000_000)
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args()
    ms = time_forward(a.rows, a.reps)
    print(f"eig_lp_forward: {a.rows} rows, {ms:.4f} ms per launch, {a.rows * 2516 / (ms * 1e-3) / 1e12:.2f} TFLOP/s")
