"""Learned warm start for the k-eigenvalue power iteration (not in the paper; an added pattern).

A 4-layer MLP (width 256, bf16 weights, FP32 accumulation; kernels in csrc/moc_mlp.cu) maps
per-region features -- the region's cross sections, a few geometry descriptors, and the instance's
cross-section perturbation -- to the region's log scalar flux per group and an estimate of k. It is
trained on converged solutions the library itself produces for perturbed instances of one geometry
(converged in FP32, then finished with FP64 outers). At solve time the prediction seeds phi, k and
the boundary flux (moc_ws_apply) and the plain power iteration converges from there; the cold start
stays the fallback and the converged plain solve is the reference result.

Everything numeric runs in the library's kernels; this module orchestrates (datasets live in
PyTorch-owned device memory) and measures.

Usage: python -m paper_2607_01591_gb300.warmstart --train 2000 --eval 200 --out result.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time
from typing import Dict, List

import numpy as np

from . import moc
from . import workloads as W

PCM = 1e-5


def lattice_geometry_features(mesh: W.Mesh, pitch: float = 1.26, guide_tubes=None) -> np.ndarray:
    """Per-region geometry descriptors of a square pin lattice centred at the origin: centroid x, y
    (scaled to [-1, 1]), distance from the pin centre (in half pitches), whether the pin is a
    guide tube, the fraction of its 8 neighbours that are, distance to the nearest lattice edge
    (scaled), and the material one-hot (3)."""
    c = mesh.centroids()
    xmin, xmax, ymin, ymax = mesh.bbox
    half = 0.5 * (xmax - xmin)
    n = int(round((xmax - xmin) / pitch))
    i = np.clip(np.floor((c[:, 0] - xmin) / pitch).astype(int), 0, n - 1)
    j = np.clip(np.floor((c[:, 1] - ymin) / pitch).astype(int), 0, n - 1)
    cx = xmin + (i + 0.5) * pitch
    cy = ymin + (j + 0.5) * pitch
    r = np.hypot(c[:, 0] - cx, c[:, 1] - cy) / (0.5 * pitch)
    gt = np.zeros((n, n))
    if guide_tubes:
        for di, dj in guide_tubes:
            gt[di + n // 2, dj + n // 2] = 1.0
    pad = np.pad(gt, 1)
    nb = sum(pad[1 + a:1 + a + n, 1 + b:1 + b + n] for a in (-1, 0, 1) for b in (-1, 0, 1) if (a, b) != (0, 0)) / 8.0
    edge = np.minimum.reduce([c[:, 0] - xmin, xmax - c[:, 0], c[:, 1] - ymin, ymax - c[:, 1]]) / half
    onehot = np.zeros((mesh.n_tri, 3))
    onehot[np.arange(mesh.n_tri), np.clip(mesh.mat, 0, 2)] = 1.0
    f = np.column_stack([c[:, 0] / half, c[:, 1] / half, r, gt[i, j], nb[i, j], edge, onehot])
    return f.astype(np.float32)


def perturbation_features(xs: W.CrossSections, base: W.CrossSections) -> np.ndarray:
    """Instance descriptor: log ratios to the base data of absorption, total scattering and
    nu*Sigma_f per material and group (0 where the base value is 0)."""
    def lr(a, b):
        with np.errstate(divide="ignore", invalid="ignore"):
            v = np.where(b > 0, np.log(np.where(b > 0, a, 1.0) / np.where(b > 0, b, 1.0)), 0.0)
        return v
    parts = [lr(xs.absorption(), base.absorption()), lr(xs.sigma_s.sum(2), base.sigma_s.sum(2)),
             lr(xs.nu_sigma_f, base.nu_sigma_f)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


class WarmStart:
    """Dataset generation, training and evaluation for one geometry."""

    def __init__(self, prob: W.Problem, base: W.CrossSections, guide_tubes=None, device: int = 0,
                 width: int = 256, seed: int = 0):
        import torch

        self.torch = torch
        self.prob = prob
        self.base = base
        self.device = device
        self.dev = f"cuda:{device}"
        self.stream = torch.cuda.Stream(device=device)
        self.G = base.n_groups
        self.R = prob.mesh.n_tri
        self.ctx32 = moc.Moc.from_problem(prob, device, "fp32", self.stream.cuda_stream, with_xs=False)
        self.ctx64 = moc.Moc.from_problem(prob, device, "fp64", self.stream.cuda_stream, with_xs=False)
        geo = lattice_geometry_features(prob.mesh, guide_tubes=guide_tubes)
        self.n_geo = geo.shape[1]
        self.geo = torch.from_numpy(geo).to(self.dev)
        self.n_glob = perturbation_features(base, base).size
        self.n_in = 3 * self.G + self.n_geo + self.n_glob
        self.n_out = self.G + 1
        self.area = None
        self.net = moc.Mlp(self.n_in, width, self.n_out, seed=seed, device=device)
        self.feat = torch.empty((self.R, self.n_in), dtype=torch.float32, device=self.dev)
        self.pred = torch.empty((self.R, self.n_out), dtype=torch.float32, device=self.dev)

    # ------------------------------------------------------------------------------ data
    def solve_reference(self, xs: W.CrossSections, polish: int = 3, tight: bool = False):
        """Converge in FP32 (|dk| <= 1e-7, fission-source change <= 1e-6), then continue in FP64 from
        that state: `polish` outers, or (tight) until |dk| <= 1e-10 and the change <= 1e-8."""
        self.ctx32.set_xs(xs)
        self.ctx32.power_iterate(1e-7, 1e-6, 20000, check_every=20, raise_on_fail=False)
        phi, k, psi = self.ctx32.get_state(with_psi=True)
        self.ctx64.set_xs(xs)
        self.ctx64.set_state(phi, k, psi)
        if tight:
            self.ctx64.power_iterate(1e-10, 1e-8, 2000, check_every=5, raise_on_fail=False)
        else:
            self.ctx64.outer(polish)
        phi64, k64 = self.ctx64.get_state()
        return phi64, k64

    def features(self, ctx, xs: W.CrossSections):
        ctx.ws_features(self.geo, self.n_geo, perturbation_features(xs, self.base), self.feat)
        return self.feat

    def make_dataset(self, instances: List[W.CrossSections], rows_per_instance: int, seed: int):
        torch = self.torch
        rng = np.random.default_rng(seed)
        n = len(instances) * rows_per_instance
        X = torch.empty((n, self.n_in), dtype=torch.float32, device=self.dev)
        Y = torch.empty((n, self.n_out), dtype=torch.float32, device=self.dev)
        ks = []
        t0 = time.perf_counter()
        for i, xs in enumerate(instances):
            phi, k = self.solve_reference(xs)
            ks.append(k)
            f = self.features(self.ctx64, xs)
            torch.cuda.synchronize(self.device)
            idx = torch.from_numpy(rng.choice(self.R, rows_per_instance, replace=False)).to(self.dev)
            s = slice(i * rows_per_instance, (i + 1) * rows_per_instance)
            X[s] = f[idx]
            tgt = np.column_stack([np.log(np.maximum(phi, 1e-300)), np.full(self.R, k)]).astype(np.float32)
            Y[s] = torch.from_numpy(tgt).to(self.dev)[idx]
        return X, Y, np.array(ks), time.perf_counter() - t0

    # ------------------------------------------------------------------------------ training
    def fit(self, X, Y, epochs: int = 4, batch: int = 8192, lr: float = 1e-3, seed: int = 0):
        torch = self.torch
        xm, xs_ = X.mean(0), X.std(0)
        ym, ys = Y.mean(0), Y.std(0)
        xs_ = torch.where(xs_ > 1e-6, xs_, torch.ones_like(xs_))
        ys = torch.where(ys > 1e-6, ys, torch.ones_like(ys))
        self.net.set_normalization(xm.cpu().numpy(), xs_.cpu().numpy(), ym.cpu().numpy(), ys.cpu().numpy())
        n = X.shape[0]
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        steps = max(1, epochs * n // batch)
        losses = []
        t0 = time.perf_counter()
        Xb = torch.empty((batch, self.n_in), dtype=torch.float32, device=self.dev)
        Yb = torch.empty((batch, self.n_out), dtype=torch.float32, device=self.dev)
        with torch.cuda.stream(self.stream):
            for s in range(steps):
                idx = torch.randint(0, n, (batch,), device=self.dev, generator=g)
                torch.index_select(X, 0, idx, out=Xb)
                torch.index_select(Y, 0, idx, out=Yb)
                lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
                want = (s % 50 == 0) or (s == steps - 1)
                loss = self.net.train_step(Xb, Yb, batch, max(lr_s, lr * 0.02), self.stream.cuda_stream, want)
                if want:
                    losses.append((s, loss))
        torch.cuda.synchronize(self.device)
        return losses, time.perf_counter() - t0

    # ------------------------------------------------------------------------------ solving
    def _iterate_to(self, ctx, k_ref: float, max_outer: int, tol: float = 5 * PCM):
        """Outers until |k - k_ref| <= tol; returns (outers, seconds of iteration)."""
        torch = self.torch
        n = 0
        t0 = time.perf_counter()
        k = float("nan")
        while n < max_outer:
            k, _ = ctx.outer(1)
            n += 1
            if abs(k - k_ref) <= tol:
                break
        return n, time.perf_counter() - t0, k

    def cold(self, ctx, xs, k_ref, max_outer=20000):
        torch = self.torch
        ctx.set_xs(xs)
        torch.cuda.synchronize(self.device)
        return self._iterate_to(ctx, k_ref, max_outer)

    def warm(self, ctx, xs, k_ref, max_outer=20000, pred_fn=None):
        """Learned start: features -> network -> iterate (timed from before inference)."""
        torch = self.torch
        ctx.set_xs(xs)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        if pred_fn is None:
            f = self.features(ctx, xs)
            self.net.forward(f, self.pred, self.R, self.stream.cuda_stream)
        else:
            self.pred.copy_(pred_fn)
        k0 = ctx.ws_apply(self.pred)
        t_inf = time.perf_counter() - t0
        n, t_it, k = self._iterate_to(ctx, k_ref, max_outer)
        return n, t_inf + t_it, k, k0, t_inf


def run(n_train: int, n_eval: int, n_eval_fp64: int, rows_per_instance: int, epochs: int, out: str,
        lattice: int = 17, seed: int = 1000):
    import torch

    if lattice == 17:
        prob = W.assembly_problem()
        gts = W.guide_tube_positions()
    else:
        prob = W.small_lattice_problem(lattice, n_azim=16, ray_spacing=0.04)
        gts = None
    base = W.synthetic_xs(["fuel", "clad", "moderator"], 7, 2)
    train = [W.perturbed_xs(base, seed + i) for i in range(n_train)]
    held = [W.perturbed_xs(base, seed + 100000 + i) for i in range(n_eval)]
    ws = WarmStart(prob, base, gts)
    X, Y, ktr, t_data = ws.make_dataset(train, rows_per_instance, seed=1)
    losses, t_fit = ws.fit(X, Y, epochs=epochs)
    # reference k of held-out instances (same solve as the training data)
    refs = [ws.solve_reference(xs, tight=True) for xs in held]
    # ablation: start from the training-mean solution (mean log flux per region, mean k)
    mean_pred = torch.empty((ws.R, ws.n_out), dtype=torch.float32, device=ws.dev)
    acc = torch.zeros((ws.R, ws.n_out), dtype=torch.float64, device=ws.dev)
    for xs in train[:min(50, n_train)]:
        phi, k = ws.solve_reference(xs)
        acc[:, :ws.G] += torch.from_numpy(np.log(phi)).to(ws.dev)
        acc[:, ws.G] += k
    mean_pred.copy_((acc / min(50, n_train)).float())
    res: Dict[str, list] = {"cold_fp32": [], "warm_fp32": [], "mean_fp32": [], "cold_fp64": [], "warm_k0_err": []}
    for i, (xs, (phi_ref, k_ref)) in enumerate(zip(held, refs)):
        n, t, k = ws.cold(ws.ctx32, xs, k_ref)
        res["cold_fp32"].append((n, t))
        n, t, k, k0, t_inf = ws.warm(ws.ctx32, xs, k_ref)
        res["warm_fp32"].append((n, t))
        res["warm_k0_err"].append(abs(k0 - k_ref))
        n, t, k, _, _ = ws.warm(ws.ctx32, xs, k_ref, pred_fn=mean_pred)
        res["mean_fp32"].append((n, t))
        if i < n_eval_fp64:
            n, t, k = ws.cold(ws.ctx64, xs, k_ref)
            res["cold_fp64"].append((n, t))

    def summ(v):
        a = np.array(v, dtype=float)
        return {"outers_mean": float(a[:, 0].mean()), "outers_median": float(np.median(a[:, 0])),
                "seconds_mean": float(a[:, 1].mean()), "n": int(a.shape[0])}

    result = {
        "workload": f"{lattice}x{lattice} lattice, {prob.mesh.n_tri} triangles, 7 groups; XS x lognormal(0.1) per material/group",
        "n_train": n_train, "n_eval": n_eval, "rows_per_instance": rows_per_instance, "epochs": epochs,
        "net": {"dims": ws.net.dims, "params": ws.net.n_params, "weights": "bf16 (FP32 master, Adam)"},
        "data_seconds": t_data, "fit_seconds": t_fit, "loss_first_last": [losses[0], losses[-1]],
        "stop": "first outer with |k - k_ref| <= 5 pcm; k_ref: FP32 to 1e-7, then FP64 to |dk| <= 1e-10",
        "cold_fp32": summ(res["cold_fp32"]), "warm_fp32": summ(res["warm_fp32"]),
        "mean_solution_fp32": summ(res["mean_fp32"]),
        "cold_fp64": summ(res["cold_fp64"]) if res["cold_fp64"] else None,
        "warm_initial_k_err_pcm_mean": float(np.mean(res["warm_k0_err"]) / PCM),
    }
    if out:
        with open(out, "w") as f:
            json.dump(result, f, indent=1)
    print(json.dumps(result), flush=True)
    return result


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--eval-fp64", type=int, default=40)
    ap.add_argument("--rows", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--lattice", type=int, default=17)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    run(a.train, a.eval, a.eval_fp64, a.rows, a.epochs, a.out, a.lattice)


if __name__ == "__main__":
    main()
