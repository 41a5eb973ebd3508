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
       [--save weights.npz]   (the trained network: FP32 master weights and standardisation)

The network the package ships (data/warmstart_assembly17.npz) was trained this way on one GB300;
`evaluate` measures it on held-out instances (bench.py's warm-start block does).
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
HERE = os.path.dirname(os.path.abspath(__file__))
SHIPPED = os.path.join(HERE, "data", "warmstart_assembly17.npz")
TRAIN_SEED = 1000            # instance i of the training set: perturbed_xs(base, TRAIN_SEED + i)
HELD_OUT_SEED = TRAIN_SEED + 100000


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

    # ------------------------------------------------------------------------------ persistence
    def save(self, path: str, meta: dict = None):
        """The network's FP32 master weights, its standardisation and its layer sizes."""
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        n = self.net.norm
        np.savez_compressed(path, params=self.net.get_params(), in_mean=n[0], in_std=n[1], out_mean=n[2],
                            out_std=n[3], dims=np.array(self.net.dims, dtype=np.int32),
                            meta=np.array(json.dumps(meta or {})))

    def load(self, path: str) -> dict:
        z = np.load(path)
        if list(z["dims"]) != list(self.net.dims):
            raise ValueError(f"{path}: network {list(z['dims'])} does not match {self.net.dims}")
        self.net.set_params(z["params"])
        self.net.set_normalization(z["in_mean"], z["in_std"], z["out_mean"], z["out_std"])
        return json.loads(str(z["meta"]))

    def time_network(self, batch: int = 8192, reps: int = 20) -> dict:
        """CUDA-event times of the network's forward pass over all regions of the geometry and of
        one training step (forward, backward, Adam) on a batch of random rows; the parameters are
        restored afterwards."""
        torch = self.torch
        p = self.net.get_params()
        norm = [v.copy() for v in self.net.norm]
        x = torch.randn((self.R, self.n_in), dtype=torch.float32, device=self.dev)
        xb = torch.randn((batch, self.n_in), dtype=torch.float32, device=self.dev)
        yb = torch.randn((batch, self.n_out), dtype=torch.float32, device=self.dev)
        st = self.stream

        def timed(fn):
            with torch.cuda.stream(st):
                fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(reps):
                    fn()
                e1.record(st)
            torch.cuda.synchronize(self.device)
            return e0.elapsed_time(e1) / reps

        fwd = timed(lambda: self.net.forward(x, self.pred, self.R, st.cuda_stream))
        trn = timed(lambda: self.net.train_step(xb, yb, batch, 1e-6, st.cuda_stream, False))
        self.net.set_params(p)
        self.net.set_normalization(*norm)
        flops = 2 * sum(a * b for a, b in zip(self.net.dims[:-1], self.net.dims[1:]))
        return {"forward_rows": self.R, "forward_ms": fwd, "forward_tflops": flops * self.R / fwd / 1e9,
                "train_batch": batch, "train_step_ms": trn, "train_tflops": 3 * flops * batch / trn / 1e9}

    def mean_solution(self, instances: List[W.CrossSections]):
        """The ablation without a network: the mean over solved training instances of the log
        flux per region and group, and of k, as a prediction in the network's output layout."""
        torch = self.torch
        acc = torch.zeros((self.R, self.n_out), dtype=torch.float64, device=self.dev)
        for xs in instances:
            phi, k = self.solve_reference(xs)
            acc[:, :self.G] += torch.from_numpy(np.log(phi)).to(self.dev)
            acc[:, self.G] += k
        return (acc / len(instances)).float()

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


def evaluate(ws: WarmStart, held: List[W.CrossSections], mean_pred, n_fp64: int) -> dict:
    """Time to |k - k_ref| <= 5 pcm on held-out instances from four starts: cold FP32, cold FP64
    (first n_fp64 instances), the training-mean solution without a network (ablation) and the
    learned start (wall time including the feature and network kernels). k_ref: FP32 to |dk| <=
    1e-7 continued in FP64 to |dk| <= 1e-10."""
    res: Dict[str, list] = {"cold_fp32": [], "warm_fp32": [], "mean_fp32": [], "cold_fp64": [], "warm_k0_err": [],
                            "mean_k0_err": [], "inference_s": []}
    for i, xs in enumerate(held):
        _, k_ref = ws.solve_reference(xs, tight=True)
        n, t, k = ws.cold(ws.ctx32, xs, k_ref)
        res["cold_fp32"].append((n, t))
        n, t, k, k0, t_inf = ws.warm(ws.ctx32, xs, k_ref)
        res["warm_fp32"].append((n, t))
        res["warm_k0_err"].append(abs(k0 - k_ref))
        res["inference_s"].append(t_inf)
        n, t, k, k0, _ = ws.warm(ws.ctx32, xs, k_ref, pred_fn=mean_pred)
        res["mean_fp32"].append((n, t))
        res["mean_k0_err"].append(abs(k0 - k_ref))
        if i < n_fp64:
            n, t, k = ws.cold(ws.ctx64, xs, k_ref)
            res["cold_fp64"].append((n, t))

    def summ(v):
        a = np.array(v, dtype=float)
        return {"outers_mean": float(a[:, 0].mean()), "outers_median": float(np.median(a[:, 0])),
                "seconds_mean": float(a[:, 1].mean()), "n": int(a.shape[0])}

    return {"stop": "first outer with |k - k_ref| <= 5 pcm; k_ref: FP32 to 1e-7, then FP64 to |dk| <= 1e-10",
            "cold_fp32": summ(res["cold_fp32"]), "warm_fp32": summ(res["warm_fp32"]),
            "mean_solution_fp32": summ(res["mean_fp32"]),
            "cold_fp64": summ(res["cold_fp64"]) if res["cold_fp64"] else None,
            "warm_initial_k_err_pcm_mean": float(np.mean(res["warm_k0_err"]) / PCM),
            "mean_solution_initial_k_err_pcm_mean": float(np.mean(res["mean_k0_err"]) / PCM),
            "inference_s_mean": float(np.mean(res["inference_s"]))}


def assembly_base():
    """The base cross sections of the assembly instances (fuel, clad, moderator; 7 groups)."""
    return W.synthetic_xs(["fuel", "clad", "moderator"], 7, 2)


def run(n_train: int, n_eval: int, n_eval_fp64: int, rows_per_instance: int, epochs: int, out: str,
        lattice: int = 17, seed: int = TRAIN_SEED, save: str = ""):
    import torch

    if lattice == 17:
        prob = W.assembly_problem()
        gts = W.guide_tube_positions()
    else:
        prob = W.small_lattice_problem(lattice, n_azim=16, ray_spacing=0.04)
        gts = None
    base = assembly_base()
    train = [W.perturbed_xs(base, seed + i) for i in range(n_train)]
    held = [W.perturbed_xs(base, seed + 100000 + i) for i in range(n_eval)]
    ws = WarmStart(prob, base, gts)
    X, Y, ktr, t_data = ws.make_dataset(train, rows_per_instance, seed=1)
    losses, t_fit = ws.fit(X, Y, epochs=epochs)
    mean_pred = ws.mean_solution(train[:min(50, n_train)])
    ev = evaluate(ws, held, mean_pred, n_eval_fp64)
    ev["network_times"] = ws.time_network()
    result = {
        "workload": f"{lattice}x{lattice} lattice, {prob.mesh.n_tri} triangles, 7 groups; XS x lognormal(0.1) per material/group",
        "n_train": n_train, "n_eval": n_eval, "rows_per_instance": rows_per_instance, "epochs": epochs,
        "net": {"dims": ws.net.dims, "params": ws.net.n_params, "weights": "bf16 (FP32 master, Adam)"},
        "data_seconds": t_data, "fit_seconds": t_fit, "loss_first_last": [losses[0], losses[-1]],
        **ev,
    }
    if save:
        ws.save(save, {"n_train": n_train, "rows_per_instance": rows_per_instance, "epochs": epochs,
                       "train_seed": seed, "lattice": lattice, "data_seconds": t_data, "fit_seconds": t_fit,
                       "loss_first_last": [losses[0], losses[-1]]})
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
    ap.add_argument("--save", default="", help="write the trained network here (.npz)")
    ap.add_argument("--time-network", action="store_true",
                    help="only time the shipped network's forward pass over the assembly's regions and a "
                         "training step (CUDA events), and print them")
    a = ap.parse_args()
    if a.time_network:
        ws = WarmStart(W.assembly_problem(), assembly_base(), W.guide_tube_positions())
        ws.load(SHIPPED)
        print(json.dumps(ws.time_network()), flush=True)
        return
    run(a.train, a.eval, a.eval_fp64, a.rows, a.epochs, a.out, a.lattice, save=a.save)


if __name__ == "__main__":
    main()
