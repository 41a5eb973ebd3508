"""Benchmark: MOC segment*polar*group updates/s on the 19-hexagon core (one GB300).

A step is one outer iteration of the whole hot path -- source update, transport sweep (tallies,
boundary-flux links, own FP32 exponential, compensated FP32 tallies), flux finalisation and the
FP64 fission/k/residual reductions -- on the seeded synthetic 19-hexagon core (1,507,650
triangles, 33 groups, 48 azimuths, TY-3 polar, 0.02 cm ray spacing, vacuum), the largest
configuration. updates per step = 2 * segments * polar * groups.

Prints one JSON line (rank 0). Under torchrun each rank runs an independent replica on its own
GPU (the sweep has no data-path exchange); value = all ranks' updates / max time. Beside the
headline the line carries, for context: the FP64 mode with its own roofline, the time to a
converged k (CMFD-accelerated, FP32 and FP64), the 17x17 assembly measured the same way with its
plain and accelerated time to k and its FP64 rate, the 3x3-assembly core and the pin cell in FP32
and FP64, the learned warm start against the cold starts and the no-network
ablation on held-out assembly instances, a DGMOC block (the assembly extruded to `--axial` planes),
host against device tracking, the hardware rate probes behind the roofline denominators and the
CPU oracle timed on a bounded sample at one thread and at all host cores.
`--impl reference` times the CPU oracle instead (one oracle outer of the sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MOC segment*polar*group updates/s"
UNIT = "updates/s"
WORKLOADS = {
    "assembly": "17x17 assembly, 39,304 triangles, 7 groups, 32 azimuths, 3 polar (TY), ray spacing 0.02 cm",
    "core": "3x3-assembly core + reflector, 608,804 triangles, 7 groups, 64 azimuths, 3 polar, ray spacing 0.01 cm",
    "hexcore": "19-hexagon core, 1,507,650 triangles, 33 groups, 48 azimuths, 3 polar, ray spacing 0.02 cm",
    "hexcore1": "central hexagon of the hex core, 79,350 triangles, 33 groups, 48 azimuths, 3 polar, ray spacing 0.02 cm",
    "hexcore7": "central 7 hexagons of the hex core, 555,450 triangles, 33 groups, 48 azimuths, 3 polar, ray spacing 0.02 cm",
    "pin": "pin cell, 200 triangles, 7 groups, 16 azimuths, 3 polar, ray spacing 0.05 cm",
}
DEFAULT_WORKLOAD = "hexcore"
# the bounded sample the CPU oracle is timed on: the central assembly of the hex core with the
# core's quadrature and cross sections (the same per-update work, 1/19 of the assemblies)
ORACLE_SAMPLE = "central hexagonal assembly of the hex core (79,350 triangles, 6.67e6 segments), 33 groups, 48 azimuths, 3 polar, 0.02 cm"


def make_problem(name: str):
    from paper_2607_01591_gb300 import workloads as W

    return {"assembly": W.assembly_problem, "core": W.core_problem, "hexcore": W.hex_core_problem,
            "hexcore7": lambda: W.hex_core_problem(n_rings=1), "hexcore1": lambda: W.hex_core_problem(n_rings=0),
            "pin": W.pin_cell_problem}[name]()


L2_FLUSH_BYTES = 512 << 20
# Algorithmic FP32 operations per update, the scope table's count: tau (2 multiplies), delta (a
# subtract and a multiply), the psi update (1), the tally FMA (1) and 8 for the exponential.
OPS_PER_UPDATE = 14
# What the kernels' own formulas execute per update: tau 1 multiply (the segment's Sigma_t l is
# shared by the polar angles), the 13-operation range-reduced 1 - e^-tau, delta 2, psi 1, tally 1.
IMPL_OPS_PER_UPDATE = 18
# FP64 peak: the nominal 1.25 TFLOP/s of the part, i.e. 0.625e12 fused multiply-adds per second
FP64_FMA_NOMINAL = 0.625e12
# DRAM bytes (read + write) and L2 sector hit rate of one sweep launch, from ncu on the named
# workload with the current kernel versions (the hex core's DRAM counters are single-pass captures
# of the full-size launch; its hit rate needs three passes, so it was captured on the seven-hexagon
# case only); absent entries are reported as null.
SWEEP_NCU = {
    ("hexcore", "fp32"): {"dram_bytes": 36.08e9 + 17.35e9, "l2_hit_pct": None},
    ("hexcore7", "fp32"): {"dram_bytes": 8.74e9 + 4.09e9, "l2_hit_pct": 61.3},
    ("assembly", "fp32"): {"dram_bytes": 82.33e6 + 2.35e6, "l2_hit_pct": 73.5},
}


def measured_rates(device: int) -> dict:
    """The library's hardware rate probes (FP32/FP64 FMA issue, L2 atomics by access shape) on this
    device, plus its multiprocessor count."""
    from paper_2607_01591_gb300 import moc

    out = {}
    for kind in moc.PROBES:
        r = moc.probe_rate(kind, device)
        out["sm_count"] = r["sm_count"]
        out[kind] = {"lane_ops_per_s": r["lane_ops_per_s"], "sectors_per_s": r["sectors_per_s"]}
    return out


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all replicas processed divided by the slowest rank's time."""
    return units_per_rank * world / seconds_max


def oracle_rate(prob, threads: int, outers: int = 1):
    """Updates/s of the CPU oracle, as it stands, over `outers` outers of `prob` on `threads`
    threads (after its track set-up, which is not timed)."""
    import oracle

    o = oracle.Oracle.from_problem(prob, threads=threads)
    o.normalise()
    t0 = time.perf_counter()
    for _ in range(outers):
        o.outer(True)
    dt = time.perf_counter() - t0
    ups = 2 * o.n_segments * len(prob.sin_theta) * prob.xs.n_groups
    return ups * outers / dt, dt, ups


def cpu_baseline(prob, name: str):
    """The oracle on the host cores: one outer of the bounded sample `prob` at one thread and at
    all cores (nproc)."""
    nproc = os.cpu_count() or 1
    v1, t1, ups = oracle_rate(prob, 1)
    vn, tn, _ = oracle_rate(prob, nproc)
    return {"value": vn, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": f"one FP64 oracle outer of the {name} ({ups:.3e} updates): {tn:.2f} s on {nproc} threads, "
                      f"{t1:.2f} s on 1 (tracks in fixed chunks, groups in turn)",
            "one_thread": {"value": v1, "s": t1}, "nproc": nproc}


def dg_cpu_baseline(nz: int = 8):
    """The oracle's DGMOC as it stands on the host cores, on a bounded sample of the DGMOC workload:
    one outer of a 3x3-pin lattice cut from the assembly's pin geometry, with the assembly's
    quadrature (32 azimuths, 0.02 cm, TY-3), extruded like the benchmark (nz planes of 10.71 cm,
    the top quarter moderator, reflective bottom, vacuum top); updates/s in the same units."""
    import oracle
    from paper_2607_01591_gb300 import workloads as W

    lat = W.small_lattice_problem(3, bc=(1, 1, 1, 1), n_azim=32, ray_spacing=0.02)
    threads = min(os.cpu_count() or 1, lat.xs.n_groups)
    o = oracle.Oracle.from_problem(lat, threads=threads)
    mat3 = np.tile(lat.mesh.mat, (nz, 1))
    mat3[nz - max(1, nz // 4):] = lat.mesh.mat.max()
    o.set_axial(np.full(nz, 10.71), mat3, bc=(1, 0))
    o.normalise()
    t0 = time.perf_counter()
    o.outer(True)
    dt = time.perf_counter() - t0
    ups = 2 * o.n_segments * len(lat.sin_theta) * lat.xs.n_groups * 2 * nz
    return {"value": ups / dt, "unit": "updates/s", "cores": threads, "kind": "oracle",
            "sample": f"one oracle DGMOC outer (FP64, one thread per group) on a 3x3-pin lattice with the "
                      f"assembly's quadrature, {nz} planes: {o.n_segments} segments, {dt:.2f} s"}


# Per DGMOC update (segment x polar x group x plane x march), FP32: the algorithmic operations of the
# closed-form 2x2 segment solution counted from its formulas (FMA = 1, the 1 - e^-x evaluation 13,
# small-angle sin/cos 10, the reciprocal 1), and the thread instructions the plane-inner sweep
# actually executes, from an ncu capture of the plane-inner sweep on the extruded assembly
DG_OPS_PER_UPDATE = 74
DG_INST_PER_UPDATE = 110.4


def dgmoc_block(moc, W, prob, device, stream, precision, nz, steps, converge=False, name="assembly"):
    """DGMOC (Sec. 2.2, Alg. 2) on the assembly extruded like the paper's 3D lattice benchmark:
    nz axial planes of 10.71 cm, the top quarter reflector (the moderator material in every
    region), reflective bottom (mid-plane symmetry) and vacuum top. Times whole outers and the
    sweep kernel alone (CUDA events on the launching stream)."""
    import torch

    n_refl = max(1, nz // 4)
    mat3 = np.tile(prob.mesh.mat, (nz, 1))
    mat3[nz - n_refl:] = prob.mesh.mat.max()
    dz = np.full(nz, 10.71)
    m = moc.Moc.from_problem(prob, device=device, precision=precision, stream=stream.cuda_stream)
    m.set_axial(dz, mat3, bc=(1, 0))
    _, ups, kpo = m.work()

    def run(k):
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.outer(k, read=False)
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    run(3)
    ms = run(steps)
    m.enable_timing(True)
    m.outer(steps, read=False)
    sweep_ms, n_sw = m.timing()
    m.enable_timing(False)
    k, _ = m.outer(0)
    ttk = None
    if converge:
        # power iteration from the flat start to |dk| <= 1e-6 and fission residual <= 1e-5 (host
        # check every 10 outers), wall time through the public API
        m.set_state(None, 1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kc, n, r, ok = m.power_iterate(tol_k=1e-6, tol_flux=1e-5, max_outer=5000, check_every=10, raise_on_fail=False)
        ttk = {"s": time.perf_counter() - t0, "outers": n, "k": kc, "residual": r, "converged": ok,
               "tolerance": "|dk| <= 1e-6, max relative fission-rate change <= 1e-5, checked every 10 outers"}
        # the same with the axial coarse-mesh acceleration (planes as coarse cells)
        m.set_dg_cmfd(8, 4, 1.0)
        m.set_state(None, 1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kc, n, r, ok = m.power_iterate(tol_k=1e-6, tol_flux=1e-5, max_outer=5000, check_every=10, raise_on_fail=False)
        ttk["accelerated"] = {"s": time.perf_counter() - t0, "outers": n, "k": kc, "residual": r, "converged": ok,
                              "acceleration": "planes as coarse cells, 8 coarse power iterations x 4 sweeps per group"}
        m.set_dg_cmfd(0)
    m.close()
    sweep_s = sweep_ms / n_sw / 1e3
    out = {"workload": f"{WORKLOADS[name]} extruded to {nz} planes x 10.71 cm ({n_refl} reflector "
                       "planes on top), reflective bottom, vacuum top, linear axial DG",
           "precision": precision, "planes": nz, "elements": nz * prob.mesh.n_tri, "updates_per_outer": ups,
           "ms_per_outer": ms / steps, "value": ups * steps / (ms / 1e3), "unit": "updates/s",
           "sweep_ms": sweep_s * 1e3, "kernel": "dg_sweep_res_kernel (plane-inner; dg_sweep_kernel when its shared memory would exceed 100 KB per block)", "k_after": k + 0.0,
           "outers_timed": steps, "gpu_launches_per_outer": kpo, "time_to_k": ttk}
    if precision != "fp64":
        peak = 152 * 128 * float(_peaks().get("sm_max_mhz", 2070.0)) * 1e6
        out["roofline"] = {"bound": "alu", "achieved": DG_OPS_PER_UPDATE * ups / sweep_s / 1e9,
                           "peak": peak / 1e9, "unit": "Gop/s", "frac": DG_OPS_PER_UPDATE * ups / sweep_s / peak,
                           "ops_per_update": DG_OPS_PER_UPDATE,
                           "issue_frac": DG_INST_PER_UPDATE * ups / sweep_s / peak,
                           "inst_per_update": DG_INST_PER_UPDATE,
                           "peak_note": "152 SMs x 128 FP32 lanes x max SM clock; issue_frac counts executed "
                                        "thread instructions (ncu) instead of algorithmic operations"}
    return out


def time_to_converged_k(moc, prob, device, stream, cmfd, plain: bool = True, pcm: float = 5.0, cmfd_tol: float = 0.0):
    """Wall time and outers of the cold-start power iteration until |k - k_ref| <= pcm * 1e-5, in
    FP32 and FP64, plain (when `plain`) and CMFD-accelerated with cmfd = (cell size, coarse power
    iterations, sweeps per group, omega). k_ref: FP32 to |dk| <= 1e-7 continued in FP64 to
    |dk| <= 1e-10, accelerated when the plain iteration is not run (the accelerated limit is the
    transport solution). cmfd_tol > 0: the accelerated runs stop each coarse power iteration once
    k and the coarse source settle to cmfd_tol (at most cmfd[1] iterations)."""
    import torch
    from paper_2607_01591_gb300 import workloads as W

    cell, n_cells = W.grid_cells(prob.mesh, cmfd[0])

    def accel(ctx):
        ctx.set_cmfd(cell, n_cells, cmfd[1], cmfd[2], cmfd[3])
        ctx.set_cmfd_tolerance(cmfd_tol)

    ref32 = moc.Moc.from_problem(prob, device=device, precision="fp32", stream=stream.cuda_stream)
    ref64 = moc.Moc.from_problem(prob, device=device, precision="fp64", stream=stream.cuda_stream)
    if not plain:
        accel(ref32)
        accel(ref64)
    ref32.power_iterate(1e-7, 1e-6, 20000, check_every=20 if plain else 2, raise_on_fail=False)
    phi, k, psi = ref32.get_state(with_psi=True)
    ref64.set_state(phi, k, psi)
    k_ref, _, _, _ = ref64.power_iterate(1e-10, 1e-8, 5000, check_every=5, raise_on_fail=False)
    out = {"k_ref": k_ref, "criterion": f"|k - k_ref| <= {pcm} pcm",
           "k_ref_from": "FP32 to |dk| <= 1e-7, continued in FP64 to |dk| <= 1e-10"
                         + ("" if plain else " (CMFD-accelerated)"),
           "cmfd": f"{cmfd[0]} cm square coarse cells ({n_cells}); per outer {cmfd[1]} coarse power iterations, "
                   f"{cmfd[2]} Gauss-Seidel sweeps per group, over-relaxation {cmfd[3]}"
                   + (f"; coarse iteration stopped once k and the coarse source settle to {cmfd_tol}" if cmfd_tol else "")}
    runs = ((("cold_fp32", ref32, False), ("cold_fp64", ref64, False)) if plain else ()) + \
        (("cold_fp32_cmfd", ref32, True), ("cold_fp64_cmfd", ref64, True))
    for name, ctx, acc in runs:
        ctx.set_xs(prob.xs)
        if acc:
            accel(ctx)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        n = 0
        while n < 20000:
            k, _ = ctx.outer(1)
            n += 1
            if abs(k - k_ref) <= pcm * 1e-5:
                break
        out[name] = {"ms": (time.perf_counter() - t0) * 1e3, "outers": n}
        if acc:
            out[name]["coarse_iterations"] = ctx.cmfd_iterations()
    ref32.close()
    ref64.close()
    return out


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle on the host cores (all of them), one outer of the bounded
    sample per step, after `warmup` untimed outers."""
    import oracle

    if rank != 0:
        return
    prob = make_problem("hexcore1")
    threads = os.cpu_count() or 1
    o = oracle.Oracle.from_problem(prob, threads=threads)
    o.normalise()
    ups = 2 * o.n_segments * len(prob.sin_theta) * prob.xs.n_groups
    for _ in range(args.warmup):
        o.outer(True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.outer(True)
    dt = time.perf_counter() - t0
    v = ups * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded mesh and cross sections)",
            "config": {"workload": WORKLOADS[DEFAULT_WORKLOAD], "updates_per_step": ups,
                       "sample": ORACLE_SAMPLE},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": v, "unit": UNIT,
                             "sample": f"{args.steps} oracle outers of the {ORACLE_SAMPLE} after {args.warmup} warm-up"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_outers(m, stream, flush, k: int, flush_l2: bool = True) -> float:
    """k outers, each bracketed by CUDA events on the library's stream (L2 flushed before each,
    untimed); returns the summed milliseconds."""
    import torch

    evs = []
    with torch.cuda.stream(stream):
        for _ in range(k):
            if flush_l2:
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.outer(1, read=False)
            e1.record(stream)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def sweep_seconds(m, stream, flush, k: int) -> float:
    """Average duration of the sweep kernel's launch, from the library's CUDA events recorded on the
    stream it launches on, over k outers."""
    m.enable_timing(True)
    timed_outers(m, stream, flush, k)
    ms, n = m.timing()
    m.enable_timing(False)
    return ms / n / 1e3


def sweep_kernel_name(prob, precision: str) -> str:
    G, P = prob.xs.n_groups, len(prob.sin_theta)
    if precision != "fp64" and P == 3 and G > 8:
        return "sweep_chunk_kernel"
    return "sweep_kernel"


def roofline(prob, m, precision: str, sweep_s: float, ups: int, workload: str, n_sm: int, rates: dict) -> dict:
    """Roofline of the sweep launch: algorithmic operations (the scope table's 14 per update)
    against the derived FP32 lane peak (FP64: the nominal FMA rate), with the HBM fraction of the
    algorithmic bytes, the L2 atomic rate and the ncu traffic beside it."""
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    G, P = prob.xs.n_groups, len(prob.sin_theta)
    R = prob.mesh.n_tri
    T, S = m.track_counts()
    Gp4 = (G + 3) // 4 * 4
    seg_b = 8 if precision != "fp64" else 12
    real_b = 4 if precision != "fp64" else 8
    tally_b = 8 if precision == "fp32" else real_b
    # segments once, region rows (Sigma_t, q/Sigma_t) and tallies once, boundary flux in and out
    alg_bytes = seg_b * S + R * Gp4 * (2 * real_b + tally_b) + 2 * T * 2 * P * Gp4 * real_b
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ops = OPS_PER_UPDATE * ups
    if precision == "fp64":
        peak, peak_note = FP64_FMA_NOMINAL, "nominal FP64 rate of the part, 1.25 TFLOP/s = 0.625e12 FMA/s (FMA = 1 op)"
        measured = rates.get("dfma", {}).get("lane_ops_per_s") if rates else None
    else:
        peak = n_sm * 128 * sm_max * 1e6
        peak_note = f"{n_sm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (derived; FMA = 1 op)"
        measured = rates.get("ffma", {}).get("lane_ops_per_s") if rates else None
    ncu = SWEEP_NCU.get((workload, precision), {})
    # L2 atomics of the launch: per (segment, sense) one tally add per group (FP32: float4 adds over
    # 4-group chunks in the chunked kernel, one FP32 add per group otherwise), plus the
    # compensation's second add in the compensated mode
    chunked = sweep_kernel_name(prob, precision) == "sweep_chunk_kernel"
    per_seg = ((G + 3) // 4 if chunked else G) * (2 if precision == "fp32" else 1)
    atom_ops = 2 * S * per_seg
    out = {"bound": "alu", "achieved": ops / sweep_s / 1e9, "peak": peak / 1e9, "unit": "Gop/s",
           "frac": ops / sweep_s / peak, "traffic": ncu.get("dram_bytes"),
           "kernel": sweep_kernel_name(prob, precision), "avg_launch_ms": sweep_s * 1e3,
           "ops_per_update": OPS_PER_UPDATE, "updates_per_launch": ups, "peak_note": peak_note,
           "impl_ops_per_update": IMPL_OPS_PER_UPDATE if precision != "fp64" else None,
           "impl_frac": IMPL_OPS_PER_UPDATE * ups / sweep_s / peak if precision != "fp64" else None,
           "frac_of_measured_fma": ops / sweep_s / measured if measured else None,
           "alg_bytes_per_launch": alg_bytes, "hbm_frac_of_measured": alg_bytes / sweep_s / 1e9 / hbm,
           "traffic_frac_of_measured_hbm": (ncu["dram_bytes"] / sweep_s / 1e9 / hbm) if ncu.get("dram_bytes") else None,
           "l2_hit_rate": ncu.get("l2_hit_pct"),
           "atomic_lane_ops_per_launch": atom_ops, "atomic_lane_ops_per_s": atom_ops / sweep_s}
    return out


def e2e_rate(m, steps: int, ups: int, world: int, local: int):
    """The metric end to end through the public API with host buffers in pinned memory: each step
    sets the FP64 state (flux, k, boundary flux) from the host, runs one outer and reads the FP64
    flux and k back; the library reads and writes the pinned arrays in place."""
    import torch
    import torch.distributed as dist

    phi_a, k0, psi_a = m.get_state(with_psi=True)
    phi0 = torch.empty(phi_a.shape, dtype=torch.float64, pin_memory=True).numpy()
    psi0 = torch.empty(psi_a.shape, dtype=torch.float64, pin_memory=True).numpy()
    phi_out = torch.empty(phi_a.shape, dtype=torch.float64, pin_memory=True).numpy()
    phi0[...] = phi_a
    psi0[...] = psi_a
    h2d = 8 * (phi0.size + psi0.size)
    d2h = 8 * phi_out.size + 8 * 8
    for _ in range(2):
        m.set_state(phi0, k0, psi0)
        m.outer(1, read=False)
        m.get_state(out=(phi_out, None))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        m.set_state(phi0, k0, psi0)
        m.outer(1, read=False)
        m.get_state(out=(phi_out, None))
    e2e_s = time.perf_counter() - t0
    value = whole_job_rate(ups * steps, world, max_over_ranks(e2e_s, world, f"cuda:{local}"))
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def workload_block(moc, prob, name, precision, local, stream, flush, steps, warmup, n_sm, rates, cmfd=None):
    """One workload measured like the headline (without the clocks and e2e): outers per second,
    the sweep's roofline, and the FP64 mode's rate."""
    from paper_2607_01591_gb300 import workloads as W

    m = moc.Moc.from_problem(prob, device=local, precision=precision, stream=stream.cuda_stream)
    _, ups, kpo = m.work()
    timed_outers(m, stream, flush, warmup)
    ms = timed_outers(m, stream, flush, steps)
    sw = sweep_seconds(m, stream, flush, steps)
    T, S = m.track_counts()
    out = {"workload": WORKLOADS[name], "precision": precision, "segments": S, "tracks": T,
           "updates_per_step": ups, "ms_per_step": ms / steps, "value": ups * steps / (ms / 1e3), "unit": UNIT,
           "roofline": roofline(prob, m, precision, sw, ups, name, n_sm, rates), "gpu_launches_per_outer": kpo}
    m.close()
    return out


def fp64_block(moc, prob, name, local, stream, flush, steps, n_sm, rates):
    """The FP64 mode of a workload: outers per second and the sweep's FP64 roofline."""
    m = moc.Moc.from_problem(prob, device=local, precision="fp64", stream=stream.cuda_stream)
    _, ups, _ = m.work()
    timed_outers(m, stream, flush, 1)
    ms = timed_outers(m, stream, flush, steps)
    sw = sweep_seconds(m, stream, flush, 1)
    out = {"value": ups * steps / (ms / 1e3), "ms_per_step": ms / steps,
           "roofline": roofline(prob, m, "fp64", sw, ups, name, n_sm, rates)}
    m.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_plain", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help=f"default: {DEFAULT_WORKLOAD} (with --dgmoc-only: the assembly, whose extruded "
                         "stack the default line's DGMOC block measures)")
    ap.add_argument("--no-time-to-k", action="store_true")
    ap.add_argument("--no-tracking", action="store_true", help="skip the host vs device tracking timing")
    ap.add_argument("--no-assembly", action="store_true", help="skip the 17x17 assembly block")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the core and pin-cell blocks (FP32 and FP64 outers of the other configurations)")
    ap.add_argument("--warm-eval", type=int, default=20, metavar="N",
                    help="held-out instances of the learned warm-start block (0 skips it)")
    ap.add_argument("--no-rates", action="store_true", help="skip the hardware rate probes")
    ap.add_argument("--aniso", type=int, default=0, metavar="L",
                    help="time outers with P_L anisotropic scattering (synthetic moments g^l Sigma_s)")
    ap.add_argument("--axial", type=int, default=8, metavar="NZ",
                    help="planes of the DGMOC measurement on the extruded assembly (0 skips it)")
    ap.add_argument("--dgmoc-only", action="store_true",
                    help="run only the DGMOC measurement (FP32 with its time to converged k, and FP64) "
                         "and print it")
    ap.add_argument("--rates-only", action="store_true",
                    help="print the hardware rate probes (FMA issue, L2 atomics) of this GPU and exit")
    ap.add_argument("--cmfd", default=None, metavar="SIZE,NOUT,NIN,OMEGA",
                    help="time CMFD-accelerated outers (square coarse cells of SIZE cm); also the "
                         "parameters of the accelerated time-to-k runs")
    ap.add_argument("--cmfd-tol", type=float, default=0.0,
                    help="stop each outer's coarse power iteration once k and the coarse source settle "
                         "to this (0: the fixed count)")
    args = ap.parse_args()
    if args.workload is None:
        args.workload = "assembly" if args.dgmoc_only else DEFAULT_WORKLOAD
    cm_defaults = {"assembly": "1.26,6,6,1.0", "core": "1.26,80,3,1.5", "hexcore": "2.52,10,5,1.0",
                   "hexcore7": "2.52,10,5,1.0", "hexcore1": "2.52,10,5,1.0", "pin": "0.63,6,6,1.0"}

    def cm_params(name, spec=None):
        f = (spec or cm_defaults[name]).split(",")
        return float(f[0]), int(f[1]), int(f[2]), float(f[3])

    cmfd = cm_params(args.workload, args.cmfd)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.warmup < 3:
        args.warmup = 3

    import torch
    import torch.distributed as dist

    from paper_2607_01591_gb300 import moc
    from paper_2607_01591_gb300 import workloads as W
    from paper_2607_01591_gb300.build import build

    if world > 1:
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    moc.load_library()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    if args.rates_only:
        with ClockSampler(local) as clk:
            rates = measured_rates(local)
        if rank == 0:
            print(json.dumps({"rates": rates, "clocks": clk.summary()}), flush=True)
        return
    prob = make_problem(args.workload)
    stream = torch.cuda.Stream(device=local)
    if args.dgmoc_only:
        blk = dgmoc_block(moc, W, prob, local, stream, args.precision, args.axial, args.steps,
                          converge=not args.no_time_to_k, name=args.workload)
        blk64 = (dgmoc_block(moc, W, prob, local, stream, "fp64", args.axial, 1, name=args.workload)
                 if args.fp64_steps > 0 else None)
        if rank == 0:
            print(json.dumps({"dgmoc": blk, "dgmoc_fp64": blk64}), flush=True)
        return
    rates = None if args.no_rates else measured_rates(local)
    m = moc.Moc.from_problem(prob, device=local, precision=args.precision, stream=stream.cuda_stream)
    if args.cmfd:
        cm_cell, cm_n = W.grid_cells(prob.mesh, cmfd[0])
        m.set_cmfd(cm_cell, cm_n, cmfd[1], cmfd[2], cmfd[3])
        m.set_cmfd_tolerance(args.cmfd_tol)
    aniso_g = None
    if args.aniso:
        # mean scattering cosines by material kind: light moderator strongly forward, heavy fuel weakly
        aniso_g = [0.4 if i == prob.xs.n_mat - 1 else 0.05 for i in range(prob.xs.n_mat)]
        m.set_scattering(W.anisotropic_moments(prob.xs, args.aniso, aniso_g))
    n_seg, ups, kpo = m.work()
    T, _ = m.track_counts()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")

    # warm-up (also builds the CUDA graphs), then the timed steps with the clocks sampled
    timed_outers(m, stream, flush, args.warmup)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = timed_outers(m, stream, flush, args.steps)
    torch.cuda.synchronize()
    ms_max = max_over_ranks(ms, world, f"cuda:{local}")
    value = whole_job_rate(ups * args.steps, world, ms_max / 1e3)

    # dominant kernel: the sweep, timed by the library's CUDA events around each launch on its stream
    sweep_s = sweep_seconds(m, stream, flush, args.steps)
    roof = roofline(prob, m, args.precision, sweep_s, ups, args.workload, n_sm, rates or {})
    e2e = e2e_rate(m, args.steps, ups, world, local)
    m.close()

    # FP64 mode on the same workload, with its own roofline (nominal FP64 FMA rate)
    fp64 = None
    if args.precision != "fp64" and args.fp64_steps > 0:
        m64 = moc.Moc.from_problem(prob, device=local, precision="fp64", stream=stream.cuda_stream)
        timed_outers(m64, stream, flush, 1)
        ms64 = timed_outers(m64, stream, flush, args.fp64_steps)
        sw64 = sweep_seconds(m64, stream, flush, 1)
        fp64 = {"value": ups * args.fp64_steps / (ms64 / 1e3), "ms_per_step": ms64 / args.fp64_steps,
                "roofline": roofline(prob, m64, "fp64", sw64, ups, args.workload, n_sm, rates or {})}
        m64.close()

    # time to converged k: outers from the cold start until |k - k_ref| <= 5 pcm (the plain
    # iteration too on the assembly, whose dominance ratio allows it)
    time_to_k = None
    if not args.no_time_to_k and args.workload in ("assembly", "core", "hexcore", "hexcore7"):
        time_to_k = time_to_converged_k(moc, prob, local, stream, cmfd, plain=args.workload == "assembly",
                                        cmfd_tol=args.cmfd_tol)

    extra = world == 1 and rank == 0
    # the 17x17 assembly measured the same way (it fits L2; its time to k plain and accelerated)
    assembly = None
    if extra and not args.no_assembly and args.workload != "assembly" and not args.aniso and not args.cmfd:
        aprob = make_problem("assembly")
        assembly = workload_block(moc, aprob, "assembly", args.precision, local, stream, flush, args.steps,
                                  args.warmup, n_sm, rates or {})
        if not args.no_time_to_k:
            assembly["time_to_k"] = time_to_converged_k(moc, aprob, local, stream, cm_params("assembly"), plain=True)

    # the other configurations of the scope table, FP32 and FP64: the 3x3-assembly core and the
    # pin cell (the assembly block above has its FP64 rate too)
    others = None
    if extra and not args.no_other_workloads and not args.aniso and not args.cmfd:
        others = {}
        for name in ("core", "pin"):
            if name == args.workload:
                continue
            oprob = make_problem(name)
            blk = workload_block(moc, oprob, name, args.precision, local, stream, flush, args.steps, args.warmup,
                                 n_sm, rates or {})
            if args.fp64_steps > 0:
                blk["fp64"] = fp64_block(moc, oprob, name, local, stream, flush, args.fp64_steps, n_sm, rates or {})
            others[name] = blk
    if assembly is not None and args.fp64_steps > 0:
        assembly["fp64"] = fp64_block(moc, make_problem("assembly"), "assembly", local, stream, flush,
                                      args.fp64_steps, n_sm, rates or {})

    # learned warm start on held-out assembly instances (the shipped network)
    warm = None
    if extra and args.warm_eval > 0 and not args.aniso and not args.cmfd:
        from paper_2607_01591_gb300 import warmstart

        warm = (warm_start_block(local, args.warm_eval) if os.path.exists(warmstart.SHIPPED)
                else {"unavailable": "no trained network at " + os.path.relpath(warmstart.SHIPPED, ROOT)})

    # DGMOC on the extruded assembly (FP32 timed; one FP64 outer for context)
    dgmoc = None
    if extra and args.axial > 0 and not args.aniso and not args.cmfd:
        aprob = make_problem("assembly")
        dgmoc = dgmoc_block(moc, W, aprob, local, stream, args.precision, args.axial, 5)
        if args.fp64_steps > 0 and args.precision != "fp64":
            d64 = dgmoc_block(moc, W, aprob, local, stream, "fp64", args.axial, 1)
            dgmoc["fp64"] = {"ms_per_outer": d64["ms_per_outer"], "value": d64["value"], "k_after": d64["k_after"]}
        if not args.no_cpu_baseline:
            dgmoc["cpu_baseline"] = dg_cpu_baseline(args.axial)

    # tracking of the headline workload: host half-edge walk vs the device walk (bit-identical tracks)
    tracking = None
    if not args.no_tracking and rank == 0:
        tr = {}
        for name in ("host", "device"):
            mt = moc.Moc(local, args.precision, stream.cuda_stream)
            mt.set_mesh(prob.mesh)
            mt.set_quadrature(prob.n_azim, prob.ray_spacing, prob.sin_theta, prob.polar_w)
            t0 = time.perf_counter()
            walk_ms = mt.generate_tracks_device() if name == "device" else None
            if name == "host":
                mt.generate_tracks()
            tr[name + "_s"] = time.perf_counter() - t0
            if walk_ms is not None:
                tr["device_walk_ms"] = walk_ms
            mt.close()
        tr["note"] = ("wall time of moc_generate_tracks (host walk, OpenMP) and moc_generate_tracks_device "
                      f"(walk on the GPU, two passes) including laydown, links, areas and upload; {os.cpu_count()} host cores")
        tracking = tr

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(make_problem("hexcore1"), ORACLE_SAMPLE)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp32_plain": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic (seeded mesh and cross sections shaped like the paper's lattice and core workloads)",
        "config": {"workload": WORKLOADS[args.workload], "precision": args.precision, "segments": n_seg, "tracks": T,
                   "updates_per_step": ups, "l2": "flushed between steps (512 MiB write, untimed)",
                   "parallelism": f"replicas x{world}",
                   "cmfd": (f"each step one CMFD-accelerated outer: {cmfd[0]} cm cells, {cmfd[1]} coarse power "
                            f"iterations x {cmfd[2]} sweeps per group, omega {cmfd[3]}") if args.cmfd else None,
                   "scattering": (f"P{args.aniso} anisotropic, Sigma_s,l = g^l Sigma_s,0, g per material {aniso_g}"
                                  if args.aniso else "isotropic")},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": kpo * args.steps,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "fp64": fp64,
        "time_to_k": time_to_k,
        "assembly": assembly,
        "other_workloads": others,
        "warm_start": warm,
        "tracking": tracking,
        "dgmoc": dgmoc,
        "rates": rates,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def warm_start_block(device: int, n_eval: int) -> dict:
    """The shipped warm-start network on n_eval held-out assembly instances (XS x lognormal(0.1)
    per material and group, seeds disjoint from training): outers and wall time to |k - k_ref| <=
    5 pcm from the cold FP64 start, the cold FP32 start, the training-mean solution without a
    network (ablation, mean over 20 training instances) and the learned FP32 start (feature and
    network kernels included)."""
    from paper_2607_01591_gb300 import warmstart
    from paper_2607_01591_gb300 import workloads as W

    base = warmstart.assembly_base()
    ws = warmstart.WarmStart(W.assembly_problem(), base, W.guide_tube_positions(), device)
    meta = ws.load(warmstart.SHIPPED)
    mean_pred = ws.mean_solution([W.perturbed_xs(base, warmstart.TRAIN_SEED + i) for i in range(20)])
    held = [W.perturbed_xs(base, warmstart.HELD_OUT_SEED + i) for i in range(n_eval)]
    r = warmstart.evaluate(ws, held, mean_pred, n_fp64=n_eval)
    r["network_times"] = ws.time_network()
    r["workload"] = WORKLOADS["assembly"] + "; XS x lognormal(0.1) per material and group"
    r["network"] = {"dims": ws.net.dims, "params": ws.net.n_params, "trained_on": meta.get("n_train"),
                    "file": os.path.relpath(warmstart.SHIPPED, ROOT)}
    r["n_eval"] = n_eval
    return r


if __name__ == "__main__":
    main()
