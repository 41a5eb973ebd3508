"""Benchmark: MOC segment*polar*group updates/s on the 17x17 assembly workload (one GB300).

A step is one outer iteration of the whole hot path: source update, transport sweep (tallies,
boundary-flux links, own FP32 exponential), flux finalisation and the FP64 fission/k/residual
reductions, on the seeded synthetic 17x17 assembly (39,304 triangles, 7 groups, 32 azimuths,
TY-3 polar, 0.02 cm ray spacing). updates per step = 2 * segments * polar * groups.

Prints one JSON line (rank 0). Under torchrun each rank runs an independent replica on its own
GPU (the sweep has no data-path exchange); value = all ranks' updates / max time. The line also
carries context measurements: the FP64 mode, the time to a converged k (plain and CMFD), host
against device tracking, and a `dgmoc` block (the assembly extruded to `--axial` planes, DGMOC
outers with their roofline and the oracle's DGMOC timed on a bounded sample); `--dgmoc-only`
prints only that block, with the time to converged k of the plain and the accelerated DGMOC.
`--impl reference` times the CPU oracle on the host cores instead (one oracle outer per step).
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
    "hexcore7": "central 7 hexagons of the hex core, 555,450 triangles, 33 groups, 48 azimuths, 3 polar, ray spacing 0.02 cm",
    "pin": "pin cell, 200 triangles, 7 groups, 16 azimuths, 3 polar, ray spacing 0.05 cm",
}
WORKLOAD = WORKLOADS["assembly"]


def make_problem(name: str):
    from paper_2607_01591_gb300 import workloads as W

    return {"assembly": W.assembly_problem, "core": W.core_problem, "hexcore": W.hex_core_problem,
            "hexcore7": lambda: W.hex_core_problem(n_rings=1), "pin": W.pin_cell_problem}[name]()
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) per launch of the sweep kernel from one ncu capture of the current kernel
# version on the assembly workload (profiles/sweep_kernel_assembly17.md); None for other workloads.
SWEEP_DRAM_BYTES = {"assembly": 82.312960e6 + 2.801920e6}


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


def cpu_baseline(prob, outers: int = 2):
    """The oracle as it stands on the host cores: `outers` outers of the full workload."""
    import oracle

    threads = min(os.cpu_count() or 1, prob.xs.n_groups)
    o = oracle.Oracle.from_problem(prob, threads=threads)
    o.normalise()
    t0 = time.perf_counter()
    for _ in range(outers):
        o.outer(True)
    dt = time.perf_counter() - t0
    ups = 2 * o.n_segments * len(prob.sin_theta) * prob.xs.n_groups
    return {"value": ups * outers / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{outers} oracle outers of the full workload (FP64, one thread per group), "
                      f"{dt:.2f} s"}


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
# actually executes, from ncu on the extruded assembly (profiles/dg_sweep_assembly17x8.md)
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


def time_to_converged_k(moc, prob, device, stream, cmfd, plain: bool = True, pcm: float = 5.0):
    """Wall time and outers of the cold-start power iteration until |k - k_ref| <= pcm * 1e-5, in
    FP32 and FP64, plain (when `plain`) and CMFD-accelerated with cmfd = (cell size, coarse power
    iterations, sweeps per group, omega). k_ref: FP32 to |dk| <= 1e-7 continued in FP64 to
    |dk| <= 1e-10, accelerated when the plain iteration is not run (the accelerated limit is the
    transport solution)."""
    import torch
    from paper_2607_01591_gb300 import workloads as W

    cell, n_cells = W.grid_cells(prob.mesh, cmfd[0])
    accel = lambda ctx: ctx.set_cmfd(cell, n_cells, cmfd[1], cmfd[2], cmfd[3])
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
                   f"{cmfd[2]} Gauss-Seidel sweeps per group, over-relaxation {cmfd[3]}"}
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
    ref32.close()
    ref64.close()
    return out


def run_reference(args, rank, world):
    from paper_2607_01591_gb300 import workloads as W
    import oracle

    if rank != 0:
        return
    prob = W.assembly_problem()
    threads = min(os.cpu_count() or 1, prob.xs.n_groups)
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
            "config": {"workload": WORKLOAD, "updates_per_step": ups},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": v, "unit": UNIT,
                             "sample": f"{args.steps} oracle outers of the full workload after {args.warmup} warm-up"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_plain", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--workload", default="assembly", choices=sorted(WORKLOADS))
    ap.add_argument("--no-time-to-k", action="store_true")
    ap.add_argument("--no-tracking", action="store_true", help="skip the host vs device tracking timing")
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
    args = ap.parse_args()
    cm_default = {"assembly": "1.26,6,6,1.0", "core": "1.26,80,3,1.5", "hexcore": "2.52,10,5,1.0", "hexcore7": "2.52,10,5,1.0",
                  "pin": "0.63,6,6,1.0"}[args.workload]
    cmp = (args.cmfd or cm_default).split(",")
    cmfd = (float(cmp[0]), int(cmp[1]), int(cmp[2]), float(cmp[3]))
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
    m = moc.Moc.from_problem(prob, device=local, precision=args.precision, stream=stream.cuda_stream)
    if args.cmfd:
        cm_cell, cm_n = W.grid_cells(prob.mesh, cmfd[0])
        m.set_cmfd(cm_cell, cm_n, cmfd[1], cmfd[2], cmfd[3])
    aniso_g = None
    if args.aniso:
        # mean scattering cosines by material kind: light moderator strongly forward, heavy fuel weakly
        aniso_g = [0.4 if i == prob.xs.n_mat - 1 else 0.05 for i in range(prob.xs.n_mat)]
        m.set_scattering(W.anisotropic_moments(prob.xs, args.aniso, aniso_g))
    n_seg, ups, kpo = m.work()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")

    def timed_steps(mm, k, flush_l2=True):
        evs = []
        with torch.cuda.stream(stream):
            for _ in range(k):
                if flush_l2:
                    flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                mm.outer(1, read=False)
                e1.record(stream)
                evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    # warm-up (also builds the CUDA graphs)
    timed_steps(m, args.warmup)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = timed_steps(m, args.steps)
    torch.cuda.synchronize()
    ms_max = max_over_ranks(ms, world, f"cuda:{local}")
    value = whole_job_rate(ups * args.steps, world, ms_max / 1e3)

    # dominant kernel: the sweep, timed by CUDA events around each launch on its stream
    m.enable_timing(True)
    timed_steps(m, args.steps)
    sweep_ms, n_sw = m.timing()
    m.enable_timing(False)
    sweep_avg_s = sweep_ms / n_sw / 1e3
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 ALU peak: 152 SMs x 128 FP32 lanes x max SM clock (instructions/s, FMA = 1)
    alu_peak = 152 * 128 * sm_max * 1e6
    ops_per_update = 19
    achieved = ops_per_update * ups / sweep_avg_s
    seg_bytes = 8 if args.precision != "fp64" else 16
    R, G, P = prob.mesh.n_tri, prob.xs.n_groups, len(prob.sin_theta)
    T, _ = m.track_counts()
    alg_bytes = seg_bytes * n_seg + R * 8 * (8 + 8) + 2 * T * 2 * P * G * 4
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))

    # end to end through the public API with host buffers in pinned memory (H2D state, outer, D2H
    # flux and k); the library reads and writes pinned arrays in place with one kernel each way
    phi_a, k0, psi_a = m.get_state(with_psi=True)
    phi0 = torch.empty(phi_a.shape, dtype=torch.float64, pin_memory=True).numpy()
    psi0 = torch.empty(psi_a.shape, dtype=torch.float64, pin_memory=True).numpy()
    phi_out = torch.empty(phi_a.shape, dtype=torch.float64, pin_memory=True).numpy()
    phi0[...] = phi_a
    psi0[...] = psi_a
    # bytes crossing the host link per step: the FP64 state read in place, the FP64 flux and the
    # scalars written back
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
    for _ in range(args.steps):
        m.set_state(phi0, k0, psi0)
        m.outer(1, read=False)
        m.get_state(out=(phi_out, None))
    e2e_s = time.perf_counter() - t0
    e2e_value = whole_job_rate(ups * args.steps, world, max_over_ranks(e2e_s, world, f"cuda:{local}"))

    # FP64 mode on the same workload (context for the FP32 numbers)
    fp64 = None
    if args.precision != "fp64" and args.fp64_steps > 0:
        m64 = moc.Moc.from_problem(prob, device=local, precision="fp64", stream=stream.cuda_stream)
        timed_steps(m64, 2)
        ms64 = timed_steps(m64, args.fp64_steps)
        fp64 = {"value": ups * args.fp64_steps / (ms64 / 1e3), "ms_per_step": ms64 / args.fp64_steps}
        m64.close()

    # time to converged k: outers from the cold start until |k - k_ref| <= 5 pcm, k_ref from FP32
    # convergence continued in FP64 to |dk| <= 1e-10 (same workload, same stream)
    time_to_k = None
    if not args.no_time_to_k and args.workload in ("assembly", "core", "hexcore"):
        time_to_k = time_to_converged_k(moc, prob, local, stream, cmfd, plain=args.workload == "assembly")

    # DGMOC on the extruded assembly (FP32 timed; one FP64 outer for context)
    dgmoc = None
    if args.axial > 0 and args.workload == "assembly":
        dgmoc = dgmoc_block(moc, W, prob, local, stream, args.precision, args.axial, 5)
        if args.fp64_steps > 0 and args.precision != "fp64":
            d64 = dgmoc_block(moc, W, prob, local, stream, "fp64", args.axial, 1)
            dgmoc["fp64"] = {"ms_per_outer": d64["ms_per_outer"], "value": d64["value"], "k_after": d64["k_after"]}
        if not args.no_cpu_baseline and world == 1:
            dgmoc["cpu_baseline"] = dg_cpu_baseline(args.axial)

    # tracking of the same workload: host half-edge walk vs the device walk (bit-identical tracks)
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
    cpu = None if args.no_cpu_baseline or world > 1 or args.workload != "assembly" else cpu_baseline(prob)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp32_plain": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic (seeded mesh and cross sections shaped like the paper's lattice workloads)",
        "config": {"workload": WORKLOADS[args.workload], "precision": args.precision, "segments": n_seg, "tracks": T,
                   "updates_per_step": ups, "l2": "flushed between steps (512 MiB write, untimed)",
                   "parallelism": f"replicas x{world}",
                   "cmfd": (f"each step one CMFD-accelerated outer: {cmfd[0]} cm cells, {cmfd[1]} coarse power "
                            f"iterations x {cmfd[2]} sweeps per group, omega {cmfd[3]}") if args.cmfd else None,
                   "scattering": (f"P{args.aniso} anisotropic, Sigma_s,l = g^l Sigma_s,0, g per material {aniso_g}"
                                  if args.aniso else "isotropic")},
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": alu_peak / 1e9, "unit": "Gop/s",
                     "frac": achieved / alu_peak,
                     "traffic": SWEEP_DRAM_BYTES.get(args.workload) if args.precision == "fp32" and not args.cmfd and not args.aniso else None,
                     "kernel": "sweep_kernel", "avg_launch_ms": sweep_avg_s * 1e3,
                     "ops_per_update": ops_per_update,
                     "peak_note": "152 SMs x 128 FP32 lanes x max SM clock (derived; FMA counted as 1 op)",
                     "hbm_frac_of_measured": alg_bytes / sweep_avg_s / 1e9 / hbm_peak,
                     "alg_bytes_per_launch": alg_bytes},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": kpo * args.steps,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "fp64": fp64,
        "time_to_k": time_to_k,
        "tracking": tracking,
        "dgmoc": dgmoc,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
