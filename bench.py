#!/usr/bin/env python
"""Benchmark of the Stokes / additive-Vanka multigrid / FGMRES hot path on GB300.

Metric: Stokes DoF/s per Vanka V-cycle, together with the FGMRES time to a
1e-8 relative residual.  One step = one FGMRES(30) solve to 1e-8,
right-preconditioned by the V(2,2) additive-Vanka cycle (every hot-path step:
residual, patch gather/solve/scatter, restriction, coarse solve, prolongation,
Arnoldi).  value = dofs x V-cycles applied / timed seconds (all ranks).

Default workload: 2048 x 2048 elements (37,769,219 dofs incl. Dirichlet rows),
10 levels, FP64, body force i.i.d. N(0,1) nodal values (seed 0), Dirichlet
velocity from the manufactured field.  Every vector (302 MB) is larger than
L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 2048] [--impl ours|reference]

With N > 1 (torchrun) each rank solves its own independent replica of the
problem (the method has no data-path exchange between problems): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes DoF/s per Vanka V-cycle + FGMRES time-to-1e-8 residual, mixed vs FP64"
UNIT = "DoF/s"
SM_COUNT = 152
ORACLE_N = 256


def dofs(n: int) -> int:
    return 2 * (2 * n + 1) ** 2 + (n + 1) ** 2


def sweep_flops(n: int) -> float:
    """Algorithmic FP64 flops of one additive Vanka sweep on an n x n grid.

    Per vertex (one patch, and one cell of owned dofs: 4 Q2 nodes x 2
    components + 1 pressure): residual 2 (2 (64 + 12) + 24) + 9 = 361 and
    weighted update 2 (9 + 6 + 6 + 4) + 16 + 2 = 68.  Patch solve (Schur
    factored, K^-1 by fast diagonalisation): the (n - 3)^2 interior patches use
    the symmetric / antisymmetric split, 2 x (4 stages x 5 vectors x 25 + 25)
    = 1050, plus 102 for dp and 100 for the z-correction: 1252; the 8n - 8
    boundary patches use full 5 x 5 per-axis factors, 2 x (4 x 25 x 10 + 25)
    = 2050, plus 202: 2252."""
    nv = (n + 1) ** 2
    ni = (n - 3) ** 2 if n >= 4 else 0
    return nv * (361.0 + 68.0) + ni * 1252.0 + (nv - ni) * 2252.0


def sweep_bytes(n: int) -> float:
    """Algorithmic bytes of one FP64 sweep: read x and b, write x."""
    return 3.0 * 8.0 * dofs(n)


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.bus_id and self.bus_id not in parts[1].lower() and parts[1].lower() not in self.bus_id:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# CPU oracle leg (subprocess, single-threaded BLAS)
# --------------------------------------------------------------------------
def oracle_worker(n: int, reps: int) -> None:
    """Time the CPU oracle's FGMRES + V(2,2) solve at n x n (prints one JSON object)."""
    import numpy as np

    import stokes_inputs as si
    from oracle import stokes_oracle as O

    t0 = time.perf_counter()
    H = O.build_hierarchy(n)
    lv = H.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 0), si.manufactured_velocity(n))
    setup = time.perf_counter() - t0
    times, its = [], []
    for _ in range(reps):
        t = time.perf_counter()
        res = O.solve(H, b)
        times.append(time.perf_counter() - t)
        its.append(res.iters)
    per = float(np.median(times))
    it = int(np.median(its))
    print(json.dumps({"n": n, "dofs": dofs(n), "solve_s": per, "iters": it, "setup_s": setup,
                      "value": dofs(n) * it / per}))


def oracle_vcycle(n: int) -> None:
    """Time the CPU oracle's set-up and one V(2,2) cycle at n x n (single thread; prints
    one JSON object).  At 2048^2 this takes minutes of set-up and about a minute per
    V-cycle, too long for the bounded CPU sample of the default run: run it on demand."""
    import resource

    import stokes_inputs as si
    from oracle import stokes_oracle as O

    t0 = time.perf_counter()
    H = O.build_hierarchy(n)
    lv = H.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 0), si.manufactured_velocity(n))
    setup = time.perf_counter() - t0
    t = time.perf_counter()
    O.vcycle(H, b)
    vc = time.perf_counter() - t
    print(json.dumps({"n": n, "dofs": dofs(n), "levels": len(H.levels), "setup_s": setup, "vcycle_s": vc,
                      "value": dofs(n) / vc, "unit": UNIT, "cores": 1,
                      "max_rss_gb": resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 1e6}))


def run_oracle(n: int, reps: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", "--n", str(n),
                        "--steps", str(reps)], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle worker failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_all_cores(n: int, procs: int) -> dict:
    """The oracle on every host core: `procs` single-threaded worker processes
    (spawned, not forked) each solve the same n x n problem at the same time;
    the aggregate is procs x dofs x V-cycles over the slowest worker's solve."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", "--n", str(n), "--steps", "1"]
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)
          for _ in range(procs)]
    outs = []
    for p in ps:
        so, se = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle worker failed:\n" + se[-2000:])
        outs.append(json.loads(so.strip().splitlines()[-1]))
    slowest = max(o["solve_s"] for o in outs)
    o = outs[0]
    return {"n": n, "dofs": o["dofs"], "iters": o["iters"], "procs": procs, "solve_s_max": slowest,
            "value": procs * o["dofs"] * o["iters"] / slowest}


# --------------------------------------------------------------------------
# distributed helpers
# --------------------------------------------------------------------------
def dist_setup(ngpus: int):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(ws, v: float, op) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allmax(ws, v: float) -> float:
    """Maximum over ranks (the slowest rank's time)."""
    import torch.distributed as dist
    return _reduce(ws, v, dist.ReduceOp.MAX if ws > 1 else None)


def allsum(ws, v: float) -> float:
    """Sum over ranks (units processed by the whole job)."""
    import torch.distributed as dist
    return _reduce(ws, v, dist.ReduceOp.SUM if ws > 1 else None)


def job_throughput(ws, units_local: float, ms_local: float) -> tuple[float, float]:
    """Whole-job units/s over replicas: units summed over ranks / max time over ranks."""
    ms = allmax(ws, ms_local)
    units = allsum(ws, units_local)
    return units / (ms * 1e-3), ms


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the finest-level sweep
# kernel at 1024 x 1024 (ncu --set full, summaries in profiles/); at other sizes the
# bench scales them by the number of dofs (the traffic of a sweep is proportional)
TRAFFIC_1024 = {
    "fp64": {"bytes": 151244032 + 45977088 + 84809216 + 172724736 + 269548032 + 56484864, "tile": "split16x16x2",
             "source": "profiles/k_vanka_own_f64_n1024.md (k_apply<double> residual + k_vanka_own<double,16,16,256,2> "
                       "+ k_colsum_update, a sweep from a non-zero iterate; "
                       "writes still in L2 at kernel end are not counted)"},
    "mixed": {"bytes": 77614592 + 7096320, "tile": "14x14",
              "source": "profiles/k_vanka_strip_f32_n1024.md (k_vanka_strip<false> interior strips; the ring "
                        "launch is not included; writes still in L2 at kernel end are not counted)"},
    "bf16": {"bytes": 76957440 + 6176256, "tile": "14x14",
             "source": "profiles/k_vanka_strip_bf16_n1024.md (k_vanka_strip<true> interior strips; the ring "
                       "launch is not included; writes still in L2 at kernel end are not counted)"},
}


def fp64_peak(dev) -> dict:
    """The FP64 peak of this GPU, measured in this run: the library's FMA-chain probe
    (stokes_measure_fp64_peak) and a cuBLAS DGEMM (4096^3, through torch.matmul),
    best of three each; the larger is the roofline denominator of the FP64 kernels."""
    import torch

    from paper_2401_06277_gb300 import stokes
    probe = stokes.stokes_measure_fp64_peak()
    n = 4096
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    a = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    b = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    dgemm = 2.0 * n ** 3 / (best * 1e-3) / 1e9
    del a, b
    return {"peak": max(probe, dgemm), "fma_probe_gflops": round(probe, 1), "dgemm_gflops": round(dgemm, 1),
            "source": "measured in this run: FP64 FMA-chain probe (stokes_measure_fp64_peak) and cuBLAS "
                      "DGEMM 4096^3 (torch.matmul), best of three each; the larger of the two"}


FP64_PEAK = None   # set once per run by run_ours


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


PRECS = {"fp64": 0, "mixed": 1, "bf16": 2}
# share of the finest-level sweeps of a V(2,2) cycle that start from a zero guess
ZERO_GUESS_SHARE = 1.0 / 4.0
# sweep configurations by stokes_level_tile: fused tiles of TX x TY vertices, or (4, 5; FP64
# only) the split sweep: 16 x 16 own-patch solves writing the corrections, then the update
# (5: compiled for two CTAs per SM)
TILE_NAMES = ["8x8", "16x8", "16x16", "14x14", "split16x16", "split16x16x2", "4x4"]


VC_REPS = 20   # graph replays of the bare V-cycle (median reported)


def time_form(args, prec_name, ws, rank, f_host, ud_host, with_e2e, smoother=0, hkw=None, n=None):
    """Time K FGMRES solves of one precision form (smoother 1: per-patch inverses, the
    paper's simple Vanka); returns the record.  The form runs on a stream of its own
    (not the legacy default stream), so that its bare V-cycle can be captured as a
    CUDA graph."""
    import torch

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        rec = _time_form(args, prec_name, ws, rank, f_host, ud_host, with_e2e, smoother, hkw, n)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    return rec


def _time_form(args, prec_name, ws, rank, f_host, ud_host, with_e2e, smoother, hkw, n):
    import torch

    import paper_2401_06277_gb300 as pkg
    from paper_2401_06277_gb300 import stokes

    dev = torch.device("cuda", torch.cuda.current_device())
    if n is None:
        n = args.n
    else:   # a secondary form timed at another size: its own seeded inputs
        import stokes_inputs as si
        f_host = torch.from_numpy(si.random_force(n, args.seed + rank))
        ud_host = torch.from_numpy(si.manufactured_velocity(n))
    N = dofs(n)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    H = pkg.Hierarchy(n, rtol=1e-8, restart=30, prec=PRECS[prec_name], tile=args.tile, smoother=smoother,
                      **(hkw or {}))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    f = f_host.to(dev)
    ud = ud_host.to(dev)
    b = H.assemble_rhs(f, ud)
    x = torch.empty_like(b)
    stream = torch.cuda.current_stream()

    def step():
        stokes.stokes_initial_guess(H.handle, b, x)
        it, rel, st = stokes.stokes_fgmres_solve(H.handle, b, x)
        return it, rel

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stokes.stokes_stats_reset(H.handle)
    stokes.stokes_stats_enable_timing(H.handle, True)
    l0 = stokes.stokes_stats_read(H.handle)["kernel_launches"]
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    clocks = ClockSampler(f"{bus:02x}:00" if isinstance(bus, int) else None)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters, rels = [], []
    for _ in range(args.steps):
        it, rel = step()
        iters.append(it)
        rels.append(rel)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    st = stokes.stokes_stats_read(H.handle)
    stokes.stokes_stats_enable_timing(H.handle, False)
    launches = st["kernel_launches"] - l0
    value, ms_max = job_throughput(ws, N * st["vcycles"], ms)
    vcycles_all = allsum(ws, st["vcycles"])
    sweep_ms = st["sweep_ms"] / max(st["sweeps_timed"], 1)
    tile = TILE_NAMES[stokes.stokes_level_tile(H.handle, H.levels - 1)]
    peaks = measured_peaks()
    sm_max = args.sm_max_mhz or peaks.get("sm_max_mhz", 2070.0)
    if (hkw or {}).get("precond") == 1:
        # no relaxation sweeps: the preconditioner is 2 x 3 V(3,3) cycles of scalar
        # multigrid (Jacobi on L and M); its cost per application is vcycle_only below
        roofline = {"bound": "hbm", "kernel": "block-triangular preconditioner (scalar multigrid on L and M)",
                    "achieved": None, "peak": peaks.get("hbm_gbs", 6780.0), "unit": "GB/s", "frac": None,
                    "traffic": None, "note": "no Vanka/Braess-Sarazin sweep to time; see vcycle_only"}
    elif smoother in (2, 3):
        # Braess-Sarazin (two Jacobi steps) per vertex: residual 361, g and diag(S) 2 x 48,
        # Jacobi step with S dp as a 21-tap vertex stencil 2 x 21 + 4, du 2 x 4 x (9 + 3) + 2 x 9:
        # ~620 flops.  Vector passes: residual 3 (x, b -> r); g 1 + 3 pressure (-> g, diag(S),
        # dp); Jacobi 4 pressure (dp, g, diag(S) -> dp); update 3 + 1 pressure
        esz = 8.0 if prec_name == "fp64" else 4.0
        fl = (n + 1) ** 2 * 620.0
        by = esz * (7.0 * dofs(n) + 8.0 * (n + 1) ** 2)
        if prec_name == "fp64":
            peak = FP64_PEAK["peak"]
            achieved = fl / (sweep_ms * 1e-3) / 1e9
            roofline = {"bound": "alu", "kernel": "Braess-Sarazin sweep (k_apply + k_bs_*, finest level)",
                        "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "GFLOP/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "peak_source": FP64_PEAK["source"],
                        "algorithmic_flops_per_launch": fl, "algorithmic_bytes_per_launch": by,
                        "hbm_gbs_achieved": round(by / (sweep_ms * 1e-3) / 1e9, 1)}
        else:
            peak = peaks.get("hbm_gbs", 6780.0)
            achieved = by / (sweep_ms * 1e-3) / 1e9
            roofline = {"bound": "hbm", "kernel": "Braess-Sarazin sweep (k_apply + k_bs_*, finest level, FP32)",
                        "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)",
                        "algorithmic_bytes_per_launch": by}
    elif smoother == 1:
        # per vertex: residual 361, dense 51 x 51 patch inverse 5202, update 68 flops;
        # bytes: the inverse (2601 doubles), x, b, x_out and the 51 corrections written and read
        fl = (n + 1) ** 2 * (361.0 + 5202.0 + 68.0)
        by = (n + 1) ** 2 * 8.0 * (2601 + 2 * 51) + sweep_bytes(n)
        peak = FP64_PEAK["peak"]
        achieved = fl / (sweep_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "kernel": "simple Vanka sweep (k_apply + k_patch_solve + k_patch_update, finest)",
                    "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "GFLOP/s",
                    "frac": round(achieved / peak, 4), "traffic": None,
                    "peak_source": FP64_PEAK["source"],
                    "algorithmic_flops_per_launch": fl, "algorithmic_bytes_per_launch": by,
                    "hbm_gbs_achieved": round(by / (sweep_ms * 1e-3) / 1e9, 1),
                    "hbm_frac": round(by / (sweep_ms * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6780.0), 4)}
    elif prec_name == "fp64":
        # the first pre-smoothing sweep of each cycle starts from zero (no residual: 361 flops
        # per vertex fewer); the timed launches average over all nu1 + nu2 sweeps
        fl = sweep_flops(n) - ZERO_GUESS_SHARE * 361.0 * (n + 1) ** 2
        peak = FP64_PEAK["peak"]
        achieved = fl / (sweep_ms * 1e-3) / 1e9
        kname = ("k_apply<double> + k_vanka_own<double,16,16> + k_colsum_update (split sweep, finest level)"
                 if tile.startswith("split")
                 else "k_vanka<double> (finest level)")
        roofline = {"bound": "alu", "kernel": kname, "achieved": round(achieved, 2),
                    "peak": round(peak, 1), "unit": "GFLOP/s", "frac": round(achieved / peak, 4),
                    "traffic": args.traffic,
                    "peak_source": FP64_PEAK["source"],
                    "fp64_peaks": {k: FP64_PEAK[k] for k in ("fma_probe_gflops", "dgemm_gflops")},
                    "nominal_gflops": round(SM_COUNT * 4 * sm_max * 1e6 / 1e9, 1),
                    "algorithmic_flops_per_launch": fl,
                    "executed_flops_note": "the kernels execute fewer FP64 flops than the algorithmic count (about "
                                           "1071 against 1681 per vertex at 1024^2, ncu: shared row transforms, the fused "
                                           "column pass and the shared last pass of the fast diagonalisation, the "
                                           "residual once per cell); profiles/k_vanka_own_f64_n1024.md",
                    "algorithmic_bytes_per_launch": sweep_bytes(n) * (3.0 - ZERO_GUESS_SHARE) / 3.0,
                    "hbm_gbs_achieved": round(sweep_bytes(n) * (3.0 - ZERO_GUESS_SHARE) / 3.0 / (sweep_ms * 1e-3) / 1e9, 1)}
    else:
        # read x and b, write x (FP32); the zero-guess sweeps do not read x
        by = (3.0 - ZERO_GUESS_SHARE) * 4.0 * N
        peak = peaks.get("hbm_gbs", 6780.0)
        achieved = by / (sweep_ms * 1e-3) / 1e9
        if tile == "14x14":
            kname = ("k_vanka_strip<true> (BF16 tcgen05 patch GEMMs) on the interior strips + k_vanka<float,14,14> "
                     "ring (finest level)" if prec_name == "bf16" else
                     "k_vanka_strip<false> (FP32 fast-diagonalisation solves) on the interior strips + "
                     "k_vanka<float,14,14> ring (finest level)")
        else:
            kname = "k_vanka<float> (finest level)"
        roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                    "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                    "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)",
                    "algorithmic_bytes_per_launch": by,
                    "fp32_gflops_achieved": round(sweep_flops(n) / (sweep_ms * 1e-3) / 1e9, 1)}
    names = TILE_NAMES
    tiles = [names[stokes.stokes_level_tile(H.handle, lv)] for lv in range(H.levels - 1, 0, -1)]
    roofline.update({"launch_ms": round(sweep_ms, 4) if st["sweeps_timed"] else None,
                     "launches_timed": st["sweeps_timed"], "tile": tile, "tiles_fine_to_coarse": tiles})
    tr = TRAFFIC_1024.get(prec_name) if smoother == 0 else None
    if tr is not None and tile == tr["tile"]:
        # DRAM bytes of one launch of the same kernel at 1024^2 (ncu capture), scaled by dofs
        roofline["traffic"] = round(tr["bytes"] * dofs(n) / dofs(1024))
        roofline["traffic_source"] = tr["source"]
    rec = {"value": value, "ms_per_step": ms_max / args.steps, "iters": iters, "relres": rels,
           "vcycles": int(vcycles_all), "ms_per_vcycle": ms_max / max(st["vcycles"], 1),
           "time_to_solution_s": ms_max / args.steps / 1e3, "roofline": roofline,
           "gpu_launches": launches, "clocks": clk, "levels": H.levels, "setup_s": t_setup}
    # the V-cycle alone (dofs per second of one preconditioner application), after the timed
    # region: one application to the assembled right-hand side captured as a CUDA graph,
    # replayed VC_REPS times after warm-up, CUDA events between replays, median interval
    z = torch.empty_like(b)
    for _ in range(2):
        stokes.stokes_vcycle_apply(H.handle, b, z)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        stokes.stokes_vcycle_apply(H.handle, b, z)
    for _ in range(3):
        graph.replay()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(VC_REPS + 1)]
    evs[0].record(stream)
    for k in range(VC_REPS):
        graph.replay()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    vc_ms = allmax(ws, statistics.median(evs[k].elapsed_time(evs[k + 1]) for k in range(VC_REPS)))
    rec["vcycle_only"] = {"ms": vc_ms, "value": ws * N / (vc_ms * 1e-3), "unit": UNIT,
                          "timing": f"median of {VC_REPS} replays of a captured CUDA graph"}
    del graph, z
    if with_e2e:
        # Every step copies its inputs (f, u_D) from pinned host memory and reads its
        # solution back.  The copies run on a second stream, double-buffered: step k + 1's
        # inputs travel while step k solves, and step k's solution returns while step
        # k + 1 solves.  The timed region holds every step's copies and compute.
        cs = torch.cuda.Stream()
        fb = [f, torch.empty_like(f)]
        udb = [ud, torch.empty_like(ud)]
        xb = [x, torch.empty_like(x)]
        xh = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(2)]
        bi = f_host.numel() * 8 + ud_host.numel() * 8
        bo = N * 8
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]    # inputs of slot s on the device
        ev_asm = [torch.cuda.Event(), torch.cuda.Event()]   # slot s's inputs consumed
        ev_sol = [torch.cuda.Event(), torch.cuda.Event()]   # slot s's solution ready
        ev_out = [torch.cuda.Event(), torch.cuda.Event()]   # slot s's solution on the host

        def copy_in(s_):
            with torch.cuda.stream(cs):
                cs.wait_event(ev_asm[s_])
                fb[s_].copy_(f_host, non_blocking=True)
                udb[s_].copy_(ud_host, non_blocking=True)
                ev_in[s_].record(cs)

        def run(steps):
            for s_ in range(2):   # no copy or solve of an earlier run still pending on the slots
                ev_asm[s_].record(stream)
                ev_out[s_].record(stream)
            copy_in(0)
            for k in range(steps):
                s_ = k % 2
                if k + 1 < steps:
                    copy_in(1 - s_)
                stream.wait_event(ev_in[s_])
                stokes.stokes_assemble_rhs(H.handle, fb[s_], udb[s_], b, n)
                ev_asm[s_].record(stream)
                stream.wait_event(ev_out[s_])   # the D2H of step k - 2 has read xb[s_]
                stokes.stokes_initial_guess(H.handle, b, xb[s_])
                stokes.stokes_fgmres_solve(H.handle, b, xb[s_])
                ev_sol[s_].record(stream)
                with torch.cuda.stream(cs):
                    cs.wait_event(ev_sol[s_])
                    xh[s_].copy_(xb[s_], non_blocking=True)
                    ev_out[s_].record(cs)
            for s_ in range(2):
                stream.wait_event(ev_out[s_])

        run(2)
        torch.cuda.synchronize()
        stokes.stokes_stats_reset(H.handle)
        barrier(ws)
        torch.cuda.synchronize()
        e0.record(stream)
        run(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        e2e_ms = allmax(ws, e0.elapsed_time(e1))
        e2e_vc = allsum(ws, stokes.stokes_stats_read(H.handle)["vcycles"])
        rec["e2e"] = {"value": N * e2e_vc / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
                      "d2h_bytes_per_step": bo, "ms_per_step": e2e_ms / args.steps,
                      "copies": "on a second stream, double-buffered: step k + 1's inputs and step k's "
                                "solution travel while the GPU solves"}
        x = xb[(args.steps - 1) % 2]
    if n == args.n:
        rec["_x"] = x.cpu()   # the last solve's solution, for the comparison across forms
    H.close()
    return rec


def solution_difference(x: "torch.Tensor", ref: "torch.Tensor", n: int) -> float:
    """max |x - ref| / max |ref| with both pressures shifted to zero mean (the pressure is
    defined up to a constant)."""
    p0 = 2 * (2 * n + 1) ** 2
    a, r = x.clone(), ref.clone()
    a[p0:] -= a[p0:].mean()
    r[p0:] -= r[p0:].mean()
    return float((a - r).abs().max() / r.abs().max())


def time_batch(args, prec_name: str) -> dict:
    """Batched form: (a) 64 right-hand sides (force seeds 1..64) on one 1024 x 1024 grid and
    (b) 32 problems with sizes drawn from {128, 256, 512, 1024} (generator seed 1000, force
    seeds 2000 + k), each set solved as one batch (lockstep FGMRES(12) to 1e-8, one CUDA graph
    per iteration).  Also times the same problems solved one after another."""
    import torch

    import stokes_inputs as si
    import paper_2401_06277_gb300 as pkg

    out = {}
    g = torch.Generator(device="cpu")
    g.manual_seed(1000)
    uneven = [int(v) for v in torch.tensor([128, 256, 512, 1024])[torch.randint(0, 4, (32,), generator=g)]]
    sets = {"rhs64_1024": ([args.batch_n] * args.batch_rhs, [1 + k for k in range(args.batch_rhs)]),
            "uneven32": (uneven, [2000 + k for k in range(32)])}
    for name, (ns, seeds) in sets.items():
        B = pkg.Batch(ns, prec=PRECS[prec_name], restart=12)
        rhs = []
        for k, (n, sd) in enumerate(zip(ns, seeds)):
            f = torch.from_numpy(si.random_force(n, sd)).cuda()
            ud = torch.from_numpy(si.manufactured_velocity(n)).cuda()
            rhs.append(B.assemble_rhs(k, f, ud))
            del f, ud
        B.solve(rhs)          # warm-up: captures the iteration graphs
        torch.cuda.synchronize()
        times, its = [], None
        for _ in range(max(1, args.batch_steps)):
            t0 = time.perf_counter()
            xs, its, rels = B.solve(rhs)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        dt = statistics.median(times)
        units = sum(dofs(n) * it for n, it in zip(ns, its))
        rec = {"problems": len(ns), "sizes": sorted(set(ns)), "solve_s": dt, "iters": its,
               "max_relres": max(rels), "value": units / dt, "unit": UNIT}
        B.close()
        del B, rhs, xs
        torch.cuda.empty_cache()
        # the same problems one after another (one hierarchy per size, graph-free path)
        seq = 0.0
        hs = {}
        for n, sd in zip(ns, seeds):
            if n not in hs:
                hs[n] = pkg.Hierarchy(n, prec=PRECS[prec_name], restart=12)
            H = hs[n]
            bb = H.assemble_rhs(torch.from_numpy(si.random_force(n, sd)).cuda(),
                                torch.from_numpy(si.manufactured_velocity(n)).cuda())
            H.solve(bb)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H.solve(bb)
            torch.cuda.synchronize()
            seq += time.perf_counter() - t0
        for H in hs.values():
            H.close()
        rec["sequential_s"] = seq
        out[name] = rec
    return out


def run_ours(args) -> None:
    import torch

    import stokes_inputs as si
    from paper_2401_06277_gb300 import build

    ws, rank, local = dist_setup(args.gpus)
    build.build()
    global FP64_PEAK
    FP64_PEAK = fp64_peak(torch.device("cuda", torch.cuda.current_device()))
    n = args.n
    N = dofs(n)
    f_host = torch.from_numpy(si.random_force(n, args.seed + rank)).pin_memory()
    ud_host = torch.from_numpy(si.manufactured_velocity(n)).pin_memory()
    main = time_form(args, args.prec, ws, rank, f_host, ud_host, with_e2e=True)
    x_ref = main.pop("_x")
    keys = ("value", "time_to_solution_s", "iters", "ms_per_vcycle", "vcycle_only", "setup_s")
    forms = {args.prec: {k: main[k] for k in keys}}

    def compare(name, o):
        # every other form solves the same right-hand side to the same tolerance: its
        # solution's difference from the headline form's (FP64: parity-tested against the oracle)
        xo = o.pop("_x", None)
        if xo is not None:
            forms[name]["solution_diff_vs_" + args.prec] = solution_difference(xo, x_ref, n)
    if not args.single_form:
        for other in PRECS:
            if other == args.prec:
                continue
            o = time_form(args, other, ws, rank, f_host, ud_host, with_e2e=False)
            forms[other] = {k: o[k] for k in keys}
            forms[other]["roofline"] = o["roofline"]
            compare(other, o)
        # the paper's simple Vanka (an explicit inverse per patch) in the FP64 form, and
        # Braess-Sarazin relaxation (the paper's comparison, Section 6.8) in FP64 and mixed FP32
        # and Schur-Uzawa with the paper's parameters (t = 1, Jacobi weight 0.4, one step)
        su = dict(bs_t=1.0, bs_omega=1.0, bs_jacobi_weight=0.4, bs_jacobi_iters=1)
        # and the block-triangular preconditioner (three V(3,3) cycles per block, Section 6.8)
        # Schur-Uzawa is not h-robust with the paper's parameters (FGMRES iterations 18 / 25 /
        # 280 at 64^2 / 256^2 / 1024^2, no convergence in 300 at 2048^2), so it is timed at 256^2
        for name, pn, sm, kw, nn in (("fp64_simple_vanka", "fp64", 1, None, None),
                                     ("fp64_braess_sarazin", "fp64", 2, None, None),
                                     ("mixed_braess_sarazin", "mixed", 2, None, None),
                                     ("fp64_block_triangular", "fp64", 0, {"precond": 1}, None),
                                     ("fp64_schur_uzawa_256", "fp64", 3, su, 256),
                                     ("bf16_wcycle", "bf16", 0, {"cycle": 2}, None)):
            o = time_form(args, pn, ws, rank, f_host, ud_host, with_e2e=False, smoother=sm, hkw=kw, n=nn)
            forms[name] = {k: o[k] for k in keys}
            forms[name]["roofline"] = o["roofline"]
            compare(name, o)
            if nn is not None:
                forms[name]["n"] = nn
    batched = None
    if not args.no_batch:
        batched = time_batch(args, "mixed")
    cpu = cpu_all = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        o = run_oracle(ORACLE_N, 1)
        cpu = {"value": o["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one FGMRES(30)+V(2,2) solve to 1e-8 at {o['n']}x{o['n']} ({o['dofs']} dofs, "
                         f"{o['iters']} V-cycles, {o['solve_s']:.2f} s; setup {o['setup_s']:.1f} s excluded), "
                         f"numpy/scipy, BLAS threads = 1"}
        procs = os.cpu_count() or 1
        oa = run_oracle_all_cores(ORACLE_N, procs)
        cpu_all = {"value": oa["value"], "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": f"{procs} concurrent single-threaded oracle processes, one FGMRES(30)+V(2,2) solve "
                             f"to 1e-8 at {oa['n']}x{oa['n']} each ({oa['iters']} V-cycles; slowest solve "
                             f"{oa['solve_s_max']:.2f} s)"}
    if rank == 0:
        prec_txt = "FP64" if args.prec == "fp64" else "FP32 V-cycle inside FP64 FGMRES"
        line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.prec == "fp64" else "f32/f64", "data": "synthetic",
                "config": {"workload": f"2D Stokes Q2-Q1, {n}x{n} elements, {prec_txt}, FGMRES(30) + V(2,2) "
                                       f"additive Vanka (omega 0.7) to 1e-8, coarse 4x4",
                           "n": n, "dofs": N, "levels": main["levels"],
                           "rhs": f"N(0,1) nodal force, seed {args.seed}",
                           "l2": "inputs larger than L2 (each vector 8*dofs bytes)",
                           "parallelism": f"replicas x{ws}"},
                "time_to_solution_s": main["time_to_solution_s"], "iters": main["iters"],
                "relres": main["relres"], "vcycles": main["vcycles"], "ms_per_vcycle": main["ms_per_vcycle"],
                "vcycle_only": main["vcycle_only"],
                "roofline": main["roofline"], "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
                "e2e": main["e2e"],
                "gpu_launches": main["gpu_launches"], "clocks": main["clocks"], "forms": forms,
                "batched": batched}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# reference arm: the CPU oracle, as it stands
# --------------------------------------------------------------------------
def run_reference(args) -> None:
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    n = ORACLE_N
    # warm-up and timed steps: each step one oracle solve at n x n
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", "--n", str(n),
                        "--steps", str(max(args.steps, 1))], capture_output=True, text=True, env=env,
                       cwd=ROOT)
    if r.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle worker failed: " + r.stderr[-300:]}))
        return
    o = json.loads(r.stdout.strip().splitlines()[-1])
    line = {"impl": "reference", "metric": METRIC, "value": o["value"], "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": o["solve_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"2D Stokes Q2-Q1, FP64, FGMRES(30) + V(2,2) additive Vanka to 1e-8; "
                                   f"CPU oracle sample at {n}x{n}", "n": n, "dofs": o["dofs"]},
            "cpu_baseline": {"value": o["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"median of {args.steps} solves at {n}x{n} ({o['iters']} V-cycles each)"},
            "e2e": {"value": o["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_kernel(args) -> None:
    """Time one kernel of the path alone on the finest level (for profiling): W + K launches."""
    import torch

    import stokes_inputs as si
    import paper_2401_06277_gb300 as pkg
    from paper_2401_06277_gb300 import build, stokes

    build.build()
    n = args.n
    H = pkg.Hierarchy(n, restart=1, tile=args.tile, prec=PRECS[args.prec], smoother=args.smoother)
    lvl = H.levels - 1
    x = torch.from_numpy(si.random_vector(n, 1)).cuda()
    b = torch.from_numpy(si.random_vector(n, 2)).cuda()
    out = torch.empty_like(b)
    if args.kernel == "sweep":
        fn = lambda: stokes.stokes_vanka_sweep(H.handle, lvl, x, b, out)
        fl, by = sweep_flops(n), sweep_bytes(n)
    elif args.kernel == "residual":
        fn = lambda: stokes.stokes_residual(H.handle, lvl, b, x, out)
        fl, by = 361.0 * (n + 1) ** 2, sweep_bytes(n)
    elif args.kernel == "solve":
        # one FGMRES(30) solve to 1e-8 of the seeded N(0,1)-force problem
        H.close()
        H = pkg.Hierarchy(n, tile=args.tile, prec=PRECS[args.prec], smoother=args.smoother)
        bb = H.assemble_rhs(torch.from_numpy(si.random_force(n, 0)).cuda(),
                            torch.from_numpy(si.manufactured_velocity(n)).cuda())

        def fn():
            stokes.stokes_initial_guess(H.handle, bb, out)
            stokes.stokes_fgmres_solve(H.handle, bb, out)
        fl, by = None, None
    else:
        fn = lambda: stokes.stokes_vcycle_apply(H.handle, b, out)
        fl, by = None, None
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    rec = {"kernel": args.kernel, "n": n, "ms": ms,
           "tile": TILE_NAMES[stokes.stokes_level_tile(H.handle, lvl)]}
    if fl:
        rec["gflops"] = fl / (ms * 1e-3) / 1e9
        rec["gbs"] = by / (ms * 1e-3) / 1e9
    print(json.dumps(rec))
    H.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sm-max-mhz", type=float, default=None)
    ap.add_argument("--traffic", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", choices=list(PRECS), default="fp64",
                    help="form of the headline line (the other form is reported under 'forms')")
    ap.add_argument("--single-form", action="store_true", help="time only the --prec form")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form timings")
    ap.add_argument("--batch-n", type=int, default=1024)
    ap.add_argument("--batch-rhs", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--oracle-worker", action="store_true")
    ap.add_argument("--oracle-vcycle", type=int, default=None, metavar="N",
                    help="time the CPU oracle's set-up and one V-cycle at N x N (single thread) and exit")
    ap.add_argument("--tile", type=int, default=-1, help="Vanka sweep configuration (-1: autotuned; 0..3 fused 8x8/16x8/16x16/14x14, 4/5 split 16x16, 6 fused 4x4)")
    ap.add_argument("--kernel", choices=["sweep", "residual", "vcycle", "solve"], default=None,
                    help="time one kernel alone on the finest level (profiling mode)")
    ap.add_argument("--smoother", type=int, choices=[0, 1, 2, 3], default=0,
                    help="profiling mode: 0 shared-inverse Vanka, 1 simple Vanka, 2 Braess-Sarazin, 3 Schur-Uzawa")
    args = ap.parse_args()
    if args.kernel:
        run_kernel(args)
        return
    if args.oracle_worker:
        oracle_worker(args.n, args.steps)
        return
    if args.oracle_vcycle:
        oracle_vcycle(args.oracle_vcycle)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
