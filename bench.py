"""Benchmark: resolvent samples per second of the full RSRR pass on one GB300.

A step is one pass of the whole hot path over the damped quadratic NEP on a 200 x 200 grid
(n = 40000, band 200), contour ellipse (-0.5+40i; 2, 30), N = 64 sampling points, L = 32
probing columns:
    rsrr_sample  (band LU + L-column solves, complex64 with FP64 refinement to eta <= tol)
    rsrr_project (Householder QR + Jacobi SVD truncation at delta = 1e-14, P_i = S^H A_i S)
    rsrr_solve   (Algorithm 1 with N_S = 500, K = 2, back-map and residuals)
value = N sampling points per step / device time per step (inputs resident on the device).
e2e   = the same metric through the public calls from pinned host buffers: rsrr_create_nep,
        rsrr_sample with the host U, project, solve with host outputs, destroy.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 the ranks run independent replicas (the sampling points of one NEP do not need a
collective; see the design notes): value = all ranks' points / max rank time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="damped quadratic NEP K + zC + z^2 M, 200x200 grid (n=40000, band 200), "
                         "ellipse (-0.5+40i; a=2, b=30), N=64, L=32",
                n=40000, band=200, N=64, L=32, N_S=500, K=2, delta=1e-14)
METRIC = "resolvent samples/sec (LU+L-RHS solve, resid<=1e-10), full RSRR pass"
UNIT = "samples/s"
FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 x max SM clock
FP64_PEAK_TFLOPS = 1.25                              # nominal FP64 rate of this part (measured 1.19)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="c64", choices=["c64", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-10, help="acceptance: eta <= tol per column")
    ap.add_argument("--grid", type=int, default=200, help="grid side (200 = the benchmark workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-points", type=int, default=0, help="points in the CPU baseline sample (0 = cores)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def workload(grid):
    import workloads
    return workloads.config1(s=grid)


def fns_of(p):
    return [(f.kind, f.params()) for f in p.fns]


def cpu_oracle_rate(prob, npts, steps=1):
    """The oracle (plain C band LU + NumPy) on the host cores: sampling points per second."""
    import oracle
    z, _, _ = oracle.contour_points(prob.gamma, prob.a, prob.b, prob.N)
    pts = list(range(npts))
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.sample(prob, points=pts, threads=os.cpu_count())
        times.append(time.perf_counter() - t0)
    return npts / statistics.median(times), times


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    prob = workload(args.grid)
    cores = os.cpu_count() or 1
    npts = args.cpu_points or min(prob.N, cores)
    import oracle
    for _ in range(args.warmup):
        oracle.sample(prob, points=list(range(min(npts, 2))), threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sample(prob, points=list(range(npts)), threads=cores)
    el = time.perf_counter() - t0
    v = npts * args.steps / el
    sample = (f"sampling phase only (band LU + L-column solves) of {npts} of the {prob.N} points per step, "
              "threads over points")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, parallelism="cpu threads"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def job_value(points_per_rank, steps, ms_local, device=None):
    """Whole-job throughput: all ranks' points over the slowest rank's time (max over ranks,
    every rank gets the same answer).  Returns (value in points/s, max ms)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    world = 1
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return points_per_rank * steps * world / (ms_max / 1e3), ms_max


def run_ours(args):
    rank, world, local = dist_env()
    import torch
    import paper_1510_07522_gb300 as rs
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prob = workload(args.grid)
    prec = (rs.RSRR_C64_IR if args.precision == "c64" else rs.RSRR_FP64) | rs.RSRR_REFINE_FULL
    stream = torch.cuda.current_stream()
    sp = __import__("ctypes").c_void_p(stream.cuda_stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    h = rs.Nep(prob.n, prob.rowptr, prob.colind, prob.vals, fns_of(prob), 0, sp)

    def step(U):
        h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, U, prec, args.tol, 20)
        h.project(WORKLOAD["delta"])
        lam, V, res = h.solve(WORKLOAD["N_S"], WORKLOAD["K"], 1e3, 4096, True)
        return h.info(), lam

    step(prob.U)
    for _ in range(args.warmup - 1):
        step(None)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    l0 = rs.lib().rsrr_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        info, lam = step(None)
        infos.append(info)
    e1.record(stream)
    barrier()
    launches = rs.lib().rsrr_kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    value, ms_max = job_value(prob.N, args.steps, ms, device="cuda")

    # ---- dominant kernel and its roofline ------------------------------------------------------
    med = lambda k: statistics.median(i[k] for i in infos)
    phases = {"sample_ms": med("ms_sample"), "project_ms": med("ms_project"), "solve_ms": med("ms_solve"),
              "factor_ms": med("ms_factor"), "trsv_ms": med("ms_trsv"),
              "project_qr_ms": med("ms_project_qr"), "project_svd_ms": med("ms_project_svd"),
              "project_basis_ms": med("ms_project_basis"), "project_gemm_ms": med("ms_project_gemm"),
              "solve_inverse_ms": med("ms_solve_inverse"), "solve_svd_ms": med("ms_solve_svd"),
              "solve_extract_ms": med("ms_solve_extract")}
    n, kl, ku = prob.n, infos[-1]["kl"], infos[-1]["ku"]
    flops_per_point = 8.0 * n * kl * (kl + ku)          # band LU with pivoting fill (real flops)
    flops_launch = flops_per_point * prob.N / max(1, infos[-1]["factor_launches"])
    fac_ms_launch = phases["factor_ms"] / max(1, infos[-1]["factor_launches"])
    achieved = flops_launch / (fac_ms_launch / 1e3) / 1e12 if fac_ms_launch > 0 else None
    roof_lu = {"kernel": "band_factor_kernel<float> (complex64 band LU, CUDA-core FFMA)", "bound": "alu",
               "achieved": achieved, "peak": FFMA_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": (achieved / FFMA_PEAK_TFLOPS) if achieved else None, "traffic": None,
               "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (no FP32 figure in the measured peaks)",
               "algorithmic": f"8 n kl (kl+ku) real flops per point x {prob.N} points per launch",
               "ms_per_step": phases["factor_ms"], "ms_per_launch": fac_ms_launch}
    zg_ms = statistics.median(i["ms_zgemm"] for i in infos)
    zg_tf = statistics.median(i["zgemm_gflop"] for i in infos) / zg_ms if zg_ms > 0 else None
    roof_zg = {"kernel": "zgemm_kernel (FP64 complex GEMM, all launches of project + solve)", "bound": "alu",
               "achieved": zg_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": (zg_tf / FP64_PEAK_TFLOPS) if zg_tf else None, "traffic": None,
               "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s); an FMA probe measured 1.19",
               "algorithmic": "8 M N K real flops per complex product", "ms_per_step": zg_ms}
    phases["zgemm_ms"] = zg_ms
    roof = roof_zg if zg_ms > phases["factor_ms"] else roof_lu

    # ---- end to end through the public calls, host buffers ------------------------------------
    e2e = None
    if not args.no_e2e:
        pin = lambda a: _pinned(torch, a)
        rowptr, colind, vals, U = pin(prob.rowptr), pin(prob.colind), pin(prob.vals), pin(np.asfortranarray(prob.U))
        h2d = rowptr.nbytes + colind.nbytes + vals.nbytes + U.nbytes
        barrier()
        d2h = 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g = rs.Nep(prob.n, rowptr, colind, vals, fns_of(prob), 0, sp)
            g.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, U, prec, args.tol, 20)
            g.project(WORKLOAD["delta"])
            lam, V, res = g.solve(WORKLOAD["N_S"], WORKLOAD["K"], 1e3, 4096, True)
            d2h = lam.nbytes + (V.nbytes if V is not None else 0) + res.nbytes
            g.close()
        barrier()
        el = time.perf_counter() - t0
        e2e_value, _ = job_value(prob.N, args.steps, 1e3 * el, device="cuda")
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        npts = args.cpu_points or min(prob.N, cores)
        v, times = cpu_oracle_rate(prob, npts)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"sampling phase only (band LU + L-column solves) of {npts} of the {prob.N} points, "
                         f"FP64 C band LU threaded over points, {times[0]:.1f} s"}
    h.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "c64+f64" if args.precision == "c64" else "c128",
                "data": "synthetic (seeded generator: grid Laplacian K, lumped M = 1 + 0.1 U(0,1), C = 0.05K + 0.02M)",
                "config": dict(WORKLOAD, parallelism=f"replicas x{world}" if world > 1 else "1 GPU",
                               tol=args.tol, precision=args.precision, refine="to working accuracy",
                               l2="inputs larger than L2 (factors 12 GB, S_hat 1.3 GB per step)"),
                "phases_ms_median": phases, "k_S": infos[-1]["k_S"], "refine_sweeps": infos[-1]["refine_sweeps"],
                "rows_kept": infos[-1]["rows_kept"],
                "jacobi_sweeps": [infos[-1]["jacobi_sweeps_project"], infos[-1]["jacobi_sweeps_solve"]],
                "max_eta": max(i["max_eta"] for i in infos), "n_eigs_inside": int(lam.size),
                "roofline": roof, "rooflines": {"band_lu": roof_lu, "zgemm": roof_zg}, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _pinned(torch, a):
    a = np.asarray(a)
    t = torch.empty(a.shape[::-1] if a.flags["F_CONTIGUOUS"] and not a.flags["C_CONTIGUOUS"] else a.shape,
                    dtype={np.dtype("int64"): torch.int64, np.dtype("int32"): torch.int32,
                           np.dtype("complex128"): torch.complex128, np.dtype("float64"): torch.float64}[a.dtype],
                    pin_memory=True)
    out = t.numpy()
    if a.flags["F_CONTIGUOUS"] and not a.flags["C_CONTIGUOUS"]:
        out = out.T
    out[...] = a
    return out


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
