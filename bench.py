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
For N > 1 the ranks run independent replicas (the sampling points of one NEP are independent
solves, so no collective is needed): value = all ranks' points / max rank time.
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

WORKLOADS = {
    "1": dict(workload="damped quadratic NEP K + zC + z^2 M, 200x200 grid (n=40000, band 200), "
                       "ellipse (-0.5+40i; a=2, b=30), N=64, L=32",
              n=40000, band=200, N=64, L=32, N_S=500, K=2, delta=1e-14, precision="c64",
              data="synthetic (seeded generator: grid Laplacian K, lumped M = 1 + 0.1 U(0,1), C = 0.05K + 0.02M)"),
    "0": dict(workload="gun-like sqrt NEP K - zM + i sqrt(z - s1^2) W1 + i sqrt(z - s2^2) W2, 30x30 grid "
                       "(n=900, band 30), circle (250; 150), N=32, L=16",
              n=900, band=30, N=32, L=16, N_S=500, K=2, delta=1e-14, precision="fp64",
              data="synthetic (seeded generator: grid Laplacian K, M = I, boundary masks W1, W2)"),
    "2": dict(workload="gun-like sqrt NEP, 400x250 grid (n=100000, band 250), circle (330; 300), N=64, L=48",
              n=100000, band=250, N=64, L=48, N_S=500, K=2, delta=1e-14, precision="c64",
              data="synthetic (seeded generator: grid Laplacian K, M = I, boundary masks W1, W2)"),
    "3": dict(workload="batch of time-delay NEPs -zI + A0 + A1 exp(-tau z): A0 the s x s grid Laplacian, "
                       "s ~ U{20..100} (n 400..10000), A1 5% random (dense LU), own circle each, N=32, L=8",
              batch=32, N=32, L=8, N_S=500, K=2, delta=1e-14, precision="c64",
              data="synthetic (seeded generator: the first members of the 256-NEP time-delay batch)"),
}
WORKLOAD = WORKLOADS["1"]
METRIC = "resolvent samples/sec (LU+L-RHS solve, resid<=1e-10), full RSRR pass"
UNIT = "samples/s"
FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 x max SM clock
FP64_PEAK_TFLOPS = 1.25                              # nominal FP64 rate of this part


def measured_peaks():
    """BF16 tensor TFLOP/s and HBM GB/s measured on this machine (MEASURED_PEAKS.json), else the
    earlier GB300 measurement used as fallback; returns (bf16, hbm, source)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 1900.0, 6800.0, "fallback (no measured peaks file)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="1", choices=sorted(WORKLOADS) + ["serve", "compare"],
                    help="1 = the benchmark workload; 0 and 2 the smaller and larger sqrt NEPs; serve = "
                         "Poisson request stream through the continuous-batching server")
    ap.add_argument("--precision", default=None, choices=["c64", "fp64"], help="default: the config's own")
    ap.add_argument("--tol", type=float, default=1e-10, help="acceptance: eta <= tol per column")
    ap.add_argument("--grid", type=int, default=0, help="grid side override (0 = the config's own size; config 3: "
                                                       "every member on an s x s grid)")
    ap.add_argument("--rates", default="1,4,16", help="serve: Poisson arrival rates, requests/s")
    ap.add_argument("--requests", type=int, default=12, help="serve: requests per rate")
    ap.add_argument("--fp64-requests", type=int, default=0,
                    help="serve: requests of the plain-FP64 one-at-a-time comparison (0 = min(requests, 40))")
    ap.add_argument("--batch", type=int, default=0, help="config 3: members of the batch (0 = the config's own)")
    ap.add_argument("--banded", action="store_true",
                    help="config 3: iterative sampler - factor only each member's grid-Laplacian band (half-width "
                         "s, natural ordering) and iterate with the full T (rsrr_set_band_preconditioner)")
    ap.add_argument("--dense", action="store_true",
                    help="config 3: the dense LU for every member (no autotuning)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 arm of the same workload")
    ap.add_argument("--no-eigs", action="store_true",
                    help="skip the pass over the same matrices with a contour that encloses eigenvalues")
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


def workload(config, grid=0):
    import workloads
    if config == "0":
        return workloads.config0(nx=grid, ny=grid) if grid else workloads.config0()
    if config == "2":
        return workloads.config2(nx=2 * grid, ny=grid) if grid else workloads.config2()
    return workloads.config1(s=grid) if grid else workloads.config1()


def fns_of(p):
    return [(f.kind, f.params()) for f in p.fns]


def line_config(W, args, prob, precision, world):
    """The `config` of the JSON line, the same for this arm and the oracle (reference) arm."""
    return dict({k: v for k, v in W.items() if k != "data"},
                parallelism=f"replicas x{world}" if world > 1 else "1 GPU",
                tol=args.tol, precision=precision, refine="to working accuracy",
                n=prob.n, N=prob.N, L=prob.L,
                l2="inputs larger than L2" if prob.n * prob.N * prob.L * 16 >= 2 * 129e6 else
                   "L2 flushed between steps (256 MB write outside the timed events)")


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
    if args.config in ("serve", "compare"):
        print(json.dumps({"impl": "reference", "unavailable": "the serving stream and the scheme comparison have "
                                                              "no oracle arm; the oracle arm times configs 0-3"}),
              flush=True)
        return
    W = WORKLOADS[args.config]
    prob = workload(args.config, args.grid)
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
    precision = args.precision or W["precision"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": W["data"], "config": line_config(W, args, prob, precision, 1),
            "timed_part": (f"the oracle's sampling phase (Algorithm 2 Steps 1-2: FP64 band LU + L-column solves) "
                           f"of {npts} of the {prob.N} points per step, on {cores} host threads; its Steps 3-5 "
                           f"are not timed, so this rate is an upper bound on the oracle's full-pass rate"),
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
    W = WORKLOADS[args.config]
    prob = workload(args.config, args.grid)
    precision = args.precision or W["precision"]
    prec = (rs.RSRR_C64_IR if precision == "c64" else rs.RSRR_FP64) | rs.RSRR_REFINE_FULL
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
        h.project(W["delta"])
        lam, V, res = h.solve(W["N_S"], W["K"], 1e3, 4096, True)
        return h.info(), lam

    step(prob.U)
    for _ in range(args.warmup - 1):
        step(None)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    l0 = rs.lib().rsrr_kernel_launches()
    # Inputs smaller than L2 (config 0) get an L2 flush between steps, outside the timed events.
    flush = None
    if prob.n * prob.N * prob.L * 16 < 2 * 129e6:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    for e0, e1 in evs:
        if flush is not None:
            flush.random_(0, 255)
        e0.record(stream)
        info, lam = step(None)
        e1.record(stream)
        infos.append(info)
    barrier()
    launches = rs.lib().rsrr_kernel_launches() - l0
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
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
    bf16_peak, _, bf16_src = measured_peaks()
    if infos[-1]["band_lu_tc"]:
        lu_peak = bf16_peak / 6.0   # 6 BF16 piece products per real product (3-piece split)
        roof_lu = {"kernel": "band_factor_tc_kernel (complex64 band LU, trailing updates on tcgen05, TMA panels)",
                   "bound": "tensor", "peak_source": f"{bf16_src}: BF16 {bf16_peak:.0f} TFLOP/s / 6 piece products "
                                                     f"per real product"}
    else:
        lu_peak = FFMA_PEAK_TFLOPS if precision == "c64" else FP64_PEAK_TFLOPS
        roof_lu = {"kernel": "band_factor_kernel<%s> (%s band LU, CUDA cores)" % (
                       ("float", "complex64") if precision == "c64" else ("double", "complex128")), "bound": "alu",
                   "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (no FP32 figure in the "
                                   "measured peaks)") if precision == "c64" else "nominal FP64 rate"}
    lu_traffic = None
    if infos[-1]["band_lu_tc"]:
        # DRAM bytes of one launch: an ncu capture of this kernel on the 100 x 100 grid (64 points,
        # kl = ku = 100) read 1.57 GB and wrote 2.74 GB, 0.979 of the compulsory bytes (band read
        # and written, stored panel blocks); scaled to this launch by the same per-point formula
        ldab = 2 * kl + ku + 1
        per_point = 2.0 * ldab * n * 8 + -(-n // 32) * 256 * 32 * 8
        lu_traffic = 0.979 * per_point * prob.N / max(1, infos[-1]["factor_launches"])
    roof_lu.update({"achieved": achieved, "peak": lu_peak, "unit": "TFLOP/s",
                    "frac": (achieved / lu_peak) if achieved else None, "traffic": lu_traffic,
                    "algorithmic": f"8 n kl (kl+ku) real flops per point x {prob.N} points per launch",
                    "ms_per_step": phases["factor_ms"], "ms_per_launch": fac_ms_launch})
    zg_ms = statistics.median(i["ms_zgemm"] for i in infos)
    tc_ms = statistics.median(i["ms_zgemm_tc"] for i in infos)
    tc_tf = statistics.median(i["zgemm_tc_gflop"] for i in infos) / tc_ms if tc_ms > 0 else None
    oz_ceiling = bf16_peak / 36.0   # 36 BF16 digit-pair products per real product
    roof_tc = {"kernel": "oz_gemm_kernel + digit images (FP64-accurate complex GEMM on tcgen05, BF16 digits)",
               "bound": "tensor", "achieved": tc_tf, "peak": oz_ceiling, "unit": "TFLOP/s",
               "frac": (tc_tf / oz_ceiling) if tc_tf else None, "traffic": None,
               "peak_source": f"{bf16_src}: BF16 {bf16_peak:.0f} TFLOP/s / 36 digit-pair products per real product",
               "algorithmic": "8 M N K real flops per complex product", "ms_per_step": tc_ms}
    jac_ms = statistics.median(i["ms_jacobi"] for i in infos)
    jac_tf = statistics.median(i["jacobi_gflop"] for i in infos) / jac_ms if jac_ms > 0 else None
    roof_jac = {"kernel": "jacobi_sweep_kernel (one-sided Jacobi, FP64, project + solve)", "bound": "alu",
                "achieved": jac_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": (jac_tf / FP64_PEAK_TFLOPS) if jac_tf else None, "traffic": None,
                "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s)",
                "algorithmic": "per sweep: 4 mb k for the column norms, 8 mb per pair whose inner product is "
                               "formed, 32 mb + 24 k per rotated pair (rotation of B and of the k-row J, new "
                               "norms); pairs and rotations counted by the kernel", "ms_per_step": jac_ms}
    # the SVD stages against a fixed count that does not grow with the sweeps: a bidiagonalising
    # SVD with both vector sets, ~4 (4 m n^2 + 8 n^3) real flops for a complex m x n (m >= n):
    # the projection's SVD of R^H (N L x rows kept) and the Hankel SVD (K k_S square)
    def gk(m, nn):
        m, nn = max(m, nn), min(m, nn)
        return 4.0 * (4.0 * m * nn * nn + 8.0 * nn ** 3)
    svd_ms = phases["project_svd_ms"] + phases["solve_svd_ms"]
    svd_work = gk(prob.N * prob.L, infos[-1]["rows_kept"]) + gk(W["K"] * infos[-1]["k_S"], W["K"] * infos[-1]["k_S"])
    svd_tf = svd_work / (svd_ms / 1e3) / 1e12 if svd_ms > 0 else None
    roof_svd = {"kernel": "SVD stages (QR preconditioner, one-sided Jacobi sweeps, vectors), project + solve",
                "bound": "alu", "achieved": svd_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": (svd_tf / FP64_PEAK_TFLOPS) if svd_tf else None, "traffic": None,
                "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s)",
                "algorithmic": "fixed count of a bidiagonalising SVD with vectors, 4 (4 m n^2 + 8 n^3) real flops "
                               "per complex m x n: R^H (N L x rows kept) and H (K k_S square)",
                "ms_per_step": svd_ms}
    phases["zgemm_ms"] = zg_ms
    phases["zgemm_tc_ms"] = tc_ms
    phases["jacobi_ms"] = jac_ms
    cands = [(phases["factor_ms"], roof_lu), (tc_ms, roof_tc), (jac_ms, roof_jac)]
    roof = max(cands, key=lambda c: c[0])[1]

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
            g.project(W["delta"])
            lam, V, res = g.solve(W["N_S"], W["K"], 1e3, 4096, True)
            eta = g.eta()   # the acceptance measure of every sample column (eta <= tol)
            d2h = lam.nbytes + (V.nbytes if V is not None else 0) + res.nbytes + eta.nbytes
            g.close()
        barrier()
        el = time.perf_counter() - t0
        e2e_value, _ = job_value(prob.N, args.steps, 1e3 * el, device="cuda")
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    h.close()
    # ---- the same workload in plain FP64 (complex128 LU and solves), the form the mixed
    # precision path is measured against, at the same acceptance eta <= tol ---------------------
    vs_fp64 = None
    if precision == "c64" and not args.no_fp64:
        prec64 = rs.RSRR_FP64 | rs.RSRR_REFINE_FULL
        g = rs.Nep(prob.n, prob.rowptr, prob.colind, prob.vals, fns_of(prob), 0, sp)

        def step64():
            g.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, prec64, args.tol, 20)
            g.project(W["delta"])
            g.solve(W["N_S"], W["K"], 1e3, 4096, True)
            return g.info()
        step64()
        k64 = max(1, min(args.steps, 2))
        barrier()
        ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k64)]
        inf64 = []
        for e0, e1 in ev64:
            if flush is not None:
                flush.random_(0, 255)
            e0.record(stream)
            inf64.append(step64())
            e1.record(stream)
        barrier()
        g.close()
        ms64 = sum(e0.elapsed_time(e1) for e0, e1 in ev64)
        v64, _ = job_value(prob.N, k64, ms64, device="cuda")
        s64 = statistics.median(i["ms_sample"] for i in inf64)
        vs_fp64 = {"value": v64, "unit": UNIT, "steps": k64, "warmup": 1, "ms_per_step": ms64 / k64,
                   "max_eta": max(i["max_eta"] for i in inf64), "k_S": inf64[-1]["k_S"],
                   "sample_ms": s64, "factor": value / v64 if v64 else None,
                   "sampling_factor": s64 / phases["sample_ms"] if phases["sample_ms"] else None,
                   "note": "the same full pass with complex128 band LU and solves (RSRR_FP64), events on "
                           "the same stream; factor = mixed-precision value / this value at the same tol"}

    # ---- the same matrices with a contour that encloses eigenvalues (the benchmark contour
    # encloses none): one full pass returning eigenpairs at full size, timed the same way, with
    # its eigenvalues against the closed form of the damped problem ----------------------------
    eig_arm = None
    if args.config == "1" and args.grid == 0 and not args.no_eigs:
        import workloads
        pb = workloads.config1b()
        g = rs.Nep(pb.n, pb.rowptr, pb.colind, pb.vals, fns_of(pb), 0, sp)

        def step_b():
            g.sample(pb.gamma, pb.a, pb.b, pb.N, pb.L, pb.U, prec, args.tol, 20)
            g.project(W["delta"])
            return g.solve(W["N_S"], W["K"], 1e3, 4096, True)
        step_b()
        kb = 2
        barrier()
        evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(kb)]
        for e0, e1 in evb:
            e0.record(stream)
            lam_b, _, res_b = step_b()
            e1.record(stream)
        barrier()
        infb = g.info()
        g.close()
        msb = sum(e0.elapsed_time(e1) for e0, e1 in evb)
        vb, _ = job_value(pb.N, kb, msb, device="cuda")
        nrm = [float(np.linalg.norm(pb.vals[i])) for i in range(pb.vals.shape[0])]
        al = np.abs(lam_b)
        scaled_res = res_b / (nrm[0] + al * nrm[1] + al ** 2 * nrm[2]) if lam_b.size else np.zeros(0)
        ex = np.asarray(pb.meta["expected"])   # closed form: the 10 lowest upper-branch eigenvalues
        ex = ex[((ex.real - pb.gamma.real) / pb.a) ** 2 + ((ex.imag - pb.gamma.imag) / pb.b) ** 2 < 1.0]
        err = max((float(np.min(np.abs(ex - l)) / abs(l)) for l in lam_b), default=None)
        eig_arm = {"workload": "the same n = 40000 damped QEP, ellipse placed around its lowest upper-branch "
                               "eigenvalues (N=64, L=32)", "value": vb, "unit": UNIT, "steps": kb,
                   "ms_per_step": msb / kb, "n_eigs_inside": int(lam_b.size),
                   "expected_inside": int(ex.size),
                   "max_scaled_residual": float(scaled_res.max()) if lam_b.size else None,
                   "max_rel_err_vs_closed_form": err, "k_S": infb["k_S"], "max_eta": infb["max_eta"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        npts = args.cpu_points or min(prob.N, cores)
        v, times = cpu_oracle_rate(prob, npts)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"sampling phase only (band LU + L-column solves) of {npts} of the {prob.N} points, "
                         f"FP64 C band LU threaded over points, {times[0]:.1f} s"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "c64+f64" if precision == "c64" else "c128",
                "data": W["data"],
                "config": line_config(W, args, prob, precision, world),
                "phases_ms_median": phases, "k_S": infos[-1]["k_S"], "refine_sweeps": infos[-1]["refine_sweeps"],
                "rows_kept": infos[-1]["rows_kept"],
                "jacobi_sweeps": [infos[-1]["jacobi_sweeps_project"], infos[-1]["jacobi_sweeps_solve"]],
                "max_eta": max(i["max_eta"] for i in infos), "n_eigs_inside": int(lam.size),
                "roofline": roof, "rooflines": {"band_lu": roof_lu, "zgemm_tc": roof_tc, "jacobi": roof_jac,
                                                "svd_stage": roof_svd},
                "vs_fp64": vs_fp64, "with_eigenpairs": eig_arm, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


SOLVE_STREAMS = 4  # config 3: streams (and host threads) for the per-NEP project / solve calls


def batch_members(count, side=0):
    import workloads
    return [workloads.config3_member(i, s=side or None) for i in range(count)]


def dense_lu_flops(n):
    return 8.0 / 3.0 * float(n) ** 3


def cpu_dense_rate(probs, seconds=15.0):
    """The oracle's dense LU solves on the host cores, on points of the smallest members until
    about `seconds` of work: flop rate, converted to samples/s at the batch's flop mix."""
    import oracle
    cores = os.cpu_count() or 1
    small = sorted(probs, key=lambda p: p.n)
    done_flops, t0, npts = 0.0, time.perf_counter(), 0
    for p in small:
        pts = list(range(min(p.N, cores)))
        el = time.perf_counter() - t0
        if npts and el + len(pts) * dense_lu_flops(p.n) / (done_flops / el) > seconds:
            break  # the next member would overrun the sample's time budget
        oracle.sample(p, points=pts, threads=cores, dense=True)
        done_flops += len(pts) * dense_lu_flops(p.n)
        npts += len(pts)
    el = time.perf_counter() - t0
    rate = done_flops / el
    mean_flops = sum(p.N * dense_lu_flops(p.n) for p in probs) / sum(p.N for p in probs)
    return rate / mean_flops, cores, (f"oracle dense LU + L-column solves on {npts} points of the smallest members "
                                      f"({el:.1f} s, {rate / 1e9:.2f} GFLOP/s), converted to samples/s at the batch's "
                                      f"mean (8/3) n^3 per point")


def run_batch(args):
    """Config 3: one rsrr_sample_batch over all members (dense LU, persistent launches), then
    rsrr_project and rsrr_solve per member."""
    rank, world, local = dist_env()
    import ctypes
    import torch
    import paper_1510_07522_gb300 as rs
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS["3"]
    B = args.batch or W["batch"]
    probs = batch_members(B, args.grid)
    precision = args.precision or W["precision"]
    prec = (rs.RSRR_C64_IR if precision == "c64" else rs.RSRR_FP64) | rs.RSRR_REFINE_FULL
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    # the handles are spread over a few streams: one batched sampling call, then each stream's
    # handles go through rsrr_project / rsrr_solve in a host thread of their own
    streams = [torch.cuda.Stream() for _ in range(SOLVE_STREAMS)]
    sps = [ctypes.c_void_p(st.cuda_stream) for st in streams]
    # default: the library's autotuner picks each member's sampler (timed on one point, cached
    # per size bucket); --banded forces the iterative sampler on the grid band, --dense the dense LU
    autotune = not (args.banded or args.dense)
    flags = rs.RSRR_NATURAL_ORDER if args.banded else (rs.RSRR_NATURAL_ORDER | rs.RSRR_AUTOTUNE if autotune else 0)

    def make(i, p, rowptr, colind, vals):
        h = rs.Nep(p.n, rowptr, colind, vals, fns_of(p), flags, sps[i % len(sps)])
        if args.banded:
            h.set_band_preconditioner(p.meta["nx"])  # the grid Laplacian: half-width s
        return h
    hs = [make(i, p, p.rowptr, p.colind, p.vals) for i, p in enumerate(probs)]
    contours = [(p.gamma, p.a, p.b) for p in probs]
    Ns, Ls = [p.N for p in probs], [p.L for p in probs]

    def finish(handles, vectors=False):
        """rsrr_project + rsrr_solve of every handle, one host thread per stream; eigenvalue counts."""
        counts = [0] * len(handles)
        out = {}

        def work(slot):
            for i in range(slot, len(handles), len(sps)):
                h = handles[i]
                h.project(W["delta"])
                lam, V, res = h.solve(W["N_S"], W["K"], 1e3, 4096, vectors)
                counts[i] = int(lam.size)
                out[i] = (lam, V, res)
        threads = [threading.Thread(target=work, args=(k,)) for k in range(len(sps))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        return counts, out

    def step(Us):
        rs.sample_batch(hs, contours, Ns, Ls, Us, prec, args.tol, 20)
        return finish(hs)[0]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    step([p.U for p in probs])
    for _ in range(args.warmup - 1):
        step(None)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    l0 = rs.lib().rsrr_kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    for e0, e1 in evs:
        e0.record(stream)
        counts = step(None)
        e1.record(stream)
        infos.append([h.info() for h in hs])
    barrier()
    launches = rs.lib().rsrr_kernel_launches() - l0
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    clk = clocks.stop()
    points = sum(Ns)
    value, ms_max = job_value(points, args.steps, ms, device="cuda")
    med = lambda key: statistics.median(sum(i[key] for i in step_infos) for step_infos in infos)
    fac_ms = statistics.median(step_infos[0]["ms_factor"] for step_infos in infos)
    launches_f = infos[-1][0]["factor_launches"]
    strategies = [i["tune_strategy"] for i in infos[-1]]
    iterative = [i["iterative_band"] >= 0 for i in infos[-1]]
    if any(iterative) and not all(iterative):
        pass  # mixed: the roofline below follows the majority
    banded_now = args.banded or (autotune and sum(iterative) * 2 > len(iterative))
    if banded_now:  # band LU of the band part, kl = ku = s: 8 n kl (kl + ku) real flops per point
        flops = sum(p.N * 8.0 * p.n * p.meta["nx"] * 2 * p.meta["nx"] for p in probs)
        fac_ms = med("ms_factor")
        launches_f = sum(i["factor_launches"] for i in infos[-1])
    else:
        flops = sum(p.N * dense_lu_flops(p.n) for p in probs)
    achieved = flops / (fac_ms / 1e3) / 1e12 if fac_ms > 0 else None
    bf16, _, src = measured_peaks()
    if banded_now:
        lu_peak = FFMA_PEAK_TFLOPS if precision == "c64" else FP64_PEAK_TFLOPS
        roof = {"kernel": "band_factor_kernel<%s> (band part of T only: the incomplete factor of the iterative "
                          "sampler)" % ("float" if precision == "c64" else "double"), "bound": "alu",
                "achieved": achieved, "peak": lu_peak, "unit": "TFLOP/s", "traffic": None,
                "peak_source": "derived FFMA rate (152 SMs x 128 lanes x 2 x 2.07 GHz)" if precision == "c64"
                else "nominal FP64 rate"}
    elif precision == "c64":
        roof = {"kernel": "dense_factor_kernel<float> (persistent dense LU, one CTA per point; trailing update "
                          "on tcgen05 BF16 tensor cores)", "bound": "tensor", "achieved": achieved, "peak": bf16,
                "unit": "TFLOP/s", "traffic": None, "peak_source": "BF16 dense, " + src,
                "split_ceiling": bf16 / 6.0,
                "split_note": "each real product is 6 BF16 piece products (3-piece split), so the algorithmic "
                              "ceiling is peak / 6"}
    else:
        roof = {"kernel": "dense_factor_kernel<double> (persistent dense LU, CUDA-core FP64)", "bound": "alu",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "traffic": None,
                "peak_source": "nominal FP64 rate"}
    roof.update({"algorithmic": (f"8 n s (2 s) real flops per point (band half-width s), {points} points in "
                                  f"{launches_f} launches") if banded_now else
                 f"(8/3) n^3 real flops per point, {points} points in {launches_f} launches",
                 "ms_per_step": fac_ms})
    roof["frac"] = achieved / roof["peak"] if achieved else None
    if "split_ceiling" in roof and achieved:
        roof["frac_of_split_ceiling"] = achieved / roof["split_ceiling"]
    phases = {"sample_ms": statistics.median(step_infos[0]["ms_sample"] for step_infos in infos),
              "factor_ms": fac_ms,
              "trsv_ms": statistics.median(step_infos[0]["ms_trsv"] for step_infos in infos),
              "project_ms": med("ms_project"), "solve_ms": med("ms_solve")}
    e2e = None
    if not args.no_e2e:
        pin = lambda a: _pinned(torch, a)
        host = [(pin(p.rowptr), pin(p.colind), pin(p.vals), pin(np.asfortranarray(p.U))) for p in probs]
        h2d = sum(sum(x.nbytes for x in t) for t in host)
        barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.steps):
            gs = [make(i, p, t[0], t[1], t[2]) for i, (p, t) in enumerate(zip(probs, host))]
            rs.sample_batch(gs, contours, Ns, Ls, [t[3] for t in host], prec, args.tol, 20)
            _, out = finish(gs, vectors=True)
            d2h = sum(lam.nbytes + V.nbytes + res.nbytes for lam, V, res in out.values())
            for g in gs:
                g.close()
        barrier()
        e2e_value, _ = job_value(points, args.steps, 1e3 * (time.perf_counter() - t0), device="cuda")
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    # ---- the same matrices with a contour that encloses eigenvalues (the benchmark contour
    # encloses none): one full pass returning eigenpairs at full size, timed the same way, with
    # its eigenvalues against the closed form of the damped problem ----------------------------
    eig_arm = None
    if args.config == "1" and args.grid == 0 and not args.no_eigs:
        import workloads
        pb = workloads.config1b()
        g = rs.Nep(pb.n, pb.rowptr, pb.colind, pb.vals, fns_of(pb), 0, sp)

        def step_b():
            g.sample(pb.gamma, pb.a, pb.b, pb.N, pb.L, pb.U, prec, args.tol, 20)
            g.project(W["delta"])
            return g.solve(W["N_S"], W["K"], 1e3, 4096, True)
        step_b()
        kb = 2
        barrier()
        evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(kb)]
        for e0, e1 in evb:
            e0.record(stream)
            lam_b, _, res_b = step_b()
            e1.record(stream)
        barrier()
        infb = g.info()
        g.close()
        msb = sum(e0.elapsed_time(e1) for e0, e1 in evb)
        vb, _ = job_value(pb.N, kb, msb, device="cuda")
        nrm = [float(np.linalg.norm(pb.vals[i])) for i in range(pb.vals.shape[0])]
        al = np.abs(lam_b)
        scaled_res = res_b / (nrm[0] + al * nrm[1] + al ** 2 * nrm[2]) if lam_b.size else np.zeros(0)
        ex = np.asarray(pb.meta["expected"])   # closed form: the 10 lowest upper-branch eigenvalues
        ex = ex[((ex.real - pb.gamma.real) / pb.a) ** 2 + ((ex.imag - pb.gamma.imag) / pb.b) ** 2 < 1.0]
        err = max((float(np.min(np.abs(ex - l)) / abs(l)) for l in lam_b), default=None)
        eig_arm = {"workload": "the same n = 40000 damped QEP, ellipse placed around its lowest upper-branch "
                               "eigenvalues (N=64, L=32)", "value": vb, "unit": UNIT, "steps": kb,
                   "ms_per_step": msb / kb, "n_eigs_inside": int(lam_b.size),
                   "expected_inside": int(ex.size),
                   "max_scaled_residual": float(scaled_res.max()) if lam_b.size else None,
                   "max_rel_err_vs_closed_form": err, "k_S": infb["k_S"], "max_eta": infb["max_eta"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sample = cpu_dense_rate(probs)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    for h in hs:
        h.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64" if precision == "c64" else "c128",
                "data": W["data"],
                "config": dict({k: v for k, v in W.items() if k != "data"}, batch=B, precision=precision,
                               n_range=[min(p.n for p in probs), max(p.n for p in probs)],
                               parallelism=f"replicas x{world}" if world > 1 else "1 GPU", tol=args.tol,
                               sampler=("iterative: band part factored (half-width s), FGMRES on the full T")
                               if args.banded else ("autotuned per member (RSRR_AUTOTUNE)" if autotune else "dense LU"),
                               l2="inputs larger than L2 (dense factors of GBs per step)"),
                "phases_ms_median": phases, "eigs_inside": counts,
                "tune_strategies": {name: strategies.count(code) for code, name in
                                    ((0, "band_tc"), (1, "band_cuda_cores"), (2, "dense"), (3, "iterative"), (-1, "untuned"))},
                "max_eta": max(i["max_eta"] for step_infos in infos for i in step_infos),
                "refine_sweeps": max(i["refine_sweeps"] for i in infos[-1]),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


SERVE_TYPES = ("0", "1", "2", "3")


def serve_requests(serve, count, seed, precision_flags):
    """`count` requests with types drawn uniformly from configs 0, 1, 2 and single members of the
    time-delay batch (seeded), each with the config's own contour, N, L and probing block."""
    import workloads
    rng = np.random.default_rng([4, seed])
    out = []
    cache = {}
    for i in range(count):
        t = SERVE_TYPES[int(rng.integers(0, len(SERVE_TYPES)))]
        if t == "3":
            p = workloads.config3_member(int(rng.integers(0, 256)), s=int(rng.integers(20, 41)))
        else:
            if t not in cache:
                cache[t] = workload(t)
            p = cache[t]
        prec = precision_flags(t)
        out.append(serve.Request(rid=i, n=p.n, rowptr=p.rowptr, colind=p.colind, vals=p.vals, fns=fns_of(p),
                                 gamma=p.gamma, a=p.a, b=p.b, N=p.N, L=p.L, U=p.U, precision=prec,
                                 N_S=500, K=2))
        out[-1].tag = t
    return out


def run_serve(args):
    """Config 4: Poisson request streams through the continuous-batching server, then the same
    requests one at a time in plain FP64 (the per-request path it is compared against)."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    import paper_1510_07522_gb300 as rs
    from paper_1510_07522_gb300 import serve
    torch.cuda.set_device(local)
    mixed = lambda t: (rs.RSRR_FP64 if t == "0" else rs.RSRR_C64_IR) | rs.RSRR_REFINE_FULL
    plain = lambda t: rs.RSRR_FP64 | rs.RSRR_REFINE_FULL
    rates = [float(r) for r in args.rates.split(",")]
    # warm-up: one request of each type through a one-slot server
    warm = serve.Server(budget_bytes=150e9, slots=1)
    serve.replay(warm, serve_requests(serve, 4, 99, mixed), [0.0] * 4)
    warm.close()
    l0 = rs.lib().rsrr_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    per_rate = []
    for k, rate in enumerate(rates):
        reqs = serve_requests(serve, args.requests, k, mixed)
        srv = serve.Server(budget_bytes=150e9, slots=4)
        t0 = time.perf_counter()
        done = serve.replay(srv, reqs, serve.poisson_arrivals(rate, len(reqs), seed=1))
        wall = time.perf_counter() - t0
        srv.close()
        st = serve.latency_stats(done)
        st.update(rate=rate, wall_s=wall, peak_inflight=srv.peak_inflight,
                  errors=sorted({r.error for r in done if r.error}),
                  by_type={t: sum(1 for r in done if r.tag == t) for t in SERVE_TYPES})
        per_rate.append(st)
    # the plain FP64 per-request path: the first requests of the last rate's stream, one at a time,
    # no overlap (bounded: FP64 requests of the larger configs take seconds each)
    n64 = args.fp64_requests or min(args.requests, 40)
    reqs = serve_requests(serve, args.requests, len(rates) - 1, plain)[:n64]
    srv = serve.Server(budget_bytes=150e9, slots=1)
    done = serve.replay(srv, reqs, serve.poisson_arrivals(rates[-1], len(reqs), seed=1))
    srv.close()
    fp64 = serve.latency_stats(done)
    fp64.update(rate=rates[-1], requests=len(reqs), errors=sorted({r.error for r in done if r.error}),
                by_type={t: sum(1 for r in done if r.tag == t) for t in SERVE_TYPES})
    clk = clocks.stop()
    launches = rs.lib().rsrr_kernel_launches() - l0
    top = per_rate[-1]
    line = {"metric": "NEPs/s and p50/p99 latency, Poisson stream of mixed NEPs (continuous batching)",
            "value": top["neps_per_s"], "unit": "NEPs/s", "n_gpus": 1, "steps": len(rates), "warmup": 1,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+f64 (config 0 requests c128)", "data": "synthetic (seeded generators of configs 0-3)",
            "config": {"workload": "serving: request types uniform over configs 0, 1 (c64+IR), 2 and time-delay "
                                   "batch members (grid side 20..40, dense LU)",
                       "requests_per_rate": args.requests, "rates": rates, "budget_GB": 150, "slots": 4,
                       "arrivals": "Poisson, seed 1", "l2": "inputs larger than L2 for configs 1 and 2"},
            "per_rate": per_rate, "fp64_per_request": fp64, "gpu_launches": int(launches), "clocks": clk,
            "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(line), flush=True)


def run_compare(args):
    """Sampling scheme against the SSRR moment scheme (K' = N and N/2) on the paper's two small
    examples with its parameters: k_S, the singular value of the projection matrix at the
    eigenvalue count, the count found and the largest eigen-residual ||T(l) v|| / ||v||."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    import paper_1510_07522_gb300 as rs
    import workloads as w
    torch.cuda.set_device(local)
    cases = [("loaded_string", dict(n=5000, N=100, L=1), 1000, 8, 32),
             ("acoustic_1d", dict(), 1000, 2, 40)]
    out = []
    for name, kw, NS, K, count in cases:
        prob = w.by_name(name, **kw)
        for Kp in (0, prob.N, prob.N // 2):
            fns = [(f.kind, f.params()) for f in prob.fns]
            h = rs.Nep(prob.n, prob.rowptr, prob.colind, prob.vals, fns)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.sample(prob.gamma, prob.a, prob.b, prob.N, prob.L, prob.U, rs.RSRR_FP64, 1e-12, 12)
            kS = h.project_moments(Kp) if Kp else h.project(1e-14)
            lam, V, res = h.solve(NS, K, 1e3, 4096, True)
            torch.cuda.synchronize()
            ms = 1e3 * (time.perf_counter() - t0)
            sig = h.sigma()
            h.close()
            out.append({"problem": name, "n": prob.n, "N": prob.N, "L": prob.L,
                        "scheme": "sampling" if Kp == 0 else "moments K'=%d" % Kp, "k_S": int(kS),
                        "sigma_count_over_sigma1": float(sig[count - 1] / sig[0]) if sig.size >= count else 0.0,
                        "eigenvalues": int(lam.size), "max_residual": float(res.max()) if res.size else None,
                        "ms": round(ms, 1)})
    print(json.dumps({"metric": "sampling vs moment scheme (k_S, sigma at the count, residuals)",
                      "data": "the paper's loaded string and Acoustic-1D examples (printed matrices)",
                      "results": out}), flush=True)


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
    elif args.config == "serve":
        run_serve(args)
    elif args.config == "compare":
        run_compare(args)
    elif args.config == "3":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
