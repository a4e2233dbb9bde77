"""Continuous-batching RSRR server on one GPU.

Requests (one NEP each: T(z) = sum_i f_i(z) A_i, contour, N, L, U) arrive at any time.  A
fixed set of worker slots, each owning a CUDA stream, runs admitted requests through the C
ABI (rsrr_create_nep -> rsrr_sample -> rsrr_project -> rsrr_solve -> rsrr_destroy).  ctypes
releases the GIL during each call, so the device work of different requests overlaps on
their streams, and a request's factors and samples stay on the device from sample to solve.

Admission: a waiting request is admitted as soon as a slot is free and its estimated device
footprint fits in what is left of the HBM budget; requests are taken in arrival order, but a
request that does not fit yet may be passed by later, smaller ones (at most `max_bypass`
times, so none starves).  A request refused by the device for lack of memory (ENOMEM) goes
back to the head of the queue, but only while other requests are in flight, whose completion can
free memory: it is not taken again before one of them completes, and after `max_retries`
refusals, or a refusal while it ran alone, it is finished with the error.
"""
from __future__ import annotations

import ctypes
import threading
import time
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import RSRR_C64_IR, RSRR_REFINE_FULL, Nep, RsrrError


def select_admissible(pending: List["Request"], free: int, max_bypass: int, completions: int = 0) -> Optional[int]:
    """Index of the oldest pending request whose footprint fits in `free` bytes, or None.
    Every older request it passes counts one bypass; a request that has been passed
    `max_bypass` times blocks everything behind it until it fits.  A request sent back after
    ENOMEM waits for `completions` (the server's count of finished requests) to pass the value
    it recorded; until then it is skipped and neither counts bypasses nor blocks."""
    for i, r in enumerate(pending):
        if r.held_until >= completions:
            continue
        if r.footprint <= free:
            for older in pending[:i]:
                if older.held_until < completions:
                    older.bypassed += 1
            return i
        if r.bypassed >= max_bypass:
            return None
    return None


def after_enomem(req: "Request", others_inflight: int, completions: int, max_retries: int) -> bool:
    """Decide what happens to a request the device refused for lack of memory.  Returns True to
    requeue it (held until one more request completes), False to finish it with the error: when
    nothing else was in flight (no completion can free memory for it) or after max_retries."""
    req.retries += 1
    if others_inflight == 0 or req.retries > max_retries:
        return False
    req.held_until = completions
    return True


def band_of(n: int, rowptr: np.ndarray, colind: np.ndarray):
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    d = colind.astype(np.int64) - rows
    return int(max(0, -d.min())), int(max(0, d.max()))


def footprint_bytes(n: int, kl: int, ku: int, N: int, L: int, nnz: int, J: int, c64: bool = True,
                    N_S: int = 500, K: int = 2) -> int:
    """An upper bound of the device memory a request holds at its peak.  The handle keeps the CSR
    values and S_hat throughout; each phase frees its own work before the next starts, so the
    peak is that plus the largest phase:
      sampling   the band factors, right-hand sides and FP64 residuals of all N points (fewer
                 when they are chunked);
      projection the QR's copy of S_hat, the digit images of its trailing block (4 bytes of image
                 per byte of matrix) and the products A_i S (k_S <= min(n, N L) columns);
      reduced    at most N_S points of T_S(z) at once and no more than 24 GiB of them (dense in band
                 storage, about 5 k_S^2 complex128 values per point), moments, Hankel matrices."""
    es = 8 if c64 else 16
    ldab = 2 * kl + ku + 1
    ldp = (32 + kl + 31) // 32 * 32
    per_point = ldab * n * es + n * ldp * es + n * L * es + n * L * 16 + nnz * 16 + n * 16
    sample = N * per_point
    s_hat = n * N * L * 16
    k = min(n, N * L)
    project = 6 * s_hat + J * n * k * 16
    per_sample = 16 * (5 * k * k + 64 * k) + k * (k + 64) + 4 * k + 64
    reduced = min(N_S * per_sample, max(per_sample, 24 << 30)) + 16 * k * k * (J + 2 * K + 4 * K * K + 8) \
        + N_S * J * 16
    persistent = s_hat + J * nnz * 16 + (64 << 20)
    return int(persistent + max(sample, project, reduced))


@dataclass
class Request:
    rid: int
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray             # complex [J, nnz]
    fns: Sequence                # [(kind, params)]
    gamma: complex
    a: float
    b: float
    N: int
    L: int
    U: np.ndarray                # complex [n, L]
    precision: int = RSRR_C64_IR | RSRR_REFINE_FULL
    tol: float = 1e-10
    delta: float = 1e-14
    N_S: int = 500
    K: int = 2
    arrival: float = 0.0
    tag: str = ""                # caller's label (request type)
    # filled in by the server
    footprint: int = 0
    t_admit: float = 0.0
    t_done: float = 0.0
    lam: Optional[np.ndarray] = None
    resid: Optional[np.ndarray] = None
    k_S: int = -1
    error: Optional[str] = None
    bypassed: int = 0
    retries: int = 0             # ENOMEM refusals so far
    held_until: int = -1         # not admitted until more than this many requests have completed

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class Server:
    def __init__(self, budget_bytes: float = 150e9, slots: int = 4, max_bypass: int = 8, device: int = 0,
                 max_retries: int = 3):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.in_use = 0
        self.max_bypass = max_bypass
        self.max_retries = max_retries
        self.completions = 0
        self.device = device
        self.pending: List[Request] = []
        self.done: List[Request] = []
        self.cv = threading.Condition()
        self.stopping = False
        self.t0 = time.perf_counter()
        self.peak_inflight = 0
        self.inflight = 0
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        for w in self.workers:
            w.start()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request) -> None:
        kl, ku = band_of(req.n, req.rowptr, req.colind)
        req.footprint = footprint_bytes(req.n, kl, ku, req.N, req.L, int(req.colind.size), int(req.vals.shape[0]),
                                        (req.precision & 0xff) == RSRR_C64_IR, req.N_S, req.K)
        if req.footprint > self.budget:
            req.error = "request larger than the whole memory budget"
            req.t_done = self.now()
            with self.cv:
                self.done.append(req)
                self.cv.notify_all()
            return
        with self.cv:
            req.arrival = self.now() if req.arrival == 0.0 else req.arrival
            self.pending.append(req)
            self.cv.notify_all()

    def _take(self) -> Optional[Request]:
        i = select_admissible(self.pending, self.budget - self.in_use, self.max_bypass, self.completions)
        return None if i is None else self.pending.pop(i)

    def _worker(self, slot: int) -> None:
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream()
        sp = ctypes.c_void_p(stream.cuda_stream)
        while True:
            with self.cv:
                req = None
                while not self.stopping:
                    req = self._take()
                    if req is not None:
                        break
                    self.cv.wait()
                if req is None:
                    return
                self.in_use += req.footprint
                self.inflight += 1
                self.peak_inflight = max(self.peak_inflight, self.inflight)
                req.t_admit = self.now()
            enomem = None
            try:
                with torch.cuda.stream(stream):
                    h = Nep(req.n, req.rowptr, req.colind, req.vals, req.fns, 0, sp)
                    try:
                        h.sample(req.gamma, req.a, req.b, req.N, req.L, req.U, req.precision, req.tol, 20)
                        req.k_S = h.project(req.delta)
                        lam, _, res = h.solve(req.N_S, req.K, 1e3, 4096, False)
                        req.lam, req.resid = lam, res
                    finally:
                        h.close()
            except RsrrError as e:
                if e.name == "ENOMEM":
                    enomem = str(e)
                else:
                    req.error = str(e)
            with self.cv:
                self.in_use -= req.footprint
                self.inflight -= 1
                if enomem is not None and after_enomem(req, self.inflight, self.completions, self.max_retries):
                    self.pending.insert(0, req)
                else:
                    if enomem is not None:
                        req.error = enomem
                    req.t_done = self.now()
                    self.done.append(req)
                    self.completions += 1
                self.cv.notify_all()

    def wait(self, count: int, timeout: float = 3600.0) -> List[Request]:
        end = time.perf_counter() + timeout
        with self.cv:
            while len(self.done) < count:
                left = end - time.perf_counter()
                if left <= 0:
                    break
                self.cv.wait(timeout=min(left, 1.0))
            return list(self.done)

    def close(self) -> None:
        with self.cv:
            self.stopping = True
            self.cv.notify_all()
        for w in self.workers:
            w.join(timeout=60)


def replay(server: Server, requests: List[Request], arrivals: Sequence[float]) -> List[Request]:
    """Submit requests at the given arrival times (seconds from now); wait for all of them."""
    start = server.now()
    for req, t in zip(requests, arrivals):
        delay = start + t - server.now()
        if delay > 0:
            time.sleep(delay)
        req.arrival = start + t
        server.submit(req)
    return server.wait(len(requests))


def poisson_arrivals(rate: float, count: int, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))


def latency_stats(reqs: List[Request]) -> dict:
    ok = [r for r in reqs if r.error is None]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(0)
    span = (max(r.t_done for r in ok) - min(r.arrival for r in ok)) if ok else 0.0
    return {"count": len(reqs), "ok": len(ok), "p50_s": float(np.percentile(lat, 50)) if ok else None,
            "p99_s": float(np.percentile(lat, 99)) if ok else None,
            "neps_per_s": (len(ok) / span) if span > 0 else None}
