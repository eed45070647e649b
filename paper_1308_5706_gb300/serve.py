"""Continuous-batching request server for wavelet analysis / synthesis jobs.

Requests of mixed band-limit L, azimuthal band-limit N and dilation lambda
arrive over time (e.g. Poisson).  An analysis request brings a real signal
f_lm (host, pinned) and leaves its wavelet coefficients W resident on the
device; a synthesis request consumes the W of an earlier analysis request
(the client's analyse -> process -> synthesise pipeline) and returns f_lm.

Scheduling (host thread, non-blocking):
  * admission: a request becomes ready when it has arrived and, for a
    synthesis, its analysis has completed; it is admitted while the HBM
    footprint of everything in flight or resident (plan workspaces, f and W
    buffers) stays under the budget, and a stream slot is free; a request
    over the budget waits (a counted deferral) while other batches run, and
    goes ahead once nothing is on the GPU, so the queue always progresses;
  * continuous batching: each free slot takes the ready requests of one
    direction (up to `max_batch`) and runs them as ONE batched launch set
    (s2dw_analysis_batch / s2dw_synthesis_batch) on its own CUDA stream, so
    work that arrives while other batches are on the GPU overlaps with them;
  * completion is observed with CUDA events; latency = completion - arrival.
Plans are pooled per (L, N, lambda, J0, precision) and reused.  A request
whose configuration has no free plan waits while one is created on a worker
thread (plan creation runs device kernels and blocks its thread for
milliseconds; the library call releases the GIL), so the scheduler keeps
launching other work meanwhile.  Results are deterministic (no atomics in the
kernels), so a request gives bit-identical output alone and in the mix.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import math
import time
from typing import Dict, List, Optional

import numpy as np

from . import binding as B
from .inputs import flm_gaussian


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                 # "analysis" | "synthesis"
    L: int
    N: int
    lam: float
    arrival: float            # seconds from the start of the run
    seed: int = 0
    parent: Optional[int] = None   # analysis request whose W a synthesis consumes
    J0: int = 0
    # filled by the server
    t_admit: float = math.nan
    t_done: float = math.nan
    f: object = None          # device f_lm (analysis input / synthesis output)
    W: object = None
    Wphi: object = None


def poisson_workload(rate: float, duration: float, seed: int, L_range=(32, 2048), N_range=(1, 8),
                     lams=(2.0, 3.0), p_synthesis=0.5, Ls=None) -> List[Request]:
    """Poisson arrivals; L uniform over the set `Ls` when given (e.g. the
    powers of two an observation pipeline uses), else log-uniform in `L_range`;
    N uniform, lambda uniform in `lams`; each synthesis request consumes the
    oldest not yet consumed analysis."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, reqs, unconsumed = 0.0, [], collections.deque()
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        rid = len(reqs)
        if unconsumed and rng.random() < p_synthesis:
            par = reqs[unconsumed.popleft()]
            reqs.append(Request(rid, "synthesis", par.L, par.N, par.lam, t, parent=par.rid))
        else:
            if Ls is not None:
                L = int(Ls[int(rng.integers(0, len(Ls)))])
            else:
                L = int(round(math.exp(rng.uniform(math.log(L_range[0]), math.log(L_range[1])))))
            N = int(rng.integers(N_range[0], N_range[1] + 1))
            N = min(N, L)
            lam = float(lams[int(rng.integers(0, len(lams)))])
            reqs.append(Request(rid, "analysis", L, N, lam, t, seed=int(rng.integers(0, 2**31))))
            unconsumed.append(rid)
    return reqs


class Server:
    def __init__(self, precision: str = "mixed", slots: int = 4, max_batch: int = 16,
                 hbm_budget: Optional[int] = None, max_pool_bytes: Optional[int] = None,
                 plan_workers: int = 2, table_L: int = 0):
        """table_L > 0: build the process-wide Wigner tables for band-limits up
        to table_L at start-up (a plan of that size is kept for the server's
        lifetime), so that no request pays for growing them."""
        import torch
        self.torch = torch
        self.precision = precision
        self.anchor = B.Plan(table_L, 1, 2.0, 0, precision) if table_L > 0 else None
        self.max_batch = min(max_batch, 64)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        free, total = torch.cuda.mem_get_info()
        self.budget = hbm_budget if hbm_budget is not None else int(free * 0.6)
        self.max_pool_bytes = max_pool_bytes if max_pool_bytes is not None else self.budget // 2
        self.pool: Dict[tuple, List[B.Plan]] = collections.defaultdict(list)
        self.pool_bytes = 0
        self.in_use = 0            # bytes of f/W buffers alive
        self.rejected = 0          # admission deferrals (budget or slots)
        self.stats = collections.Counter()
        self.workers = concurrent.futures.ThreadPoolExecutor(max_workers=max(1, plan_workers))
        self.creating: Dict[tuple, List[concurrent.futures.Future]] = collections.defaultdict(list)

    # ---- plans -------------------------------------------------------------
    def _key(self, r: Request):
        return (r.L, r.N, r.lam, r.J0, self.precision)

    def _take_plan(self, r: Request) -> Optional[B.Plan]:
        """A free plan of r's configuration, or None (one is then being made)."""
        key = self._key(r)
        lst = self.pool[key]
        if lst:
            self.stats["plan_take"] += 1
            p = lst.pop()
            self.pool_bytes -= p.info["workspace_bytes"]
            return p
        if not self.creating[key]:
            self.stats["plan_create"] += 1
            self.creating[key].append(self.workers.submit(self._make_plan, r.L, r.N, r.lam, r.J0))
        return None

    def _make_plan(self, L, N, lam, J0):
        t0 = time.perf_counter()
        p = B.Plan(L, N, lam, J0, self.precision)
        return p, time.perf_counter() - t0

    def _collect_plans(self):
        for key, futs in self.creating.items():
            for fu in [f for f in futs if f.done()]:
                futs.remove(fu)
                p, dt = fu.result()
                self.stats["plan_create_s"] += dt
                self.pool[key].append(p)
                self.pool_bytes += p.info["workspace_bytes"]

    def prewarm(self, reqs: List[Request], per_key: int = 1) -> float:
        """Create `per_key` plans for every configuration in `reqs` ahead of
        serving (plan creation computes kernels and tables on the device and
        blocks the host thread for milliseconds).  Returns the seconds spent."""
        t0 = time.perf_counter()
        for key in sorted({self._key(r) for r in reqs}):
            L, N, lam, J0, prec = key
            while len(self.pool[key]) < per_key:
                self._give_plan(B.Plan(L, N, lam, J0, prec))
        return time.perf_counter() - t0

    def _give_plan(self, p: B.Plan):
        self.pool[(p.L, p.N, p.lam, p.J0, p.precision)].append(p)
        self.pool_bytes += p.info["workspace_bytes"]
        while self.pool_bytes > self.max_pool_bytes:
            k = next((k for k, v in self.pool.items() if v), None)
            if k is None:
                break
            q = self.pool[k].pop(0)
            self.pool_bytes -= q.info["workspace_bytes"]
            q.close()

    def _footprint(self, r: Request) -> int:
        el = 4 if self.precision == "mixed" else 8
        n = 2 * r.L - 1
        J = B_jmax(r.L, r.lam) - r.J0
        w = ((J + 1) * r.N * 2 * r.L * n + 2 * r.L * n) * el
        f = r.L * r.L * 2 * el
        ws = 0 if self.pool.get(self._key(r)) else _workspace_estimate(r, el)
        return (w + f if r.kind == "analysis" else f) + ws

    # ---- run ---------------------------------------------------------------
    def run(self, reqs: List[Request], keep_outputs: bool = False, time_scale: float = 1.0, payload=None):
        """Serve `reqs`; `payload(r)` gives an analysis request's f_lm as a pinned
        host tensor (the bytes a client sends; by default generated from r.seed
        when the request is admitted)."""
        torch = self.torch
        cd = torch.complex64 if self.precision == "mixed" else torch.complex128
        rd = torch.float32 if self.precision == "mixed" else torch.float64
        by_id = {r.rid: r for r in reqs}
        pending = collections.deque(sorted(reqs, key=lambda r: r.arrival))
        ready: List[Request] = []
        busy = [None] * len(self.streams)      # per slot: (event, batch, plans, t_launch)
        consumers = collections.Counter(r.parent for r in reqs if r.parent is not None)
        done_count = 0
        t0 = time.perf_counter()
        while done_count < len(reqs):
            now = (time.perf_counter() - t0) / time_scale
            # completions
            for s, b in enumerate(busy):
                if b is not None and b[0].query():
                    ev, batch, plans = b[0], b[1], b[2]
                    tdone = (time.perf_counter() - t0) / time_scale
                    for r, p in zip(batch, plans):
                        r.t_done = tdone
                        self._give_plan(p)
                        done_count += 1
                        # buffers leave the server's account once consumed (kept
                        # outputs are handed to the caller and stop counting too)
                        if r.kind == "synthesis":
                            par = by_id[r.parent]
                            consumers[par.rid] -= 1
                            if consumers[par.rid] == 0:
                                self.in_use -= _nbytes(par.W) + _nbytes(par.Wphi)
                                if not keep_outputs:
                                    par.W = par.Wphi = None
                            self.in_use -= _nbytes(r.f)
                            if not keep_outputs:
                                r.f = None
                        elif consumers[r.rid] == 0:  # an analysis no synthesis consumes
                            self.in_use -= _nbytes(r.W) + _nbytes(r.Wphi)
                            if not keep_outputs:
                                r.W = r.Wphi = None
                    busy[s] = None
            self._collect_plans()
            # arrivals -> ready (synthesis waits for its analysis)
            while pending and pending[0].arrival <= now:
                ready.append(pending.popleft())
            # admission + batched launch on each free slot
            for s in range(len(self.streams)):
                if busy[s] is not None or not ready:
                    continue
                kind = None
                batch: List[Request] = []
                plans: List[B.Plan] = []
                budget_left = self.budget - self.in_use - self.pool_bytes
                for r in list(ready):
                    if r.kind == "synthesis" and not (by_id[r.parent].t_done <= now):
                        continue
                    if (kind is not None and r.kind != kind) or len(batch) >= self.max_batch:
                        continue
                    fp = self._footprint(r)
                    # over the budget: wait while other work runs (it frees memory);
                    # with nothing on the GPU the request goes ahead, so the queue
                    # always progresses (resident W that waits for its synthesis is
                    # not work in flight)
                    running = any(b is not None for b in busy)
                    if fp > budget_left and (batch or running):
                        self.rejected += 1
                        continue
                    p = self._take_plan(r)
                    if p is None:
                        continue
                    kind = r.kind
                    batch.append(r)
                    plans.append(p)
                    budget_left -= fp
                if not batch:
                    continue
                for r in batch:
                    ready.remove(r)
                stream = self.streams[s]
                with torch.cuda.stream(stream):
                    if kind == "analysis":
                        for r, p in zip(batch, plans):
                            fh = payload(r) if payload is not None else \
                                torch.from_numpy(flm_gaussian(r.L, r.seed, "cl")).to(cd).pin_memory()
                            r.f = torch.empty(r.L * r.L, dtype=cd, device="cuda")
                            r.f.copy_(fh, non_blocking=True)
                            r.W = torch.empty(p.w_shape, dtype=rd, device="cuda")
                            r.Wphi = torch.empty(p.wphi_shape, dtype=rd, device="cuda")
                            self.in_use += _nbytes(r.f) + _nbytes(r.W) + _nbytes(r.Wphi)
                        B.s2dw_analysis_batch([p.handle for p in plans], [r.f for r in batch],
                                              [r.W for r in batch], [r.Wphi for r in batch], stream)
                        for r in batch:  # the input f is read by the launch set on this stream
                            self.in_use -= _nbytes(r.f)
                            if not keep_outputs:
                                r.f = None
                    else:
                        for r in batch:
                            r.f = torch.empty(r.L * r.L, dtype=cd, device="cuda")
                            self.in_use += _nbytes(r.f)
                        B.s2dw_synthesis_batch([p.handle for p in plans], [by_id[r.parent].W for r in batch],
                                               [by_id[r.parent].Wphi for r in batch], [r.f for r in batch],
                                               stream)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                for r in batch:
                    r.t_admit = now
                self.stats["batches"] += 1
                self.stats["batched_jobs"] += len(batch)
                busy[s] = (ev, batch, plans)
            if all(b is None for b in busy) and not ready and pending:
                wait = pending[0].arrival - (time.perf_counter() - t0) / time_scale
                if wait > 0:
                    time.sleep(min(wait * time_scale, 0.002))
            else:
                time.sleep(0.0001)
        wall = (time.perf_counter() - t0) / time_scale
        return self.report(reqs, wall)

    def report(self, reqs, wall):
        lat = np.array([r.t_done - r.arrival for r in reqs]) * 1e3
        return {"requests": len(reqs), "wall_s": wall, "transforms_per_s": len(reqs) / wall,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "mean": float(lat.mean()), "max": float(lat.max())},
                "admission_deferrals": self.rejected, "batches": self.stats["batches"],
                "mean_batch": self.stats["batched_jobs"] / max(1, self.stats["batches"]),
                "plans_created": self.stats["plan_create"], "plans_taken_from_pool": self.stats["plan_take"],
                "plan_create_s": round(self.stats["plan_create_s"], 3),
                "plan_create_ms_mean": round(1e3 * self.stats["plan_create_s"] / max(1, self.stats["plan_create"]), 3)}

    def close(self):
        self.workers.shutdown(wait=True)
        self._collect_plans()
        for lst in self.pool.values():
            for p in lst:
                p.close()
        self.pool.clear()
        if self.anchor is not None:
            self.anchor.close()
            self.anchor = None


def _nbytes(t) -> int:
    return 0 if t is None else t.numel() * t.element_size()


def B_jmax(L: int, lam: float) -> int:
    J, p = 0, 1.0
    while p < L:
        p *= lam
        J += 1
    return J


def _workspace_estimate(r: Request, el: int) -> int:
    # conservative: Fourier cubes, beta outputs and synthesis partials of a plan
    L, N = r.L, r.N
    return int(2 * (3 * N * L * L + 2 * N * 2 * L * L) * el + (L // 32 + 1) * L * L * 2 * el + 2 * L * N * L * el)
