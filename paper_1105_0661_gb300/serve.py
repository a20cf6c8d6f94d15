"""Streaming block server: continuous batching of concurrent observations on one GPU.

Several observations (each its own plan: tables and device-resident FIR/shift history) deliver
blocks over time.  The server admits a block as soon as

  * its observation has no block on the GPU (the FIR history makes an observation's blocks
    sequential), and
  * the device-memory budget has room for the block's working set (input staging, output, and
    the corner-turned scratch, drawn from a shared pool so observations share memory),

and then enqueues, on the observation's own CUDA stream, the host-to-device copy of the block, the
fused path (lbf_run_block_ws) and the device-to-host copy of the beams.  Blocks of different
observations therefore overlap on the device while others wait for memory; completions free their
slot and the next waiting block is admitted.  Latency is measured per block from its arrival to the
host seeing its completion event, and reported as p50/p99 against the real-time block period.

All computation runs in the CUDA library; this module schedules and accounts memory.
"""

from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class BlockResult:
    obs: int
    index: int
    arrival: float
    admitted: float
    done: float

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Obs:
    oid: int
    plan: object
    stream: object
    host_in: object          # pinned host tensor holding this observation's block bytes
    host_out: object         # pinned host tensor receiving its beams
    queue: list = field(default_factory=list)   # (arrival, index) waiting, in order
    busy: bool = False
    results: list = field(default_factory=list)
    outputs: list = field(default_factory=list)


class Pool:
    """Device buffers reused across blocks, accounted against a byte budget.

    Buffers are kept by size class and handed out again instead of being freed, so the steady
    state of the server makes no device allocations."""

    def __init__(self, device, budget_bytes: int):
        import torch
        self.torch = torch
        self.device = device
        self.budget = int(budget_bytes)
        self.held = 0          # bytes of buffers currently handed out (in-flight blocks)
        self.reserved = 0      # bytes owned permanently (plans)
        self.free = {}         # nbytes -> [tensor]

    def fits(self, nbytes: int) -> bool:
        return self.reserved + self.held + nbytes <= self.budget

    def take(self, nbytes: int):
        lst = self.free.get(nbytes)
        t = lst.pop() if lst else self.torch.empty(max(nbytes, 16), dtype=self.torch.uint8, device=self.device)
        self.held += nbytes
        return t

    def give(self, t, nbytes: int):
        self.held -= nbytes
        self.free.setdefault(nbytes, []).append(t)


class Server:
    """Continuous-batching server of observation blocks on one GPU."""

    def __init__(self, device, budget_bytes: int, keep_outputs: bool = False):
        import torch
        self.torch = torch
        self.device = device
        self.pool = Pool(device, budget_bytes)
        self.obs: dict[int, _Obs] = {}
        self.inflight = []          # (event, obs, index, arrival, admitted, buffers)
        self.keep_outputs = keep_outputs

    # -- observations
    def add(self, oid: int, plan, host_in, host_out):
        d = plan.dims
        plan_bytes = plan.device_bytes()
        if self.pool.reserved + plan_bytes > self.pool.budget:
            raise MemoryError(f"observation {oid}: plan needs {plan_bytes} B beyond the budget")
        self.pool.reserved += plan_bytes
        need = d.in_bytes + d.out_bytes + d.workspace_bytes
        if self.pool.reserved + need > self.pool.budget:
            raise MemoryError(f"observation {oid}: one block needs {need} B beyond the budget")
        self.obs[oid] = _Obs(oid, plan, self.torch.cuda.Stream(device=self.device), host_in, host_out)

    def block_bytes(self, oid: int) -> int:
        d = self.obs[oid].plan.dims
        return d.in_bytes + d.out_bytes + d.workspace_bytes

    # -- arrivals and scheduling
    def arrive(self, oid: int, index: int, t: float):
        self.obs[oid].queue.append((t, index))

    def _admit(self, now: float):
        # oldest waiting block first, across observations
        cands = sorted((o.queue[0][0], o.oid) for o in self.obs.values() if o.queue and not o.busy)
        for _, oid in cands:
            o = self.obs[oid]
            d = o.plan.dims
            if not self.pool.fits(d.in_bytes + d.out_bytes + d.workspace_bytes):
                continue
            arrival, index = o.queue.pop(0)
            bufs = [(self.pool.take(n), n) for n in (d.in_bytes, d.out_bytes, d.workspace_bytes)]
            d_in, d_out, d_ws = (b[0] for b in bufs)
            with self.torch.cuda.stream(o.stream):
                d_in[:d.in_bytes].copy_(o.host_in.view(self.torch.uint8)[:d.in_bytes], non_blocking=True)
                o.plan.run_block_ws(d_in, d_out, d_ws, o.stream)
                o.host_out.view(self.torch.uint8)[:d.out_bytes].copy_(d_out[:d.out_bytes], non_blocking=True)
                ev = self.torch.cuda.Event()
                ev.record(o.stream)
            o.busy = True
            self.inflight.append((ev, o, index, arrival, now, bufs))

    def _reap(self, now: float):
        still = []
        for item in self.inflight:
            ev, o, index, arrival, admitted, bufs = item
            if ev.query():
                done = time.perf_counter()
                o.results.append(BlockResult(o.oid, index, arrival, admitted, done))
                if self.keep_outputs:
                    o.outputs.append(o.host_out.clone())
                for t, n in bufs:
                    self.pool.give(t, n)
                o.busy = False
            else:
                still.append(item)
        self.inflight = still

    def run(self, schedule, poll_s: float = 2e-4):
        """Serve a schedule of (arrival_offset_s, oid, index) in real time; returns the results."""
        events = list(schedule)
        heapq.heapify(events)
        t0 = time.perf_counter()
        while events or self.inflight or any(o.queue for o in self.obs.values()):
            now = time.perf_counter()
            while events and t0 + events[0][0] <= now:
                off, oid, index = heapq.heappop(events)
                self.arrive(oid, index, t0 + off)
            self._reap(now)
            self._admit(now)
            if not self.inflight and events and not any(o.queue for o in self.obs.values()):
                time.sleep(max(0.0, min(poll_s * 10, t0 + events[0][0] - time.perf_counter())))
            else:
                time.sleep(poll_s)
        wall = time.perf_counter() - t0
        res = [r for o in self.obs.values() for r in o.results]
        return res, wall


def poisson_schedule(n_obs: int, n_blocks: int, period_s: float, rng: np.random.Generator):
    """Arrival offsets with Poisson jitter: per observation, block k arrives at
    k * period + J_k with J_k exponential of mean period/4 (late by a random amount, never early),
    observations staggered uniformly over one period."""
    out = []
    for oid in range(n_obs):
        phase = rng.uniform(0, period_s)
        for k in range(n_blocks):
            out.append((phase + k * period_s + rng.exponential(period_s / 4), oid, k))
    return out


def latency_summary(results, period_s: float) -> dict:
    lat = np.array([r.latency for r in results])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max()), "period_s": period_s, "blocks": int(lat.size),
            "late_blocks": int(np.sum(lat > period_s))}
