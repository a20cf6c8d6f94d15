"""Streaming block server: continuous batching of concurrent observations on one GPU.

Several observations deliver blocks over time.  Each observation is served by a few chunk plans,
one per contiguous range of its subbands (subbands are independent given their own FIR/shift
history, so the chunks together give exactly the beams of one plan over the whole block).  A block
is admitted as soon as

  * its observation has fewer than two blocks on the GPU (the FIR history makes an observation's
    blocks sequential on its compute stream, but block k + 1 may already upload while block k is
    being processed), and
  * the device-memory budget has room for the block's input and output buffers (drawn from a
    shared pool, so observations share memory); among the admissible blocks the one that arrived
    first goes first.

An admitted block is pipelined over three streams of its observation: chunk c is uploaded (one
strided copy out of the whole host block, lbf_upload_subbands), filtered and beam-formed
(lbf_run_block_ws) and downloaded (lbf_download_subbands) while chunk c + 1 is uploading, so a
block's latency is about one upload plus the last chunk's kernels and download, not the sum of
the whole block's upload, kernels and download.  Blocks of different observations overlap on the
device.  Latency is measured per block from its arrival to the host seeing its last download
complete, and reported as p50/p99 against the real-time block period.

All computation runs in the CUDA library; this module schedules, accounts memory and orders the
copies.
"""

from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np

MAX_INFLIGHT_PER_OBS = 2


@dataclass
class BlockResult:
    obs: int
    index: int
    arrival: float
    admitted: float
    done: float
    upload_gbs: float = 0.0   # host-to-device rate of this block's own uploads (CUDA events)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Chunk:
    plan: object
    first: int               # first subband of the chunk in the observation


@dataclass
class _Obs:
    oid: int
    chunks: list
    n_subbands: int
    s_h2d: object            # upload stream
    s_comp: object           # kernel stream (the chunks' histories advance in order here)
    s_d2h: object            # download stream
    ws: object               # device workspace shared by the chunks (they run one after another)
    host_in: object          # default pinned host input / output of a block (whole observation)
    host_out: object
    queue: list = field(default_factory=list)   # (arrival, index, host_in, host_out) waiting, in order
    inflight: int = 0
    results: list = field(default_factory=list)
    outputs: list = field(default_factory=list)

    @property
    def busy(self) -> bool:
        return self.inflight > 0


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
        self.reserved = 0      # bytes owned permanently (plans and workspaces)
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


def subband_ranges(n_subbands: int, n_chunks: int):
    """n_chunks contiguous, nearly equal subband ranges (first, count) covering n_subbands."""
    k = max(1, min(int(n_chunks), int(n_subbands)))
    edges = [round(i * n_subbands / k) for i in range(k + 1)]
    return [(edges[i], edges[i + 1] - edges[i]) for i in range(k)]


class Server:
    """Continuous-batching server of observation blocks on one GPU."""

    def __init__(self, device, budget_bytes: int, keep_outputs: bool = False):
        import torch
        self.torch = torch
        self.device = device
        self.pool = Pool(device, budget_bytes)
        self.obs: dict[int, _Obs] = {}
        self.inflight = []          # (done event, obs, index, arrival, admitted, buffers, host_out, upload events)
        self.keep_outputs = keep_outputs

    # -- observations
    def add(self, oid: int, chunk_plans, n_subbands: int, host_in, host_out):
        """Observation `oid` served by `chunk_plans`: a list of (plan, first_subband) covering its
        n_subbands subbands in order (one plan is the whole observation as a single chunk).  Plans
        are created with an external workspace; host_in / host_out are the default pinned host
        buffers of a whole block."""
        chunks = [_Chunk(p, int(f)) for p, f in chunk_plans]
        assert sum(c.plan.dims.n_subbands for c in chunks) == n_subbands
        plan_bytes = sum(c.plan.device_bytes() for c in chunks)
        ws_bytes = max(c.plan.dims.workspace_bytes for c in chunks)
        if self.pool.reserved + plan_bytes + ws_bytes > self.pool.budget:
            raise MemoryError(f"observation {oid}: plans need {plan_bytes + ws_bytes} B beyond the budget")
        self.pool.reserved += plan_bytes + ws_bytes
        ws = self.torch.empty(max(ws_bytes, 256), dtype=self.torch.uint8, device=self.device)
        o = _Obs(oid, chunks, int(n_subbands), *(self.torch.cuda.Stream(device=self.device) for _ in range(3)),
                 ws, host_in, host_out)
        self.obs[oid] = o
        if self.pool.reserved + self.block_bytes(oid) > self.pool.budget:
            raise MemoryError(f"observation {oid}: one block needs {self.block_bytes(oid)} B beyond the budget")

    def block_bytes(self, oid: int) -> int:
        """Pool bytes one block of observation oid holds while in flight (inputs and outputs)."""
        return sum(c.plan.dims.in_bytes + c.plan.dims.out_bytes for c in self.obs[oid].chunks)

    # -- arrivals and scheduling
    def arrive(self, oid: int, index: int, t: float, host_in=None, host_out=None):
        """Block `index` of observation oid arrived at time t (host buffers default to the
        observation's own)."""
        self.obs[oid].queue.append((t, index, host_in, host_out))

    def _enqueue(self, o: _Obs, host_in, host_out):
        torch = self.torch
        bufs = []
        up0 = torch.cuda.Event(enable_timing=True)
        up0.record(o.s_h2d)
        for c in o.chunks:
            d = c.plan.dims
            d_in, d_out = self.pool.take(d.in_bytes), self.pool.take(d.out_bytes)
            bufs += [(d_in, d.in_bytes), (d_out, d.out_bytes)]
            c.plan.upload_subbands(host_in, o.n_subbands, c.first, d_in, o.s_h2d)
            ev_in = torch.cuda.Event()
            ev_in.record(o.s_h2d)
            o.s_comp.wait_event(ev_in)
            c.plan.run_block_ws(d_in, d_out, o.ws, o.s_comp)
            ev_k = torch.cuda.Event()
            ev_k.record(o.s_comp)
            o.s_d2h.wait_event(ev_k)
            c.plan.download_subbands(d_out, o.n_subbands, c.first, host_out, o.s_d2h)
        up1 = torch.cuda.Event(enable_timing=True)
        up1.record(o.s_h2d)
        done = torch.cuda.Event()
        done.record(o.s_d2h)
        return done, bufs, (up0, up1)

    def _admit(self, now: float):
        # earliest arrival first, across observations
        cands = sorted((o.queue[0][0], o.oid) for o in self.obs.values()
                       if o.queue and o.inflight < MAX_INFLIGHT_PER_OBS)
        for _, oid in cands:
            o = self.obs[oid]
            if not self.pool.fits(self.block_bytes(oid)):
                continue
            arrival, index, h_in, h_out = o.queue.pop(0)
            h_in = o.host_in if h_in is None else h_in
            h_out = o.host_out if h_out is None else h_out
            ev, bufs, up = self._enqueue(o, h_in, h_out)
            o.inflight += 1
            self.inflight.append((ev, o, index, arrival, now, bufs, h_out, up))

    def _reap(self, now: float):
        still = []
        for item in self.inflight:
            ev, o, index, arrival, admitted, bufs, h_out, up = item
            if ev.query():
                done = time.perf_counter()
                up_s = up[0].elapsed_time(up[1]) / 1e3
                nbytes = sum(c.plan.dims.in_bytes for c in o.chunks)
                o.results.append(BlockResult(o.oid, index, arrival, admitted, done,
                                             nbytes / up_s / 1e9 if up_s > 0 else 0.0))
                if self.keep_outputs:
                    o.outputs.append(h_out.clone())
                for t, n in bufs:
                    self.pool.give(t, n)
                o.inflight -= 1
            else:
                still.append(item)
        self.inflight = still

    def idle(self) -> bool:
        return not self.inflight and not any(o.queue for o in self.obs.values())

    def step(self):
        now = time.perf_counter()
        self._reap(now)
        self._admit(now)

    def run(self, schedule, poll_s: float = 2e-4):
        """Serve a schedule of (arrival_offset_s, oid, index) in real time; returns the results and
        the wall time.  `busy_s` afterwards holds the time during which at least one block was
        waiting or in flight (the GPU and its copy engines had work)."""
        events = list(schedule)
        heapq.heapify(events)
        t0 = time.perf_counter()
        self.busy_s = 0.0
        last = t0
        while events or not self.idle():
            now = time.perf_counter()
            if not self.idle():
                self.busy_s += now - last
            last = now
            while events and t0 + events[0][0] <= now:
                off, oid, index = heapq.heappop(events)
                self.arrive(oid, index, t0 + off)
            self.step()
            if self.idle() and events:
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
    out = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "max_s": float(lat.max()), "period_s": period_s, "blocks": int(lat.size),
           "late_blocks": int(np.sum(lat > period_s))}
    up = np.array([r.upload_gbs for r in results if r.upload_gbs > 0])
    if up.size:   # the host link as the blocks' own uploads saw it (shared with other jobs)
        out["block_upload_gbs"] = {"p50": float(np.percentile(up, 50)), "min": float(up.min()),
                                   "max": float(up.max())}
    return out
