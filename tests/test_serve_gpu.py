"""Streaming server: concurrent observations of different shapes, admitted by a memory budget, give
each observation the same beams alone and in the mix; a budget that fits one block at a time still
serves everything (blocks wait for memory instead of failing)."""

import numpy as np
import pytest

from oracle import lbf_oracle as O
from synth import generate as G

torch = pytest.importorskip("torch")

N = 256


def _obs_specs():
    rng = np.random.default_rng(21)
    specs = []
    for oid, (S, F, B, out, bits, prec) in enumerate([(12, 3, 5, "I", 16, "fp32"), (24, 2, 70, "IQUV", 8, "fp16tc"),
                                                      (16, 4, 130, "I", 16, "fp16tc"), (8, 2, 9, "IQUV", 16, "fp32")]):
        xyz = G.lofar_positions(rng, S // 2, S - S // 2)
        wl = G.Workload(f"obs{oid}", xyz, G.subband_centres(F, 120e6 + 10e6 * oid), G.hex_beam_grid(B, 0.05),
                        (0.3, 0.4), 64 * N, 16 if out == "I" else 4, out, sample_bits=bits,
                        sigma=32.0 if bits == 16 else 8.0, source="tone")
        specs.append((wl, prec))
    return specs


def _make_server(dev, specs, budget, blocks):
    from paper_1105_0661_gb300 import Plan
    from paper_1105_0661_gb300.serve import Server
    srv = Server(dev, budget, keep_outputs=True)
    host = {}
    for oid, (wl, prec) in specs:
        plan = Plan.from_workload(wl, precision=prec, external_workspace=True)
        h_in = torch.empty(plan.dims.in_bytes, dtype=torch.uint8, pin_memory=True)
        h_out = torch.empty(plan.dims.out_bytes, dtype=torch.uint8, pin_memory=True)
        srv.add(oid, plan, h_in, h_out)
        host[oid] = (h_in, blocks[oid])
    return srv, host


def _serve(srv, host, schedule):
    """Run the schedule, loading each block's bytes into its observation's pinned input just
    before it can be admitted (blocks of one observation are sequential)."""
    # the server copies h_in at admission; feed block k when block k-1 has completed
    order = {}
    for off, oid, k in sorted(schedule):
        order.setdefault(oid, []).append(k)
    import time
    results = []
    pending = sorted(schedule)
    t0 = time.perf_counter()
    while pending or srv.inflight or any(o.queue for o in srv.obs.values()):
        now = time.perf_counter()
        while pending and t0 + pending[0][0] <= now:
            off, oid, k = pending[0]
            o = srv.obs[oid]
            if o.busy or o.queue:      # the previous block still owns the pinned input
                break
            h_in, blocks = host[oid]
            h_in.copy_(torch.from_numpy(blocks[k].reshape(-1).view(np.uint8)))
            srv.arrive(oid, k, t0 + off)
            pending.pop(0)
        srv._reap(now)
        srv._admit(now)
        time.sleep(1e-4)
    return {oid: [x.view(torch.float32).numpy().copy() for x in o.outputs] for oid, o in srv.obs.items()}


@pytest.mark.gpu
def test_alone_equals_mixed_and_budget_serialises():
    from paper_1105_0661_gb300 import build_lib
    build_lib.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    specs = _obs_specs()
    nblk = 3
    blocks = {oid: [G.make_block(wl, seed=oid, block_index=k) for k in range(nblk)] for oid, (wl, _) in enumerate(specs)}
    alone = {}
    for oid, spec in enumerate(specs):
        srv, host = _make_server(dev, [(oid, spec)], 8 << 30, blocks)
        alone[oid] = _serve(srv, host, [(0.001 * k, oid, k) for k in range(nblk)])[oid]
    # all together, interleaved arrivals, generous budget: blocks of different observations overlap
    srv, host = _make_server(dev, list(enumerate(specs)), 8 << 30, blocks)
    sched = [(0.002 * k + 0.0005 * oid, oid, k) for oid in range(len(specs)) for k in range(nblk)]
    mixed = _serve(srv, host, sched)
    for oid in alone:
        assert len(mixed[oid]) == nblk
        for k in range(nblk):
            a, m = alone[oid][k], mixed[oid][k]
            assert np.array_equal(a, m), (oid, k)
    # a budget that admits only one block at a time (plans + the largest block) still serves all
    from paper_1105_0661_gb300 import Plan
    need = 0
    plans = 0
    for wl, prec in specs:
        p = Plan.from_workload(wl, precision=prec, external_workspace=True)
        need = max(need, p.dims.in_bytes + p.dims.out_bytes + p.dims.workspace_bytes)
        plans += p.device_bytes()
        p.close()
    srv, host = _make_server(dev, list(enumerate(specs)), plans + need, blocks)
    tight = _serve(srv, host, sched)
    for oid in alone:
        for k in range(nblk):
            assert np.array_equal(alone[oid][k], tight[oid][k]), (oid, k)
    assert srv.pool.held == 0


@pytest.mark.gpu
def test_served_beams_match_the_oracle():
    from paper_1105_0661_gb300 import build_lib
    build_lib.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    wl, prec = _obs_specs()[0]
    blocks = {0: [G.make_block(wl, seed=5, block_index=k) for k in range(2)]}
    srv, host = _make_server(dev, [(0, (wl, prec))], 8 << 30, blocks)
    outs = _serve(srv, host, [(0.0, 0, 0), (0.001, 0, 1)])[0]
    ob = O.observation_from_workload(wl)
    for k in range(2):
        ref = ob.run_block(blocks[0][k])
        got = outs[k].reshape(ref.shape).astype(np.float64)
        assert (np.abs(got - ref) / ref).max() <= 1e-5


def test_schedule_and_latency_summary():
    from paper_1105_0661_gb300.serve import BlockResult, latency_summary, poisson_schedule
    rng = np.random.default_rng(0)
    sch = poisson_schedule(3, 5, 1.0, rng)
    assert len(sch) == 15
    for off, oid, k in sch:
        assert off >= k * 1.0          # jitter only delays a block
    res = [BlockResult(0, k, 0.0, 0.0, 0.1 * (k + 1)) for k in range(10)]
    s = latency_summary(res, 1.0)
    assert s["blocks"] == 10 and s["late_blocks"] == 0
    assert abs(s["p50_s"] - 0.55) < 1e-9 and s["max_s"] == pytest.approx(1.0)
