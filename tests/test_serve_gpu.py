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


def _make_server(dev, specs, budget, n_chunks=2):
    """A server with each observation split into n_chunks subband chunks."""
    from paper_1105_0661_gb300 import Plan
    from paper_1105_0661_gb300.serve import Server, subband_ranges
    srv = Server(dev, budget, keep_outputs=True)
    for oid, (wl, prec) in specs:
        chunks = [(Plan.from_workload(wl.subset(list(range(f, f + n))), precision=prec, external_workspace=True), f)
                  for f, n in subband_ranges(wl.n_subbands, n_chunks)]
        in_b = sum(p.dims.in_bytes for p, _ in chunks)
        out_b = sum(p.dims.out_bytes for p, _ in chunks)
        srv.add(oid, chunks, wl.n_subbands, torch.empty(in_b, dtype=torch.uint8, pin_memory=True),
                torch.empty(out_b, dtype=torch.uint8, pin_memory=True))
    return srv


def _serve(srv, blocks, schedule):
    """Run the schedule in real time; every block has its own pinned input (loaded with its bytes
    up front) and output, so blocks of one observation may be in flight together."""
    import time
    feeds = {}
    for off, oid, k in schedule:
        h_in = torch.from_numpy(blocks[oid][k].reshape(-1).view(np.uint8)).pin_memory()
        h_out = torch.empty_like(srv.obs[oid].host_out).pin_memory()
        feeds[(oid, k)] = (h_in, h_out)
    pending = sorted(schedule)
    t0 = time.perf_counter()
    while pending or not srv.idle():
        now = time.perf_counter()
        while pending and t0 + pending[0][0] <= now:
            off, oid, k = pending.pop(0)
            h_in, h_out = feeds[(oid, k)]
            srv.arrive(oid, k, t0 + off, h_in, h_out)
        srv.step()
        time.sleep(1e-4)
    out = {}
    for oid, o in srv.obs.items():
        order = sorted(range(len(o.results)), key=lambda i: o.results[i].index)
        out[oid] = [o.outputs[i].view(torch.float32).numpy().copy() for i in order]
    return out


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
        srv = _make_server(dev, [(oid, spec)], 8 << 30, n_chunks=1)     # whole observation, one chunk
        alone[oid] = _serve(srv, blocks, [(0.001 * k, oid, k) for k in range(nblk)])[oid]
    # all together, in chunks, interleaved arrivals (two blocks of an observation may overlap),
    # generous budget: blocks of different observations overlap
    srv = _make_server(dev, list(enumerate(specs)), 8 << 30)
    sched = [(0.002 * k + 0.0005 * oid, oid, k) for oid in range(len(specs)) for k in range(nblk)]
    mixed = _serve(srv, blocks, sched)
    for oid in alone:
        assert len(mixed[oid]) == nblk
        for k in range(nblk):
            a, m = alone[oid][k], mixed[oid][k]
            assert np.array_equal(a, m), (oid, k)
    # a budget that admits only the largest block at a time still serves everything, in order
    reserved, need = srv.pool.reserved, max(srv.block_bytes(oid) for oid in srv.obs)
    srv = _make_server(dev, list(enumerate(specs)), reserved + need)
    tight = _serve(srv, blocks, sched)
    for oid in alone:
        for k in range(nblk):
            assert np.array_equal(alone[oid][k], tight[oid][k]), (oid, k)
    assert srv.pool.held == 0


@pytest.mark.gpu
@pytest.mark.parametrize("which,tol", [(0, 1e-5), (1, 1e-3)])
def test_served_beams_match_the_oracle(which, tol):
    """Served in three subband chunks with two blocks in flight: an FP32 observation (Stokes I,
    per element within 1e-5) and a tensor-core one (IQUV, within 1e-3 of I) against the oracle."""
    from paper_1105_0661_gb300 import build_lib
    build_lib.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    wl, prec = _obs_specs()[which]
    wl = wl.subset([0, 1, 0])              # three subbands (the first repeated): three chunks
    blocks = {0: [G.make_block(wl, seed=5, block_index=k) for k in range(3)]}
    srv = _make_server(dev, [(0, (wl, prec))], 8 << 30, n_chunks=3)
    outs = _serve(srv, blocks, [(0.0, 0, 0), (0.0005, 0, 1), (0.001, 0, 2)])[0]
    ob = O.observation_from_workload(wl)
    for k in range(3):
        ref = ob.run_block(blocks[0][k])
        got = outs[k].reshape(ref.shape).astype(np.float64)
        I = ref[:, 0]
        assert (np.abs(got[:, 0] - I) / I).max() <= tol, k
        if ref.shape[1] == 4:
            assert (np.abs(got[:, 1:] - ref[:, 1:]) / I[:, None]).max() <= tol, k


def test_subband_ranges_cover_the_observation():
    from paper_1105_0661_gb300.serve import subband_ranges
    for F, k in [(1, 4), (3, 3), (244, 4), (61, 4), (7, 2)]:
        r = subband_ranges(F, k)
        assert r[0][0] == 0 and sum(n for _, n in r) == F and all(n > 0 for _, n in r)
        assert all(r[i][0] + r[i][1] == r[i + 1][0] for i in range(len(r) - 1))


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
