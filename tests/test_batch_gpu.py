"""Batches: one persistent grouped launch per stage for a block of every plan gives exactly the
beams each plan gives alone (same item bodies), over consecutive blocks; the same holds when the
batch block is replayed as a CUDA graph and after autotuning."""

import numpy as np
import pytest

from synth import generate as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 256


def _specs():
    rng = np.random.default_rng(31)
    out = []
    for i, (S, F, B, outk, bits, T) in enumerate([(12, 3, 1, "I", 16, 40 * N), (20, 2, 17, "IQUV", 8, 64 * N),
                                                  (33, 1, 130, "I", 16, 48 * N), (8, 4, 6, "V", 16, 32 * N),
                                                  (64, 1, 40, "IQUV", 8, 64 * N),
                                                  # odd M: the FP32 corner turn without tensor stores
                                                  (10, 2, 3, "V", 16, 41 * N)]):
        xyz = G.lofar_positions(rng, S // 2, S - S // 2)
        wl = G.Workload(f"b{i}", xyz, G.subband_centres(F, 130e6 + 5e6 * i), G.hex_beam_grid(B, 0.05), (0.3, 0.4),
                        T, 4 if outk != "V" else 1, outk, sample_bits=bits, sigma=32.0 if bits == 16 else 8.0,
                        source="tone")
        out.append(wl)
    return out


def _out(plan, dev):
    return torch.empty(plan.dims.out_bytes // 4, dtype=torch.float32, device=dev)


def test_batch_equals_separate_runs():
    from paper_1105_0661_gb300 import Batch, Plan, build_lib
    build_lib.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    wls = _specs()
    solo = [Plan.from_workload(wl) for wl in wls]
    grouped = [Plan.from_workload(wl) for wl in wls]
    batch = Batch(grouped)
    nblk = 6
    blocks = [[torch.from_numpy(G.make_block(wl, seed=i, block_index=k)).to(dev) for k in range(nblk)]
              for i, wl in enumerate(wls)]
    so = [_out(p, dev) for p in solo]
    bo = [_out(p, dev) for p in grouped]
    d_in = [torch.empty_like(blocks[i][0]) for i in range(len(wls))]
    for k in range(nblk):
        for i, p in enumerate(solo):
            p.run_block(blocks[i][k], so[i])
        for i in range(len(wls)):
            d_in[i].copy_(blocks[i][k])
        if k < 2:
            batch.run(d_in, bo)                   # grouped launches
        else:
            if k == 2:
                batch.capture(d_in, bo)           # then graph replays with fixed buffers
            batch.launch()
        torch.cuda.synchronize()
        for i in range(len(wls)):
            assert torch.equal(so[i], bo[i]), (k, i)
    # autotune restarts every stream: compare with fresh plans from the first block on
    info = batch.tune(d_in, bo, reps=2)
    assert info["best_spc"] in (0, 64, 256, 1024) and len(info["candidates"]) in (4, 7, 10)
    assert info["best_mid_variant"] in {c["mid_variant"] for c in info["candidates"]}
    fresh = [Plan.from_workload(wl) for wl in wls]
    fo = [_out(p, dev) for p in fresh]
    for k in range(2):
        for i in range(len(wls)):
            fresh[i].run_block(blocks[i][k], fo[i])
            d_in[i].copy_(blocks[i][k])
        batch.run(d_in, bo)
        torch.cuda.synchronize()
        for i in range(len(wls)):
            r, g = fo[i].double().cpu().numpy(), bo[i].double().cpu().numpy()
            scale = np.abs(r).max()
            assert np.max(np.abs(g - r)) <= 1e-5 * scale, (k, i)
    batch.close()


def test_batch_with_tensor_core_plans_equals_separate_runs():
    """Tensor-core plans (Stokes I, IQUV with the incoherent beam, voltages) and FP32 plans in one
    batch: grouped filter bank writing the FP16 planes, then one persistent tensor-core launch per
    class of output kind and integration length (here the two IQUV plans, of 20 and 64 stations,
    share one, the second in the two-product form); every output equals the same plan run alone,
    block after block, also as graph replays."""
    from paper_1105_0661_gb300 import Batch, Plan, build_lib
    build_lib.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    wls = _specs()
    kinds = [dict(), dict(precision="fp16tc"), dict(precision="fp16tc", incoherent_beam=True),
             dict(precision="fp16tc"), dict(precision="fp16tc2"), dict()]
    assert len(kinds) == len(wls)
    solo = [Plan.from_workload(wl, **kw) for wl, kw in zip(wls, kinds)]
    grouped = [Plan.from_workload(wl, **kw) for wl, kw in zip(wls, kinds)]
    batch = Batch(grouped)
    nblk = 4
    blocks = [[torch.from_numpy(G.make_block(wl, seed=40 + i, block_index=k)).to(dev) for k in range(nblk)]
              for i, wl in enumerate(wls)]
    so = [_out(p, dev) for p in solo]
    bo = [_out(p, dev) for p in grouped]
    d_in = [torch.empty_like(blocks[i][0]) for i in range(len(wls))]
    for k in range(nblk):
        for i, p in enumerate(solo):
            p.run_block(blocks[i][k], so[i])
        for i in range(len(wls)):
            d_in[i].copy_(blocks[i][k])
        if k < 2:
            batch.run(d_in, bo)
        else:
            if k == 2:
                batch.capture(d_in, bo)
            batch.launch()
        torch.cuda.synchronize()
        for i in range(len(wls)):
            assert torch.equal(so[i], bo[i]), (k, i)
    for p in grouped:
        assert p.device_status() == 0
    batch.close()


def test_batch_of_sixteen_uneven_observations_matches_the_oracle():
    """The batched workload's 16 sub-observations (stations 12-64, subbands 8-244, beams 1-512,
    int8 or int16, drawn from default_rng(1..16)), scaled down to 16 spectra per block: tuned,
    captured as CUDA graphs and replayed, then every observation's first block is compared with
    the FP64 oracle on sampled subbands and channels -- FP32 plans per element within 1e-5 on
    Stokes I, tensor-core plans (64 beams or more) within 1e-3."""
    from oracle import lbf_oracle as O
    from paper_1105_0661_gb300 import Batch, Plan, build_lib
    from synth.device import make_block_device
    build_lib.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    wls = G.batch_workloads(16, 16 * N)
    prec = ["fp16tc" if (wl.n_beams >= 64 and wl.n_stations <= 64) else "fp32" for wl in wls]
    plans = [Plan.from_workload(wl, precision=pr) for wl, pr in zip(wls, prec)]
    kinds = {p.dims.bf_kernel for p in plans}
    assert {1, 3} <= kinds                     # the few-beam FP32 kernel and the tensor cores
    d_in = [make_block_device(wl, seed=i + 1, device=dev) for i, wl in enumerate(wls)]
    d_out = [_out(p, dev) for p in plans]
    batch = Batch(plans)
    channels = [0, 1, 31, 127, 128, 160, 254, 255]
    worst = {"fp32": 0.0, "fp16tc": 0.0}
    refs = {}

    def check(label):
        for i, (wl, p, pr) in enumerate(zip(wls, plans, prec)):
            assert p.device_status() == 0
            ob = O.observation_from_workload(wl)
            got = d_out[i].view(p.shape("stokes"))                      # [B][1][F][N][M/Q]
            for f in sorted({0, wl.n_subbands - 1}):
                if (i, f) not in refs:
                    blk_f = d_in[i][:, f].cpu().numpy()                 # [S][T][P][2]
                    refs[(i, f)] = ob.run_block_sampled(blk_f, f, channels)   # [B][1][nc][M/Q]
                ref = refs[(i, f)]
                g = got[:, :, f][:, :, channels].double().cpu().numpy()
                I = ref[:, 0]
                assert np.all(I > 0)
                err = float((np.abs(g[:, 0] - I) / I).max())
                worst[pr] = max(worst[pr], err)
                assert err <= (1e-5 if pr == "fp32" else 1e-3), (label, wl.name, pr, f, err)

    # grouped persistent launches (the default), replayed as a graph: block 0 of every stream
    batch.capture(d_in, d_out)
    assert batch.launches() < 16               # grouped: far fewer than 3 launches per observation
    batch.launch()
    torch.cuda.synchronize()
    check("grouped")
    # the tuned tile shapes and launch mode (tuning restarts every stream), again as a graph
    batch.tune(d_in, d_out, reps=1)
    batch.capture(d_in, d_out)
    batch.launch()
    torch.cuda.synchronize()
    check("tuned")
    print(f"batch of 16 vs oracle: max Stokes I rel err FP32 {worst['fp32']:.2e}, tensor cores {worst['fp16tc']:.2e}")
    batch.close()


def test_batch_larger_than_one_launch_table():
    """70 small observations of one class (int16, FP32, Stokes I, few-beam): a grouped launch
    holds at most 64 observations, so the class runs as two launches each numbering its own work
    items; every output equals the same plan run alone, over two blocks."""
    from paper_1105_0661_gb300 import Batch, Plan, build_lib
    build_lib.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(7)
    wls = []
    for i in range(70):
        S, F, B = 2 + i % 5, 1 + i % 3, 1 + i % 4
        xyz = G.lofar_positions(rng, S // 2, S - S // 2)
        wls.append(G.Workload(f"m{i}", xyz, G.subband_centres(F, 120e6 + 1e6 * i), G.hex_beam_grid(B, 0.05),
                              (0.3, 0.4), 32 * N, 4, "I", sample_bits=16, sigma=32.0, source="tone"))
    solo = [Plan.from_workload(wl) for wl in wls]
    grouped = [Plan.from_workload(wl) for wl in wls]
    assert {p.dims.bf_kernel for p in grouped} == {1}
    batch = Batch(grouped)
    d_in = [torch.empty((wl.n_stations, wl.n_subbands, wl.block_samples, 2, 2), dtype=torch.int16, device=dev)
            for wl in wls]
    so = [_out(p, dev) for p in solo]
    bo = [_out(p, dev) for p in grouped]
    for k in range(2):
        for i, wl in enumerate(wls):
            d_in[i].copy_(torch.from_numpy(G.make_block(wl, seed=i, block_index=k)))
            solo[i].run_block(d_in[i], so[i])
        batch.run(d_in, bo)
        torch.cuda.synchronize()
        for i in range(len(wls)):
            assert torch.equal(so[i], bo[i]), (k, i)
    assert batch.launches() < 70
    batch.close()
