"""Parity at the workloads' full sizes, in the launch configuration bench.py times.

* the tiny observation (8 stations, 1 subband at 150 MHz, 65536 samples, 4 beams, Stokes I over 4
  spectra): every output element against the oracle;
* the LOFAR-scale observation (48 stations x 244 subbands x 196608 samples, 127 beams, Stokes I
  over 16): sampled (subband, channel) outputs that the oracle evaluates one by one, plus
  properties that hold at any size.
"""

import numpy as np
import pytest

from oracle import lbf_oracle as O
from synth import generate as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    from paper_1105_0661_gb300 import build_lib
    build_lib.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _check_I(got, ref, tol=1e-5):
    assert np.all(ref > 0)
    err = np.abs(got - ref) / ref
    assert err.max() <= tol, f"max rel err {err.max():.3e}"
    return err.max()


def test_tiny_observation_every_output(dev):
    from paper_1105_0661_gb300 import Plan
    wl = G.workload_tiny(0)
    plan = Plan.from_workload(wl)
    assert plan.dims.bf_kernel == 1            # few-beam kernel for 4 beams
    ob = O.observation_from_workload(wl)
    out = torch.empty(plan.shape("stokes"), dtype=torch.float32, device=dev)
    assert out.shape == (4, 1, 1, 256, 64)     # 4 beams x 256 channels x 64 time bins
    for bi in range(2):
        blk = G.make_block(wl, seed=0, block_index=bi)
        plan.run_block(torch.from_numpy(blk).to(dev), out)
        _check_I(out.cpu().numpy().astype(np.float64), ob.run_block(blk))
    plan.close()


def test_tiny_observation_tone_is_in_beam0(dev):
    """The injected tone (channel 160, beam 0's direction) dominates beam 0 in its channel."""
    from paper_1105_0661_gb300 import Plan
    wl = G.workload_tiny(0)
    plan = Plan.from_workload(wl)
    out = torch.empty(plan.shape("stokes"), dtype=torch.float32, device=dev)
    plan.run_block(torch.from_numpy(G.make_block(wl, seed=0)).to(dev), out)
    p = out[:, 0, 0, :, 8:].mean(dim=-1).cpu().numpy()          # [B, N] after the FIR fill
    assert np.argmax(p[0]) == 160
    assert p[0, 160] > 2.0 * p[1:, 160].max()
    plan.close()


def test_lofar_full_size_sampled(dev):
    from paper_1105_0661_gb300 import Plan
    from synth.device import make_block_device
    wl = G.workload_lofar_fp32(0)
    plan = Plan.from_workload(wl)
    assert plan.dims.bf_kernel == 2            # many-beam kernel for 127 beams
    d_in = make_block_device(wl, seed=0, device=dev)
    out = torch.empty(plan.shape("stokes"), dtype=torch.float32, device=dev)
    plan.run_block(d_in, out)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all()) and bool((out > 0).all())
    ob = O.observation_from_workload(wl)
    chans = [0, 1, 127, 128, 160, 255]
    for f in (0, 121, 243):
        blk_f = d_in[:, f].cpu().numpy()
        ref = ob.run_block_sampled(blk_f, f, chans)                  # [B, 1, nc, M/Q]
        got = out[:, :, f][:, :, chans].double().cpu().numpy()
        _check_I(got, ref)
    plan.close()


@pytest.mark.parametrize("bits", [8, 16])
def test_lofar1024_tensor_core_full_size_sampled(dev, bits):
    """The precision form at full size (48 stations x 244 subbands x 196608 samples, 1024 beams,
    Stokes IQUV over 16, FP16 tensor cores): sampled (subband, channel) outputs against the oracle,
    Stokes I within 1e-3 relative and Q, U, V within 1e-3 of I."""
    from paper_1105_0661_gb300 import Plan
    from synth.device import make_block_device
    wl = G.workload_lofar_tc(bits, 0)
    plan = Plan.from_workload(wl, precision="fp16tc")
    assert plan.dims.bf_kernel == 3
    d_in = make_block_device(wl, seed=0, device=dev)
    out = torch.empty(plan.shape("stokes"), dtype=torch.float32, device=dev)
    plan.run_block(d_in, out)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    ob = O.observation_from_workload(wl)
    chans = [0, 127, 128, 255]
    for f in (0, 243):
        ref = ob.run_block_sampled(d_in[:, f].cpu().numpy(), f, chans)        # [B, 4, nc, M/Q]
        got = out[:, :, f][:, :, chans].double().cpu().numpy()
        I = ref[:, 0]
        assert np.all(I > 0)
        eI = (np.abs(got[:, 0] - I) / I).max()
        eq = (np.abs(got[:, 1:] - ref[:, 1:]) / I[:, None]).max()
        print(f"bits={bits} f={f}: Stokes I max rel err {eI:.2e}, QUV/I {eq:.2e}")
        assert eI <= 1e-3 and eq <= 1e-3
    del out
    plan.close()


def test_pulsar_chain_full_size_sampled(dev):
    """The pulsar pipeline at full size (48 stations x 244 subbands x 196608 samples, 127 beams):
    voltages of the whole block -> channel-level dedispersion (256-point runs) -> Stokes I over 16,
    against the oracle's one-by-one evaluation of sampled (subband, channel) series."""
    from paper_1105_0661_gb300 import Plan
    from synth.device import make_block_device
    wl = G.workload_lofar_fp32(0)
    wl_v = G.Workload(**{**wl.__dict__, "output": "V"})
    pv, ps = Plan.from_workload(wl_v), Plan.from_workload(wl)
    d_in = make_block_device(wl, seed=0, device=dev)
    vol = torch.empty(pv.shape("vol"), dtype=torch.complex64, device=dev)
    pv.run_block(d_in, vol)
    dm = 5e3                                      # large enough to rotate the 3 Hz sub-channels
    pv.dedisperse(dm, 256, vol, vol)
    out = torch.empty(ps.shape("stokes"), dtype=torch.float32, device=dev)
    ps.stokes(vol, out)
    torch.cuda.synchronize()
    del vol
    ob_v = O.observation_from_workload(wl_v)
    chans = [0, 128, 255]
    rate = wl.sample_rate_hz / 256
    for f in (0, 243):
        v = ob_v.run_block_sampled(d_in[:, f].cpu().numpy(), f, chans)          # [B, nc, P, M]
        for i, c in enumerate(chans):
            v[:, i] = O.dedisperse_series(v[:, i], ob_v.f0[f] + ob_v.df[c], rate, dm, 256)
        p = O.stokes_from_voltages(v[:, :, 0], v[:, :, 1], "I")                  # [1, B, nc, M]
        ref = np.moveaxis(O.integrate(p, wl.int_factor), 0, 1)                   # [B, 1, nc, M/Q]
        got = out[:, :, f][:, :, chans].double().cpu().numpy()
        _check_I(got, ref)
    pv.close()
    ps.close()
