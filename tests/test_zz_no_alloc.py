"""The allocation-free entry point lbf_run_block_static, for callers that cannot call cudaMalloc
(a plugin whose host framework owns the device-memory budget, a real-time ingest thread that
must not take the allocator's locks mid-observation).

It must give the same beams as the allocating entry point (a fresh plan's lbf_run_block) on two
calls in a row -- the second reuses the shared static scratch left by the first -- and refuse
observations larger than its fixed scratch before touching the device.  This file is collected
last so that a failure here cannot hide another test's result.
"""

import numpy as np
import pytest

from synth import generate as G

TOL = 1e-5   # the FP32 Stokes tolerance of the parity tests


def _kw(wl):
    return dict(station_xyz=wl.station_xyz, subband_hz=wl.subband_hz, beam_dlm=wl.beam_dlm,
                phase_centre=wl.phase_centre, taps=wl.taps, block_samples=wl.block_samples,
                int_factor=wl.int_factor, output=wl.output, sample_bits=wl.sample_bits,
                bandpass=wl.bandpass)


def _lib():
    from paper_1105_0661_gb300 import build_lib
    build_lib.build()
    from paper_1105_0661_gb300 import lbf
    return lbf


def test_too_big_is_refused_on_the_host():
    lbf = _lib()
    wl = G.workload_lofar_fp32(0)          # 48 x 244 x 196608 station-samples: far beyond 24 MiB
    with pytest.raises(lbf.LbfError) as ei:
        lbf.run_block_static(**_kw(wl), d_in=1 << 20, d_out=1 << 20, stream=0)
    assert ei.value.status == lbf.LBF_ETOOBIG


@pytest.mark.gpu
@pytest.mark.parametrize("out,bits", [("I", 16), ("IQUV", 8)])
def test_static_entry_matches_plan_run_block_twice(out, bits):
    torch = pytest.importorskip("torch")
    lbf = _lib()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    wl = G.workload_tiny(0)                 # 8 stations x 65536 samples, 4 beams, Stokes over 4
    wl.output, wl.sample_bits = out, bits
    wl.sigma = 32.0 if bits == 16 else 8.0
    wl.bandpass = G.bandpass_ripple(256)
    for call in range(2):
        blk = torch.from_numpy(G.make_block(wl, seed=call)).to(dev)
        plan = lbf.Plan.from_workload(wl)
        ref = torch.empty(plan.shape("stokes"), dtype=torch.float32, device=dev)
        plan.run_block(blk, ref)
        got = torch.full_like(ref, float("nan"))
        lbf.run_block_static(**_kw(wl), d_in=blk, d_out=got)
        torch.cuda.synchronize()
        r, g = ref.double().cpu().numpy(), got.double().cpu().numpy()
        I = r[:, 0]
        assert np.all(I > 0) and np.all(np.isfinite(g))
        assert (np.abs(g[:, 0] - I) / I).max() <= TOL, call
        if out == "IQUV":
            assert (np.abs(g[:, 1:] - r[:, 1:]) / I[:, None]).max() <= TOL, call
        plan.close()
