"""The allocation-free entry point lbf_run_block_static, for callers that cannot call cudaMalloc
(a plugin whose host framework owns the device-memory budget, a real-time ingest thread that
must not take the allocator's locks mid-observation).

It must give the same beams as the allocating entry point (a fresh plan's lbf_run_block) on two
calls in a row -- the second reuses the shared static scratch left by the first -- and the same
beams as the FP64 oracle; it must refuse observations larger than its fixed scratch before
touching the device, and the binding must refuse buffers too short for the block.  This file is
collected last so that a failure here cannot hide another test's result.
"""

import numpy as np
import pytest

from oracle import lbf_oracle as O
from synth import generate as G

TOL = 1e-5   # the FP32 tolerance of the parity tests (Stokes per element, voltages relative RMS)


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


def _status(lbf, **kw):
    """Status of a call with integer stand-ins for the device buffers (no device is touched: the
    size limits are checked first, and a CPU-only host then fails the device-pointer check)."""
    try:
        lbf.run_block_static(d_in=1 << 20, d_out=1 << 20, stream=0, **kw)
        return lbf.LBF_OK
    except lbf.LbfError as e:
        return e.status


def _one_station(F, T, B=1):
    return dict(station_xyz=np.zeros((1, 3)), subband_hz=G.subband_centres(F, 120e6),
                beam_dlm=np.zeros((B, 2)), phase_centre=(0.3, 0.4), taps=G.kaiser_sinc_taps(16, 256),
                block_samples=T, int_factor=1, output="I", sample_bits=16)


def test_too_big_is_refused_on_the_host():
    lbf = _lib()
    wl = G.workload_lofar_fp32(0)          # 48 x 244 x 196608 station-samples: far beyond 24 MiB
    assert _status(lbf, **_kw(wl)) == lbf.LBF_ETOOBIG


def test_each_scratch_limit_is_exact():
    """Each of the three limits, one step over (LBF_ETOOBIG) and at or just under it (accepted by
    the size checks; without a GPU the call then fails the device-pointer check, LBF_EINVAL)."""
    lbf = _lib()
    wl = G.workload_tiny(0)
    wl.subband_hz = G.subband_centres(3, 150e6)
    # corner-turned block: S*F*T*16 bytes <= 24 MiB, i.e. S*F*T <= 1572864 station-samples
    wl.block_samples = 65536                 # 8 x 3 x 65536 = 1572864 exactly
    assert _status(lbf, **_kw(wl)) == lbf.LBF_EINVAL
    wl.block_samples = 65536 + 4 * 256       # the next block size with M a multiple of Q = 4
    assert _status(lbf, **_kw(wl)) == lbf.LBF_ETOOBIG
    # history: S*F*H*8 bytes <= 4 MiB with H = 15*256 + d_max = 3840 for one station
    assert _status(lbf, **_one_station(136, 256)) == lbf.LBF_EINVAL      # 4177920 bytes
    assert _status(lbf, **_one_station(137, 256)) == lbf.LBF_ETOOBIG     # 4208640 bytes
    # weight tables: 16 bytes per (beam, station) plus the fixed tables, <= 4 MiB
    assert _status(lbf, **_one_station(1, 256, B=200000)) == lbf.LBF_EINVAL
    assert _status(lbf, **_one_station(1, 256, B=300000)) == lbf.LBF_ETOOBIG


def test_short_buffers_are_refused_before_the_call():
    """The C entry point cannot measure raw device pointers, so the binding checks the tensors'
    sizes against the block's input and output sizes and raises before calling the library."""
    torch = pytest.importorskip("torch")
    lbf = _lib()
    wl = G.workload_tiny(0)
    S, F, T, B = wl.n_stations, wl.n_subbands, wl.block_samples, wl.n_beams
    in_bytes = S * F * T * 8
    out_bytes = B * F * 256 * (T // 256 // wl.int_factor) * 4
    good_in = torch.empty(in_bytes, dtype=torch.uint8)
    good_out = torch.empty(out_bytes, dtype=torch.uint8)
    with pytest.raises(ValueError):
        lbf.run_block_static(**_kw(wl), d_in=good_in[:-1], d_out=good_out, stream=0)
    with pytest.raises(ValueError):
        lbf.run_block_static(**_kw(wl), d_in=good_in, d_out=good_out[:-4], stream=0)
    wl.output = "V"
    with pytest.raises(ValueError):   # voltages need B x F x T x 2 pols x 8 bytes
        lbf.run_block_static(**_kw(wl), d_in=good_in, d_out=good_out, stream=0)


def _compare(lbf, torch, wl, blk, dev, variant):
    """One static call against a fresh plan's run_block and against the oracle."""
    plan = lbf.Plan.from_workload(wl, bf_variant=variant)
    stokes = wl.output != "V"
    shape, dt = (plan.shape("stokes"), torch.float32) if stokes else (plan.shape("vol"), torch.complex64)
    d_in = torch.from_numpy(blk).to(dev)
    ref = torch.empty(shape, dtype=dt, device=dev)
    plan.run_block(d_in, ref)
    got = torch.full_like(ref, float("nan"))
    lbf.run_block_static(**_kw(wl), d_in=d_in, d_out=got, bf_variant=variant)
    torch.cuda.synchronize()
    r = ref.cpu().numpy().astype(np.complex128 if not stokes else np.float64)
    g = got.cpu().numpy().astype(np.complex128 if not stokes else np.float64)
    o = O.observation_from_workload(wl).run_block(blk)
    plan.close()
    assert np.all(np.isfinite(g))
    if stokes:
        I = r[:, 0]
        assert np.all(I > 0)
        errs = [(np.abs(g[:, 0] - I) / I).max(), (np.abs(g[:, 0] - o[:, 0]) / o[:, 0]).max()]
        if wl.output == "IQUV":
            errs += [(np.abs(g[:, 1:] - r[:, 1:]) / I[:, None]).max(),
                     (np.abs(g[:, 1:] - o[:, 1:]) / o[:, :1]).max()]
        return max(errs)
    def rel_rms(a, b):
        num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=(2, 3, 4)))
        return (num / np.sqrt(np.sum(np.abs(b) ** 2, axis=(2, 3, 4)))).max()
    return max(rel_rms(g, r), rel_rms(g, o))


@pytest.mark.gpu
@pytest.mark.parametrize("out,bits,variant", [("I", 16, "auto"), ("IQUV", 8, "auto"), ("I", 16, "many"),
                                              ("V", 16, "auto"), ("V", 8, "many")])
def test_static_entry_matches_plan_run_block_twice(out, bits, variant):
    torch = pytest.importorskip("torch")
    lbf = _lib()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    wl = G.workload_tiny(0)                 # 8 stations x 65536 samples, 4 beams, Stokes over 4
    wl.output, wl.sample_bits = out, bits
    wl.sigma = 32.0 if bits == 16 else 8.0
    wl.bandpass = G.bandpass_ripple(256)
    if out == "V":
        wl.block_samples = 64 * 256         # voltages of 64 spectra: a small oracle case
    for call in range(2):
        blk = G.make_block(wl, seed=call)
        err = _compare(lbf, torch, wl, blk, dev, variant)
        print(f"static {out} i{bits} {variant} call {call}: max error vs run_block and oracle {err:.2e}")
        assert err <= TOL, call


@pytest.mark.gpu
def test_static_entry_at_the_corner_turn_limit():
    """8 stations x 3 subbands x 65536 samples fill the 24 MiB corner-turned scratch exactly."""
    torch = pytest.importorskip("torch")
    lbf = _lib()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    wl = G.workload_tiny(0)
    wl.subband_hz = G.subband_centres(3, 150e6)
    assert wl.n_stations * wl.n_subbands * wl.block_samples * 16 == 24 << 20
    err = _compare(lbf, torch, wl, G.make_block(wl, seed=5), dev, "auto")
    print(f"static at the scratch limit: max error {err:.2e}")
    assert err <= TOL
