"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle on the same seeded inputs.

Tolerances (FP32 path):
  * corner turn / transposes: exact;
  * integer shift decisions: exact;
  * filter-bank output, delay-compensated channels and beam voltages: relative RMS error
    ||got - ref|| / ||ref|| <= 1e-5 per (subband, station) or (beam, subband);
  * Stokes I: |got - ref| <= 1e-5 * ref per element (I > 0);
  * Stokes Q, U, V (they cross zero): |got - ref| <= 1e-5 * I_ref per element.
"""

import numpy as np
import pytest

from oracle import lbf_oracle as O
from synth import generate as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 256
TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    from paper_1105_0661_gb300 import build_lib
    build_lib.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _plan(wl, **over):
    from paper_1105_0661_gb300 import Plan
    return Plan.from_workload(wl, **over)


def _wl(S=8, F=2, T=40 * N, B=5, Q=4, out="I", bits=16, seed=0, long_baselines=True, bp=True):
    """A small observation that spans several CTA tiles with a ragged tail (M = 40 spectra)."""
    rng = np.random.default_rng(seed)
    xyz = G.lofar_positions(rng, S // 2, S - S // 2) if long_baselines else G.disc_positions(rng, S, 1000.0)
    wl = G.Workload("parity", xyz, G.subband_centres(F, 120e6), G.hex_beam_grid(B, 0.05), (0.3, 0.4), T, Q, out,
                    sample_bits=bits, sigma=32.0 if bits == 16 else 8.0, source="tone")
    if bp:
        wl.bandpass = G.bandpass_ripple(N)
    return wl


def _rel_rms(got, ref, axes):
    num = np.sqrt(np.sum(np.abs(got - ref) ** 2, axis=axes))
    den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=axes))
    return num / den


def _to_dev(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def _check_stokes(got, ref, tol=TOL):
    """got/ref [B][nS][F][N][Mq]."""
    I = ref[:, 0]
    assert np.all(I > 0)
    eI = np.abs(got[:, 0] - I) / I
    assert eI.max() <= tol, f"Stokes I max rel err {eI.max():.3e}"
    if ref.shape[1] == 4:
        eq = np.abs(got[:, 1:] - ref[:, 1:]) / I[:, None]
        assert eq.max() <= tol, f"Stokes QUV max err/I {eq.max():.3e}"


# ----------------------------------------------------------------------------- geometry
def test_integer_shifts_match_oracle(dev):
    for wl in (G.workload_tiny(0), G.workload_lofar_fp32(0), _wl(S=12, seed=3)):
        p = _plan(wl.subset([0]) if wl.n_subbands > 1 else wl, block_samples=N, int_factor=1)
        n, d = p.shifts()
        ob = O.observation_from_workload(wl)
        assert np.array_equal(n, ob.n_shift) and np.array_equal(d, ob.d_shift)
        assert p.dims.d_max == ob.d_max and p.dims.history_samples == ob.H
        p.close()


# ----------------------------------------------------------------------------- a1-a3 filter bank
@pytest.mark.parametrize("bits", [16, 8])
def test_ppf_matches_oracle_over_two_blocks(dev, bits):
    wl = _wl(bits=bits)
    p = _plan(wl)
    ob = O.observation_from_workload(wl)
    assert ob.d_max > 3
    chan = torch.empty(p.shape("chan"), dtype=torch.complex64, device=dev)
    for bi in range(2):
        blk = G.make_block(wl, seed=1, block_index=bi)
        p.ppf(_to_dev(blk, dev), chan)
        ref = ob.ppf(blk)
        got = chan.cpu().numpy().astype(np.complex128)
        err = _rel_rms(got, ref, (2, 3, 4))
        assert err.max() <= TOL, (bi, err.max())
    p.close()


def test_ppf_streaming_equals_one_long_block(dev):
    """Three blocks with device-resident history equal one block three times as long."""
    wl = _wl(T=16 * N, F=1)
    wl3 = _wl(T=48 * N, F=1)
    p1, p3 = _plan(wl), _plan(wl3)
    big = G.make_block(wl3, seed=2)
    c3 = torch.empty(p3.shape("chan"), dtype=torch.complex64, device=dev)
    p3.ppf(_to_dev(big, dev), c3)
    c1 = torch.empty(p1.shape("chan"), dtype=torch.complex64, device=dev)
    parts = []
    for i in range(3):
        p1.ppf(_to_dev(big[:, :, i * 16 * N:(i + 1) * 16 * N], dev), c1)
        parts.append(c1.cpu().numpy())
    assert np.array_equal(np.concatenate(parts, axis=3), c3.cpu().numpy())
    p1.close(); p3.close()


def test_reset_state_restarts_the_stream(dev):
    wl = _wl(F=1, T=16 * N)
    p = _plan(wl)
    blk = _to_dev(G.make_block(wl, seed=4), dev)
    chan = torch.empty(p.shape("chan"), dtype=torch.complex64, device=dev)
    p.ppf(blk, chan)
    first = chan.clone()
    p.ppf(blk, chan)
    assert not torch.equal(first, chan)
    p.reset_state()
    p.ppf(blk, chan)
    assert torch.equal(first, chan)
    p.close()


# ----------------------------------------------------------------------------- a4 delay + corner turn
def test_delay_correct_matches_oracle(dev):
    wl = _wl()
    p = _plan(wl)
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(5)
    shp = p.shape("chan")
    chan = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    ct = torch.empty(p.shape("ct"), dtype=torch.complex64, device=dev)
    p.delay_correct(_to_dev(chan, dev), ct)
    ref = ob.delay_correct(chan.astype(np.complex128))
    got = ct.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
    p.close()


def test_corner_turn_is_exact_transpose(dev):
    """With no delays (phase centre at zenith, stations in the ground plane) and a unit bandpass,
    delay_correct is a pure transpose [F][S][P][M][N] -> [F][N][S][P][M]: exact."""
    wl = _wl(bp=False)
    wl.phase_centre = (0.0, 0.0)
    p = _plan(wl)
    rng = np.random.default_rng(6)
    shp = p.shape("chan")
    chan = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    ct = torch.empty(p.shape("ct"), dtype=torch.complex64, device=dev)
    p.delay_correct(_to_dev(chan, dev), ct)
    assert np.array_equal(ct.cpu().numpy(), np.ascontiguousarray(np.transpose(chan, (0, 4, 1, 2, 3))))
    p.close()


# ----------------------------------------------------------------------------- a5-a6 beam former
@pytest.mark.parametrize("variant,B", [("few", 5), ("many", 5), ("many", 133), ("few", 19), ("many64", 5),
                                       ("many64", 64), ("many64", 133), ("few", 12), ("few", 28), ("few", 44)])
def test_beamform_voltages_match_oracle(dev, variant, B):
    wl = _wl(B=B, out="V")
    p = _plan(wl, bf_variant=variant)
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(7)
    shp = p.shape("ct")
    ct = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    vol = torch.empty(p.shape("vol"), dtype=torch.complex64, device=dev)
    p.beamform(_to_dev(ct, dev), vol)
    ref = ob.beamform(ct.astype(np.complex128))
    err = _rel_rms(vol.cpu().numpy().astype(np.complex128), ref, (2, 3, 4))
    assert err.max() <= TOL, err.max()
    p.close()


@pytest.mark.parametrize("B,kernel", [(8, 1), (32, 1), (33, 4), (64, 4), (65, 2), (127, 2), (154, 4), (200, 2),
                                      (269, 4), (472, 2)])
def test_automatic_beam_former_choice(dev, B, kernel):
    """AUTO: the few-beam kernel up to 32 beams, then the many-beam tile (128 beams: kernel 2, 64
    beams: kernel 4) that leaves the fewest tile slots empty (a 64-beam slot weighed 1.15)."""
    wl = _wl(B=B, F=1, T=16 * N)
    p = _plan(wl)
    assert p.dims.bf_kernel == kernel
    p.close()


# ----------------------------------------------------------------------------- a7 Stokes
# M a multiple of 4 takes the four-spectra-per-lane kernel (ragged last unit group at M = 100,
# several lane passes at M = 160); M = 66 and 70 take the one-spectrum-per-lane kernel.
@pytest.mark.parametrize("out,Q,M", [("I", 1, 64), ("I", 8, 64), ("IQUV", 4, 64), ("IQUV", 32, 64), ("I", 2, 64),
                                     ("I", 4, 100), ("IQUV", 16, 160), ("I", 32, 160),
                                     ("I", 2, 66), ("IQUV", 1, 70)])
def test_stokes_matches_oracle(dev, out, Q, M):
    wl = _wl(T=M * N, out=out, Q=Q, B=3)
    p = _plan(wl)
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(8)
    shp = p.shape("vol")
    vol = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    p.stokes(_to_dev(vol, dev), o)
    _check_stokes(o.cpu().numpy().astype(np.float64), ob.stokes(vol.astype(np.complex128)))
    p.close()


@pytest.mark.parametrize("variant", ["few", "many", "many64"])
@pytest.mark.parametrize("out,Q", [("I", 4), ("IQUV", 16), ("I", 1), ("IQUV", 2), ("I", 32), ("IQUV", 8)])
def test_beamform_stokes_epilogue_matches_oracle(dev, variant, out, Q):
    wl = _wl(T=64 * N, out=out, Q=Q, B=6)
    p = _plan(wl, bf_variant=variant)
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(9)
    shp = p.shape("ct")
    ct = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    p.beamform_stokes(_to_dev(ct, dev), o)
    _check_stokes(o.cpu().numpy().astype(np.float64), ob.stokes(ob.beamform(ct.astype(np.complex128))))
    p.close()


# ----------------------------------------------------------------------------- a1-a7 fused
@pytest.mark.parametrize("variant", ["few", "many", "many64"])
@pytest.mark.parametrize("out,bits", [("I", 16), ("IQUV", 16), ("V", 16), ("I", 8)])
def test_run_block_matches_oracle(dev, variant, out, bits):
    wl = _wl(out=out, bits=bits, Q=4 if out != "V" else 1)
    p = _plan(wl, bf_variant=variant)
    ob = O.observation_from_workload(wl)
    shape = p.shape("stokes") if out != "V" else p.shape("vol")
    o = torch.empty(shape, dtype=torch.float32 if out != "V" else torch.complex64, device=dev)
    for bi in range(2):
        blk = G.make_block(wl, seed=10, block_index=bi)
        p.run_block(_to_dev(blk, dev), o)
        ref = ob.run_block(blk)
        got = o.cpu().numpy().astype(np.float64 if out != "V" else np.complex128)
        if out == "V":
            assert _rel_rms(got, ref, (2, 3, 4)).max() <= TOL
        else:
            _check_stokes(got, ref)
    p.close()


@pytest.mark.parametrize("B,out", [(12, "I"), (20, "I"), (30, "I"), (12, "IQUV"), (16, "V")])
def test_few_beam_kernel_beam_counts_match_oracle(dev, B, out):
    """The few-beam kernel takes 16 beams per CTA for 9-16 and 25-32 beams of Stokes I and 8
    otherwise: both forms, with a partly filled last beam group, against the oracle over two
    blocks."""
    wl = _wl(B=B, out=out, Q=4 if out != "V" else 1)
    p = _plan(wl, bf_variant="few")
    assert p.dims.bf_kernel == 1
    ob = O.observation_from_workload(wl)
    shape = p.shape("stokes") if out != "V" else p.shape("vol")
    o = torch.empty(shape, dtype=torch.float32 if out != "V" else torch.complex64, device=dev)
    for bi in range(2):
        blk = G.make_block(wl, seed=14, block_index=bi)
        p.run_block(_to_dev(blk, dev), o)
        ref = ob.run_block(blk)
        got = o.cpu().numpy().astype(np.float64 if out != "V" else np.complex128)
        if out == "V":
            assert _rel_rms(got, ref, (2, 3, 4)).max() <= TOL
        else:
            _check_stokes(got, ref)
    p.close()


def test_fused_equals_split_chain(dev):
    """run_block == ppf -> delay_correct -> beamform_stokes bit for bit (same arithmetic), and
    == ppf -> delay_correct -> beamform -> stokes within FP32 rounding."""
    wl = _wl(out="IQUV", Q=4)
    pf, ps = _plan(wl), _plan(wl)
    blk = _to_dev(G.make_block(wl, seed=11), dev)
    o1 = torch.empty(pf.shape("stokes"), dtype=torch.float32, device=dev)
    pf.run_block(blk, o1)
    chan = torch.empty(ps.shape("chan"), dtype=torch.complex64, device=dev)
    ct = torch.empty(ps.shape("ct"), dtype=torch.complex64, device=dev)
    o2 = torch.empty_like(o1)
    ps.ppf(blk, chan)
    ps.delay_correct(chan, ct)
    ps.beamform_stokes(ct, o2)
    assert torch.equal(o1, o2)
    vol = torch.empty(ps.shape("vol"), dtype=torch.complex64, device=dev)
    o3 = torch.empty_like(o1)
    ps.beamform(ct, vol)
    ps.stokes(vol, o3)
    I = o1[:, 0]
    assert ((o3[:, 0] - I).abs() / I).max().item() < 1e-5
    pf.close(); ps.close()


# ----------------------------------------------------------------------------- edge cases
def test_degenerate_single_everything(dev):
    """S = 1, B = 1, one spectrum per block (T = N), Q = 1."""
    wl = _wl(S=1, F=1, T=N, B=1, Q=1, long_baselines=False)
    for variant in ("few", "many", "many64"):
        p = _plan(wl, bf_variant=variant)
        ob = O.observation_from_workload(wl)
        o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
        for bi in range(3):
            blk = G.make_block(wl, seed=12, block_index=bi)
            p.run_block(_to_dev(blk, dev), o)
            ref = ob.run_block(blk)
            _check_stokes(o.cpu().numpy().astype(np.float64), ref)
        p.close()


def test_empty_block_is_a_no_op(dev):
    wl = _wl(T=0, F=1)
    p = _plan(wl)
    assert p.dims.n_spectra == 0 and p.dims.out_bytes == 0
    x = torch.zeros(16, dtype=torch.int16, device=dev)
    o = torch.zeros(4, dtype=torch.float32, device=dev)
    p.run_block(x, o)
    p.ppf(x, o)
    assert torch.count_nonzero(o).item() == 0
    p.close()


def test_host_pointer_rejected(dev):
    from paper_1105_0661_gb300 import LbfError
    wl = _wl(F=1, T=16 * N)
    p = _plan(wl)
    host = torch.zeros(p.shape("in"), dtype=torch.int16)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    with pytest.raises(LbfError) as ei:
        p.run_block(host, o)
    assert ei.value.status == 1
    with pytest.raises(ValueError):
        p.stokes(o, o)   # a Stokes-sized buffer is far too short to be read as voltages
    p.close()


def test_maximum_paper_geometry(dev):
    """64 stations (the paper's maximum, Section 3) x 8 beams x Q 16, int8, many-beam kernel."""
    wl = _wl(S=64, F=1, T=32 * N, B=8, Q=16, bits=8)
    p = _plan(wl, bf_variant="many")
    ob = O.observation_from_workload(wl)
    blk = G.make_block(wl, seed=13)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    p.run_block(_to_dev(blk, dev), o)
    _check_stokes(o.cpu().numpy().astype(np.float64), ob.run_block(blk))
    p.close()


# ----------------------------------------------------------------------------- incoherent beam
# the tensor-core cases also cover windows longer than a thread's 8 spectra (Q = 16, 32) and a
# last group of 8 spectra that runs past M (M = 36)
@pytest.mark.parametrize("variant,prec,bits,out,tol,M,Q", [
    ("few", "fp32", 16, "IQUV", TOL, 64, 4), ("many", "fp32", 8, "I", TOL, 64, 4),
    ("many64", "fp32", 16, "IQUV", TOL, 64, 4),
    ("auto", "fp16tc", 16, "IQUV", 1e-3, 64, 4), ("auto", "fp16tc", 8, "I", 1e-3, 64, 4),
    ("auto", "fp16tc", 16, "I", 1e-3, 96, 32), ("auto", "fp16tc", 16, "IQUV", 1e-3, 36, 2),
    ("auto", "fp16tc", 8, "I", 1e-3, 80, 16)])
def test_incoherent_beam_matches_oracle(dev, variant, prec, bits, out, tol, M, Q):
    """LBF_FLAG_INCOHERENT_BEAM: beam index B of the Stokes output is the incoherent beam
    (Section 3); the coherent beams are unchanged."""
    wl = _wl(S=16, B=6 if variant == "few" else 70, out=out, bits=bits, Q=Q, T=M * N)
    p = _plan(wl, bf_variant=variant, precision=prec, incoherent_beam=True)
    ob = O.observation_from_workload(wl, incoherent_beam=True)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    assert o.shape[0] == wl.n_beams + 1
    for bi in range(2):
        blk = G.make_block(wl, seed=20, block_index=bi)
        p.run_block(_to_dev(blk, dev), o)
        _check_stokes(o.cpu().numpy().astype(np.float64), ob.run_block(blk), tol)
    p.close()


# ----------------------------------------------------------------------------- superstation beam former
@pytest.mark.parametrize("M", [40, 41])   # even M: two spectra per thread; odd M: one
def test_superstation_matches_oracle(dev, M):
    wl = _wl(S=12, F=2, T=M * N) if M % 4 == 0 else _wl(S=12, F=2, T=M * N, out="V", Q=1)
    p = _plan(wl)
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(40)
    shp = p.shape("ct")
    ct = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    d_ct = _to_dev(ct, dev)
    for groups in (np.array([0, 0, 1, 1, 1, 2, 0, 2, 1, 0, 2, 2]), np.zeros(12, dtype=int), np.arange(12)):
        G_ = int(groups.max()) + 1
        ss = torch.empty((wl.n_subbands, N, G_, 2, M), dtype=torch.complex64, device=dev)
        p.superstation(groups, d_ct, ss)
        ref = ob.superstation(ct.astype(np.complex128), groups)
        got = ss.cpu().numpy().astype(np.complex128)
        if G_ == 12:
            assert np.array_equal(got, ct.astype(np.complex128))
        else:
            assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref))
    p.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16tc"])
def test_host_buffer_calls_pipeline_in_order(dev, prec):
    """lbf_run_block_host on a stream of blocks enqueued back to back (no synchronisation between
    calls, shared device staging buffers): the upload of block k+1 overlaps block k's kernels, and
    every block still gives exactly the outputs of the device-buffer path, and the oracle's."""
    wl = _wl(S=16, B=70, out="IQUV", Q=4, T=64 * N)
    p_host = _plan(wl, precision=prec)
    p_dev = _plan(wl, precision=prec)
    ob = O.observation_from_workload(wl)
    nblk = 3
    blocks = [G.make_block(wl, seed=30, block_index=k) for k in range(nblk)]
    h_in = [torch.from_numpy(b).pin_memory() for b in blocks]
    h_out = [torch.empty(p_host.shape("stokes"), dtype=torch.float32).pin_memory() for _ in range(nblk)]
    d_in = torch.empty(blocks[0].shape, dtype=torch.int16, device=dev)
    d_out = torch.empty(p_host.shape("stokes"), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    for k in range(nblk):
        p_host.run_block_host(h_in[k], h_out[k], d_in, d_out, stream)
    stream.synchronize()
    o = torch.empty(p_dev.shape("stokes"), dtype=torch.float32, device=dev)
    tol = TOL if prec == "fp32" else 1e-3
    for k in range(nblk):
        p_dev.run_block(_to_dev(blocks[k], dev), o)
        assert torch.equal(o.cpu(), h_out[k]), k
        _check_stokes(h_out[k].numpy().astype(np.float64), ob.run_block(blocks[k]), tol)
    p_host.close()
    p_dev.close()


@pytest.mark.parametrize("prec,nblk,out,bits", [("fp32", 3, "IQUV", 16), ("fp16tc", 4, "IQUV", 16),
                                              ("fp32", 1, "IQUV", 16), ("fp32", 2, "V", 8), ("fp16tc", 3, "V", 16)])
def test_multi_block_host_call_matches_per_block_path(dev, prec, nblk, out, bits):
    """lbf_run_blocks_host: n blocks from host buffers in one call, uploads alternating between two
    device buffers and overlapping the previous block's kernels, downloads overlapping the next
    block's filter bank.  Every block equals the device-buffer path bit for bit (the same kernels on
    the same inputs) and the oracle within tolerance; a second call continues the stream."""
    wl = _wl(S=16, B=70, out=out, Q=4, T=64 * N, bits=bits)
    p_host = _plan(wl, precision=prec)
    p_dev = _plan(wl, precision=prec)
    ob = O.observation_from_workload(wl)
    blocks = [G.make_block(wl, seed=31, block_index=k) for k in range(2 * nblk)]
    kind, dt = ("vol", torch.complex64) if out == "V" else ("stokes", torch.float32)
    h_in = [torch.from_numpy(b).pin_memory() for b in blocks]
    h_out = [torch.empty(p_host.shape(kind), dtype=dt).pin_memory() for _ in blocks]
    d_in0 = torch.empty(blocks[0].shape, dtype=torch.from_numpy(blocks[0]).dtype, device=dev)
    d_in1 = torch.empty_like(d_in0) if nblk > 1 else None
    d_out = torch.empty(p_host.shape(kind), dtype=dt, device=dev)
    stream = torch.cuda.Stream(device=dev)
    p_host.run_blocks_host(h_in[:nblk], h_out[:nblk], d_in0, d_in1, d_out, stream)
    p_host.run_blocks_host(h_in[nblk:], h_out[nblk:], d_in0, d_in1, d_out, stream)
    stream.synchronize()
    o = torch.empty(p_dev.shape(kind), dtype=dt, device=dev)
    tol = TOL if prec == "fp32" else 1e-3
    for k in range(2 * nblk):
        p_dev.run_block(_to_dev(blocks[k], dev), o)
        assert torch.equal(o.cpu(), h_out[k]), k
        ref = ob.run_block(blocks[k])
        if out == "V":
            err = _rel_rms(h_out[k].numpy().astype(np.complex128), ref, (2, 3, 4))
            assert err.max() <= (TOL if prec == "fp32" else 1e-4), (k, err.max())
        else:
            _check_stokes(h_out[k].numpy().astype(np.float64), ref, tol)
    from paper_1105_0661_gb300.lbf import LbfError
    with pytest.raises(LbfError):   # two blocks need two distinct input buffers
        p_host.run_blocks_host(h_in[:2], h_out[:2], d_in0, d_in0, d_out, stream)
    p_host.close()
    p_dev.close()


@pytest.mark.parametrize("bits,prec", [(16, "fp32"), (8, "fp32"), (16, "fp16tc")])
def test_input_not_16_byte_aligned_gives_the_same_block(dev, bits, prec):
    """The filter bank copies in-block tiles as 16-byte pieces when the input is 16-byte aligned and
    one sample at a time otherwise: an input that starts one sample word past a 16-byte boundary
    (still word-aligned, as the ABI requires) takes the second path and must give the same bits."""
    wl = _wl(S=6, F=2, T=40 * N, B=5, Q=4, bits=bits)
    p_a = _plan(wl, precision=prec)
    p_b = _plan(wl, precision=prec)
    blk = G.make_block(wl, seed=12, block_index=0)
    word = 8 if bits == 16 else 4
    flat = torch.from_numpy(np.ascontiguousarray(blk)).view(torch.uint8).reshape(-1)
    raw = torch.zeros(flat.numel() + 16, dtype=torch.uint8, device=dev)
    raw[word:word + flat.numel()].copy_(flat.to(dev))
    d_mis = raw[word:word + flat.numel()].view(torch.from_numpy(blk).dtype).view(blk.shape)
    assert d_mis.data_ptr() % 16 == word
    o_a = torch.empty(p_a.shape("stokes"), dtype=torch.float32, device=dev)
    o_b = torch.empty_like(o_a)
    for bi in range(2):   # the second block also reads the history written from the first
        if bi == 1:
            blk = G.make_block(wl, seed=12, block_index=1)
            raw[word:word + flat.numel()].copy_(torch.from_numpy(np.ascontiguousarray(blk)).view(torch.uint8).reshape(-1).to(dev))
        p_a.run_block(_to_dev(blk, dev), o_a)
        p_b.run_block(d_mis, o_b)
        assert torch.equal(o_a, o_b), bi
    p_a.close()
    p_b.close()


# ----------------------------------------------------------------------------- failure detection
def test_filter_bank_bounded_wait_expires_reports_and_context_survives(dev):
    """Failure detection without a GPU fault, FP32 path: one filter-bank CTA issues none of its
    input copies, so its halves wait on ring barriers that nothing completes.  The waits expire,
    the CTA records code 4 (the filter bank's input) and returns, lbf_device_status reports it and
    clears it, and the next launch on the same plan and context matches the oracle."""
    import time
    wl = _wl(S=8, F=2, T=64 * N, B=5, Q=4)
    p = _plan(wl)
    ob = O.observation_from_workload(wl)
    blk = G.make_block(wl, seed=4)
    d_in = _to_dev(blk, dev)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    assert p.device_status() == 0
    p.debug_stall_next(1)               # filter-bank CTA 1 (a spectrum chunk of one stream) copies nothing
    t0 = time.perf_counter()
    p.run_block(d_in, o)
    code = p.device_status()            # synchronises
    elapsed = time.perf_counter() - t0
    print(f"stalled filter bank: code {code}, {elapsed:.2f} s")
    assert code == 4
    assert elapsed < 30.0
    assert p.device_status() == 0       # the error word was cleared
    p.reset_state()                     # the stalled launch advanced the history
    p.run_block(d_in, o)
    assert p.device_status() == 0
    _check_stokes(o.cpu().numpy().astype(np.float64), ob.run_block(blk))
    p.close()
