"""Tensor-core (tcgen05, FP16 operands, FP32 accumulation) beam former against the FP64 oracle.

Bar (precision form): Stokes I within 1e-3 relative per element; Q, U, V within 1e-3 of I.
Both sample widths use two FP16 planes of the filtered spectrum (hi + lo).  The maximum errors seen are
printed so that the error of each output is reported.
"""

import time

import numpy as np
import pytest

from oracle import lbf_oracle as O
from synth import generate as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 256
TOL = 1e-3


@pytest.fixture(scope="module")
def dev():
    from paper_1105_0661_gb300 import build_lib
    build_lib.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _wl(S=48, F=2, T=64 * N, B=130, Q=16, out="I", bits=16, seed=0):
    rng = np.random.default_rng(seed)
    wl = G.Workload("tc", G.lofar_positions(rng, S // 2, S - S // 2), G.subband_centres(F, 120e6),
                    G.hex_beam_grid(B, 0.05), (0.3, 0.4), T, Q, out, sample_bits=bits,
                    sigma=32.0 if bits == 16 else 8.0, source="tone")
    wl.bandpass = G.bandpass_ripple(N)
    return wl


def _errors(got, ref):
    I = ref[:, 0]
    assert np.all(I > 0)
    eI = float((np.abs(got[:, 0] - I) / I).max())
    eq = float((np.abs(got[:, 1:] - ref[:, 1:]) / I[:, None]).max()) if ref.shape[1] == 4 else 0.0
    return eI, eq


@pytest.mark.parametrize("S,bits,out,B,M,variant", [(48, 16, "I", 130, 64, "auto"), (48, 8, "IQUV", 127, 80, "auto"),
                                                    (16, 16, "IQUV", 64, 64, "auto"), (64, 16, "I", 256, 48, "auto"),
                                                    (8, 8, "I", 5, 64, "many"), (8, 8, "I", 5, 64, "auto"),
                                                    (24, 16, "IQUV", 8, 64, "auto"), (24, 16, "I", 9, 64, "auto")])
def test_tc_beamform_stokes_matches_oracle(dev, S, bits, out, B, M, variant):
    """A tensor-core plan uses the tensor cores only where the beam count makes the beam former a
    dense contraction: up to 8 beams (AUTO) it runs the bandwidth-bound few-beam kernel (1); MANY
    forces the tensor-core kernel (3) even for 5 beams, which leaves the beam block mostly empty."""
    from paper_1105_0661_gb300 import Plan
    Q = 16
    wl = _wl(S=S, B=B, out=out, bits=bits, T=M * N, Q=Q)
    p = Plan.from_workload(wl, precision="fp16tc", bf_variant=variant)
    assert p.dims.bf_kernel == (1 if (variant == "auto" and B <= 8) else 3)
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(1)
    shp = p.shape("ct")
    ct = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    p.beamform_stokes(torch.from_numpy(ct).to(dev), o)
    assert p.device_status() == 0
    ref = ob.stokes(ob.beamform(ct.astype(np.complex128)))
    eI, eq = _errors(o.cpu().numpy().astype(np.float64), ref)
    print(f"TC S={S} bits={bits} {out} B={B} M={M}: Stokes I max rel err {eI:.2e}, QUV/I {eq:.2e}")
    assert eI <= TOL and eq <= TOL
    p.close()


@pytest.mark.parametrize("bits,out", [(16, "I"), (8, "IQUV")])
def test_tc_run_block_matches_oracle(dev, bits, out):
    from paper_1105_0661_gb300 import Plan
    wl = _wl(bits=bits, out=out, T=96 * N)
    p = Plan.from_workload(wl, precision="fp16tc")
    ob = O.observation_from_workload(wl)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    for bi in range(2):
        blk = G.make_block(wl, seed=2, block_index=bi)
        p.run_block(torch.from_numpy(blk).to(dev), o)
        assert p.device_status() == 0
        eI, eq = _errors(o.cpu().numpy().astype(np.float64), ob.run_block(blk))
        print(f"TC run_block bits={bits} {out} block {bi}: I {eI:.2e} QUV/I {eq:.2e}")
        assert eI <= TOL and eq <= TOL
    p.close()


def test_tc_equals_fp32_path_within_precision_bar(dev):
    from paper_1105_0661_gb300 import Plan
    wl = _wl(out="IQUV", T=64 * N)
    blk = torch.from_numpy(G.make_block(wl, seed=3)).to(dev)
    outs = []
    for prec in ("fp32", "fp16tc"):
        p = Plan.from_workload(wl, precision=prec)
        o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
        p.run_block(blk, o)
        outs.append(o.double().cpu().numpy())
        p.close()
    eI, eq = _errors(outs[1], outs[0])
    assert eI <= TOL and eq <= TOL


@pytest.mark.parametrize("Q,out", [(1, "IQUV"), (2, "I"), (4, "IQUV"), (8, "I"), (32, "IQUV"), (32, "I")])
def test_tc_every_integration_length(dev, Q, out):
    """Each integration length Q in {1, 2, 4, 8, 16, 32} has its own epilogue; M = 96 spectra leave
    the last 64-spectrum tile half empty, and 200 beams leave the second beam block partial."""
    from paper_1105_0661_gb300 import Plan
    wl = _wl(S=24, B=200, out=out, bits=16, T=96 * N, Q=Q)
    p = Plan.from_workload(wl, precision="fp16tc")
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(Q)
    shp = p.shape("ct")
    ct = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    p.beamform_stokes(torch.from_numpy(ct).to(dev), o)
    assert p.device_status() == 0
    ref = ob.stokes(ob.beamform(ct.astype(np.complex128)))
    eI, eq = _errors(o.cpu().numpy().astype(np.float64), ref)
    print(f"TC Q={Q} {out}: Stokes I max rel err {eI:.2e}, QUV/I {eq:.2e}")
    assert eI <= TOL and eq <= TOL
    p.close()


def test_bounded_wait_expires_reports_and_context_survives(dev):
    """Failure detection without a GPU fault: the loads of one work item are never issued, so the
    MMA warp waits on a barrier that nothing completes.  The wait expires, the kernel records the
    role and returns, lbf_device_status reports it (and clears it), and the next launch on the
    same plan and context matches the oracle."""
    from paper_1105_0661_gb300 import Plan
    wl = _wl(S=16, F=1, B=70, T=64 * N, Q=16, out="I")
    p = Plan.from_workload(wl, precision="fp16tc")
    ob = O.observation_from_workload(wl)
    blk = G.make_block(wl, seed=9)
    d_in = torch.from_numpy(blk).to(dev)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    assert p.device_status() == 0
    p.debug_stall_next(0)               # the CTA that owns work item 0 loads nothing
    t0 = time.perf_counter()
    p.run_block(d_in, o)
    code = p.device_status()            # synchronises
    elapsed = time.perf_counter() - t0
    print(f"stalled launch: role code {code}, {elapsed:.2f} s")
    # the MMA role gives up waiting for its loads; the epilogue, polling with the same bound for
    # the accumulator those loads would have produced, can expire first: either role is correct
    assert code in (2, 3)
    assert elapsed < 30.0
    assert p.device_status() == 0       # the error word was cleared
    p.reset_state()                     # the stalled launch advanced the history
    p.run_block(d_in, o)
    assert p.device_status() == 0
    eI, eq = _errors(o.cpu().numpy().astype(np.float64), ob.run_block(blk))
    assert eI <= TOL
    p.close()


@pytest.mark.parametrize("S,B,M,Q,out", [(1, 1, 16, 16, "I"), (3, 3, 32, 1, "IQUV"), (64, 129, 16, 8, "IQUV")])
def test_tc_degenerate_shapes(dev, S, B, M, Q, out):
    """One station (Kpad 16, a single K step), a single beam, fewer spectra than one 32-spectrum
    tile (the second tile of the pair is all padding), and the largest station count with one
    beam past a 128-beam block."""
    from paper_1105_0661_gb300 import Plan
    wl = _wl(S=S, B=B, out=out, bits=16, T=M * N, Q=Q, F=1)
    p = Plan.from_workload(wl, precision="fp16tc")
    ob = O.observation_from_workload(wl)
    blk = G.make_block(wl, seed=S + B)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    p.run_block(torch.from_numpy(blk).to(dev), o)
    assert p.device_status() == 0
    eI, eq = _errors(o.cpu().numpy().astype(np.float64), ob.run_block(blk))
    print(f"TC S={S} B={B} M={M} Q={Q} {out}: I {eI:.2e} QUV/I {eq:.2e}")
    assert eI <= TOL and eq <= TOL
    p.close()


def _vol_rel_rms(got, ref):
    """max over (beam, subband) of the relative RMS error of [B][F][N][P][M] voltages"""
    num = np.sqrt(np.sum(np.abs(got - ref) ** 2, axis=(2, 3, 4)))
    den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(2, 3, 4)))
    return float((num / den).max())


@pytest.mark.parametrize("S,B,M,bits", [(48, 130, 80, 16), (16, 70, 64, 8), (8, 5, 47, 16)])
def test_tc_voltages_match_oracle(dev, S, B, M, bits):
    """Complex-voltage output from the tensor cores (run_block, plan output V): beam voltages
    [B][F][N][P][M] within 1e-4 relative RMS per (beam, subband); M = 47 takes the unaligned
    store path and a ragged last tile."""
    from paper_1105_0661_gb300 import Plan
    wl = _wl(S=S, B=B, out="V", bits=bits, T=M * N, Q=1)
    p = Plan.from_workload(wl, precision="fp16tc")
    ob = O.observation_from_workload(wl)
    blk = G.make_block(wl, seed=11)
    vol = torch.empty(p.shape("vol"), dtype=torch.complex64, device=dev)
    p.run_block(torch.from_numpy(blk).to(dev), vol)
    assert p.device_status() == 0
    err = _vol_rel_rms(vol.cpu().numpy().astype(np.complex128), ob.run_block(blk))
    print(f"TC voltages S={S} B={B} M={M} bits={bits}: max rel RMS {err:.2e}")
    assert err <= 1e-4
    p.close()


def test_tc_split_beamform_voltages(dev):
    """lbf_beamform on a tensor-core plan (corner-turned input converted to the FP16 scratch)."""
    from paper_1105_0661_gb300 import Plan
    wl = _wl(S=48, B=130, out="I", T=64 * N, Q=16)
    p = Plan.from_workload(wl, precision="fp16tc")
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(5)
    shp = p.shape("ct")
    ct = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    vol = torch.empty(p.shape("vol"), dtype=torch.complex64, device=dev)
    p.beamform(torch.from_numpy(ct).to(dev), vol)
    assert p.device_status() == 0
    err = _vol_rel_rms(vol.cpu().numpy().astype(np.complex128), ob.beamform(ct.astype(np.complex128)))
    print(f"TC split beamform: max rel RMS {err:.2e}")
    assert err <= 1e-4
    p.close()


def test_tc2_voltages_within_the_weight_rounding_bound(dev):
    """Two-product form (weights rounded to FP16 once, spectrum split hi + lo): every beam voltage
    lies within the bound its arithmetic sets,
        |V - V_ref| <= (sqrt(2) 2^-12 + 1e-5) sum_s |Y_s|,
    i.e. the FP16 rounding of each weight component (at most 2^-12 for |x| < 1) plus 1e-5 for the
    sincos of the reduced phase and the FP32 accumulation; the three-product form of the same plan
    stays far inside it."""
    from paper_1105_0661_gb300 import Plan
    wl = _wl(S=48, B=130, out="I", T=64 * N, Q=16)
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(6)
    ratios = {}
    for prec in ("fp16tc2", "fp16tc"):
        p = Plan.from_workload(wl, precision=prec)
        assert p.dims.bf_kernel == 3
        shp = p.shape("ct")                                   # [F][N][S][P][M]
        if not ratios:
            ct = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
            y = ct.astype(np.complex128)
            ref = ob.beamform(y)                              # [B][F][N][P][M]
            bound = (np.sqrt(2.0) * 2.0 ** -12 + 1e-5) * np.abs(y).sum(axis=2)[None]
        vol = torch.empty(p.shape("vol"), dtype=torch.complex64, device=dev)
        p.beamform(torch.from_numpy(ct).to(dev), vol)
        assert p.device_status() == 0
        err = np.abs(vol.cpu().numpy().astype(np.complex128) - ref)
        ratios[prec] = float((err / bound).max())
        p.close()
    print(f"voltage error / weight-rounding bound: two products {ratios['fp16tc2']:.3f}, "
          f"three products {ratios['fp16tc']:.2e}")
    assert ratios["fp16tc2"] <= 1.0
    assert ratios["fp16tc"] <= 0.05


@pytest.mark.parametrize("bits,out", [(16, "I"), (8, "IQUV")])
def test_tc2_run_block_matches_oracle(dev, bits, out):
    """Two-product form against the FP64 oracle over two blocks: Stokes I within 1e-3 relative RMS
    per (beam, subband) row, Q, U, V within 1e-3 of I's RMS; the per-element maximum is printed
    (the weight rounding is not scaled down on single elements of beams that cancel a source)."""
    from paper_1105_0661_gb300 import Plan
    wl = _wl(bits=bits, out=out, T=96 * N)
    p = Plan.from_workload(wl, precision="fp16tc2")
    assert p.dims.bf_kernel == 3
    ob = O.observation_from_workload(wl)
    o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
    for bi in range(2):
        blk = G.make_block(wl, seed=2, block_index=bi)
        p.run_block(torch.from_numpy(blk).to(dev), o)
        assert p.device_status() == 0
        got, ref = o.cpu().numpy().astype(np.float64), ob.run_block(blk)   # [B][nS][F][N][M/Q]
        I = ref[:, 0]
        rms_I = np.sqrt(np.sum((got[:, 0] - I) ** 2, axis=(2, 3)) / np.sum(I ** 2, axis=(2, 3)))
        rms_q = 0.0
        if ref.shape[1] == 4:
            num = np.sqrt(np.sum((got[:, 1:] - ref[:, 1:]) ** 2, axis=(3, 4)))
            rms_q = float((num / np.sqrt(np.sum(I ** 2, axis=(2, 3)))[:, None]).max())
        eI, eq = _errors(got, ref)
        print(f"TC2 run_block bits={bits} {out} block {bi}: I rel RMS {rms_I.max():.2e} (per element max {eI:.2e}), "
              f"QUV/I rel RMS {rms_q:.2e} (max {eq:.2e})")
        assert rms_I.max() <= TOL and rms_q <= TOL
    p.close()


@pytest.mark.parametrize("S,out,Q,B,M", [(64, "I", 16, 130, 48), (48, "V", 1, 70, 47), (24, "IQUV", 32, 64, 96),
                                         (8, "IQUV", 1, 9, 40), (33, "I", 8, 200, 64)])
def test_tc2_shapes_match_oracle(dev, S, out, Q, B, M):
    """Two-product form over the kernel's corners: 64 stations (the two weight sets then fill all
    512 TMEM columns), voltages and 32-spectrum windows (two epilogue warps per lane quadrant),
    single-spectrum windows (scalar sums), ragged beam blocks and spectra.  Voltages within 1e-3
    relative RMS per (beam, subband); Stokes I within 1e-3 relative RMS per (beam, subband) row,
    Q, U, V within 1e-3 of I's RMS."""
    from paper_1105_0661_gb300 import Plan
    wl = _wl(S=S, B=B, out=out, Q=Q, T=M * N)
    p = Plan.from_workload(wl, precision="fp16tc2", bf_variant="many")
    assert p.dims.bf_kernel == 3
    ob = O.observation_from_workload(wl)
    blk = G.make_block(wl, seed=12)
    ref = ob.run_block(blk)
    if out == "V":
        vol = torch.empty(p.shape("vol"), dtype=torch.complex64, device=dev)
        p.run_block(torch.from_numpy(blk).to(dev), vol)
        assert p.device_status() == 0
        err = _vol_rel_rms(vol.cpu().numpy().astype(np.complex128), ref)
        print(f"TC2 voltages S={S} B={B} M={M}: max rel RMS {err:.2e}")
        assert err <= TOL
    else:
        o = torch.empty(p.shape("stokes"), dtype=torch.float32, device=dev)
        p.run_block(torch.from_numpy(blk).to(dev), o)
        assert p.device_status() == 0
        got = o.cpu().numpy().astype(np.float64)
        I = ref[:, 0]
        rms_I = np.sqrt(np.sum((got[:, 0] - I) ** 2, axis=(2, 3)) / np.sum(I ** 2, axis=(2, 3)))
        rms_q = 0.0
        if ref.shape[1] == 4:
            num = np.sqrt(np.sum((got[:, 1:] - ref[:, 1:]) ** 2, axis=(3, 4)))
            rms_q = float((num / np.sqrt(np.sum(I ** 2, axis=(2, 3)))[:, None]).max())
        print(f"TC2 S={S} {out} Q={Q} B={B} M={M}: I rel RMS {rms_I.max():.2e}, QUV/I {rms_q:.2e}")
        assert rms_I.max() <= TOL and rms_q <= TOL
    p.close()
