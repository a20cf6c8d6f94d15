"""Channel-level dedispersion (Section 4.4) on the GPU against the FP64 oracle.

Bar: the FP32 path's voltage tolerance (relative RMS <= 1e-5 per (beam, subband)); Stokes of
dedispersed voltages per element <= 1e-5 relative.  Subband centres of 12-30 MHz make the chirp
phase reach many cycles inside a 763 Hz channel, so the phase reduction is exercised.
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
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _wl(M, B=5, F=2, S=6, out="V", Q=1, f0=12e6):
    rng = np.random.default_rng(7)
    return G.Workload("dd", G.lofar_positions(rng, S // 2, S - S // 2), G.subband_centres(F, f0),
                      G.hex_beam_grid(B, 0.05), (0.3, 0.4), M * N, Q, out, source="tone")


def _rel_rms(got, ref, axes):
    return np.sqrt(np.sum(np.abs(got - ref) ** 2, axis=axes) / np.sum(np.abs(ref) ** 2, axis=axes))


@pytest.mark.parametrize("K,M,dm,inplace", [(2, 64, 3e3, False), (16, 64, 3e3, True), (64, 64, 8e3, False),
                                            (4096, 4096, 2e3, True), (256, 768, 0.0, False),
                                            (256, 768, 4e3, True), (256, 256, 9e3, False)])
def test_dedisperse_matches_oracle(dev, K, M, dm, inplace):
    from paper_1105_0661_gb300 import Plan
    wl = _wl(M, B=2 if M > 1000 else 5, F=1 if M > 1000 else 2)
    p = Plan.from_workload(wl)
    ob = O.observation_from_workload(wl)
    rng = np.random.default_rng(K)
    shp = p.shape("vol")
    vol = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(np.complex64)
    d_in = torch.from_numpy(vol).to(dev)
    d_out = d_in if inplace else torch.empty_like(d_in)
    p.dedisperse(dm, K, d_in, d_out)
    got = d_out.cpu().numpy().astype(np.complex128)
    ref = ob.dedisperse(vol.astype(np.complex128), dm, K)
    err = _rel_rms(got, ref, axes=(2, 3, 4))
    print(f"K={K} M={M} DM={dm}: max rel RMS {err.max():.2e}")
    assert err.max() <= TOL
    if dm == 0.0:
        assert _rel_rms(got, vol.astype(np.complex128), axes=(2, 3, 4)).max() <= TOL
    p.close()


def test_dedisperse_rejects_bad_lengths(dev):
    from paper_1105_0661_gb300 import LbfError, Plan
    wl = _wl(48)
    p = Plan.from_workload(wl)
    v = torch.zeros(p.shape("vol"), dtype=torch.complex64, device=dev)
    for K in (0, 1, 3, 32, 8192):           # 32 does not divide M = 48; 8192 is above the bound
        with pytest.raises(LbfError):
            p.dedisperse(1.0, K, v, v)
    with pytest.raises(LbfError):
        p.dedisperse(float("nan"), 16, v, v)
    p.close()


def test_beamform_dedisperse_stokes_chain_matches_oracle(dev):
    """run_block (voltages) -> dedisperse -> stokes through the C-ABI equals the oracle's chain."""
    from paper_1105_0661_gb300 import Plan
    wl_v = _wl(64, B=4, F=2, S=8, out="V", f0=20e6)
    wl_s = _wl(64, B=4, F=2, S=8, out="IQUV", Q=4, f0=20e6)
    pv, ps = Plan.from_workload(wl_v), Plan.from_workload(wl_s)
    ob_v, ob_s = O.observation_from_workload(wl_v), O.observation_from_workload(wl_s)
    blk = G.make_block(wl_v, seed=3)
    vol = torch.empty(pv.shape("vol"), dtype=torch.complex64, device=dev)
    pv.run_block(torch.from_numpy(blk).to(dev), vol)
    pv.dedisperse(5e3, 16, vol, vol)
    out = torch.empty(ps.shape("stokes"), dtype=torch.float32, device=dev)
    ps.stokes(vol, out)
    got = out.cpu().numpy().astype(np.float64)
    ref = ob_s.stokes(ob_v.dedisperse(ob_v.run_block(blk), 5e3, 16))
    I = ref[:, 0]
    assert np.all(I > 0)
    eI = (np.abs(got[:, 0] - I) / I).max()
    eq = (np.abs(got[:, 1:] - ref[:, 1:]) / I[:, None]).max()
    print(f"chain: Stokes I max rel err {eI:.2e}, QUV/I {eq:.2e}")
    assert eI <= TOL and eq <= TOL
    pv.close()
    ps.close()
