"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each check is a function taking an Observation class, so that the mutation tests at the bottom can
plant a plausible mistake in a subclass (on the CPU) and show that some pin fails.
"""

import os

import numpy as np
import pytest

from oracle import lbf_oracle as O
from synth import generate as G

N, L = 256, 16
TS = 1.0 / G.SUBBAND_RATE_HZ
TAPS = G.kaiser_sinc_taps(L, N)


def _obs(cls=O.Observation, xyz=None, f0=(150e6,), beams=((0.0, 0.0),), pc=(0.0, 0.0), taps=TAPS,
         bp=None, Q=1, output="V", n=N, l=L):
    xyz = np.zeros((1, 3)) if xyz is None else np.asarray(xyz, dtype=np.float64)
    return cls(xyz, np.asarray(f0), np.asarray(beams), pc, taps, bp, n_channels=n, n_taps=l,
               int_factor=Q, output=output)


def _bins(chan):
    """Undo the channel order: X[..., k] with k the FFT bin, from chan[..., c]."""
    n = chan.shape[-1]
    k = np.arange(n)
    return chan[..., (k + n // 2) % n]


def _stations_with_shifts(ks, frac=0.2, l0=0.3):
    """Stations on the x axis whose phase-centre delay (l0, 0) is -(k - frac) samples."""
    ks = np.asarray(ks, dtype=np.float64)
    x = (ks - frac) * O.C_LIGHT * TS / l0
    return np.stack([x, np.zeros_like(x), np.zeros_like(x)], axis=1)


# ----------------------------------------------------------------------------- DFT (Section 4.2)
def check_dft_is_numpy_fft(mod=O):
    rng = np.random.default_rng(1)
    for n in (8, 16, 256):
        v = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
        X = mod.dft(v)
        ref = np.fft.fft(v, axis=-1)
        assert np.max(np.abs(X - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_dft_is_numpy_fft():
    """Library special case: the definition equals numpy's FFT (same sign, no normalisation)."""
    check_dft_is_numpy_fft()


def test_dft_parseval():
    rng = np.random.default_rng(2)
    v = rng.standard_normal((4, N)) + 1j * rng.standard_normal((4, N))
    X = O.dft(v)
    assert np.allclose(N * np.sum(np.abs(v) ** 2, -1), np.sum(np.abs(X) ** 2, -1), rtol=1e-12)


# ----------------------------------------------------------------------------- FIR (Section 4.2)
def check_impulse_reproduces_taps(cls=O.Observation):
    """An impulse at sample a*N + p0 gives v_m[p0] = h[(a - m + L - 1) N + p0], zero elsewhere."""
    ob = _obs(cls)
    T = 32 * N
    a, p0, amp = 5, 37, 1000.0
    x = np.zeros((1, 1, T, 2), dtype=np.complex128)
    x[0, 0, a * N + p0, 0] = amp
    chan = ob.ppf(x)                                   # [F, S, P, M, N]
    v = np.fft.ifft(_bins(chan[0, 0, 0]), axis=-1)      # [M, N] FIR output recovered
    exp = np.zeros_like(v)
    h = np.asarray(TAPS, dtype=np.float64).reshape(L, N)
    for m in range(a, a + L):
        exp[m, p0] = amp * h[a - m + L - 1, p0]
    assert np.max(np.abs(v - exp)) <= 1e-9 * amp
    assert np.max(np.abs(chan[0, 0, 1])) == 0.0


def test_impulse_reproduces_taps():
    check_impulse_reproduces_taps()


def test_dc_input_gives_sum_of_taps_in_centre_channel():
    """Closed form: a constant input x = a gives channel N/2 (baseband DC) = a * sum(h) in steady state."""
    ob = _obs()
    T = 24 * N
    x = np.full((1, 1, T, 2), 100.0 + 0j)
    chan = ob.ppf(x)
    hsum = float(np.sum(TAPS.astype(np.float64)))
    ss = chan[0, 0, :, L - 1:, :]                       # spectra with a full window
    assert np.allclose(ss[..., N // 2], 100.0 * hsum, rtol=1e-12, atol=1e-9)
    assert abs(hsum - 1.0) < 1e-5
    assert np.all(np.abs(ss[..., N // 2]) > 1e3 * np.max(np.abs(np.delete(ss, N // 2, axis=-1))))


def check_tone_lands_in_its_channel(cls=O.Observation):
    """A baseband tone at k0 * fs/N appears in channel N/2 + k0 (ascending frequency) with
    amplitude a * sum(h) and no phase drift across spectra."""
    for k0 in (32, -40, 0, 127):
        ob = _obs(cls)
        T = 24 * N
        j = np.arange(T)
        x = np.zeros((1, 1, T, 2), dtype=np.complex128)
        x[0, 0, :, 1] = 50.0 * np.exp(2j * np.pi * k0 * j / N)
        chan = ob.ppf(x)[0, 0, 1, L - 1:]               # pol Y, steady state [M', N]
        c = N // 2 + k0
        hsum = float(np.sum(TAPS.astype(np.float64)))
        assert np.allclose(chan[:, c], 50.0 * hsum, rtol=1e-10)
        assert np.argmax(np.abs(chan[0])) == c


def test_tone_lands_in_its_channel():
    check_tone_lands_in_its_channel()


def check_identity_taps_reproduce_shifted_input(cls=O.Observation):
    """Brute-force index check of the integer shift: with h[(L-1)N + p] = 1 (all other taps 0)
    the filter output is v_m[p] = x'[mN + p] = x[mN + p - d_s], zeros before the stream start,
    and the second block continues from the first block's tail."""
    taps = np.zeros(L * N, dtype=np.float32)
    taps[(L - 1) * N:] = 1.0
    ks = [0, 3, 7, 1]
    ob = _obs(cls, xyz=_stations_with_shifts(ks), pc=(0.3, 0.0), taps=taps)
    rng = np.random.default_rng(3)
    T = 4 * N
    blocks = [rng.integers(-100, 100, (4, 1, T, 2, 2)).astype(np.int16) for _ in range(2)]
    stream = np.concatenate([O.unpack(b) for b in blocks], axis=2)            # [S, 1, 2T, P]
    for bi, blk in enumerate(blocks):
        chan = ob.ppf(blk)
        v = np.fft.ifft(_bins(chan[0]), axis=-1)                            # [S, P, M, N]
        for s, k in enumerate(ks):
            d = k                      # a station reached k samples early is delayed by k
            j = bi * T + np.arange(T) - d
            exp = np.where(j >= 0, stream[s, 0, np.clip(j, 0, None), :].T, 0)  # [P, T]
            got = v[s].reshape(2, T)
            assert np.max(np.abs(got - exp)) < 1e-9, (bi, s)


def test_identity_taps_reproduce_shifted_input():
    check_identity_taps_reproduce_shifted_input()


def test_shift_readings():
    """n_s = round-half-away(tau/Ts) and d_s = max(n) - n_s >= 0."""
    ob = _obs(xyz=_stations_with_shifts([0, 3, 7, 1]), pc=(0.3, 0.0))
    assert list(ob.n_shift) == [0, -3, -7, -1]
    assert list(ob.d_shift) == [0, 3, 7, 1]
    assert list(O.round_half_away(np.array([0.5, -0.5, 1.49, -2.5]))) == [1, -1, 1, -3]


def test_streaming_blocks_equal_one_block():
    """Brute force: three consecutive blocks with carried history equal one block of 3T samples."""
    wl = G.workload_tiny(0)
    wl.block_samples = 8 * N
    xyz = G.lofar_positions(np.random.default_rng(4), 3, 3)   # long baselines: shifts > 0
    one = _obs(xyz=xyz, pc=(0.3, 0.4))
    three = _obs(xyz=xyz, pc=(0.3, 0.4))
    assert one.d_max > 5
    rng = np.random.default_rng(5)
    big = rng.integers(-200, 200, (6, 1, 24 * N, 2, 2)).astype(np.int16)
    ref = one.ppf(big)
    parts = [three.ppf(big[:, :, i * 8 * N:(i + 1) * 8 * N]) for i in range(3)]
    got = np.concatenate(parts, axis=3)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_brute_force_tiny_filter_bank():
    """Pure-loop evaluation of the FIR/DFT definition on a tiny case (N = 8, L = 3)."""
    n, l = 8, 3
    rng = np.random.default_rng(6)
    taps = rng.standard_normal(n * l).astype(np.float32)
    xyz = _stations_with_shifts([0, 2])
    ob = _obs(xyz=xyz, pc=(0.3, 0.0), taps=taps, n=n, l=l)
    T = 6 * n
    blocks = [rng.integers(-50, 50, (2, 1, T, 2, 2)).astype(np.int16) for _ in range(2)]
    stream = np.concatenate([O.unpack(b) for b in blocks], axis=2)
    h = taps.astype(np.float64)
    for bi, blk in enumerate(blocks):
        chan = ob.ppf(blk)
        for s, d in enumerate(ob.d_shift):
            for p_ in range(2):
                for m in range(T // n):
                    v = np.zeros(n, dtype=np.complex128)
                    for p in range(n):
                        for t in range(l):
                            j = bi * T + (m - (l - 1) + t) * n + p - d
                            if j >= 0:
                                v[p] += h[t * n + p] * stream[s, 0, j, p_]
                    for c in range(n):
                        k = (c - n // 2) % n
                        X = sum(v[p] * np.exp(-2j * np.pi * p * k / n) for p in range(n))
                        assert abs(chan[0, s, p_, m, c] - X) < 1e-9


# ----------------------------------------------------------------------------- delay, weights, beam
def check_single_station_unit_weight_reproduces_channelised_input(cls=O.Observation):
    """S = 1 at the array origin, beam at the phase centre: the beam is the channelised input
    times the bandpass of its channel (Sections 3, 4.3)."""
    bp = G.bandpass_ripple(N)
    for bpv in (None, bp):
        ob = _obs(cls, pc=(0.3, 0.4), bp=bpv)
        blk = G.make_block(G.Workload("t", np.zeros((1, 3)), np.array([150e6]), np.zeros((1, 2)),
                                      (0.3, 0.4), 8 * N, 1, "V"), seed=7)
        chan = ob.ppf(blk, advance=False)
        vol = ob.beamform(ob.delay_correct(chan))          # [B, F, N, P, M]
        exp = np.transpose(chan[:, 0], (0, 3, 1, 2)) * (1.0 if bpv is None else bp.astype(np.float64)[None, :, None, None])
        assert np.max(np.abs(vol[0] - exp)) <= 1e-12 * np.max(np.abs(exp))


def test_single_station_unit_weight_reproduces_channelised_input():
    check_single_station_unit_weight_reproduces_channelised_input()


def test_zero_delay_beam_is_station_sum():
    """Phase centre at zenith, stations in the ground plane, beam at the centre: every delay is 0,
    so the beam is the plain sum over stations of bandpass-corrected channels."""
    rng = np.random.default_rng(8)
    xyz = G.disc_positions(rng, 5, 3000.0)
    bp = G.bandpass_ripple(N)
    ob = _obs(xyz=xyz, pc=(0.0, 0.0), bp=bp, f0=(120e6, 130e6))
    assert np.all(ob.d_shift == 0)
    blk = rng.integers(-300, 300, (5, 2, 4 * N, 2, 2)).astype(np.int16)
    chan = ob.ppf(blk, advance=False)
    vol = ob.beamform(ob.delay_correct(chan))[0]               # [F, N, P, M]
    # linearity: the filter bank of the station sum equals the sum of the station filter banks
    summed = O.unpack(blk).sum(axis=0, keepdims=True)
    ob1 = _obs(xyz=np.zeros((1, 3)), pc=(0.0, 0.0), bp=bp, f0=(120e6, 130e6))
    exp = np.transpose(ob1.ppf(summed)[:, 0], (0, 3, 1, 2)) * bp.astype(np.float64)[None, :, None, None]
    assert np.max(np.abs(vol - exp)) <= 1e-10 * np.max(np.abs(exp))


def check_tone_at_beam_gains_S_squared(cls=O.Observation):
    """Noise-free plane-wave tone from beam b's direction, long baselines (integer shifts of many
    samples), tone off the band centre: after delay compensation and weighting every station adds
    in phase, so |V_b|^2 = S^2 |a|^2 (sum(h))^2 exactly in the tone channel; the other beams lose."""
    rng = np.random.default_rng(9)
    xyz = G.lofar_positions(rng, 6, 10, 1000.0, 80000.0)
    S = xyz.shape[0]
    beams = G.hex_beam_grid(7, 0.05)
    wl = G.Workload("t", xyz, np.array([140e6, 150.3e6]), beams, (0.3, 0.4), 16 * N, 1, "V")
    ob = _obs(cls, xyz=xyz, f0=wl.subband_hz, beams=beams, pc=(0.3, 0.4), output="V")
    assert ob.d_max >= 10
    b_src, k0, amp = 3, 32, 20.0
    hsum = float(np.sum(TAPS.astype(np.float64)))
    for bi in range(2):
        x = G.tone_signal(wl, amp, k0, G.source_direction(wl, b_src), bi)[..., None] * np.ones(2)
        vol = ob.run_block(x)
    c = N // 2 + k0
    p = np.abs(vol[:, :, c]) ** 2                                   # [B, F, P, M]
    assert np.allclose(p[b_src], (S * amp * hsum) ** 2, rtol=1e-9)
    others = np.delete(p, b_src, axis=0)
    assert np.max(others) < 0.5 * (S * amp * hsum) ** 2


def test_tone_at_beam_gains_S_squared():
    check_tone_at_beam_gains_S_squared()


def test_noise_adds_incoherently():
    """Off-source noise: every beam has E|V|^2 = S * P_noise * sum(h^2) (incoherent sum), while the
    tone in its beam has S^2 |a|^2 (the N_stations^2 coherent gain), statistically."""
    rng = np.random.default_rng(10)
    xyz = G.lofar_positions(rng, 8, 8)
    S = xyz.shape[0]
    beams = G.hex_beam_grid(3, 0.05)
    sigma = 30.0
    wl = G.Workload("t", xyz, np.array([150e6]), beams, (0.3, 0.4), 64 * N, 1, "V", sigma=sigma,
                    snr=0.1, source="tone")
    ob = O.observation_from_workload(wl)
    blk0 = G.make_block(wl, seed=11, block_index=0, source="noise")
    ob.run_block(blk0)
    blk1 = G.make_block(wl, seed=11, block_index=1, source="noise")
    vol = ob.run_block(blk1)
    p = np.mean(np.abs(vol) ** 2, axis=(0, 3, 4))               # [F, N] over beams, pols, spectra
    h2 = float(np.sum(TAPS.astype(np.float64) ** 2))
    exp = S * 2 * sigma ** 2 * h2
    mid = p[0, 16:-16]                                            # avoid band edges (filter roll-off)
    assert abs(np.mean(mid) / exp - 1.0) < 0.03


# ----------------------------------------------------------------------------- Stokes (Section 4.5)
def check_stokes_closed_forms(stokes=O.stokes_from_voltages):
    X = np.array([1.0 + 0j, 1 + 1j, 0j, 3 - 2j])
    Y = np.array([1j, 1.0 + 0j, 2.0 + 0j, 0.5 + 4j])
    s = stokes(X, Y, "IQUV")
    exp = []
    for x, y in zip(X, Y):
        xx, yy = abs(x) ** 2, abs(y) ** 2
        z = x * np.conj(y)
        exp.append([xx + yy, xx - yy, 2 * z.real, 2 * z.imag])
    assert np.allclose(s.T, np.array(exp))
    assert np.allclose(s[:, 0], [2.0, 0.0, 0.0, -2.0])   # X = 1, Y = i: V = 2 Im(1 * conj(i)) = -2
    assert np.allclose(stokes(X, Y, "I")[0], s[0])


def test_stokes_closed_forms():
    check_stokes_closed_forms()


def test_stokes_fully_polarised_identity():
    """Invariant: for a single (unintegrated) sample I^2 = Q^2 + U^2 + V^2."""
    rng = np.random.default_rng(12)
    X = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    Y = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    I, Qs, U, V = O.stokes_from_voltages(X, Y, "IQUV")
    assert np.allclose(I ** 2, Qs ** 2 + U ** 2 + V ** 2, rtol=1e-12)


def check_integration_sums_consecutive_spectra(integrate=O.integrate):
    p = np.arange(2 * 32, dtype=np.float64).reshape(2, 32)
    for q in (1, 2, 4, 8, 16):
        r = integrate(p, q)
        assert r.shape == (2, 32 // q)
        assert r[1, 1] == sum(p[1, q + i] for i in range(q))


def test_integration_sums_consecutive_spectra():
    """Brute force: the integrated Stokes sample is the sum (not the mean) of Q consecutive spectra."""
    check_integration_sums_consecutive_spectra()


def test_run_block_stokes_matches_stokes_of_voltages_and_sampled_path():
    """The whole path equals its parts, and the one-by-one sampled evaluation equals the full one."""
    wl = G.workload_tiny(0)
    wl.block_samples = 32 * N
    wl.bandpass = G.bandpass_ripple(N)
    for out in ("I", "IQUV", "V"):
        wl.output = out
        ob = O.observation_from_workload(wl)
        blk = G.make_block(wl, seed=0)
        full = ob.run_block(blk)
        ob.reset()
        vol = ob.beamform(ob.delay_correct(ob.ppf(blk)))
        if out != "V":
            assert np.allclose(full, ob.stokes(vol))
        ob2 = O.observation_from_workload(wl)
        ch = [0, 77, 128, 160, 255]
        smp = ob2.run_block_sampled(blk[:, 0], 0, ch)
        ref = full[:, :, 0][:, :, ch] if out != "V" else full[:, 0][:, ch]
        assert np.max(np.abs(smp - ref)) <= 1e-10 * np.max(np.abs(ref))


# ----------------------------------------------------------------------------- paper's rates
def _golden_rates(golden_dir):
    rows = {}
    for line in open(os.path.join(golden_dir, "paper_rates.txt")):
        if line.strip() and not line.startswith("#"):
            name, val, unit = line.split()[:3]
            rows[name] = (float(val), unit)
    return rows


def test_paper_rates_from_oracle_volumes(golden_dir):
    """The oracle's input and output volumes reproduce the rates the paper prints (Section 1,
    Section 2.2, Section 4.6, Table 1): 8-byte dual-pol int16 station samples, and per beam FP32
    complex voltages, FP32 IQUV and FP32 Stokes I at the subband sample rate."""
    g = _golden_rates(golden_dir)
    nsub = int(g["n_subbands"][0])
    assert round(G.SUBBAND_RATE_HZ / 1e3) == g["subband_rate_khz"][0]
    T = 2 * N
    seconds = T / G.SUBBAND_RATE_HZ
    wl = G.Workload("r", np.zeros((1, 3)), np.array([150e6]), np.zeros((1, 2)), (0.0, 0.0), T, 1, "V")
    blk = G.make_block(wl, seed=0)
    per_station = blk[0, 0].nbytes * 8 / seconds * nsub / 1e9

    def close(val, printed):
        step = 10.0 ** (np.floor(np.log10(printed)) - (1 if printed < 10 else 0))
        return abs(val - printed) <= step

    assert close(per_station, g["per_station_input"][0])
    for st, key in ((64, "station_input_64st"), (24, "station_input_24st"), (4, "station_input_4st")):
        assert close(st * per_station, g[key][0]), key
    for out, key in (("V", "beam_rate_voltages"), ("IQUV", "beam_rate_iquv"), ("I", "beam_rate_stokes_i")):
        ob = _obs(output=out, Q=1)
        res = ob.run_block(blk)
        bits = 64 if out == "V" else 32                        # FP32 complex / FP32 real output
        rate = res[0].size * bits / seconds * nsub / 1e9
        assert close(rate, g[key][0]), (key, rate)


# ----------------------------------------------------------------------------- mutation checks
class _ResidualUsesFullDelay(O.Observation):
    def delay_phase(self):
        return (self.f0[None, :, None] + self.df[None, None, :]) * self.tau[:, None, None]


class _ShiftWrongWay(O.Observation):
    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.d_shift = self.d_max - self.d_shift


class _WeightsUseCentreFrequency(O.Observation):
    def weights(self, f, channels=None):
        c = np.arange(self.N) if channels is None else np.asarray(channels)
        fc = self.f0[f] + 0.0 * self.df[c]
        return np.exp(2j * np.pi * fc[:, None, None] * self.beam_delays()[None])


class _TapsTimeReversed(O.Observation):
    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.h = self.h[::-1].copy()


class _WeightsConjugated(O.Observation):
    """Weights with the phase sign of the DFT (exp(-2 pi i f tau)) instead of the delay's."""
    def weights(self, f, channels=None):
        return np.conj(super().weights(f, channels))


class _ChannelsInBinOrder(O.Observation):
    """Channels left in FFT-bin order (no (k + N/2) mod N reorder to ascending frequency)."""
    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.k_of_c = np.arange(self.N)


class _BandpassByFftBin(O.Observation):
    """The bandpass indexed by FFT bin k instead of channel c = (k + N/2) mod N."""
    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.bp = np.roll(self.bp, self.N // 2)


@pytest.mark.parametrize("cls,check", [
    (_ResidualUsesFullDelay, check_tone_at_beam_gains_S_squared),
    (_ShiftWrongWay, check_identity_taps_reproduce_shifted_input),
    (_WeightsUseCentreFrequency, check_tone_at_beam_gains_S_squared),
    (_TapsTimeReversed, check_impulse_reproduces_taps),
    (_BandpassByFftBin, check_single_station_unit_weight_reproduces_channelised_input),
    (_WeightsConjugated, check_tone_at_beam_gains_S_squared),
    (_ChannelsInBinOrder, check_tone_lands_in_its_channel),
])
def test_pins_catch_planted_mistakes(cls, check):
    with pytest.raises(AssertionError):
        check(cls)


def test_pins_catch_wrong_stokes_v_sign():
    """V = 2 Im(X conj Y) as printed (Section 4.5); the conjugate convention -2 Im(X conj Y) fails."""
    def flipped(X, Y, kind):
        out = O.stokes_from_voltages(X, Y, kind)
        if kind == "IQUV":
            out = out.copy()
            out[3] = -out[3]
        return out
    with pytest.raises(AssertionError):
        check_stokes_closed_forms(flipped)


def test_pins_catch_integration_as_mean():
    with pytest.raises(AssertionError):
        check_integration_sums_consecutive_spectra(lambda p, q: O.integrate(p, q) / q)


def test_pins_catch_wrong_fft_sign(monkeypatch):
    monkeypatch.setattr(O, "dft_matrix", lambda n: np.exp(+2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n))
    with pytest.raises(AssertionError):
        check_dft_is_numpy_fft(O)
    with pytest.raises(AssertionError):
        check_tone_lands_in_its_channel()


# ----------------------------------------------------------------------------- incoherent beam (Section 3)
def test_incoherent_single_station_equals_coherent_centre_beam():
    """S = 1 at the origin, beam at the phase centre: the incoherent beam (Stokes of the unweighted
    station signal) equals the coherent beam."""
    wl = G.Workload("t", np.zeros((1, 3)), np.array([150e6]), np.zeros((1, 2)), (0.3, 0.4), 16 * N, 4, "IQUV")
    ob = O.observation_from_workload(wl, incoherent_beam=True)
    out = ob.run_block(G.make_block(wl, seed=3))
    assert out.shape[0] == 2
    assert np.allclose(out[1], out[0], rtol=1e-12, atol=0)


def test_incoherent_beam_ignores_delay_phases():
    """The delay phase has unit modulus and is common to both pols of a station, so the incoherent
    Stokes parameters equal those of the bandpass-corrected channels without any phase."""
    rng = np.random.default_rng(13)
    xyz = G.lofar_positions(rng, 4, 4)
    bp = G.bandpass_ripple(N)
    ob = _obs(xyz=xyz, pc=(0.3, 0.4), bp=bp, output="IQUV", Q=4)
    blk = rng.integers(-300, 300, (8, 1, 16 * N, 2, 2)).astype(np.int16)
    chan = ob.ppf(blk, advance=False)                                   # [F, S, P, M, N]
    inc = ob.incoherent(ob.delay_correct(chan))
    y = chan * bp.astype(np.float64)                                    # no phase
    p = O.stokes_from_voltages(y[:, :, 0], y[:, :, 1], "IQUV")          # [4, F, S, M, N]
    ref = O.integrate(np.moveaxis(p.sum(axis=2), -1, 2), 4)             # [4, F, N, M/Q]
    assert np.allclose(inc, ref, rtol=1e-10, atol=1e-6)


def test_incoherent_beam_keeps_an_off_axis_source():
    """Wide field of view (Section 3): a noise-free tone far outside the coherent beam still gives
    the incoherent beam S |a|^2 per pol and spectrum in its channel, while the coherent beam at the
    phase centre gets far less than the S^2 |a|^2 it would get on source."""
    rng = np.random.default_rng(14)
    xyz = G.lofar_positions(rng, 6, 10)
    S = xyz.shape[0]
    wl = G.Workload("t", xyz, np.array([150e6]), np.zeros((1, 2)), (0.3, 0.4), 16 * N, 4, "I")
    ob = O.observation_from_workload(wl, incoherent_beam=True)
    amp, k0 = 20.0, 32
    hsum = float(np.sum(TAPS.astype(np.float64)))
    far = (0.3 + np.radians(2.0), 0.4 - np.radians(1.5))
    for bi in range(2):
        x = G.tone_signal(wl, amp, k0, far, bi)[..., None] * np.ones(2)
        out = ob.run_block(x)
    c = N // 2 + k0
    inc = out[1, 0, 0, c]                                  # [M/Q]
    assert np.allclose(inc, S * 2 * 4 * (amp * hsum) ** 2, rtol=1e-9)
    assert np.max(out[0, 0, 0, c]) < 0.25 * S * np.min(inc)


# ----------------------------------------------------------------------------- superstation (Section 4.2)
def test_superstation_of_all_stations_is_the_phase_centre_beam():
    """One group holding every station equals the tied-array beam pointed at the phase centre
    (unit weights); singleton groups reproduce the stations."""
    rng = np.random.default_rng(15)
    xyz = G.lofar_positions(rng, 5, 5)
    ob = _obs(xyz=xyz, pc=(0.3, 0.4), beams=((0.0, 0.0),), bp=G.bandpass_ripple(N))
    blk = rng.integers(-200, 200, (10, 1, 8 * N, 2, 2)).astype(np.int16)
    ct = ob.delay_correct(ob.ppf(blk, advance=False))
    one = ob.superstation(ct, np.zeros(10, dtype=int))             # [F, N, 1, P, M]
    beam = ob.beamform(ct)                                          # [1, F, N, P, M]
    assert np.max(np.abs(one[:, :, 0] - beam[0])) <= 1e-10 * np.max(np.abs(beam))
    ident = ob.superstation(ct, np.arange(10))
    assert np.array_equal(ident, ct)
    two = ob.superstation(ct, np.array([0, 1] * 5))
    assert np.allclose(two[:, :, 0], ct[:, :, 0::2].sum(axis=2)) and np.allclose(two[:, :, 1], ct[:, :, 1::2].sum(axis=2))


# ----------------------------------------------------------------------------- dedispersion (Section 4.4)
def test_dedispersion_zero_dm_is_identity_and_runs_keep_their_norm():
    rng = np.random.default_rng(40)
    x = rng.standard_normal((3, 256)) + 1j * rng.standard_normal((3, 256))
    assert np.allclose(O.dedisperse_series(x, 120e6, 762.939453125, 0.0, 64), x, atol=1e-12)
    y = O.dedisperse_series(x, 30e6, 762.939453125, 5e3, 64)
    # unimodular chirp: Parseval per run of k samples
    assert np.allclose(np.linalg.norm(y.reshape(3, 4, 64), axis=-1), np.linalg.norm(x.reshape(3, 4, 64), axis=-1))
    # phi is linear in DM, so -DM applies the conjugate chirp and undoes +DM
    assert np.allclose(O.dedisperse_series(y, 30e6, 762.939453125, -5e3, 64), x, atol=1e-10)


def test_dedispersion_aligns_wave_packets_dispersed_by_the_cold_plasma_delay_law():
    """Independent of the chirp formula: two narrow-band wave packets at sub-channel frequencies
    nu1, nu2 arrive at T0 + K_DM DM (1/(f+nu)^2 - 1/f^2) (the textbook delay law t = K_DM DM / f^2).
    After dedispersion both envelopes peak at T0; with the chirp's sign flipped they move apart."""
    rate, k, f_c, dm = 762.939453125, 1024, 10e6, 40.0
    m = np.arange(k)
    t0 = 512.0
    peaks, flipped = [], []
    for jbin in (-268, 268):                      # nu = +-199.7 Hz, exactly on FFT bins
        nu = jbin * rate / k
        delay = O.K_DM * dm * (1.0 / (f_c + nu) ** 2 - 1.0 / f_c ** 2) * rate   # in samples
        assert abs(delay) > 40
        env = np.exp(-0.5 * ((m - t0 - delay) / 16.0) ** 2)
        x = env * np.exp(2j * np.pi * jbin * m / k)
        peaks.append(np.argmax(np.abs(O.dedisperse_series(x, f_c, rate, dm, k))))
        flipped.append(np.argmax(np.abs(O.dedisperse_series(x, f_c, rate, -dm, k))))
    assert all(abs(p - t0) <= 1 for p in peaks), peaks
    assert abs(flipped[0] - flipped[1]) > 150, flipped


def test_dedispersion_phase_derivative_is_the_relative_delay():
    """d phi / d nu = K_DM DM (1/f^2 - 1/(f + nu)^2), checked by central differences."""
    f_c, dm = 50e6, 123.0
    nu = np.linspace(-300.0, 300.0, 7)
    h = 1e-3
    num = (O.dedispersion_phase(f_c, nu + h, dm) - O.dedispersion_phase(f_c, nu - h, dm)) / (2 * h)
    ref = O.K_DM * dm * (1.0 / f_c ** 2 - 1.0 / (f_c + nu) ** 2)
    assert np.allclose(num, ref, rtol=1e-6, atol=1e-18)
