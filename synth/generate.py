"""Seeded generators for station layouts, beam grids, filter taps and station voltage blocks.

Sample layout of a block (the station-side format of Section 3: each sample is two complex
16-bit integers, the X and Y polarisations):

    block[s, f, t, pol, ri]    int16 (or int8), ri = 0 real / 1 imaginary

i.e. per station, per subband, a time series of dual-polarisation complex samples, the order in
which a station emits its data.

The sky model used for the injected sources is the plain-wave picture of Section 3 (Fig. 2): a
source in direction (l, m) reaches a station at position (x, y, z) at time offset
-(x*l + y*m + z*n)/c relative to the array origin.  The generator carries its own copy of that
geometry because it is the *physics of the input*, not part of the beam former.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SUBBAND_RATE_HZ = 195312.5  # Section 3: 195 kHz subbands; complex sample rate of one subband
C_LIGHT = 299792458.0


# ----------------------------------------------------------------------------- geometry
def disc_positions(rng: np.random.Generator, n: int, radius_m: float) -> np.ndarray:
    """Stations uniform in a disc of the given radius, in the local ground plane (z = 0)."""
    r = radius_m * np.sqrt(rng.random(n))
    th = 2.0 * np.pi * rng.random(n)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n)], axis=1)


def lofar_positions(rng: np.random.Generator, n_core: int = 24, n_remote: int = 24,
                    core_radius_m: float = 1000.0, max_radius_m: float = 80000.0) -> np.ndarray:
    """A LOFAR-like layout (Section 3: a dense core plus stations at increasing distance).

    Core stations are uniform in a disc of `core_radius_m`; remote stations have a radius that is
    log-uniform between `core_radius_m` and `max_radius_m` and a uniform position angle.
    """
    core = disc_positions(rng, n_core, core_radius_m)
    lr = rng.uniform(np.log(core_radius_m), np.log(max_radius_m), n_remote)
    th = 2.0 * np.pi * rng.random(n_remote)
    r = np.exp(lr)
    remote = np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n_remote)], axis=1)
    return np.concatenate([core, remote], axis=0)


def square_beam_grid(n_side: int, pitch_deg: float) -> np.ndarray:
    """Tied-array beam offsets on an n_side x n_side square grid centred on the phase centre.

    Offsets are direction-cosine differences (dl, dm) taken as the grid angle in radians; beam 0
    is the (-, -) corner, beams run fastest along l.
    """
    idx = np.arange(n_side) - (n_side - 1) / 2.0
    out = [(np.radians(ix * pitch_deg), np.radians(iy * pitch_deg)) for iy in idx for ix in idx]
    return np.asarray(out, dtype=np.float64)


def hex_beam_grid(n_beams: int, pitch_deg: float) -> np.ndarray:
    """The first `n_beams` points of a centred hexagonal grid, in ring order (centre first).

    Ring k holds 6k points, so 6 rings give 1 + 3*6*7 = 127 beams (Fig. 3 shows tied-array beams
    as hexagons filling a station beam).
    """
    dirs = [(1, 0), (1, -1), (0, -1), (-1, 0), (-1, 1), (0, 1)]
    pts = [(0, 0)]
    k = 1
    while len(pts) < n_beams:
        q, r = -k, k  # start corner of ring k
        for d in range(6):
            for _ in range(k):
                pts.append((q, r))
                q, r = q + dirs[d][0], r + dirs[d][1]
        k += 1
    pts = pts[:n_beams]
    out = [(np.radians(pitch_deg * (q + 0.5 * r)), np.radians(pitch_deg * (np.sqrt(3.0) / 2.0) * r))
           for q, r in pts]
    return np.asarray(out, dtype=np.float64).reshape(n_beams, 2)


def subband_centres(n: int, f_start_hz: float = 110e6, rate_hz: float = SUBBAND_RATE_HZ) -> np.ndarray:
    """Contiguous subbands of `rate_hz` width starting at `f_start_hz`: centre j = f0 + (j + 1/2)*rate."""
    return f_start_hz + (np.arange(n) + 0.5) * rate_hz


# ----------------------------------------------------------------------------- filter tables
def kaiser_sinc_taps(n_taps: int = 16, n_channels: int = 256, beta: float = 9.0) -> np.ndarray:
    """Poly-phase prototype: a Kaiser-windowed sinc of n_taps*n_channels points, sum 1, float32.

    h[n] = w_kaiser(n; beta) * sinc((n - (LN-1)/2) / N), normalised to sum(h) = 1.  The filter is a
    convention (the paper does not print its filter); both sides receive these taps as data.
    """
    LN = n_taps * n_channels
    n = np.arange(LN, dtype=np.float64)
    h = np.kaiser(LN, beta) * np.sinc((n - (LN - 1) / 2.0) / n_channels)
    h /= h.sum()
    return h.astype(np.float32)


def bandpass_ripple(n_channels: int = 256, depth: float = 0.1, cycles: float = 3.0) -> np.ndarray:
    """A synthetic station-filter ripple to exercise the per-channel bandpass correction."""
    c = np.arange(n_channels, dtype=np.float64)
    return (1.0 + depth * np.cos(2.0 * np.pi * cycles * c / n_channels)).astype(np.float32)


# ----------------------------------------------------------------------------- workloads
@dataclass
class Workload:
    """Shape and geometry of one observation (all FP64 except taps/bandpass, which are float32)."""
    name: str
    station_xyz: np.ndarray          # [S, 3] metres, local ENU
    subband_hz: np.ndarray           # [F] subband centre frequencies
    beam_dlm: np.ndarray             # [B, 2] direction-cosine offsets from the phase centre
    phase_centre: tuple              # (l0, m0)
    block_samples: int               # T, samples per station per subband per block
    int_factor: int                  # Q, spectra summed per Stokes output
    output: str                      # 'V' (voltages), 'I', or 'IQUV'
    sample_bits: int = 16            # 16 or 8
    sigma: float = 32.0              # per-component noise sigma in integer units
    n_channels: int = 256
    n_taps: int = 16
    sample_rate_hz: float = SUBBAND_RATE_HZ
    taps: np.ndarray = field(default=None)
    bandpass: np.ndarray = field(default=None)
    source: str = "tone"             # 'tone', 'pulse' or 'noise'
    snr: float = 0.1

    def __post_init__(self):
        if self.taps is None:
            self.taps = kaiser_sinc_taps(self.n_taps, self.n_channels)
        if self.bandpass is None:
            self.bandpass = np.ones(self.n_channels, dtype=np.float32)

    @property
    def n_stations(self) -> int:
        return int(self.station_xyz.shape[0])

    @property
    def n_subbands(self) -> int:
        return int(self.subband_hz.shape[0])

    @property
    def n_beams(self) -> int:
        return int(self.beam_dlm.shape[0])

    @property
    def n_spectra(self) -> int:
        return self.block_samples // self.n_channels

    def station_samples(self) -> int:
        return self.n_stations * self.n_subbands * self.block_samples

    def subset(self, subbands) -> "Workload":
        """The same observation restricted to a list of subband indices."""
        sb = np.asarray(self.subband_hz)[np.asarray(subbands)]
        return Workload(**{**self.__dict__, "subband_hz": sb, "name": f"{self.name}[sb{list(subbands)}]"})


def workload_tiny(seed: int = 0) -> Workload:
    """8 stations in a 2 km disc, 1 subband at 150 MHz, 65536 int16 samples, 4 beams on a 0.5 deg
    square grid, Stokes I integrated over 4 spectra, tone at beam 0 with SNR 0.1."""
    rng = np.random.default_rng(seed)
    return Workload(name="tiny-8st-1sb-4beam-I4", station_xyz=disc_positions(rng, 8, 1000.0),
                    subband_hz=np.array([150e6]), beam_dlm=square_beam_grid(2, 0.5),
                    phase_centre=(0.3, 0.4), block_samples=65536, int_factor=4, output="I",
                    source="tone")


def workload_lofar_fp32(seed: int = 0) -> Workload:
    """48 stations (24 core in a 2 km disc, 24 remote log-uniform to 80 km), 244 subbands over
    110-158 MHz, 196608-sample blocks, 127 beams on a 6-ring hex grid of 0.05 deg pitch, Stokes I
    integrated over 16 spectra, pulsed source at beam 0."""
    rng = np.random.default_rng(seed)
    return Workload(name="lofar-48st-244sb-127beam-I16", station_xyz=lofar_positions(rng),
                    subband_hz=subband_centres(244), beam_dlm=hex_beam_grid(127, 0.05),
                    phase_centre=(0.3, 0.4), block_samples=196608, int_factor=16, output="I",
                    source="pulse")


def workload_lofar_tc(sample_bits: int = 8, seed: int = 0) -> Workload:
    """The 48-station observation in the many-beam form: 1024 hex beams, Stokes IQUV over 16."""
    wl = workload_lofar_fp32(seed)
    wl.name = f"lofar-48st-244sb-1024beam-IQUV16-i{sample_bits}"
    wl.beam_dlm = hex_beam_grid(1024, 0.05)
    wl.output = "IQUV"
    wl.sample_bits = sample_bits
    wl.sigma = 8.0 if sample_bits == 8 else 32.0
    return wl


# ----------------------------------------------------------------------------- station signals
def batch_workloads(n: int = 16, block_samples: int = 65536) -> list:
    """The batched workload: n sub-observations with stations 12-64, subbands 8-244, beams 1-512
    (log-uniform), int8 or int16 samples, drawn from numpy.random.default_rng(i) for i = 1..n,
    otherwise as the tiny observation (Stokes I over 4 spectra, tone at beam 0)."""
    out = []
    for i in range(1, n + 1):
        rng = np.random.default_rng(i)
        S = int(rng.integers(12, 65))
        F = int(rng.integers(8, 245))
        B = int(np.exp(rng.uniform(0.0, np.log(512.0))))
        bits = 8 if rng.random() < 0.5 else 16
        xyz = lofar_positions(rng, S // 2, S - S // 2)
        out.append(Workload(f"sub{i}-{S}st-{F}sb-{B}beam-i{bits}", xyz, subband_centres(F, 110e6),
                            hex_beam_grid(B, 0.05), (0.3, 0.4), block_samples, 4, "I", sample_bits=bits,
                            sigma=8.0 if bits == 8 else 32.0, source="tone"))
    return out


def small_batch_workloads(n: int = 64, block_samples: int = 16384, seed: int = 5) -> list:
    """Many small observations (the regime where one grouped launch beats per-observation
    launches): stations 8-16, subbands 2-8, beams 1-8, int16, Stokes I over 4, drawn in turn from
    numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        S, F, B = int(rng.integers(8, 17)), int(rng.integers(2, 9)), int(rng.integers(1, 9))
        xyz = lofar_positions(rng, S // 2, S - S // 2)
        out.append(Workload(f"small{i}-{S}st-{F}sb-{B}beam", xyz, subband_centres(F, 120e6 + 1e6 * i),
                            hex_beam_grid(B, 0.05), (0.3, 0.4), block_samples, 4, "I", sample_bits=16,
                            sigma=32.0, source="tone"))
    return out


def _arrival_offset(xyz: np.ndarray, l: float, m: float) -> np.ndarray:
    """Arrival-time offset (s) of a plane wave from direction (l, m) at each station (sky model)."""
    n = np.sqrt(max(0.0, 1.0 - l * l - m * m))
    return -(xyz[:, 0] * l + xyz[:, 1] * m + xyz[:, 2] * n) / C_LIGHT


def source_direction(wl: Workload, beam: int = 0) -> tuple:
    return (wl.phase_centre[0] + wl.beam_dlm[beam, 0], wl.phase_centre[1] + wl.beam_dlm[beam, 1])


def tone_signal(wl: Workload, amp: float, chan_offset: int, direction, block_index: int) -> np.ndarray:
    """Complex baseband tone, [S, F, T], identical in both polarisations.

    A tone at baseband frequency df = chan_offset * fs/N (sky frequency f0 + df) from `direction`
    arrives at station s as amp * exp(2 pi i df t) * exp(-2 pi i (f0 + df) tau_s), t the absolute
    sample time (so consecutive blocks continue the same tone).
    """
    T = wl.block_samples
    ts = 1.0 / wl.sample_rate_hz
    df = chan_offset * wl.sample_rate_hz / wl.n_channels
    tau = _arrival_offset(wl.station_xyz, *direction)
    t = (block_index * T + np.arange(T)) * ts
    f_sky = wl.subband_hz + df
    phase = np.exp(-2j * np.pi * f_sky[None, :] * tau[:, None])          # [S, F]
    return amp * phase[:, :, None] * np.exp(2j * np.pi * df * t)[None, None, :]


def pulse_signal(wl: Workload, rng: np.random.Generator, direction, power: float,
                 period_s: float = 0.033, duty: float = 0.05, block_index: int = 0) -> np.ndarray:
    """Gated complex noise (a pulsar-like source, no dispersion), [S, F, T].

    The source signal p(t) is complex Gaussian noise of the given power, switched on for the first
    `duty` of every `period_s`.  Station s receives p(t - tau_s) * exp(-2 pi i f0 tau_s); the
    fractional delay is applied as a phase ramp over the block's FFT (circular wrap accepted).
    """
    S, F, T = wl.n_stations, wl.n_subbands, wl.block_samples
    ts = 1.0 / wl.sample_rate_hz
    t = (block_index * T + np.arange(T)) * ts
    gate = (np.mod(t, period_s) < duty * period_s).astype(np.float64)
    sig = np.sqrt(power / 2.0)
    tau = _arrival_offset(wl.station_xyz, *direction)
    nu = np.fft.fftfreq(T, ts)
    out = np.empty((S, F, T), dtype=np.complex128)
    for f in range(F):
        p = gate * (rng.standard_normal(T) + 1j * rng.standard_normal(T)) * sig
        P = np.fft.fft(p)
        for s in range(S):
            out[s, f] = np.fft.ifft(P * np.exp(-2j * np.pi * (wl.subband_hz[f] + nu) * tau[s]))
    return out


def quantise(x: np.ndarray, bits: int) -> np.ndarray:
    """Round a complex [S, F, T, P] array to the station integer format [S, F, T, P, 2]."""
    lim = (1 << (bits - 1)) - 1
    ri = np.stack([x.real, x.imag], axis=-1)
    q = np.clip(np.rint(ri), -lim - 1, lim)
    return q.astype(np.int16 if bits == 16 else np.int8)


def make_block(wl: Workload, seed: int = 0, block_index: int = 0, source: str | None = None,
               noise: bool = True) -> np.ndarray:
    """One block of station data, [S, F, T, 2, 2] int16/int8, seeded by (seed, block_index).

    Complex Gaussian noise of per-component sigma `wl.sigma`, plus the workload's source at beam
    0's direction: a tone at channel offset +32 (SNR `wl.snr` = tone power / noise power), or a
    pulsed source; then rounded to nearest and clamped to the integer range.
    """
    source = wl.source if source is None else source
    rng = np.random.default_rng([seed, block_index])
    S, F, T = wl.n_stations, wl.n_subbands, wl.block_samples
    x = np.zeros((S, F, T, 2), dtype=np.complex128)
    if noise:
        g = rng.standard_normal((S, F, T, 2, 2)) * wl.sigma
        x += g[..., 0] + 1j * g[..., 1]
    p_noise = 2.0 * wl.sigma ** 2
    direction = source_direction(wl, 0)
    if source == "tone":
        x += tone_signal(wl, np.sqrt(wl.snr * p_noise), 32, direction, block_index)[..., None]
    elif source == "pulse":
        x += pulse_signal(wl, rng, direction, wl.snr * p_noise, block_index=block_index)[..., None]
    elif source != "noise":
        raise ValueError(f"unknown source {source!r}")
    return quantise(x, wl.sample_bits)
