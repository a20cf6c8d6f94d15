"""FP64 CPU oracle of the LOFAR station-to-beam path (Mol & Romein, "The LOFAR Beam Former").

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may import this module.  The CUDA library never calls it, shares no code, tables or constants
with it, and must fail loudly when its own extension is missing rather than fall back here.

Everything is float64 / complex128 and written as the plain definition of each step, in the order
of the paper's pipeline (Section 4 and Fig. 4): integer-sample shift and int->float conversion
(Sections 3, 4.2), poly-phase filter bank = FIR + FFT into channels (Section 4.2), sub-sample delay
compensation by a per-sample complex multiply plus bandpass correction (Sections 3, 4.3), tied-array
beam forming as a weighted sum over stations with weights that depend on channel frequency,
station position and beam direction (Sections 3, 4.3), and Stokes I / IQUV with time integration
(Sections 3, 4.5, 5.1).  Library primitives used as steps: numpy matmul (the DFT as a product with
the DFT matrix, the beam sum as a product with the weight matrix), exp, sum.

Readings where the paper is silent (each also listed in the design notes):
  * delays: plane wave, tau_s(l, m) = -(x l + y m + z n)/c relative to the array origin;
  * integer shift: n_s = round-half-away(tau_s / Ts) for the phase centre, d_s = max(n) - n_s,
    x'_s[j] = x_s[j - d_s]; samples before the start of the stream are zero;
  * FIR (window-presum form, h[0] on the oldest sample):
        v_m[p] = sum_{t=0}^{L-1} h[tN + p] * x'[(m - (L-1) + t) N + p];
  * FFT: X_m[k] = sum_p v_m[p] exp(-2 pi i p k / N), unnormalised; channel c = (k + N/2) mod N, so
    channels run in ascending frequency with baseband offset df_c = (c - N/2) fs/N;
  * delay compensation: Y = X * bp[c] * exp(+2 pi i [f0 tau_s + df_c (tau_s - n_s Ts)]);
  * weights: w[b, s] = exp(+2 pi i f_c (tau_s(beam b) - tau_s(phase centre))), f_c = f0 + df_c;
  * Stokes: as printed in Section 4.5 (V = 2 Im(X conj(Y))); integration sums Q spectra;
  * channel-level dedispersion (Section 4.4): k-point FFT per run of k spectra of a channel, the
    textbook coherent-dedispersion chirp, inverse FFT (no overlap between runs).

Parity pins: every function here is pinned by tests marked not-gpu against closed forms, library
special cases, invariants and the paper's printed rates; none is "parity unpinned".
"""

from __future__ import annotations

import numpy as np

C_LIGHT = 299792458.0  # m/s


# ----------------------------------------------------------------------------- geometry (Section 3)
def plane_wave_delay(xyz: np.ndarray, l: float, m: float) -> np.ndarray:
    """Geometric delay tau_s (s) of each station for direction cosines (l, m).

    Section 3 (Fig. 2): a source's signal reaches different antennas at different times; for a
    plane wave from (l, m, n = sqrt(1 - l^2 - m^2)) a station at (x, y, z) sees it earlier by
    (x l + y m + z n)/c than the array origin.
    """
    n = np.sqrt(max(0.0, 1.0 - l * l - m * m))
    return -(xyz[:, 0] * l + xyz[:, 1] * m + xyz[:, 2] * n) / C_LIGHT


def round_half_away(x: np.ndarray) -> np.ndarray:
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def integer_shifts(tau: np.ndarray, ts: float):
    """Sample-level delay compensation (Section 3): n_s = round(tau_s / Ts), d_s = max(n) - n_s."""
    n = round_half_away(tau / ts).astype(np.int64)
    d = n.max() - n if n.size else n
    return n, d


def unpack(block: np.ndarray) -> np.ndarray:
    """Station integers [S, F, T, P, 2] -> complex128 [S, F, T, P] (Section 4.2 conversion step).

    A complex array [S, F, T, P] is accepted as already converted (noise-free pin inputs)."""
    if np.iscomplexobj(block):
        return block.astype(np.complex128)
    b = block.astype(np.float64)
    return b[..., 0] + 1j * b[..., 1]


def dft_matrix(n: int) -> np.ndarray:
    """F[p, k] = exp(-2 pi i p k / n): the unnormalised forward DFT as a matrix."""
    p = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(p, p) / n)


def dft(v: np.ndarray) -> np.ndarray:
    """X[..., k] = sum_p v[..., p] exp(-2 pi i p k / N), the definition, as a matrix product."""
    return v @ dft_matrix(v.shape[-1])


def stokes_from_voltages(X: np.ndarray, Y: np.ndarray, kind: str) -> np.ndarray:
    """Section 4.5: I = X conj X + Y conj Y, Q = X conj X - Y conj Y, U = 2 Re(X conj Y),
    V = 2 Im(X conj Y).  Returns [nS, ...] with nS = 1 ('I') or 4 ('IQUV')."""
    xx = (X * np.conj(X)).real
    yy = (Y * np.conj(Y)).real
    I = xx + yy
    if kind == "I":
        return I[None]
    xy = X * np.conj(Y)
    return np.stack([I, xx - yy, 2.0 * xy.real, 2.0 * xy.imag])


def integrate(p: np.ndarray, q: int) -> np.ndarray:
    """Time integration (Section 5.1, factors 1..16): sum of q consecutive spectra, last axis."""
    m = p.shape[-1]
    assert m % q == 0
    return p.reshape(p.shape[:-1] + (m // q, q)).sum(axis=-1)


# ----------------------------------------------------------------------------- dedispersion (Section 4.4)
# Dispersion constant of the cold-plasma delay law t(f) = K_DM * DM / f^2 (DM in pc cm^-3, f in Hz,
# t in s): 4.148808e3 s MHz^2 = 4.148808e15 s Hz^2 (Lorimer & Kramer, Handbook of Pulsar Astronomy,
# 2005, eq. 4.7).  The paper names the chirp but prints no formula; this constant and the transfer
# function below are the textbook coherent-dedispersion filter of Hankins & Rickett (1975).
K_DM = 4.148808e15


def dedispersion_phase(f_centre: float, nu: np.ndarray, dm: float) -> np.ndarray:
    """Phase in cycles of the interstellar medium's transfer function at sky frequency
    f_centre + nu: phi(nu) = K_DM DM nu^2 / (f_centre^2 (f_centre + nu)).  Its derivative is
    K_DM DM (1/f_centre^2 - 1/(f_centre + nu)^2), the extra dispersion delay of frequency
    f_centre + nu relative to f_centre (with a sign, since a delay tau multiplies a spectrum by
    exp(-2 pi i nu tau))."""
    nu = np.asarray(nu, dtype=np.float64)
    return K_DM * dm * nu * nu / (f_centre * f_centre * (f_centre + nu))


def dedisperse_series(x: np.ndarray, f_centre: float, channel_rate_hz: float, dm: float, k: int) -> np.ndarray:
    """Channel-level dedispersion (Section 4.4) of complex series x[..., M] sampled at
    channel_rate_hz (one spectrum per sample) around sky frequency f_centre: every run of k
    consecutive samples is transformed by a k-point FFT into sub-channels of width
    channel_rate_hz / k, multiplied by the chirp exp(-2 pi i phi(nu_j)) that undoes the dispersion
    (nu_j = j channel_rate/k for j < k/2, (j - k) channel_rate/k otherwise), and transformed back
    (inverse FFT, scaled by 1/k).  M must be a multiple of k.  Library FFTs serve as the steps."""
    x = np.asarray(x, dtype=np.complex128)
    M = x.shape[-1]
    assert M % k == 0
    j = np.arange(k)
    nu = np.where(j < k // 2, j, j - k) * (channel_rate_hz / k)
    chirp = np.exp(-2j * np.pi * dedispersion_phase(f_centre, nu, dm))
    runs = x.reshape(x.shape[:-1] + (M // k, k))
    y = np.fft.ifft(np.fft.fft(runs, axis=-1) * chirp, axis=-1)
    return y.reshape(x.shape)


# ----------------------------------------------------------------------------- one observation
class Observation:
    """State and tables of one observation; `run_block` processes consecutive blocks.

    Array layouts (the same layouts the library documents):
      block  [S][F][T][P][2] int          station samples
      chan   [F][S][P][M][N] complex       filter-bank output, channel-ordered (ppf)
      ct     [F][N][S][P][M] complex       delay-compensated, corner-turned (delay_correct)
      vol    [B][F][N][P][M] complex       tied-array beam voltages (beamform)
      out    [B][nS][F][N][M/Q] real       Stokes, integrated (stokes)
    """

    def __init__(self, station_xyz, subband_hz, beam_dlm, phase_centre, taps, bandpass=None,
                 n_channels=256, n_taps=16, sample_rate_hz=195312.5, int_factor=1, output="I",
                 incoherent_beam=False):
        self.xyz = np.asarray(station_xyz, dtype=np.float64).reshape(-1, 3)
        self.f0 = np.asarray(subband_hz, dtype=np.float64).reshape(-1)
        self.beam_dlm = np.asarray(beam_dlm, dtype=np.float64).reshape(-1, 2)
        self.l0, self.m0 = float(phase_centre[0]), float(phase_centre[1])
        self.N, self.L = int(n_channels), int(n_taps)
        self.h = np.asarray(taps, dtype=np.float64).reshape(self.L, self.N)  # h[t, p] = h[tN + p]
        bp = np.ones(self.N) if bandpass is None else np.asarray(bandpass, dtype=np.float64)
        self.bp = bp.reshape(self.N)
        self.fs = float(sample_rate_hz)
        self.ts = 1.0 / self.fs
        self.Q = int(int_factor)
        self.output = output
        self.incoherent_beam = bool(incoherent_beam)   # Stokes output gains beam B: incoherent
        self.S, self.F, self.B = self.xyz.shape[0], self.f0.shape[0], self.beam_dlm.shape[0]
        # geometry for the phase centre (sample shift + sub-sample phase) and for each beam
        self.tau = plane_wave_delay(self.xyz, self.l0, self.m0)
        self.n_shift, self.d_shift = integer_shifts(self.tau, self.ts)
        self.d_max = int(self.d_shift.max()) if self.S else 0
        self.H = (self.L - 1) * self.N + self.d_max
        c = np.arange(self.N)
        self.df = (c - self.N // 2) * (self.fs / self.N)              # channel baseband offsets
        self.k_of_c = (c - self.N // 2) % self.N                        # FFT bin of channel c
        self.reset()

    # -- state
    def reset(self):
        """Zero history: samples before the start of the stream are zero."""
        self.history = np.zeros((self.S, self.F, self.H, 2), dtype=np.complex128)

    # -- a1..a3: integer shift, conversion, FIR, FFT (Sections 3, 4.2)
    def ppf(self, block: np.ndarray, advance: bool = True) -> np.ndarray:
        x = unpack(block)                                               # [S, F, T, P]
        S, F, T, P = x.shape
        N, L, H = self.N, self.L, self.H
        assert T % N == 0
        M = T // N
        ext = np.concatenate([self.history, x], axis=2)                  # E = [history | block]
        chan = np.empty((F, S, P, M, N), dtype=np.complex128)
        for s in range(S):
            # x'[j] = x[j - d_s]; block-relative index j of x' sits at E[H + j - d_s].  Spectrum m
            # reads x'[(m - L + 1) N .. (m + 1) N - 1].
            start = H - int(self.d_shift[s]) - (L - 1) * N
            seg = ext[s, :, start:start + (M + L - 1) * N, :]           # [F, (M+L-1)N, P]
            frames = seg.reshape(F, M + L - 1, N, P)
            v = np.zeros((F, M, N, P), dtype=np.complex128)
            for t in range(L):
                v += self.h[t][None, None, :, None] * frames[:, t:t + M]
            X = dft(np.moveaxis(v, 2, 3))                                # [F, M, P, N] bins k
            chan[:, s] = np.moveaxis(X[..., self.k_of_c], 1, 2)          # [F, P, M, N] channels c
        if advance:
            self.history = ext[:, :, T:T + H, :].copy()
        return chan

    # -- a4: delay compensation + bandpass + corner turn (Sections 3, 4.3)
    def delay_phase(self) -> np.ndarray:
        """phi[s, f, c] in cycles = f0_f tau_s + df_c (tau_s - n_s Ts)."""
        resid = self.tau - self.n_shift * self.ts
        return (self.f0[None, :, None] * self.tau[:, None, None]
                + self.df[None, None, :] * resid[:, None, None])

    def delay_correct(self, chan: np.ndarray) -> np.ndarray:
        g = self.bp[None, None, :] * np.exp(2j * np.pi * self.delay_phase())   # [S, F, N]
        y = chan * np.transpose(g, (1, 0, 2))[:, :, None, None, :]              # [F, S, P, M, N]
        return np.ascontiguousarray(np.transpose(y, (0, 4, 1, 2, 3)))           # [F, N, S, P, M]

    # -- a5: weights (Sections 3, 4.3)
    def beam_delays(self) -> np.ndarray:
        """dtau[b, s] = tau_s(beam b direction) - tau_s(phase centre)."""
        out = np.empty((self.B, self.S))
        for b in range(self.B):
            out[b] = plane_wave_delay(self.xyz, self.l0 + self.beam_dlm[b, 0],
                                      self.m0 + self.beam_dlm[b, 1]) - self.tau
        return out

    def weights(self, f: int, channels=None) -> np.ndarray:
        """w[c, b, s] = exp(+2 pi i f_c dtau[b, s]) for subband f."""
        c = np.arange(self.N) if channels is None else np.asarray(channels)
        fc = self.f0[f] + self.df[c]
        return np.exp(2j * np.pi * fc[:, None, None] * self.beam_delays()[None])

    # -- a6: tied-array beam former (Section 4.3)
    def beamform(self, ct: np.ndarray, channels=None) -> np.ndarray:
        """V = sum_s w Y for the corner-turned block ct [F][n][S][P][M]; `channels` lists the
        channel index of each of the n rows (default: all N channels)."""
        F, N, S, P, M = ct.shape
        vol = np.empty((self.B, F, N, P, M), dtype=np.complex128)
        for f in range(F):
            w = self.weights(f, channels)                                  # [n, B, S]
            v = w @ ct[f].reshape(N, S, P * M)                             # [N, B, P*M]
            vol[:, f] = np.transpose(v.reshape(N, self.B, P, M), (1, 0, 2, 3))
        return vol

    def incoherent(self, ct: np.ndarray) -> np.ndarray:
        """Incoherent beam (Section 3): Stokes of the unweighted station signals, summed over
        stations as powers; returns [nS][F][N][M/Q]."""
        p = stokes_from_voltages(ct[:, :, :, 0], ct[:, :, :, 1], "IQUV" if self.output == "IQUV" else "I")
        return integrate(p.sum(axis=3), self.Q)

    def superstation(self, ct: np.ndarray, group_of_station) -> np.ndarray:
        """Superstation beam former (Section 4.2): the delay-compensated signals of the stations of
        each group summed with unit weight, as if the group were one station.
        ct [F][N][S][P][M] -> [F][N][G][P][M], G = max(group) + 1."""
        grp = np.asarray(group_of_station)
        G = int(grp.max()) + 1
        out = np.zeros(ct.shape[:2] + (G,) + ct.shape[3:], dtype=np.complex128)
        for s in range(ct.shape[2]):
            out[:, :, grp[s]] += ct[:, :, s]
        return out

    # -- channel-level dedispersion of beam voltages (Section 4.4)
    def dedisperse(self, vol: np.ndarray, dm: float, k: int) -> np.ndarray:
        """vol [B][F][N][P][M] -> the same layout, each (beam, subband, channel, pol) series
        dedispersed around its channel's sky frequency f0_f + df_c at the channel rate fs/N."""
        out = np.empty(vol.shape, dtype=np.complex128)
        for f in range(vol.shape[1]):
            for c in range(vol.shape[2]):
                out[:, f, c] = dedisperse_series(vol[:, f, c], self.f0[f] + self.df[c], self.fs / self.N, dm, k)
        return out

    # -- a7: Stokes + integration (Sections 4.5, 5.1)
    def stokes(self, vol: np.ndarray) -> np.ndarray:
        p = stokes_from_voltages(vol[:, :, :, 0], vol[:, :, :, 1], self.output)   # [nS, B, F, N, M]
        return np.ascontiguousarray(np.moveaxis(integrate(p, self.Q), 0, 1))      # [B, nS, F, N, M/Q]

    # -- the whole path for one block
    def run_block(self, block: np.ndarray, channel_group: int = 32) -> np.ndarray:
        ct = self.delay_correct(self.ppf(block))
        if self.output == "V":
            return self.beamform(ct)
        # channels are independent; evaluating them in groups only bounds the memory of the
        # intermediate voltages (B x group x P x M) for many-beam observations
        parts = [self.stokes(self.beamform(ct[:, c0:c0 + channel_group],
                                           np.arange(c0, min(c0 + channel_group, self.N))))
                 for c0 in range(0, self.N, channel_group)]
        out = np.concatenate(parts, axis=3)
        if self.incoherent_beam:
            out = np.concatenate([out, self.incoherent(ct)[None]], axis=0)
        return out

    # -- selected (subband, channel) outputs of one block from zero history, computed one by one
    def run_block_sampled(self, block_f: np.ndarray, f: int, channels) -> np.ndarray:
        """Outputs of subband `f` for the listed channels only, first block of a fresh stream.

        block_f is the [S][T][P][2] slice of subband f.  The FIR is evaluated in full; the DFT is
        evaluated only at the bins of the listed channels (rows of the same DFT definition).
        Returns [B][nS][len(channels)][M/Q] (or [B][len][P][M] voltages).
        """
        ch = np.asarray(channels)
        x = unpack(block_f)                                              # [S, T, P]
        S, T, P = x.shape
        N, L = self.N, self.L
        M = T // N
        Hz = np.zeros((S, self.H, P), dtype=np.complex128)
        ext = np.concatenate([Hz, x], axis=1)
        k = self.k_of_c[ch]
        Fk = np.exp(-2j * np.pi * np.outer(np.arange(N), k) / N)          # [N, nc]
        resid = self.tau - self.n_shift * self.ts
        ct = np.empty((len(ch), S, P, M), dtype=np.complex128)
        for s in range(S):
            start = self.H - int(self.d_shift[s]) - (L - 1) * N
            frames = ext[s, start:start + (M + L - 1) * N, :].reshape(M + L - 1, N, P)
            v = np.zeros((M, N, P), dtype=np.complex128)
            for t in range(L):
                v += self.h[t][None, :, None] * frames[t:t + M]
            X = np.einsum("mnp,nk->kpm", v, Fk)                            # [nc, P, M]
            phi = self.f0[f] * self.tau[s] + self.df[ch] * resid[s]
            ct[:, s] = X * (self.bp[ch] * np.exp(2j * np.pi * phi))[:, None, None]
        w = self.weights(f, ch)                                           # [nc, B, S]
        vol = (w @ ct.reshape(len(ch), S, P * M)).reshape(len(ch), self.B, P, M)
        vol = np.transpose(vol, (1, 0, 2, 3))                             # [B, nc, P, M]
        if self.output == "V":
            return vol
        p = stokes_from_voltages(vol[:, :, 0], vol[:, :, 1], self.output)   # [nS, B, nc, M]
        return np.moveaxis(integrate(p, self.Q), 0, 1)                    # [B, nS, nc, M/Q]


def observation_from_workload(wl, **over) -> Observation:
    """(`over` may also set incoherent_beam.)"""
    return _observation_from_workload(wl, **over)


def _observation_from_workload(wl, **over) -> Observation:
    """Build an Observation from a synth.Workload-like object (attributes only, no import)."""
    kw = dict(station_xyz=wl.station_xyz, subband_hz=wl.subband_hz, beam_dlm=wl.beam_dlm,
              phase_centre=wl.phase_centre, taps=wl.taps, bandpass=wl.bandpass,
              n_channels=wl.n_channels, n_taps=wl.n_taps, sample_rate_hz=wl.sample_rate_hz,
              int_factor=wl.int_factor, output=wl.output)
    kw.update(over)
    return Observation(**kw)
