"""Seeded generation of full-size station blocks directly in device memory (torch).

The LOFAR-scale observation (48 stations x 244 subbands x 196608 samples = 18.4 GB of int16 per
block) is too large to synthesise on the host in a test or benchmark, so it is drawn on the GPU
with a seeded torch generator, one station at a time.  The signal model is the one of
synth.generate: complex Gaussian noise of per-component sigma plus a source at beam 0's direction
(a pulsed source: gated complex noise, 5 % duty in a 33 ms period, fractional station delays
applied as a phase ramp over the block's FFT; or a plane-wave tone at channel offset +32),
rounded to nearest and clamped to the integer range.  Same seed, shape and device -> same block.
"""

from __future__ import annotations

import math

import numpy as np

from .generate import C_LIGHT, Workload, source_direction


def make_block_device(wl: Workload, seed: int, device, source: str | None = None):
    import torch

    source = wl.source if source is None else source
    S, F, T = wl.n_stations, wl.n_subbands, wl.block_samples
    ts = 1.0 / wl.sample_rate_hz
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    dtype = torch.int16 if wl.sample_bits == 16 else torch.int8
    lim = (1 << (wl.sample_bits - 1)) - 1
    out = torch.empty((S, F, T, 2, 2), dtype=dtype, device=device)
    l, m = source_direction(wl, 0)
    n = math.sqrt(max(0.0, 1.0 - l * l - m * m))
    xyz = wl.station_xyz
    arrival = -(xyz[:, 0] * l + xyz[:, 1] * m + xyz[:, 2] * n) / C_LIGHT     # sky model, s
    p_noise = 2.0 * wl.sigma ** 2
    f0 = torch.tensor(np.asarray(wl.subband_hz), dtype=torch.float64, device=device)
    tt = torch.arange(T, device=device, dtype=torch.float64) * ts
    P = None
    if source == "pulse":
        gate = (torch.remainder(tt, 0.033) < 0.05 * 0.033).to(torch.float32)
        amp = math.sqrt(wl.snr * p_noise / 2.0)
        pr = torch.randn((F, T), generator=gen, device=device) * amp
        pi = torch.randn((F, T), generator=gen, device=device) * amp
        P = torch.fft.fft(torch.complex(pr * gate, pi * gate), dim=-1)       # [F, T]
        nu = torch.fft.fftfreq(T, d=ts, device=device, dtype=torch.float64)
    elif source == "tone":
        df = 32 * wl.sample_rate_hz / wl.n_channels
        a_tone = math.sqrt(wl.snr * p_noise)
    elif source != "noise":
        raise ValueError(f"unknown source {source!r}")
    for s in range(S):
        x = torch.randn((F, T, 2, 2), generator=gen, device=device) * wl.sigma
        if source == "pulse":
            ph = -2.0 * math.pi * (f0[:, None] + nu[None, :]) * arrival[s]
            ramp = torch.polar(torch.ones_like(ph), torch.remainder(ph, 2 * math.pi)).to(torch.complex64)
            sig = torch.fft.ifft(P * ramp, dim=-1)
        elif source == "tone":
            ph = 2.0 * math.pi * (df * tt[None, :] - (f0[:, None] + df) * arrival[s])
            sig = torch.polar(torch.full_like(ph, a_tone), torch.remainder(ph, 2 * math.pi)).to(torch.complex64)
        if source != "noise":
            x[..., 0] += sig.real[..., None]
            x[..., 1] += sig.imag[..., None]
        out[s] = torch.clamp(torch.round(x), -lim - 1, lim).to(dtype)
        del x
    return out
