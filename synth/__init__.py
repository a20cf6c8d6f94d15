"""Seeded synthetic inputs for the LOFAR station-to-beam path.

This package holds the input side only: station layouts, beam grids, subband centre frequencies,
the FIR prototype taps, a bandpass shape and the station voltage streams (noise, a plane-wave
tone, a pulsed source).  None of the beam former's own arithmetic (integer shift, filter bank,
delay compensation, weights, beam sum, Stokes) lives here.  Both the FP64 oracle and the CUDA
library consume what these functions return; neither is imported from here.
"""

from .generate import (  # noqa: F401
    SUBBAND_RATE_HZ,
    Workload,
    bandpass_ripple,
    disc_positions,
    hex_beam_grid,
    kaiser_sinc_taps,
    lofar_positions,
    make_block,
    square_beam_grid,
    subband_centres,
    workload_lofar_fp32,
    workload_lofar_tc,
    workload_tiny,
)
