"""Python binding of the C-ABI in include/lbf.h (argument marshalling only).

Every step of the path runs in the CUDA library liblbf.so; this module only converts a plan's
configuration to the C struct, torch tensors to device pointers and torch streams to cudaStream_t.
Importing it without the built library raises: there is no fallback path.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbf.so")

LBF_OK, LBF_EINVAL, LBF_ENOMEM, LBF_ECUDA, LBF_ESTATE, LBF_ETIMEOUT, LBF_EBUSY, LBF_EUNSUPPORTED, LBF_ETOOBIG = range(9)
OUTPUTS = {"V": 0, "I": 1, "IQUV": 4}
PRECISIONS = {"fp32": 0, "fp16tc": 1, "fp16tc2": 2}
BF_VARIANTS = {"auto": 0, "few": 1, "many": 2, "many64": 3}

# Every symbol include/lbf.h declares; the test suite checks the library exports all of them.
EXPORTED = ("lbf_plan", "lbf_plan_destroy", "lbf_plan_dims", "lbf_plan_shifts", "lbf_reset_state",
            "lbf_ppf", "lbf_delay_correct", "lbf_beamform", "lbf_beamform_stokes", "lbf_stokes",
            "lbf_run_block", "lbf_run_block_ws", "lbf_run_block_host", "lbf_run_blocks_host",
            "lbf_upload_subbands", "lbf_download_subbands", "lbf_trace_begin", "lbf_trace_end",
            "lbf_device_status", "lbf_debug_stall_next", "lbf_run_block_static", "lbf_superstation", "lbf_dedisperse",
            "lbf_batch_create", "lbf_batch_destroy",
            "lbf_batch_run", "lbf_batch_capture", "lbf_batch_launch", "lbf_batch_launches", "lbf_batch_tune",
            "lbf_measure_fp32_peak", "lbf_status_string", "lbf_version")


class LbfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}")


class _Config(ctypes.Structure):
    _fields_ = [
        ("n_stations", ctypes.c_int32), ("n_subbands", ctypes.c_int32), ("n_channels", ctypes.c_int32),
        ("n_taps", ctypes.c_int32), ("n_beams", ctypes.c_int32), ("block_samples", ctypes.c_int32),
        ("int_factor", ctypes.c_int32), ("sample_bits", ctypes.c_int32), ("output", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("bf_variant", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("sample_rate_hz", ctypes.c_double), ("phase_centre_l", ctypes.c_double),
        ("phase_centre_m", ctypes.c_double),
        ("station_xyz_m", ctypes.POINTER(ctypes.c_double)),
        ("subband_centre_hz", ctypes.POINTER(ctypes.c_double)),
        ("beam_dlm", ctypes.POINTER(ctypes.c_double)),
        ("fir_taps", ctypes.POINTER(ctypes.c_float)),
        ("bandpass", ctypes.POINTER(ctypes.c_float)),
    ]


class _Trace(ctypes.Structure):
    _fields_ = [("n_kernels", ctypes.c_int32), ("launches", ctypes.c_int32 * 16),
                ("total_ms", ctypes.c_double * 16), ("names", (ctypes.c_char * 32) * 16),
                ("dropped", ctypes.c_int32)]


class _Tuning(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int32), ("spc", ctypes.c_int32 * 10), ("mid_variant", ctypes.c_int32 * 10),
                ("ms", ctypes.c_double * 10), ("best_spc", ctypes.c_int32), ("best_mid_variant", ctypes.c_int32),
                ("best_ms", ctypes.c_double)]


class _AluPeak(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int32), ("ffma_ms", ctypes.c_double), ("ffma2_ms", ctypes.c_double),
                ("ffma_tflops", ctypes.c_double), ("ffma2_tflops", ctypes.c_double)]


class _Dims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "n_stations", "n_subbands", "n_channels", "n_taps", "n_beams", "block_samples", "int_factor",
        "n_spectra", "n_stokes", "d_max", "history_samples", "bf_kernel")] + \
        [(n, ctypes.c_size_t) for n in (
            "in_bytes", "chan_bytes", "ct_bytes", "vol_bytes", "out_bytes", "stokes_bytes",
            "workspace_bytes", "plan_bytes")]


_lib = None


def load_library() -> ctypes.CDLL:
    """Load liblbf.so (built in-tree by build_lib.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"liblbf.so not built at {LIB_PATH}; run paper_1105_0661_gb300.build_lib.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)
        sig = {
            "lbf_plan": ([ctypes.POINTER(_Config), ctypes.POINTER(vp)], ctypes.c_int),
            "lbf_plan_destroy": ([vp], ctypes.c_int),
            "lbf_plan_dims": ([vp, ctypes.POINTER(_Dims)], ctypes.c_int),
            "lbf_plan_shifts": ([vp, i32p, i32p], ctypes.c_int),
            "lbf_reset_state": ([vp, vp], ctypes.c_int),
            "lbf_ppf": ([vp, vp, vp, vp], ctypes.c_int),
            "lbf_delay_correct": ([vp, vp, vp, vp], ctypes.c_int),
            "lbf_beamform": ([vp, vp, vp, vp], ctypes.c_int),
            "lbf_beamform_stokes": ([vp, vp, vp, vp], ctypes.c_int),
            "lbf_stokes": ([vp, vp, vp, vp], ctypes.c_int),
            "lbf_run_block": ([vp, vp, vp, vp], ctypes.c_int),
            "lbf_run_block_ws": ([vp, vp, vp, vp, ctypes.c_size_t, vp], ctypes.c_int),
            "lbf_run_block_host": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
            "lbf_run_blocks_host": ([vp, ctypes.c_int32, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp, vp],
                                    ctypes.c_int),
            "lbf_upload_subbands": ([vp, vp, ctypes.c_int32, ctypes.c_int32, vp, vp], ctypes.c_int),
            "lbf_download_subbands": ([vp, vp, ctypes.c_int32, ctypes.c_int32, vp, vp], ctypes.c_int),
            "lbf_trace_begin": ([vp, ctypes.c_int32], ctypes.c_int),
            "lbf_trace_end": ([vp, ctypes.POINTER(_Trace)], ctypes.c_int),
            "lbf_device_status": ([vp, i32p], ctypes.c_int),
            "lbf_debug_stall_next": ([vp, ctypes.c_int64], ctypes.c_int),
            "lbf_superstation": ([vp, i32p, ctypes.c_int32, vp, vp, vp], ctypes.c_int),
            "lbf_dedisperse": ([vp, ctypes.c_double, ctypes.c_int32, vp, vp, vp], ctypes.c_int),
            "lbf_run_block_static": ([ctypes.POINTER(_Config), vp, vp, vp], ctypes.c_int),
            "lbf_batch_create": ([ctypes.POINTER(vp), ctypes.c_int32, ctypes.POINTER(vp)], ctypes.c_int),
            "lbf_batch_destroy": ([vp], ctypes.c_int),
            "lbf_batch_run": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp], ctypes.c_int),
            "lbf_batch_capture": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp], ctypes.c_int),
            "lbf_batch_launch": ([vp, vp], ctypes.c_int),
            "lbf_batch_launches": ([vp, i32p], ctypes.c_int),
            "lbf_batch_tune": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, ctypes.c_int32,
                                ctypes.POINTER(_Tuning)], ctypes.c_int),
            "lbf_measure_fp32_peak": ([ctypes.c_int32, vp, ctypes.POINTER(_AluPeak)], ctypes.c_int),
            "lbf_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "lbf_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes, fn.restype = args, res
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load_library().lbf_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != LBF_OK:
        raise LbfError(status, where)


def _ptr(t, need: int = 0) -> int:
    """Address of a contiguous torch tensor holding at least `need` bytes (or an int address,
    taken as is).  The size check keeps a short buffer from reaching a kernel."""
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    nbytes = t.numel() * t.element_size()
    if nbytes < need:
        raise ValueError(f"buffer holds {nbytes} bytes, the call needs {need}")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


@dataclass
class Dims:
    n_stations: int
    n_subbands: int
    n_channels: int
    n_taps: int
    n_beams: int
    block_samples: int
    int_factor: int
    n_spectra: int
    n_stokes: int
    d_max: int
    history_samples: int
    bf_kernel: int
    in_bytes: int
    chan_bytes: int
    ct_bytes: int
    vol_bytes: int
    out_bytes: int
    stokes_bytes: int
    workspace_bytes: int
    plan_bytes: int


class Plan:
    """One observation: tables, device-resident FIR/shift history and run_block scratch.

    precision: "fp32" (SIMT), "fp16tc" (tensor cores, three FP16 products) or "fp16tc2" (tensor
    cores, two products: FP16 weights); bf_variant: "auto", "few", "many" (128-beam tiles) or
    "many64" (lbf_config's fields of the same names)."""

    def __init__(self, station_xyz, subband_hz, beam_dlm, phase_centre, taps, block_samples,
                 int_factor=1, output="I", sample_bits=16, bandpass=None, n_channels=256, n_taps=16,
                 sample_rate_hz=195312.5, precision="fp32", bf_variant="auto", external_workspace=False,
                 incoherent_beam=False):
        lib = load_library()
        self._keep = [np.ascontiguousarray(station_xyz, dtype=np.float64).reshape(-1, 3),
                      np.ascontiguousarray(subband_hz, dtype=np.float64).reshape(-1),
                      np.ascontiguousarray(beam_dlm, dtype=np.float64).reshape(-1, 2),
                      np.ascontiguousarray(taps, dtype=np.float32).reshape(-1),
                      None if bandpass is None else np.ascontiguousarray(bandpass, dtype=np.float32).reshape(-1)]
        xyz, f0, dlm, h, bp = self._keep
        cfg = _Config()
        cfg.n_stations, cfg.n_subbands, cfg.n_beams = xyz.shape[0], f0.shape[0], dlm.shape[0]
        cfg.n_channels, cfg.n_taps = n_channels, n_taps
        cfg.block_samples, cfg.int_factor, cfg.sample_bits = block_samples, int_factor, sample_bits
        cfg.output = OUTPUTS[output]
        cfg.precision = PRECISIONS[precision]
        cfg.bf_variant = BF_VARIANTS[bf_variant]
        cfg.flags = (1 if external_workspace else 0) | (2 if incoherent_beam else 0)
        self.incoherent_beam = bool(incoherent_beam)
        cfg.sample_rate_hz = sample_rate_hz
        cfg.phase_centre_l, cfg.phase_centre_m = float(phase_centre[0]), float(phase_centre[1])
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        cfg.station_xyz_m = xyz.ctypes.data_as(dp)
        cfg.subband_centre_hz = f0.ctypes.data_as(dp)
        cfg.beam_dlm = dlm.ctypes.data_as(dp)
        cfg.fir_taps = h.ctypes.data_as(fp)
        cfg.bandpass = bp.ctypes.data_as(fp) if bp is not None else ctypes.cast(None, fp)
        self.output = output
        self.sample_bits = sample_bits
        handle = ctypes.c_void_p()
        _check(lib.lbf_plan(ctypes.byref(cfg), ctypes.byref(handle)), "lbf_plan")
        self._h = handle
        self._lib = lib
        d = _Dims()
        _check(lib.lbf_plan_dims(self._h, ctypes.byref(d)), "lbf_plan_dims")
        self.dims = Dims(**{n: getattr(d, n) for n, _ in _Dims._fields_})

    @classmethod
    def from_workload(cls, wl, **over):
        kw = dict(station_xyz=wl.station_xyz, subband_hz=wl.subband_hz, beam_dlm=wl.beam_dlm,
                  phase_centre=wl.phase_centre, taps=wl.taps, block_samples=wl.block_samples,
                  int_factor=wl.int_factor, output=wl.output, sample_bits=wl.sample_bits,
                  bandpass=wl.bandpass, n_channels=wl.n_channels, n_taps=wl.n_taps,
                  sample_rate_hz=wl.sample_rate_hz)
        kw.update(over)
        return cls(**kw)

    # -- shapes of the documented layouts
    def shape(self, which: str):
        d = self.dims
        S, F, T, N, M, B = d.n_stations, d.n_subbands, d.block_samples, d.n_channels, d.n_spectra, d.n_beams
        return {"in": (S, F, T, 2, 2), "chan": (F, S, 2, M, N), "ct": (F, N, S, 2, M),
                "vol": (B, F, N, 2, M),
                "stokes": (B + (1 if self.incoherent_beam and d.n_stokes else 0), d.n_stokes, F, N,
                           M // d.int_factor if d.n_stokes else 0)}[which]

    def shifts(self):
        S = self.dims.n_stations
        n = (ctypes.c_int32 * S)()
        dd = (ctypes.c_int32 * S)()
        _check(self._lib.lbf_plan_shifts(self._h, n, dd), "lbf_plan_shifts")
        return np.array(n[:], dtype=np.int64), np.array(dd[:], dtype=np.int64)

    # -- entry points (device pointers / torch CUDA tensors)
    def reset_state(self, stream=None):
        _check(self._lib.lbf_reset_state(self._h, _stream(stream)), "lbf_reset_state")

    def ppf(self, d_in, d_chan, stream=None):
        d = self.dims
        _check(self._lib.lbf_ppf(self._h, _ptr(d_in, d.in_bytes), _ptr(d_chan, d.chan_bytes),
                                 _stream(stream)), "lbf_ppf")

    def delay_correct(self, d_chan, d_ct, stream=None):
        d = self.dims
        _check(self._lib.lbf_delay_correct(self._h, _ptr(d_chan, d.chan_bytes), _ptr(d_ct, d.ct_bytes),
                                           _stream(stream)), "lbf_delay_correct")

    def beamform(self, d_ct, d_vol, stream=None):
        d = self.dims
        _check(self._lib.lbf_beamform(self._h, _ptr(d_ct, d.ct_bytes), _ptr(d_vol, d.vol_bytes),
                                      _stream(stream)), "lbf_beamform")

    def beamform_stokes(self, d_ct, d_out, stream=None):
        d = self.dims
        _check(self._lib.lbf_beamform_stokes(self._h, _ptr(d_ct, d.ct_bytes), _ptr(d_out, d.stokes_bytes),
                                             _stream(stream)), "lbf_beamform_stokes")

    def stokes(self, d_vol, d_out, stream=None):
        d = self.dims
        _check(self._lib.lbf_stokes(self._h, _ptr(d_vol, d.vol_bytes), _ptr(d_out, d.stokes_bytes),
                                    _stream(stream)), "lbf_stokes")

    def run_block(self, d_in, d_out, stream=None):
        d = self.dims
        _check(self._lib.lbf_run_block(self._h, _ptr(d_in, d.in_bytes), _ptr(d_out, d.out_bytes),
                                       _stream(stream)), "lbf_run_block")

    def run_block_ws(self, d_in, d_out, d_ws, stream=None):
        """run_block with a caller-provided scratch buffer (>= dims.workspace_bytes)."""
        d = self.dims
        nbytes = d_ws.numel() * d_ws.element_size() if not isinstance(d_ws, int) else d.workspace_bytes
        _check(self._lib.lbf_run_block_ws(self._h, _ptr(d_in, d.in_bytes), _ptr(d_out, d.out_bytes),
                                          _ptr(d_ws, d.workspace_bytes), nbytes, _stream(stream)),
               "lbf_run_block_ws")

    def device_bytes(self) -> int:
        """Device memory the plan itself holds (tables, history, and its scratch unless external)."""
        return self.dims.plan_bytes

    def run_block_host(self, h_in, h_out, d_in, d_out, stream=None):
        """H2D copy of h_in, the fused path on `stream`, D2H copy into h_out; the copies run on the
        plan's copy streams (the next block's upload overlaps this block's kernels) and `stream`
        waits for the download.  Synchronise `stream` before reading h_out or reusing h_in."""
        d = self.dims
        _check(self._lib.lbf_run_block_host(self._h, _ptr(h_in, d.in_bytes), _ptr(h_out, d.out_bytes),
                                            _ptr(d_in, d.in_bytes), _ptr(d_out, d.out_bytes),
                                            _stream(stream)), "lbf_run_block_host")

    def run_blocks_host(self, h_ins, h_outs, d_in0, d_in1, d_out, stream=None):
        """len(h_ins) consecutive blocks from host buffers, pipelined (uploads alternate between
        d_in0 and d_in1 and overlap the previous block's kernels); `stream` waits for the last
        download.  Synchronise `stream` before reading the h_outs or reusing the h_ins."""
        d = self.dims
        n = len(h_ins)
        if len(h_outs) != n:
            raise ValueError("h_ins and h_outs differ in length")
        arr_in = (ctypes.c_void_p * max(n, 1))(*[_ptr(h, d.in_bytes) for h in h_ins])
        arr_out = (ctypes.c_void_p * max(n, 1))(*[_ptr(h, d.out_bytes) for h in h_outs])
        d1 = _ptr(d_in1, d.in_bytes) if d_in1 is not None else None
        _check(self._lib.lbf_run_blocks_host(self._h, n, arr_in, arr_out, _ptr(d_in0, d.in_bytes), d1,
                                             _ptr(d_out, d.out_bytes), _stream(stream)), "lbf_run_blocks_host")

    def upload_subbands(self, h_in, n_subbands_full, first_subband, d_in, stream=None):
        """Asynchronous strided copy of subbands [first, first + F) of a whole host block
        [S][n_subbands_full][T][P][2] into this (chunk) plan's device input block."""
        d = self.dims
        full = d.in_bytes // d.n_subbands * int(n_subbands_full)
        _check(self._lib.lbf_upload_subbands(self._h, _ptr(h_in, full), int(n_subbands_full), int(first_subband),
                                             _ptr(d_in, d.in_bytes), _stream(stream)), "lbf_upload_subbands")

    def download_subbands(self, d_out, n_subbands_full, first_subband, h_out, stream=None):
        """Asynchronous strided copy of this (chunk) plan's output into the rows of a whole host
        output laid out for n_subbands_full subbands."""
        d = self.dims
        full = d.out_bytes // d.n_subbands * int(n_subbands_full)
        _check(self._lib.lbf_download_subbands(self._h, _ptr(d_out, d.out_bytes), int(n_subbands_full),
                                               int(first_subband), _ptr(h_out, full), _stream(stream)),
               "lbf_download_subbands")

    def dedisperse(self, dm, fft_len, d_vol_in, d_vol_out, stream=None):
        """Channel-level dedispersion (Section 4.4) of voltages [B][F][N][P][M] (may be in place)."""
        d = self.dims
        _check(self._lib.lbf_dedisperse(self._h, float(dm), int(fft_len), _ptr(d_vol_in, d.vol_bytes),
                                        _ptr(d_vol_out, d.vol_bytes), _stream(stream)), "lbf_dedisperse")

    def superstation(self, group_of_station, d_ct, d_ss, stream=None):
        """Sum the delay-compensated stations of each group (Section 4.2); d_ss is
        [F][N][G][P][M] cf32 with G = max(group) + 1."""
        grp = np.ascontiguousarray(group_of_station, dtype=np.int32).reshape(-1)
        G = int(grp.max()) + 1
        d = self.dims
        need = d.ct_bytes // d.n_stations * G
        _check(self._lib.lbf_superstation(self._h, grp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), G,
                                          _ptr(d_ct, d.ct_bytes), _ptr(d_ss, need), _stream(stream)),
               "lbf_superstation")

    def device_status(self) -> int:
        """Synchronise and return the role code of a device-side wait that gave up since the last
        call (0 = none; 1 loads, 2 MMA, 3 epilogue, 4 filter-bank input) and clear it.  A wait that gave up
        (LBF_ETIMEOUT) is reported through the code; other failures raise."""
        code = ctypes.c_int32(0)
        st = self._lib.lbf_device_status(self._h, ctypes.byref(code))
        if st != LBF_ETIMEOUT:
            _check(st, "lbf_device_status")
        return code.value

    def debug_stall_next(self, item: int = 0):
        """Failure-detection test: the next tensor-core launch stops loading at work item `item`; on an
        FP32 plan, filter-bank CTA `item` of the next fused launch issues none of its input copies."""
        _check(self._lib.lbf_debug_stall_next(self._h, int(item)), "lbf_debug_stall_next")

    def trace_begin(self, max_launches: int = 4096):
        _check(self._lib.lbf_trace_begin(self._h, int(max_launches)), "lbf_trace_begin")

    def trace_end(self) -> dict:
        """Per-kernel {name: (launches, total_ms)} of the launches since trace_begin."""
        t = _Trace()
        _check(self._lib.lbf_trace_end(self._h, ctypes.byref(t)), "lbf_trace_end")
        out = {}
        for k in range(t.n_kernels):
            if t.launches[k]:
                out[t.names[k].value.decode()] = (int(t.launches[k]), float(t.total_ms[k]))
        out["_dropped"] = int(t.dropped)
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several plans run together: one persistent grouped launch per stage for a block of every
    plan (lbf_batch_*), optionally replayed as a CUDA graph and autotuned."""

    def __init__(self, plans):
        lib = load_library()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib.lbf_batch_create(arr, len(self.plans), ctypes.byref(h)), "lbf_batch_create")
        self._h, self._lib = h, lib

    def _bufs(self, d_ins, d_outs):
        ins = (ctypes.c_void_p * len(self.plans))(*[_ptr(x, p.dims.in_bytes) for x, p in zip(d_ins, self.plans)])
        outs = (ctypes.c_void_p * len(self.plans))(*[_ptr(x, p.dims.out_bytes) for x, p in zip(d_outs, self.plans)])
        return ins, outs

    def run(self, d_ins, d_outs, stream=None):
        ins, outs = self._bufs(d_ins, d_outs)
        _check(self._lib.lbf_batch_run(self._h, ins, outs, _stream(stream)), "lbf_batch_run")

    def capture(self, d_ins, d_outs, stream=None):
        ins, outs = self._bufs(d_ins, d_outs)
        _check(self._lib.lbf_batch_capture(self._h, ins, outs, _stream(stream)), "lbf_batch_capture")

    def launch(self, stream=None):
        _check(self._lib.lbf_batch_launch(self._h, _stream(stream)), "lbf_batch_launch")

    def launches(self) -> int:
        """Kernel launches of one batch block (as the tables were last filled)."""
        n = ctypes.c_int32(0)
        _check(self._lib.lbf_batch_launches(self._h, ctypes.byref(n)), "lbf_batch_launches")
        return n.value

    def tune(self, d_ins, d_outs, reps=3, stream=None) -> dict:
        ins, outs = self._bufs(d_ins, d_outs)
        t = _Tuning()
        _check(self._lib.lbf_batch_tune(self._h, ins, outs, _stream(stream), int(reps), ctypes.byref(t)),
               "lbf_batch_tune")
        n = t.n_candidates
        return {"candidates": [{"spc": t.spc[i], "mid_variant": t.mid_variant[i], "ms": t.ms[i]} for i in range(n)],
                "best_spc": t.best_spc, "best_mid_variant": t.best_mid_variant, "best_ms": t.best_ms}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_peak(reps: int = 5, stream=None) -> dict:
    """Measured FP32 SIMT throughput of the current device (lbf_measure_fp32_peak): scalar FFMA
    and packed FP32x2 forms, TFLOP/s at 2 flop per lane FMA; synchronous."""
    r = _AluPeak()
    _check(load_library().lbf_measure_fp32_peak(int(reps), _stream(stream), ctypes.byref(r)),
           "lbf_measure_fp32_peak")
    return {"sms": r.sms, "ffma_tflops": r.ffma_tflops, "ffma2_tflops": r.ffma2_tflops,
            "ffma_ms": r.ffma_ms, "ffma2_ms": r.ffma2_ms}


def plan_status(cfg_kwargs) -> int:
    """Status lbf_plan returns for a configuration (validation only; LBF_OK needs a GPU)."""
    try:
        Plan(**cfg_kwargs).close()
        return LBF_OK
    except LbfError as e:
        return e.status


def run_block_static(station_xyz, subband_hz, beam_dlm, phase_centre, taps, block_samples, d_in, d_out,
                     int_factor=1, output="I", sample_bits=16, bandpass=None, sample_rate_hz=195312.5,
                     bf_variant="auto", stream=None):
    """One block through lbf_run_block_static, the entry point that allocates no device memory:
    for callers that cannot call cudaMalloc (a host framework that owns the device-memory budget,
    a real-time thread that must not take the allocator's locks).  The block is processed as the
    first block of a new stream; its scratch is a fixed 32 MiB device array shared by all calls,
    so calls whose device work overlaps must not be issued.  Raises LbfError(LBF_ETOOBIG) when the
    observation exceeds that scratch."""
    lib = load_library()
    keep = [np.ascontiguousarray(station_xyz, dtype=np.float64).reshape(-1, 3),
            np.ascontiguousarray(subband_hz, dtype=np.float64).reshape(-1),
            np.ascontiguousarray(beam_dlm, dtype=np.float64).reshape(-1, 2),
            np.ascontiguousarray(taps, dtype=np.float32).reshape(-1),
            None if bandpass is None else np.ascontiguousarray(bandpass, dtype=np.float32).reshape(-1)]
    xyz, f0, dlm, h, bp = keep
    cfg = _Config()
    cfg.n_stations, cfg.n_subbands, cfg.n_beams = xyz.shape[0], f0.shape[0], dlm.shape[0]
    cfg.n_channels, cfg.n_taps = 256, 16
    cfg.block_samples, cfg.int_factor, cfg.sample_bits = block_samples, int_factor, sample_bits
    cfg.output, cfg.precision, cfg.bf_variant, cfg.flags = OUTPUTS[output], 0, BF_VARIANTS[bf_variant], 0
    cfg.sample_rate_hz = sample_rate_hz
    cfg.phase_centre_l, cfg.phase_centre_m = float(phase_centre[0]), float(phase_centre[1])
    dp, fp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    cfg.station_xyz_m = xyz.ctypes.data_as(dp)
    cfg.subband_centre_hz = f0.ctypes.data_as(dp)
    cfg.beam_dlm = dlm.ctypes.data_as(dp)
    cfg.fir_taps = h.ctypes.data_as(fp)
    cfg.bandpass = bp.ctypes.data_as(fp) if bp is not None else ctypes.cast(None, fp)
    # the kernels read and write whole blocks: a short buffer must not reach them
    S, F, B = cfg.n_stations, cfg.n_subbands, cfg.n_beams
    T, M = int(block_samples), int(block_samples) // 256
    in_bytes = S * F * T * (8 if sample_bits == 16 else 4)
    if output == "V":
        out_bytes = B * F * T * 2 * 8                               # [B][F][N][P][M] cf32
    else:
        n_stokes = 1 if output == "I" else 4
        out_bytes = B * n_stokes * F * 256 * (M // int_factor) * 4  # [B][nS][F][N][M/Q] f32
    _check(lib.lbf_run_block_static(ctypes.byref(cfg), _ptr(d_in, in_bytes), _ptr(d_out, out_bytes),
                                    _stream(stream)), "lbf_run_block_static")
