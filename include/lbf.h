/*
 * lbf.h -- C ABI of the GB300 LOFAR station-to-beam library.
 *
 * The library computes the beam-forming pipeline of Mol & Romein, "The LOFAR Beam Former:
 * Implementation and Performance Analysis" (Sections 3 and 4): per subband a poly-phase filter
 * bank (16-tap FIR + 256-point FFT into channels, Section 4.2), per-station delay compensation as
 * an integer sample shift plus a per-sample phase rotation with bandpass correction (Sections 3,
 * 4.3), the tied-array beam former -- a complex weighted sum over stations per beam, channel,
 * polarisation and sample, with weights depending on channel frequency, station position and
 * beam direction (Section 4.3) -- and Stokes I or IQUV with time integration (Sections 4.5, 5.1).
 *
 * Conventions shared by every call
 *   - All sample/beam buffers are DEVICE pointers owned by the caller; the library never frees
 *     them.  Every call is asynchronous on the caller's CUDA stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream) unless stated otherwise.
 *   - A plan owns device copies of its tables (taps, bandpass, delays) and its device-resident
 *     state: the FIR/shift history of every (station, subband) stream and the run_block scratch.
 *   - Every call returns lbf_status; nothing is thrown across the ABI.  Bad arguments give
 *     LBF_EINVAL before any device work is enqueued.  A launch error, or an asynchronous error
 *     from earlier work, gives LBF_ECUDA.
 *   - One plan is one stream of blocks: calls on a plan must not overlap in time (use one plan
 *     per concurrent observation / stream).
 *
 * Array layouts (row-major, rightmost index fastest; cf32 = interleaved complex float32):
 *   in    [S][F][T][P][2]     int16 or int8   station samples (Section 3: each sample is two complex
 *                                              16-bit integers, X and Y polarisation); P = 2
 *   chan  [F][S][P][M][N]     cf32            filter-bank output, channel c (ascending frequency)
 *   ct    [F][N][S][P][M]     cf32            delay-compensated, bandpass-corrected, corner-turned
 *   vol   [B][F][N][P][M]     cf32            tied-array beam voltages (complex-voltages pipeline)
 *   out   [B][nS][F][N][M/Q]  float32         Stokes I (nS = 1) or IQUV (nS = 4), integrated
 *   with S stations, F subbands, T samples per block, N = 256 channels, M = T/N spectra,
 *   B beams, Q the integration factor.
 *
 * Definitions (the readings used where the paper is silent):
 *   tau_s(l,m) = -(x_s l + y_s m + z_s sqrt(1-l^2-m^2))/c       plane-wave geometric delay
 *   n_s = round-half-away(tau_s(l0,m0)/Ts), d_s = max_s n_s - n_s     integer shift (Section 3)
 *   x'_s[j] = x_s[j - d_s]                   samples before the first block are zero
 *   v_m[p] = sum_{t<16} h[tN+p] x'[(m-15+t)N + p]                    FIR, h[0] on the oldest sample
 *   X_m[k] = sum_p v_m[p] exp(-2 pi i p k/N),  channel c = (k + N/2) mod N,  df_c = (c-N/2) fs/N
 *   Y = X * bp[c] * exp(+2 pi i (f0_f tau_s + df_c (tau_s - n_s Ts)))        (Sections 3, 4.3)
 *   w[b,s] = exp(+2 pi i (f0_f + df_c)(tau_s(l0+dl_b, m0+dm_b) - tau_s(l0,m0)))  (Section 4.3)
 *   V_b = sum_s w[b,s] Y_s;  I = |X|^2+|Y|^2, Q = |X|^2-|Y|^2, U = 2Re(X conj Y), V = 2Im(X conj Y)
 *   (Section 4.5), each summed over Q consecutive spectra (Section 5.1).
 */
#ifndef LBF_H
#define LBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBF_OK = 0,
  LBF_EINVAL = 1,      /* bad argument, shape, NULL pointer or unsupported combination */
  LBF_ENOMEM = 2,      /* device allocation failed */
  LBF_ECUDA = 3,       /* a CUDA runtime error (launch or earlier asynchronous error) */
  LBF_ESTATE = 4,      /* plan in an unusable state (e.g. destroyed, or device mismatch) */
  LBF_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
  LBF_EBUSY = 6,       /* resource temporarily unavailable */
  LBF_EUNSUPPORTED = 7, /* valid request this library does not implement */
  LBF_ETOOBIG = 8       /* request exceeds the fixed scratch of lbf_run_block_static */
} lbf_status;

typedef enum { LBF_I8 = 8, LBF_I16 = 16 } lbf_sample_bits;

/* Pipelines of Section 3: complex voltages, Stokes I, Stokes IQUV. */
typedef enum { LBF_VOLTAGES = 0, LBF_STOKES_I = 1, LBF_STOKES_IQUV = 4 } lbf_output;

/* Arithmetic of the beam former (the precision form of the beam former, Section 4.3 computed on
 * tensor cores): FP32 SIMT; FP16 tensor cores with three products (spectrum and weights both split
 * hi + lo: Whi Yhi + Wlo Yhi + Whi Ylo, FP32 accumulation, errors ~1e-6 relative); or FP16 tensor
 * cores with two products (spectrum split hi + lo, weights rounded to FP16 once: Whi Yhi + Whi Ylo,
 * two thirds of the MMA work; the weight rounding, <= 2^-12 per component, leaves Stokes I within
 * ~7e-4 relative RMS on the test observations, more on single elements of beams that cancel a
 * strong source). */
typedef enum { LBF_FP32 = 0, LBF_FP16_TC = 1, LBF_FP16_TC2 = 2 } lbf_precision;

/* Beam-former kernel choice: AUTO picks the bandwidth-bound few-beam kernel for B <= 8 (tensor-core
 * precisions) or B <= 32 (FP32), and otherwise the tensor-core kernel (LBF_FP16_TC, LBF_FP16_TC2)
 * or the register-tiled FP32 many-beam kernel with the beam tile -- 128 (MANY) or 64 (MANY64)
 * beams per CTA -- that leaves the fewest tile slots empty (a 64-beam slot weighed as 1.15 of a
 * 128-beam one).  With
 * LBF_FP16_TC or LBF_FP16_TC2, MANY and MANY64 both select the tensor-core kernel. */
typedef enum { LBF_BF_AUTO = 0, LBF_BF_FEW = 1, LBF_BF_MANY = 2, LBF_BF_MANY64 = 3 } lbf_bf_variant;

/* The plan does not allocate the run_block scratch; the caller passes one to lbf_run_block_ws
 * (several plans can then share scratch buffers, as a serving loop does). */
#define LBF_FLAG_EXTERNAL_WORKSPACE 1
/* The Stokes output gains one beam, index B: the incoherent beam (Section 3) -- the Stokes
 * parameters of the unweighted station signals summed over stations as powers, i.e. the wide
 * field of view of the stations -- formed by lbf_run_block, lbf_run_block_ws and
 * lbf_beamform_stokes (not by lbf_stokes, which has no station data).  Stokes outputs only. */
#define LBF_FLAG_INCOHERENT_BEAM 2

typedef struct lbf_config {
  int32_t n_stations;     /* S >= 1 */
  int32_t n_subbands;     /* F >= 1 */
  int32_t n_channels;     /* N; the library supports 256 */
  int32_t n_taps;         /* L; the library supports 16 */
  int32_t n_beams;        /* B >= 1 */
  int32_t block_samples;  /* T >= 0, a multiple of N (T = 0: every call is a no-op) */
  int32_t int_factor;     /* Q in {1,2,4,8,16,32}; for Stokes outputs M = T/N must be a multiple */
  int32_t sample_bits;    /* 16 (int16) or 8 (int8) */
  int32_t output;         /* lbf_output */
  int32_t precision;      /* lbf_precision */
  int32_t bf_variant;     /* lbf_bf_variant */
  int32_t flags;          /* LBF_FLAG_* bits (0 for lbf_run_block_static) */
  double sample_rate_hz;  /* fs of one subband (195312.5 for LOFAR's 195 kHz subbands) */
  double phase_centre_l;  /* direction cosines (l0, m0) of the phase centre */
  double phase_centre_m;
  const double *station_xyz_m;     /* HOST [S][3] station positions, metres, local ENU */
  const double *subband_centre_hz; /* HOST [F] sky frequency of each subband's centre */
  const double *beam_dlm;          /* HOST [B][2] beam offsets (dl, dm) from the phase centre */
  const float *fir_taps;           /* HOST [L*N] prototype filter, h[t*N + p] */
  const float *bandpass;           /* HOST [N] per-channel bandpass correction, NULL = all ones */
} lbf_config;

typedef struct lbf_dims {
  int32_t n_stations, n_subbands, n_channels, n_taps, n_beams, block_samples, int_factor;
  int32_t n_spectra;          /* M = T / N */
  int32_t n_stokes;           /* nS: 1 (I), 4 (IQUV), 0 (voltages) */
  int32_t d_max;              /* largest integer shift d_s, in samples */
  int32_t history_samples;    /* H = (L-1) N + d_max samples kept per (station, subband) */
  int32_t bf_kernel;          /* beam former the plan uses: 1 few-beam, 2 many-beam FP32 (128-beam
                                 tiles), 3 tensor core, 4 many-beam FP32 (64-beam tiles) */
  size_t in_bytes;            /* bytes of one input block */
  size_t chan_bytes;          /* bytes of a chan buffer */
  size_t ct_bytes;            /* bytes of a ct buffer */
  size_t vol_bytes;           /* bytes of a vol buffer */
  size_t out_bytes;           /* bytes of one run_block output (vol_bytes for voltages) */
  size_t stokes_bytes;        /* bytes of a Stokes buffer [B (+1 incoherent)][nS][F][N][M/Q]
                                 (0 for voltages) */
  size_t workspace_bytes;     /* device scratch lbf_run_block needs (held by the plan unless
                                 LBF_FLAG_EXTERNAL_WORKSPACE) */
  size_t plan_bytes;          /* device memory the plan itself holds (tables, history, scratch) */
} lbf_dims;

typedef struct lbf_plan_s *lbf_plan_t;

/* Create a plan (Section 4 pipeline for one observation).  Validates `cfg`, computes the FP64
 * geometry on the host (phase-centre delays tau_s, integer shifts n_s and d_s, beam delay
 * differences), copies the tables to the current CUDA device, allocates the history (zeroed: the
 * stream starts with zero samples) and the run_block scratch.  Synchronous.  The config's host
 * arrays are copied; the caller keeps ownership.  On error *out is set to NULL.
 * With precision LBF_FP16_TC the many-beam beam former runs on the tensor cores (tcgen05, FP16
 * operands, FP32 accumulation): the filtered spectrum of either sample width feeds it as two FP16
 * planes (hi = fp16(X), lo = fp16(X - hi)) and the weights are split the same way, three products
 * per tile, writing Stokes or beam voltages; it needs S <= 64.  In lbf_run_block the planes hold
 * the spectrum before the delay phase and bandpass, which the weights carry instead (the same
 * linear map; Section 4.3's correction, applied once per weight); lbf_beamform and
 * lbf_beamform_stokes take an already corrected block.  LBF_FP16_TC2 is the same
 * with FP16 weights only (two products per tile).  The tensor cores are used
 * only where the beam count makes the beam former a dense contraction: with bf_variant AUTO and
 * B <= 8 beams, or bf_variant FEW, a tensor-core plan runs the bandwidth-bound FP32 few-beam
 * kernel on the FP32 corner-turned block instead (lbf_plan_dims reports bf_kernel 1); with MANY,
 * or AUTO and B > 8, it runs the tensor-core kernel (bf_kernel 3).
 * Errors: LBF_EINVAL (bad config), LBF_EUNSUPPORTED (N != 256, L != 16, or a tensor-core plan with
 * S > 64), LBF_ENOMEM, LBF_ECUDA. */
lbf_status lbf_plan(const lbf_config *cfg, lbf_plan_t *out);

/* Release every device buffer of the plan (synchronises the device first). NULL is a no-op. */
lbf_status lbf_plan_destroy(lbf_plan_t plan);

/* Sizes and derived dimensions of a plan (host only, no device work). */
lbf_status lbf_plan_dims(lbf_plan_t plan, lbf_dims *out);

/* Copy the integer shifts n_s and d_s (Section 3 sample-level delay compensation) of the S
 * stations to the HOST arrays n_shift[S] and d_shift[S] (either may be NULL). */
lbf_status lbf_plan_shifts(lbf_plan_t plan, int32_t *n_shift, int32_t *d_shift);

/* Zero the FIR/shift history on `stream`: the next block starts a new stream of samples. */
lbf_status lbf_reset_state(lbf_plan_t plan, void *stream);

/* Steps a1-a3: integer shift + int->float conversion + 16-tap FIR + 256-point FFT (Sections 3,
 * 4.2) of one block.  d_in: device `in` layout; d_chan: device `chan` layout (written).
 * Advances the plan's history by one block. */
lbf_status lbf_ppf(lbf_plan_t plan, const void *d_in, void *d_chan, void *stream);

/* Step a4: sub-sample delay compensation (phase rotation) + bandpass + corner turn (Sections 3,
 * 4.3).  d_chan: device `chan` layout (read); d_ct: device `ct` layout (written).  Stateless. */
lbf_status lbf_delay_correct(lbf_plan_t plan, const void *d_chan, void *d_ct, void *stream);

/* Steps a5-a6: weights generated on the device (FP64 phase, reduced to one cycle, FP32 sincos)
 * and the tied-array beam sum (Section 4.3).  d_ct: device `ct` (read); d_vol: device `vol`
 * layout (written).  Stateless.  A tensor-core plan converts `ct` into its FP16 scratch first
 * (not available with LBF_FLAG_EXTERNAL_WORKSPACE: LBF_EUNSUPPORTED). */
lbf_status lbf_beamform(lbf_plan_t plan, const void *d_ct, void *d_vol, void *stream);

/* Steps a5-a7 fused: beam former with the Stokes/integration epilogue (Sections 4.3, 4.5, 5.1).
 * d_ct: device `ct` (read); d_out: device `out` layout (written).  Requires a Stokes output. */
lbf_status lbf_beamform_stokes(lbf_plan_t plan, const void *d_ct, float *d_out, void *stream);

/* Step a7: Stokes I/IQUV (as configured) with integration over Q spectra (Sections 4.5, 5.1).
 * d_vol: device `vol` (read); d_out: device `out` layout (written).  Requires a Stokes output. */
lbf_status lbf_stokes(lbf_plan_t plan, const void *d_vol, float *d_out, void *stream);

/* lbf_run_block with caller-provided scratch: d_ws (device, >= workspace_bytes of lbf_plan_dims,
 * 256-byte aligned) is used for this call only and may be shared with other plans between calls.
 * Works for every plan; a plan created with LBF_FLAG_EXTERNAL_WORKSPACE can only run blocks
 * this way.  Errors as lbf_run_block, LBF_EINVAL for a short or misaligned workspace. */
lbf_status lbf_run_block_ws(lbf_plan_t plan, const void *d_in, void *d_out, void *d_ws, size_t ws_bytes,
                            void *stream);

/* Steps a1-a7 for one block, fused: filter bank with the delay/bandpass/corner-turn epilogue into
 * the plan's scratch, then the beam former with the Stokes epilogue (or voltages).  d_in: device
 * `in`; d_out: device `out` (Stokes) or `vol` (voltages).  Advances the history by one block.
 * Equal, within FP32 rounding, to lbf_ppf -> lbf_delay_correct -> lbf_beamform -> lbf_stokes. */
lbf_status lbf_run_block(lbf_plan_t plan, const void *d_in, void *d_out, void *stream);

/* Superstation beam former (Section 4.2: combine several stations as if they were one): the
 * delay-compensated signals of the stations of each group summed with unit weight.
 * group_of_station: HOST [S], values in [0, n_groups); d_ct: device `ct` [F][N][S][P][M];
 * d_ss: device [F][N][n_groups][P][M] cf32 (the corner-turned layout with groups in place of
 * stations).  Synchronises `stream` while the group table is uploaded.  Stateless. */
lbf_status lbf_superstation(lbf_plan_t plan, const int32_t *group_of_station, int32_t n_groups, const void *d_ct,
                            void *d_ss, void *stream);

/* Channel-level dedispersion (Section 4.4) of beam voltages.  Every run of fft_len consecutive
 * spectra of each (beam, subband, channel, pol) series is transformed by an fft_len-point FFT into
 * sub-channels nu_j = j (fs/N)/fft_len (j - fft_len for j >= fft_len/2), multiplied by the
 * coherent-dedispersion chirp exp(-2 pi i K_DM DM nu^2 / (f_c^2 (f_c + nu))) with f_c the channel's
 * sky frequency f0_f + (c - N/2) fs/N and K_DM = 4.148808e15 s Hz^2 (cold-plasma delay
 * t = K_DM DM / f^2), and transformed back (inverse FFT scaled by 1/fft_len).  Runs do not overlap
 * (each is circular).  Apply it to the output of lbf_beamform, before lbf_stokes.
 * d_vol_in, d_vol_out: device [B][F][N][P][M] cf32, 16-byte aligned; they may be the same buffer.
 * dm: dispersion measure in pc cm^-3 (finite; 0 leaves the data unchanged up to rounding).
 * fft_len: a power of two in [2, 4096] that divides M.
 * Errors: LBF_EINVAL (fft_len, dm or pointers), LBF_ESTATE, LBF_ECUDA.  Stateless; enqueued on
 * `stream`. */
lbf_status lbf_dedisperse(lbf_plan_t plan, double dm, int32_t fft_len, const void *d_vol_in, void *d_vol_out,
                          void *stream);

/* lbf_run_block with HOST buffers: the copy h_in -> d_in (in_bytes), the fused path d_in -> d_out
 * on `stream`, and the copy d_out -> h_out (out_bytes), one cudaMemcpyAsync each.  The copies run
 * on two streams of the plan, ordered by events: a block's upload starts as soon as the previous
 * block's kernels have read d_in, so it overlaps that block's beam former; `stream` waits for the
 * download before anything enqueued on it later.  h_in/h_out should be page-locked (cudaHostAlloc
 * / pinned) for the copies to be asynchronous; d_in/d_out are caller-owned device staging buffers
 * of the documented sizes, reused across calls.  Returns once the work is enqueued; h_in must stay
 * unchanged and h_out unread until `stream` has passed this call (e.g. cudaStreamSynchronize).
 * Not available for plans with LBF_FLAG_EXTERNAL_WORKSPACE (LBF_EINVAL). */
lbf_status lbf_run_block_host(lbf_plan_t plan, const void *h_in, void *h_out, void *d_in, void *d_out,
                              void *stream);

/* n consecutive blocks of the stream from HOST buffers, pipelined: the result equals n calls of
 * lbf_run_block_host (block k from h_in[k] into h_out[k], the history advancing n times).
 * Block k is uploaded into d_in0 (k even) or d_in1 (k odd), so its upload overlaps the kernels of
 * block k - 1 and waits only for block k - 2 to have read that buffer; the kernels run on a
 * stream of the plan; block k's download overlaps block k + 1's filter bank, and block k + 1's
 * first write of d_out waits for it.  Everything is ordered after the work already on `stream`,
 * and `stream` waits for the last download: once `stream` has passed the call, every h_out[k] is
 * complete and every h_in[k] may be reused.  Returns once the work is enqueued.
 * h_in, h_out: HOST arrays of n pointers (in_bytes / out_bytes each; page-locked for asynchronous
 * copies; entries may repeat).  d_in0, d_in1: distinct device buffers of in_bytes (d_in1 unused
 * and may be NULL when n == 1); d_out: device buffer of out_bytes.  All caller-owned.
 * Errors: LBF_EINVAL (n < 0, NULL arrays or entries, bad or equal device buffers, or a plan with
 * LBF_FLAG_EXTERNAL_WORKSPACE), LBF_ESTATE, LBF_ECUDA.  n == 0 does nothing. */
lbf_status lbf_run_blocks_host(lbf_plan_t plan, int32_t n, const void *const *h_in, void *const *h_out,
                               void *d_in0, void *d_in1, void *d_out, void *stream);

/* Transport of a subband range between a whole block in HOST memory and a plan that covers only
 * that range (a "chunk" plan: the same observation restricted to subbands [first_subband,
 * first_subband + F) of n_subbands_full).  Subbands are independent given their own history, so a
 * block processed as chunks gives exactly the beams of the whole block, and a serving loop can
 * upload chunk k + 1 while chunk k is filtered and beam-formed.  Each call is one asynchronous
 * strided copy on `stream` (h_in / h_out should be page-locked).
 * lbf_upload_subbands: h_in [S][n_subbands_full][T][P][2] -> d_in, the chunk's `in` block
 *   [S][F][T][P][2] (in_bytes of the chunk plan).
 * lbf_download_subbands: d_out, the chunk's `out` (Stokes [B (+1)][nS][F][N][M/Q]) or `vol`
 *   ([B][F][N][P][M]) -> the same rows of h_out, laid out for n_subbands_full subbands.
 * Errors: LBF_EINVAL (range outside the full block, NULL or non-device buffers), LBF_ESTATE,
 * LBF_ECUDA. */
lbf_status lbf_upload_subbands(lbf_plan_t chunk, const void *h_in, int32_t n_subbands_full, int32_t first_subband,
                               void *d_in, void *stream);
lbf_status lbf_download_subbands(lbf_plan_t chunk, const void *d_out, int32_t n_subbands_full, int32_t first_subband,
                                 void *h_out, void *stream);

/* Kernel timing trace (CUDA events around every kernel the plan launches).
 * lbf_trace_begin allocates event pairs for up to `max_launches` launches and starts recording;
 * lbf_trace_end synchronises on the recorded events, writes per-kernel totals to `out` and frees
 * the events.  While no trace is active the calls record nothing. */
typedef struct lbf_trace {
  int32_t n_kernels;           /* entries used in the arrays below */
  int32_t launches[16];        /* launches per kernel */
  double total_ms[16];         /* summed event time per kernel */
  char names[16][32];          /* kernel names: ppf, ppf_ct, hist_update, delay_ct, bf_few, bf_many,
                                  stokes, ppf_ct16, bf_tc, ct_to_ct16, incoherent_ct16,
                                  dedisperse, superstation */
  int32_t dropped;             /* launches not recorded because max_launches was reached */
} lbf_trace;
lbf_status lbf_trace_begin(lbf_plan_t plan, int32_t max_launches);
lbf_status lbf_trace_end(lbf_plan_t plan, lbf_trace *out);

/* Synchronises the device and reports whether a bounded device-side wait (tensor-core pipeline
 * barriers) gave up since the last call: LBF_ETIMEOUT (the results of the affected launch are
 * invalid; *code, if given, receives the role that gave up: 1 tensor-core loads, 2 MMA, 3 epilogue,
 * 4 the filter bank's input copies).  Code 5 (returned as LBF_ECUDA) means the filter bank found
 * its dynamic shared memory not 128-byte aligned for its tensor stores and wrote no output.
 * Otherwise LBF_OK.  The error word is cleared. */
lbf_status lbf_device_status(lbf_plan_t plan, int32_t *code);

/* Failure-detection test hook for the bounded device-side waits.  One-shot; the launch's output
 * is invalid afterwards, lbf_device_status reports LBF_ETIMEOUT and the context stays usable.
 *  - Tensor-core plan: the next tensor-core beam-former launch (lbf_run_block, lbf_run_block_ws,
 *    lbf_run_block_host or lbf_beamform_stokes) issues no loads from work item `item` on, so the
 *    CTA that owns that item waits on a barrier that nothing completes: the wait expires after a
 *    bounded number of polls (well under a second), the CTA records the MMA role in the plan's
 *    error word, lets its own copies and MMAs finish, frees its tensor memory and returns.
 *    item: a work item index in [0, F * 256 * ceil(B / 128)).
 *  - FP32 plan: in the next fused launch (lbf_run_block, lbf_run_block_ws, lbf_run_block_host),
 *    filter-bank CTA `item` (stream s * F + f and spectrum chunk, in [0, S * F * chunks)) issues
 *    none of its input copies; its waits for them expire, it records code 4 (the filter bank's
 *    input) and returns.  An index past the end never stalls.
 * Errors: LBF_EINVAL, LBF_ESTATE. */
lbf_status lbf_debug_stall_next(lbf_plan_t plan, int64_t item);

/* lbf_run_block without any device allocation, for callers that cannot call cudaMalloc (for
 * example a plugin whose host framework owns the device-memory budget, or a real-time ingest
 * thread that must not take the allocator's locks mid-observation).  The paper has no
 * counterpart: it is a deployment variant of the fused FP32 path.
 *
 * Processes ONE block of `cfg` as the first block of a new stream (zero history), exactly as a
 * fresh plan's lbf_run_block would (FP32 precision only): d_in is the device `in` block, d_out
 * the device `out` (Stokes) or `vol` (voltages) buffer, both caller-owned; the call enqueues its
 * work on `stream` and returns.  All other device memory -- tables, zero history and the
 * corner-turned scratch -- lives in one file-scope device array of 32 MiB that every GPU loading
 * the library holds until the process exits; the call allocates nothing (no cudaMalloc/cudaFree,
 * no allocating library routine).  Limits: S*F*T*16 bytes <= 24 MiB (e.g. S*F*T <= 1572864
 * station-samples), S*F*((L-1)N + d_max)*sample-bytes <= 4 MiB, and the weight tables
 * (about 4*F*B*S + 12*B*S bytes) <= 4 MiB; beyond them it returns LBF_ETOOBIG before touching the
 * device.  The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  The address is kept
 * for the life of the process, so the entry point must not be called on a device after
 * cudaDeviceReset of that device.  Every call shares the array and overwrites the previous call's
 * contents (the zero history is cleared on each call); calls whose device work overlaps in time
 * race on it.  The host-side staging of the tables is process-wide as well and is serialised by a
 * lock, so concurrent calls from several host threads are safe on the host side (their device
 * work still races unless it is ordered, e.g. on one stream).  The caller's buffers must hold
 * S*F*T*sample-bytes (d_in) and the Stokes or voltage output size (d_out); the C entry point
 * cannot check raw device pointers for length.  Other errors as lbf_plan/lbf_run_block:
 * LBF_EINVAL, LBF_EUNSUPPORTED, LBF_ECUDA. */
lbf_status lbf_run_block_static(const lbf_config *cfg, const void *d_in, void *d_out, void *stream);

/* ---- Batches: several observations processed together (Section 7: independent observations can
 * run in parallel as long as resources allow).  One block of every plan of
 * a batch runs as ONE persistent grouped launch per stage -- filter bank (with the delay / bandpass
 * / corner-turn epilogue), history update, beam former with its Stokes epilogue (one launch per
 * FP32 beam-former kernel in use, each at its own residency) -- instead of three launches per
 * plan; CTAs take work items from a shared counter, so uneven observations load-balance.
 * Tensor-core plans join the grouped filter bank and history update; then ONE persistent
 * tensor-core launch per class of output kind and integration length walks the work items of all
 * the class's plans (up to 32 plans per launch).  Plans of a batch must use their own scratch (no
 * LBF_FLAG_EXTERNAL_WORKSPACE), be on the current device and be in at most one active batch;
 * their history advances exactly as with lbf_run_block.  d_in[i] / d_out[i] are plan i's device
 * `in` and `out` (or `vol`) buffers. */
typedef struct lbf_batch_s *lbf_batch_t;

typedef struct lbf_batch_tuning {
  int32_t n_candidates;         /* candidates timed (4, 7 or 10) */
  int32_t spc[10];              /* spectra per filter-bank work item of each candidate; 0: the
                                   per-plan mode (each plan's own filter bank and FP32 beam former
                                   inside the batch graph, the tensor-core stage still grouped) */
  int32_t mid_variant[10];      /* beam-former choice: 0 each plan's own; 1 plans with 9..64 beams
                                   switched between the few- and many-beam kernels; 2 FP32 plans
                                   with more than 8 beams switched between 128- and 64-beam tiles */
  double ms[10];                /* mean time of one batch block per candidate */
  int32_t best_spc, best_mid_variant;
  double best_ms;
} lbf_batch_tuning;

lbf_status lbf_batch_create(const lbf_plan_t *plans, int32_t n, lbf_batch_t *out);
lbf_status lbf_batch_destroy(lbf_batch_t batch);

/* One block of every plan: grouped launches on `stream`.  Synchronises `stream` first (the
 * launch tables are staged in pinned host memory). */
lbf_status lbf_batch_run(lbf_batch_t batch, const void *const *d_in, void *const *d_out, void *stream);

/* Capture the batch block for these buffers as CUDA graphs (one per history parity) and make
 * lbf_batch_launch replay them: a whole batch block becomes a single graph launch.  Any
 * lbf_batch_run or lbf_batch_tune call drops the graphs. */
lbf_status lbf_batch_capture(lbf_batch_t batch, const void *const *d_in, void *const *d_out, void *stream);
lbf_status lbf_batch_launch(lbf_batch_t batch, void *stream);

/* Kernel launches of one batch block as the tables were last filled (by lbf_batch_run,
 * lbf_batch_capture or lbf_batch_tune): one grouped filter-bank launch per class of sample width
 * and output form, the grouped history update, one grouped FP32 beam-former launch per class of
 * beam-former kernel, output kind and CTAs per SM, one tensor-core launch per class of output kind
 * and integration length (per 32 plans), and one incoherent-beam kernel per tensor-core plan that
 * forms it.  Host only. */
lbf_status lbf_batch_launches(lbf_batch_t batch, int32_t *n_launches);

/* Autotune the batch's tile shapes on these buffers: spectra per filter-bank work item (64, 256,
 * 1024: a quarter, half or all of a stream's block) times the beam-former choice (each plan's own; for plans with 9..64 beams the few- or
 * many-beam kernel; for FP32 plans with more than 8 beams the 128- or 64-beam tile) in grouped
 * persistent launches, then the best of these as per-plan launches of the FP32 stages; each
 * candidate is timed over `reps` blocks with CUDA events, the fastest is kept.  The candidate runs use the plans'
 * histories, so every plan's stream is restarted (history zeroed) afterwards.  `out` may be NULL. */
lbf_status lbf_batch_tune(lbf_batch_t batch, const void *const *d_in, void *const *d_out, void *stream,
                          int32_t reps, lbf_batch_tuning *out);

/* ---- Measurement (roofline denominators, not a step of the paper's path).
 * The FP32 SIMT throughput of the current device, measured: kernels of independent FMA chains on
 * every SM (four 256-thread CTAs per SM, 16 chains per thread), each timed with CUDA events on
 * `stream` over `reps` launches after one warm-up, in two forms -- scalar FFMA and packed FP32x2
 * (fma.rn.f32x2) -- keeping the fastest launch of each.  The paper rates its beam-former kernel
 * against the FPU's peak (Section 4.3); this gives the GPU's peak at the clocks it runs at now.
 * Synchronous (waits for its own launches).  Errors: LBF_EINVAL (reps outside 1..100 or NULL
 * out), LBF_ECUDA. */
typedef struct lbf_alu_peak {
  int32_t sms;              /* streaming multiprocessors of the device */
  double ffma_ms;           /* fastest launch, scalar FFMA form */
  double ffma2_ms;          /* fastest launch, packed FP32x2 form */
  double ffma_tflops;       /* 2 flop per lane FMA over the fastest launch */
  double ffma2_tflops;
} lbf_alu_peak;
lbf_status lbf_measure_fp32_peak(int32_t reps, void *stream, lbf_alu_peak *out);

/* Human-readable name of a status code (static string). */
const char *lbf_status_string(lbf_status s);

/* Library version string (static). */
const char *lbf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBF_H */
