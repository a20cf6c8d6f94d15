// C-ABI layer: plan creation (host FP64 geometry, device tables and state) and the entry points
// declared in include/lbf.h.  No compute happens here; every step of the path is a kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lbf.h"
#include "lbf_internal.cuh"
#include "plan.h"

namespace {

constexpr uint32_t kMagic = lbf::kPlanMagic;
constexpr double kC = 299792458.0;         // m/s

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return nullptr;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

}  // namespace

namespace lbf {

// The filter bank's store boxes over a plane [F*N][Mt][kpad][P][32]: dims (64 halves of a K row,
// kpad rows, Mt tiles, F*N channel rows); a box is 16 spectra of one pol (32 bytes) x the two rows
// of a station x 1 tile x the 256 channels of a subband, laid out [channel][row][spectrum] in
// shared memory.
cudaError_t encode_ct16_store_map(void *map, void *base, int kpad, int M, long long fc_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t mb = (cuuint64_t)tc_tiles(M);
  const cuuint64_t dims[4] = {64, (cuuint64_t)kpad, mb, (cuuint64_t)fc_rows};
  const cuuint64_t strides[3] = {128, (cuuint64_t)kpad * 128, mb * kpad * 128};
  const cuuint32_t box[4] = {16, 2, 1, (cuuint32_t)kN};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  CUresult r = encode(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, base, dims, strides, box,
                      elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The FP32 corner turn as FP32 elements: dims (2M re/im values of a (station, pol) row, P, S,
// F*N channel rows); a box is 16 spectra (128 bytes) x 1 x 1 x nch channels, laid out
// [channel][spectrum] in shared memory.  The strides are multiples of 16 bytes only for even M.
cudaError_t encode_ct32_store_map(void *map, void *base, int S, int M, long long fc_rows, int nch) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  if (M % 2 != 0 || nch < 1 || nch > kN) return cudaErrorInvalidValue;
  const cuuint64_t row = (cuuint64_t)M * 8;   // bytes of one (station, pol) row
  const cuuint64_t dims[4] = {(cuuint64_t)M * 2, 2, (cuuint64_t)S, (cuuint64_t)fc_rows};
  const cuuint64_t strides[3] = {row, 2 * row, 2 * row * (cuuint64_t)S};
  const cuuint32_t box[4] = {32, 1, 1, (cuuint32_t)nch};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  CUresult r = encode(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box,
                      elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace lbf

namespace {

// Plane-wave geometric delay, evaluated left to right with no contraction so that the integer
// shift decisions are reproducible: -(x l + y m + z n) / c with n = sqrt(max(0, 1 - l^2 - m^2)).
double plane_wave_delay(const double *xyz, double l, double m) {
  double nn = 1.0 - l * l - m * m;
  const double n = std::sqrt(nn > 0.0 ? nn : 0.0);
  const double dot = xyz[0] * l + xyz[1] * m + xyz[2] * n;
  return -dot / kC;
}

double round_half_away(double x) {
  const double a = std::floor(std::fabs(x) + 0.5);
  return x < 0 ? -a : (x > 0 ? a : 0.0);
}

bool is_pow2_upto32(int q) { return q == 1 || q == 2 || q == 4 || q == 8 || q == 16 || q == 32; }

lbf_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LBF_OK;
  if (e == cudaErrorMemoryAllocation) return LBF_ENOMEM;
  return LBF_ECUDA;
}

template <typename T>
cudaError_t upload(T **dst, const T *src, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  return src ? cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice) : cudaSuccess;
}

void release(lbf_plan_s *p) {
  cudaFree(p->taps); cudaFree(p->twiddle); cudaFree(p->bandpass); cudaFree(p->dshift);
  cudaFree(p->tau); cudaFree(p->resid); cudaFree(p->f0); cudaFree(p->dtau);
  cudaFree(p->hist[0]); cudaFree(p->hist[1]); cudaFree(p->ws);
  cudaFree(p->phase0); cudaFree(p->step); cudaFree(p->phase0g); cudaFree(p->stepg);
  cudaFree(p->ct16[0]); cudaFree(p->d_err); cudaFree(p->ss_members); cudaFree(p->ss_offs);
  if (p->h2d) cudaStreamDestroy(p->h2d);
  if (p->d2h) cudaStreamDestroy(p->d2h);
  if (p->cs) cudaStreamDestroy(p->cs);
  for (cudaEvent_t ev : {p->ev_in_free, p->ev_in_ready, p->ev_out_ready, p->ev_out_done, p->ev_start,
                         p->ev_in_free2[0], p->ev_in_free2[1]})
    if (ev) cudaEventDestroy(ev);
}

lbf_status validate(const lbf_config *c) {
  if (!c) return LBF_EINVAL;
  if (c->n_stations < 1 || c->n_subbands < 1 || c->n_beams < 1) return LBF_EINVAL;
  if (c->n_channels < 1 || c->n_taps < 1) return LBF_EINVAL;
  if (c->block_samples < 0 || c->block_samples % c->n_channels != 0) return LBF_EINVAL;
  if (c->sample_bits != 16 && c->sample_bits != 8) return LBF_EINVAL;
  if (c->output != LBF_VOLTAGES && c->output != LBF_STOKES_I && c->output != LBF_STOKES_IQUV) return LBF_EINVAL;
  if (c->precision != LBF_FP32 && c->precision != LBF_FP16_TC && c->precision != LBF_FP16_TC2) return LBF_EINVAL;
  if (c->bf_variant < LBF_BF_AUTO || c->bf_variant > LBF_BF_MANY64) return LBF_EINVAL;
  if ((c->flags & ~(LBF_FLAG_EXTERNAL_WORKSPACE | LBF_FLAG_INCOHERENT_BEAM)) != 0) return LBF_EINVAL;
  if ((c->flags & LBF_FLAG_INCOHERENT_BEAM) && c->output == LBF_VOLTAGES) return LBF_EINVAL;
  if (!is_pow2_upto32(c->int_factor)) return LBF_EINVAL;
  const int M = c->block_samples / c->n_channels;
  if (c->output != LBF_VOLTAGES && M % c->int_factor != 0) return LBF_EINVAL;
  if (!(c->sample_rate_hz > 0.0) || !std::isfinite(c->sample_rate_hz)) return LBF_EINVAL;
  if (!std::isfinite(c->phase_centre_l) || !std::isfinite(c->phase_centre_m)) return LBF_EINVAL;
  if (!c->station_xyz_m || !c->subband_centre_hz || !c->beam_dlm || !c->fir_taps) return LBF_EINVAL;
  for (int i = 0; i < 3 * c->n_stations; ++i) if (!std::isfinite(c->station_xyz_m[i])) return LBF_EINVAL;
  for (int i = 0; i < c->n_subbands; ++i) if (!std::isfinite(c->subband_centre_hz[i])) return LBF_EINVAL;
  for (int i = 0; i < 2 * c->n_beams; ++i) if (!std::isfinite(c->beam_dlm[i])) return LBF_EINVAL;
  if (c->n_channels != lbf::kN || c->n_taps != lbf::kL) return LBF_EUNSUPPORTED;
  if (c->precision != LBF_FP32 && c->n_stations > lbf::tc_max_stations()) return LBF_EUNSUPPORTED;
  if ((c->bf_variant == LBF_BF_MANY || c->bf_variant == LBF_BF_MANY64) && c->precision == LBF_FP32 &&
      c->n_stations > lbf::many_beam_max_stations())
    return LBF_EUNSUPPORTED;
  // index arithmetic: per-plan sizes must keep grid dimensions in range
  const long long ctas = (long long)c->n_subbands * lbf::kN * ((c->n_beams + 7) / 8);
  if (ctas >= (1LL << 31)) return LBF_EUNSUPPORTED;
  return LBF_OK;
}

bool valid_plan(lbf_plan_t p) { return p && p->magic == kMagic; }

// TMA descriptor of one FP16 plane [F*N][Mt][kpad][P][32] (Mt = tc_tiles(M), an even number of
// tiles of 32 spectra; a tile's kpad K rows hold the two pols side by side, 128 bytes per row, so
// a tile is one contiguous kpad x 128-byte region): boxes of two tiles, 128-byte swizzle.
cudaError_t encode_ct16_map(CUtensorMap *map, void *base, int kpad, int M, long long fc_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t mb = (cuuint64_t)lbf::tc_tiles(M);
  const cuuint64_t dims[4] = {64, (cuuint64_t)kpad, mb, (cuuint64_t)fc_rows};
  const cuuint64_t strides[3] = {128, (cuuint64_t)kpad * 128, mb * kpad * 128};
  const cuuint32_t box[4] = {64, (cuuint32_t)kpad, 2, 1};   // two tiles: all K rows of 64 spectra
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, base, dims, strides, box, elem,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

lbf::Ct16Out ct16_out(lbf_plan_t p) {
  lbf::Ct16Out o;
  o.hi = p->ct16[0];
  o.lo = p->planes > 1 ? static_cast<unsigned char *>(p->ct16[0]) + p->ct16_bytes : nullptr;
  o.kpad = p->kpad;
  return o;
}

// Descriptors of the FP16 planes of a tensor-core scratch at `ws` (hi, then lo).
cudaError_t encode_planes(lbf_plan_t p, void *ws, CUtensorMap *maps) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < p->planes && e == cudaSuccess; ++i)
    e = encode_ct16_map(&maps[i], static_cast<unsigned char *>(ws) + i * p->ct16_bytes, p->kpad, p->M,
                        (long long)p->F * p->N);
  return e;
}

// Device pointer check (host-only query): rejects host pointers before any launch.
bool device_ptr(const void *p, size_t align) {
  if (!p || (reinterpret_cast<uintptr_t>(p) % align) != 0) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

lbf_status check_call(lbf_plan_t p) {
  if (!valid_plan(p)) return LBF_ESTATE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBF_ECUDA;
  if (dev != p->device) return LBF_ESTATE;
  return LBF_OK;
}

enum KernelId { K_PPF = 0, K_PPF_CT, K_HIST, K_DELAY, K_BF_FEW, K_BF_MANY, K_STOKES, K_PPF_CT16, K_BF_TC,
                K_CT16, K_INC16, K_DEDISP, K_SS, K_BF_MANY64, K_COUNT };
static_assert(K_COUNT <= 16, "lbf_trace holds 16 kernels");
const char *const kKernelNames[K_COUNT] = {"ppf", "ppf_ct", "hist_update", "delay_ct", "bf_few", "bf_many",
                                           "stokes", "ppf_ct16", "bf_tc", "ct_to_ct16", "incoherent_ct16",
                                           "dedisperse", "superstation", "bf_many64"};

// Launch through `fn`, bracketed by trace events when a trace is active.
template <typename Fn>
cudaError_t traced(lbf_plan_t p, int kernel, cudaStream_t st, Fn &&fn) {
  if (!p->tracing) return fn();
  if (p->trace_used >= p->trace.size()) {
    ++p->trace_dropped;
    return fn();
  }
  auto &slot = p->trace[p->trace_used++];
  slot.kernel = kernel;
  cudaError_t e = cudaEventRecord(slot.a, st);
  if (e != cudaSuccess) return e;
  e = fn();
  if (e != cudaSuccess) return e;
  return cudaEventRecord(slot.b, st);
}

void trace_free(lbf_plan_t p) {
  for (auto &s : p->trace) { cudaEventDestroy(s.a); cudaEventDestroy(s.b); }
  p->trace.clear();
  p->trace_used = 0;
  p->trace_dropped = 0;
  p->tracing = false;
}

int bf_kernel_id(lbf_plan_t p) { return p->variant == 1 ? K_BF_FEW : p->variant == 3 ? K_BF_MANY64 : K_BF_MANY; }

// The fused path on device buffers (a1-a7).  `ws` is the scratch of this call: the FP32
// corner-turned block, or the FP16 planes of a tensor-core plan (with `maps` their descriptors).
// input_read (optional) is recorded once d_in has been read; the first kernel that writes d_out
// waits for out_free (optional).
cudaError_t run_block_device(lbf_plan_t p, const void *d_in, void *d_out, void *ws, const CUtensorMap *maps,
                             cudaStream_t st, cudaEvent_t input_read = nullptr, cudaEvent_t out_free = nullptr) {
  lbf::Geometry g = p->geometry();
  const void *h = p->hist[p->cur];
  void *nh = p->hist[p->cur ^ 1];
  if (p->tc) {
    // the filter bank writes the FP16 planes before the delay phase and bandpass; the
    // tensor-core weights carry both (folded tables), the incoherent beam the bandpass
    g.ct16_raw = 1;
    lbf::Ct16Out o;
    o.hi = ws;
    o.lo = p->planes > 1 ? static_cast<unsigned char *>(ws) + p->ct16_bytes : nullptr;
    o.kpad = p->kpad;
    cudaError_t e = traced(p, K_PPF_CT16, st, [&] { return lbf::launch_ppf(g, p->bits, d_in, h, nullptr, nullptr, st, &o); });
    if (e == cudaSuccess) e = traced(p, K_HIST, st, [&] { return lbf::launch_hist_update(g, p->bits, d_in, h, nh, st); });
    if (e == cudaSuccess && input_read) e = cudaEventRecord(input_read, st);
    if (e == cudaSuccess && out_free) e = cudaStreamWaitEvent(st, out_free, 0);
    if (e != cudaSuccess) return e;
    p->cur ^= 1;
    if (p->inc) {
      e = traced(p, K_INC16, st, [&] { return lbf::launch_incoherent_ct16(g, p->out_kind, o, (float *)d_out, st); });
      if (e != cudaSuccess) return e;
    }
    return traced(p, K_BF_TC, st, [&] {
      const long long stall = p->stall_item;
      p->stall_item = -1;
      return lbf::launch_bf_tc(g, p->out_kind, &maps[0], &maps[1], (float *)d_out, p->d_err, st, stall); });
  }
  float2 *ct = static_cast<float2 *>(ws);
  g.ppf_stall = p->stall_item;   // failure-detection test hook (one-shot)
  p->stall_item = -1;
  cudaError_t e = traced(p, K_PPF_CT, st, [&] { return lbf::launch_ppf(g, p->bits, d_in, h, nullptr, ct, st); });
  if (e == cudaSuccess) e = traced(p, K_HIST, st, [&] { return lbf::launch_hist_update(g, p->bits, d_in, h, nh, st); });
  if (e == cudaSuccess && input_read) e = cudaEventRecord(input_read, st);
  if (e == cudaSuccess && out_free) e = cudaStreamWaitEvent(st, out_free, 0);
  if (e != cudaSuccess) return e;
  p->cur ^= 1;
  return traced(p, bf_kernel_id(p), st,
                [&] { return lbf::launch_beamform(g, p->variant, p->out_kind, ct, d_out, st); });
}

// The plan's own scratch (tensor-core planes are contiguous: hi then lo).
void *own_ws(lbf_plan_t p) { return p->tc ? p->ct16[0] : static_cast<void *>(p->ws); }

}  // namespace

extern "C" {

const char *lbf_status_string(lbf_status s) {
  switch (s) {
    case LBF_OK: return "LBF_OK";
    case LBF_EINVAL: return "LBF_EINVAL: invalid argument";
    case LBF_ENOMEM: return "LBF_ENOMEM: device allocation failed";
    case LBF_ECUDA: return "LBF_ECUDA: CUDA runtime error";
    case LBF_ESTATE: return "LBF_ESTATE: plan in an unusable state";
    case LBF_ETIMEOUT: return "LBF_ETIMEOUT: device wait timed out";
    case LBF_EBUSY: return "LBF_EBUSY: resource busy";
    case LBF_EUNSUPPORTED: return "LBF_EUNSUPPORTED: not supported by this library";
    case LBF_ETOOBIG: return "LBF_ETOOBIG: exceeds the fixed scratch of the allocation-free entry point";
  }
  return "LBF_?: unknown status";
}

const char *lbf_version(void) { return "lbf 0.1 (sm_103a)"; }

lbf_status lbf_plan(const lbf_config *cfg, lbf_plan_t *out) {
  if (!out) return LBF_EINVAL;
  *out = nullptr;
  lbf_status v = validate(cfg);
  if (v != LBF_OK) return v;
  lbf_plan_s *p = new (std::nothrow) lbf_plan_s();
  if (!p) return LBF_ENOMEM;
  p->S = cfg->n_stations; p->F = cfg->n_subbands; p->N = cfg->n_channels; p->L = cfg->n_taps;
  p->B = cfg->n_beams; p->T = cfg->block_samples; p->M = p->T / p->N; p->Q = cfg->int_factor;
  p->bits = cfg->sample_bits; p->fs = cfg->sample_rate_hz; p->word = p->bits == 16 ? 8 : 4;
  p->out_kind = cfg->output == LBF_STOKES_I ? lbf::OUT_STOKES_I
              : cfg->output == LBF_STOKES_IQUV ? lbf::OUT_STOKES_IQUV : lbf::OUT_VOLTAGES;
  p->nS = cfg->output == LBF_STOKES_I ? 1 : cfg->output == LBF_STOKES_IQUV ? 4 : 0;
  if (cfg->bf_variant == LBF_BF_AUTO)
    p->variant = lbf::auto_bf_variant(p->B, p->S);
  else
    p->variant = cfg->bf_variant;
  // Tensor cores only where the beam count makes the beam former a dense contraction: a
  // tensor-core plan with few beams (AUTO and B <= 8, or FEW asked for) runs the bandwidth-bound
  // few-beam kernel on the FP32 corner-turned block instead (Section 4.3: few beams stream the
  // stations once; many beams reuse each station sample across beams).
  const bool tc_asked = cfg->precision != LBF_FP32;
  const bool tc_few = tc_asked && (cfg->bf_variant == LBF_BF_FEW || (cfg->bf_variant == LBF_BF_AUTO && p->B <= 8));
  if (tc_few) p->variant = 1;

  // ---- FP64 geometry on the host (Section 3: delays, integer shifts, beam delay differences)
  const double ts = 1.0 / p->fs;
  const double l0 = cfg->phase_centre_l, m0 = cfg->phase_centre_m;
  std::vector<double> tau(p->S), resid(p->S), dtau((size_t)p->B * p->S);
  p->n_shift.resize(p->S);
  p->d_shift.resize(p->S);
  long long nmax = 0;
  for (int s = 0; s < p->S; ++s) {
    tau[s] = plane_wave_delay(cfg->station_xyz_m + 3 * s, l0, m0);
    const double n = round_half_away(tau[s] / ts);
    if (!(std::fabs(n) < 1e6)) { delete p; return LBF_EUNSUPPORTED; }
    p->n_shift[s] = (int32_t)n;
    nmax = (s == 0 || p->n_shift[s] > nmax) ? p->n_shift[s] : nmax;
  }
  for (int s = 0; s < p->S; ++s) {
    p->d_shift[s] = (int32_t)(nmax - p->n_shift[s]);
    p->d_max = p->d_shift[s] > p->d_max ? p->d_shift[s] : p->d_max;
    resid[s] = tau[s] - (double)p->n_shift[s] * ts;
  }
  for (int b = 0; b < p->B; ++b)
    for (int s = 0; s < p->S; ++s)
      dtau[(size_t)b * p->S + s] =
          plane_wave_delay(cfg->station_xyz_m + 3 * s, l0 + cfg->beam_dlm[2 * b], m0 + cfg->beam_dlm[2 * b + 1]) - tau[s];
  p->H = (p->L - 1) * p->N + p->d_max;

  std::vector<float2> tw(p->N);
  for (int n = 0; n < p->N; ++n) {
    const double a = 2.0 * M_PI * (double)n / (double)p->N;
    tw[n] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  std::vector<float> bp(p->N, 1.0f);
  if (cfg->bandpass) std::memcpy(bp.data(), cfg->bandpass, sizeof(float) * p->N);

  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = upload(&p->taps, cfg->fir_taps, (size_t)p->L * p->N);
  if (e == cudaSuccess) e = upload(&p->twiddle, tw.data(), tw.size());
  if (e == cudaSuccess) e = upload(&p->bandpass, bp.data(), bp.size());
  if (e == cudaSuccess) e = upload(&p->dshift, (const int *)p->d_shift.data(), (size_t)p->S);
  if (e == cudaSuccess) e = upload(&p->tau, tau.data(), tau.size());
  if (e == cudaSuccess) e = upload(&p->resid, resid.data(), resid.size());
  if (e == cudaSuccess) e = upload(&p->f0, cfg->subband_centre_hz, (size_t)p->F);
  if (e == cudaSuccess) e = upload(&p->dtau, dtau.data(), dtau.size());
  if (e == cudaSuccess) e = upload<float>(&p->phase0, nullptr, (size_t)p->F * p->B * p->S);
  if (e == cudaSuccess) e = upload<float>(&p->step, nullptr, (size_t)p->B * p->S);
  if (e == cudaSuccess) e = lbf::launch_phase_tables(p->F, p->B, p->S, p->fs, p->f0, p->dtau, p->phase0, p->step, 0);
  p->hist_bytes = (size_t)p->S * p->F * p->H * p->word;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMalloc(&p->hist[i], p->hist_bytes ? p->hist_bytes : 16);
    if (e == cudaSuccess) e = cudaMemset(p->hist[i], 0, p->hist_bytes ? p->hist_bytes : 16);
  }
  p->tc = tc_asked && !tc_few;
  p->tc_wlo = cfg->precision == LBF_FP16_TC2 ? 0 : 1;
  if (p->tc) {   // weight tables with the delay compensation folded in, for the fused path
    if (e == cudaSuccess) e = upload<float>(&p->phase0g, nullptr, (size_t)p->F * p->B * p->S);
    if (e == cudaSuccess) e = upload<float>(&p->stepg, nullptr, (size_t)p->B * p->S);
    if (e == cudaSuccess)
      e = lbf::launch_phase_tables(p->F, p->B, p->S, p->fs, p->f0, p->dtau, p->phase0g, p->stepg, 0, p->tau,
                                   p->resid);
  }
  p->external_ws = (cfg->flags & LBF_FLAG_EXTERNAL_WORKSPACE) != 0;
  p->inc = (cfg->flags & LBF_FLAG_INCOHERENT_BEAM) ? 1 : 0;
  if (e == cudaSuccess) e = cudaMalloc((void **)&p->ss_members, sizeof(int) * p->S);
  if (e == cudaSuccess) e = cudaMalloc((void **)&p->ss_offs, sizeof(int) * (p->S + 1));
  if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (p->tc) {
    // FP16 planes [F*N][Mb][kpad][P][32], hi then lo in one buffer; pad rows k >= 2S and pad
    // spectra m >= M stay zero.  Both sample widths keep a lo plane: an 8-bit sample is exact in
    // FP16, but its filtered, delay-corrected spectrum is not, and a beam summed with cancellation
    // magnifies that rounding past 1e-3 on Stokes I.
    p->kpad = lbf::tc_kpad(p->S);
    p->planes = 2;
    p->ct16_bytes = (size_t)p->F * p->N * p->kpad * lbf::tc_tiles(p->M) * 64 * 2;
    p->ws_need = p->planes * p->ct16_bytes;
    if (!p->external_ws && e == cudaSuccess) {
      e = cudaMalloc(&p->ct16[0], p->ws_need ? p->ws_need : 16);
      if (e == cudaSuccess) e = cudaMemset(p->ct16[0], 0, p->ws_need ? p->ws_need : 16);
      if (e == cudaSuccess && p->M > 0) e = encode_planes(p, p->ct16[0], p->tmap);
    }
  } else {
    p->ws_need = (size_t)p->F * p->N * p->S * lbf::kP * p->M * sizeof(float2);
  }
  // FP32 corner-turned scratch of FP32 plans (unless the caller provides it per call)
  p->ws_bytes = (p->tc || p->external_ws) ? 0 : p->ws_need;
  if (e == cudaSuccess) e = cudaMalloc((void **)&p->ws, p->ws_bytes ? p->ws_bytes : 16);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    release(p);
    delete p;
    cudaGetLastError();
    return cuda_status(e);
  }
  *out = p;
  return LBF_OK;
}

lbf_status lbf_plan_destroy(lbf_plan_t p) {
  if (!p) return LBF_OK;
  if (!valid_plan(p)) return LBF_ESTATE;
  cudaDeviceSynchronize();
  trace_free(p);
  release(p);
  p->magic = 0;
  delete p;
  return LBF_OK;
}

lbf_status lbf_plan_dims(lbf_plan_t p, lbf_dims *d) {
  if (!valid_plan(p)) return LBF_ESTATE;
  if (!d) return LBF_EINVAL;
  std::memset(d, 0, sizeof(*d));
  d->n_stations = p->S; d->n_subbands = p->F; d->n_channels = p->N; d->n_taps = p->L;
  d->n_beams = p->B; d->block_samples = p->T; d->int_factor = p->Q; d->n_spectra = p->M;
  d->n_stokes = p->nS; d->d_max = p->d_max; d->history_samples = p->H;
  d->bf_kernel = p->tc ? 3 : p->variant == 3 ? 4 : p->variant;
  const size_t cplx = (size_t)p->S * p->F * lbf::kP * p->T * sizeof(float2);
  d->in_bytes = (size_t)p->S * p->F * p->T * p->word;
  d->chan_bytes = cplx;
  d->ct_bytes = cplx;
  d->vol_bytes = (size_t)p->B * p->F * lbf::kP * p->T * sizeof(float2);
  d->stokes_bytes = p->nS ? (size_t)(p->B + p->inc) * p->nS * p->F * p->N * (p->M / p->Q) * sizeof(float) : 0;
  d->out_bytes = p->nS ? d->stokes_bytes : d->vol_bytes;
  d->workspace_bytes = p->ws_need;
  d->plan_bytes = 2 * p->hist_bytes + (p->external_ws ? 0 : p->ws_need) +
                  sizeof(float) * ((size_t)p->F * p->B * p->S + (size_t)p->B * p->S + (size_t)p->L * p->N + p->N) +
                  sizeof(double) * ((size_t)p->B * p->S + 2 * (size_t)p->S + p->F) + sizeof(float2) * p->N;
  return LBF_OK;
}

lbf_status lbf_plan_shifts(lbf_plan_t p, int32_t *n_shift, int32_t *d_shift) {
  if (!valid_plan(p)) return LBF_ESTATE;
  if (n_shift) std::memcpy(n_shift, p->n_shift.data(), sizeof(int32_t) * p->S);
  if (d_shift) std::memcpy(d_shift, p->d_shift.data(), sizeof(int32_t) * p->S);
  return LBF_OK;
}

lbf_status lbf_reset_state(lbf_plan_t p, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < 2; ++i) {
    cudaError_t e = cudaMemsetAsync(p->hist[i], 0, p->hist_bytes ? p->hist_bytes : 16, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  p->cur = 0;
  return LBF_OK;
}

lbf_status lbf_ppf(lbf_plan_t p, const void *d_in, void *d_chan, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_in, p->word) || !device_ptr(d_chan, 8)) return LBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const lbf::Geometry g = p->geometry();
  const void *h = p->hist[p->cur];
  void *nh = p->hist[p->cur ^ 1];
  cudaError_t e = traced(p, K_PPF, st, [&] { return lbf::launch_ppf(g, p->bits, d_in, h, (float2 *)d_chan, nullptr, st); });
  if (e == cudaSuccess) e = traced(p, K_HIST, st, [&] { return lbf::launch_hist_update(g, p->bits, d_in, h, nh, st); });
  if (e != cudaSuccess) return cuda_status(e);
  p->cur ^= 1;
  return LBF_OK;
}

lbf_status lbf_delay_correct(lbf_plan_t p, const void *d_chan, void *d_ct, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_chan, 8) || !device_ptr(d_ct, 8)) return LBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const lbf::Geometry g = p->geometry();
  return cuda_status(traced(p, K_DELAY, st, [&] { return lbf::launch_delay_ct(g, (const float2 *)d_chan, (float2 *)d_ct, st); }));
}

lbf_status lbf_beamform(lbf_plan_t p, const void *d_ct, void *d_vol, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_ct, 8) || !device_ptr(d_vol, 8)) return LBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const lbf::Geometry g = p->geometry();
  if (p->tc) {   // the tensor-core beam former writing voltages, from the plan's FP16 scratch
    if (p->external_ws) return LBF_EUNSUPPORTED;
    const lbf::Ct16Out o = ct16_out(p);
    cudaError_t e = traced(p, K_CT16, st, [&] { return lbf::launch_ct_to_ct16(g, (const float2 *)d_ct, o, st); });
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(traced(p, K_BF_TC, st, [&] {
      const long long stall = p->stall_item;
      p->stall_item = -1;
      return lbf::launch_bf_tc(g, lbf::OUT_VOLTAGES, &p->tmap[0], &p->tmap[1], static_cast<float *>(d_vol), p->d_err,
                               st, stall); }));
  }
  return cuda_status(traced(p, bf_kernel_id(p), st, [&] {
    return lbf::launch_beamform(g, p->variant, lbf::OUT_VOLTAGES, (const float2 *)d_ct, d_vol, st); }));
}

lbf_status lbf_beamform_stokes(lbf_plan_t p, const void *d_ct, float *d_out, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (p->nS == 0) return LBF_EINVAL;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_ct, 8) || !device_ptr(d_out, 4)) return LBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const lbf::Geometry g = p->geometry();
  if (p->tc) {
    if (p->external_ws) return LBF_EUNSUPPORTED;
    const lbf::Ct16Out o = ct16_out(p);
    cudaError_t e = traced(p, K_CT16, st, [&] { return lbf::launch_ct_to_ct16(g, (const float2 *)d_ct, o, st); });
    if (e == cudaSuccess && p->inc)
      e = traced(p, K_INC16, st, [&] { return lbf::launch_incoherent_ct16(g, p->out_kind, o, d_out, st); });
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(traced(p, K_BF_TC, st, [&] {
      const long long stall = p->stall_item;
      p->stall_item = -1;
      return lbf::launch_bf_tc(g, p->out_kind, &p->tmap[0], &p->tmap[1], d_out, p->d_err, st, stall); }));
  }
  return cuda_status(traced(p, bf_kernel_id(p), st, [&] {
    return lbf::launch_beamform(g, p->variant, p->out_kind, (const float2 *)d_ct, d_out, st); }));
}

lbf_status lbf_stokes(lbf_plan_t p, const void *d_vol, float *d_out, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (p->nS == 0) return LBF_EINVAL;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_vol, 8) || !device_ptr(d_out, 4)) return LBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const lbf::Geometry g = p->geometry();
  return cuda_status(traced(p, K_STOKES, st, [&] { return lbf::launch_stokes(g, p->out_kind, (const float2 *)d_vol, d_out, st); }));
}

lbf_status lbf_run_block(lbf_plan_t p, const void *d_in, void *d_out, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (p->M == 0) return LBF_OK;
  if (p->external_ws) return LBF_EINVAL;
  if (!device_ptr(d_in, p->word) || !device_ptr(d_out, p->nS ? 4 : 8)) return LBF_EINVAL;
  return cuda_status(run_block_device(p, d_in, d_out, own_ws(p), p->tmap, (cudaStream_t)stream));
}

lbf_status lbf_run_block_ws(lbf_plan_t p, const void *d_in, void *d_out, void *d_ws, size_t ws_bytes,
                            void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_in, p->word) || !device_ptr(d_out, p->nS ? 4 : 8)) return LBF_EINVAL;
  if (ws_bytes < p->ws_need || !device_ptr(d_ws, 256)) return LBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  CUtensorMap maps[2];
  if (p->tc) {
    cudaError_t e = encode_planes(p, d_ws, maps);
    // pad rows k in [2S, kpad) of each (subband, channel, spectrum block) must read as zero
    const size_t row = 128;   // bytes of one K row
    const size_t blocks = (size_t)p->F * p->N * lbf::tc_tiles(p->M);
    for (int i = 0; i < p->planes && e == cudaSuccess && p->kpad > 2 * p->S; ++i)
      e = cudaMemset2DAsync(static_cast<unsigned char *>(d_ws) + i * p->ct16_bytes + 2 * p->S * row,
                            p->kpad * row, 0, (p->kpad - 2 * p->S) * row, blocks, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return cuda_status(run_block_device(p, d_in, d_out, d_ws, maps, st));
}

lbf_status lbf_run_block_host(lbf_plan_t p, const void *h_in, void *h_out, void *d_in, void *d_out,
                              void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (p->M == 0) return LBF_OK;
  if (!h_in || !h_out || p->external_ws) return LBF_EINVAL;
  if (!device_ptr(d_in, p->word) || !device_ptr(d_out, p->nS ? 4 : 8)) return LBF_EINVAL;
  lbf_dims d;
  lbf_plan_dims(p, &d);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!p->h2d) {   // first call: the plan's copy streams and events
    e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&p->ev_in_free, &p->ev_in_ready, &p->ev_out_ready, &p->ev_out_done})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
  }
  // upload once the previous block's kernels have read d_in (its history update), so that the
  // upload overlaps that block's beam former
  e = cudaStreamWaitEvent(p->h2d, p->ev_in_free, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_in, h_in, d.in_bytes, cudaMemcpyHostToDevice, p->h2d);
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_in_ready, p->h2d);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ev_in_ready, 0);
  if (e == cudaSuccess) e = run_block_device(p, d_in, d_out, own_ws(p), p->tmap, st, p->ev_in_free);
  // download on its own stream; `stream` then waits for it, so later work on `stream` (and the
  // next block's kernels, which rewrite d_out) follow the copy
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_out_ready, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, p->ev_out_ready, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_out, d.out_bytes, cudaMemcpyDeviceToHost, p->d2h);
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_out_done, p->d2h);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ev_out_done, 0);
  return cuda_status(e);
}

lbf_status lbf_run_blocks_host(lbf_plan_t p, int32_t n, const void *const *h_in, void *const *h_out, void *d_in0,
                               void *d_in1, void *d_out, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (n < 0 || (n > 0 && (!h_in || !h_out)) || p->external_ws) return LBF_EINVAL;
  if (n == 0 || p->M == 0) return LBF_OK;
  for (int k = 0; k < n; ++k)
    if (!h_in[k] || !h_out[k]) return LBF_EINVAL;
  void *const din[2] = {d_in0, d_in1};
  if (!device_ptr(d_in0, p->word) || !device_ptr(d_out, p->nS ? 4 : 8)) return LBF_EINVAL;
  if (n > 1 && (!device_ptr(d_in1, p->word) || d_in1 == d_in0)) return LBF_EINVAL;
  lbf_dims d;
  lbf_plan_dims(p, &d);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!p->h2d) {
    e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&p->ev_in_free, &p->ev_in_ready, &p->ev_out_ready, &p->ev_out_done})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (!p->cs) {
    e = cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&p->ev_start, &p->ev_in_free2[0], &p->ev_in_free2[1]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
  }
  // everything after the work already on `stream` (and after this plan's earlier host calls,
  // which `stream` waits for)
  e = cudaEventRecord(p->ev_start, st);
  for (cudaStream_t q : {p->h2d, p->cs, p->d2h})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q, p->ev_start, 0);
  // the input buffers have no pending reads from an earlier call (those finished before ev_start)
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventRecord(p->ev_in_free2[i], p->cs);
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_out_done, p->d2h);
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    void *di = din[k & 1];
    // upload block k into its buffer once block k - 2 (the buffer's last reader) has read it
    e = cudaStreamWaitEvent(p->h2d, p->ev_in_free2[k & 1], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(di, h_in[k], d.in_bytes, cudaMemcpyHostToDevice, p->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_in_ready, p->h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->cs, p->ev_in_ready, 0);
    // kernels of block k; its first write of d_out waits for block k - 1's download
    if (e == cudaSuccess) e = run_block_device(p, di, d_out, own_ws(p), p->tmap, p->cs, p->ev_in_free2[k & 1],
                                               p->ev_out_done);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_out_ready, p->cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, p->ev_out_ready, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out[k], d_out, d.out_bytes, cudaMemcpyDeviceToHost, p->d2h);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_out_done, p->d2h);
  }
  // a later lbf_run_block_host upload waits for these kernels' reads; `stream` passes this call
  // once the last download (and so every kernel and copy) is done
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_in_free, p->cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ev_out_done, 0);
  return cuda_status(e);
}

lbf_status lbf_upload_subbands(lbf_plan_t p, const void *h_in, int32_t n_subbands_full, int32_t first_subband,
                               void *d_in, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (!h_in || n_subbands_full < p->F || first_subband < 0 || first_subband > n_subbands_full - p->F) return LBF_EINVAL;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_in, p->word)) return LBF_EINVAL;
  // rows: stations; a row of the full block holds n_subbands_full streams, the chunk's p->F of them
  const size_t stream_bytes = (size_t)p->T * p->word;
  const unsigned char *src = static_cast<const unsigned char *>(h_in) + (size_t)first_subband * stream_bytes;
  return cuda_status(cudaMemcpy2DAsync(d_in, (size_t)p->F * stream_bytes, src, (size_t)n_subbands_full * stream_bytes,
                                       (size_t)p->F * stream_bytes, (size_t)p->S, cudaMemcpyHostToDevice,
                                       (cudaStream_t)stream));
}

lbf_status lbf_download_subbands(lbf_plan_t p, const void *d_out, int32_t n_subbands_full, int32_t first_subband,
                                 void *h_out, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (!h_out || n_subbands_full < p->F || first_subband < 0 || first_subband > n_subbands_full - p->F) return LBF_EINVAL;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_out, p->nS ? 4 : 8)) return LBF_EINVAL;
  // rows: (beam, Stokes parameter) of [B (+1)][nS][F][N][M/Q], or beams of [B][F][N][P][M]
  const size_t rows = p->nS ? (size_t)(p->B + p->inc) * p->nS : (size_t)p->B;
  const size_t sub_bytes = p->nS ? (size_t)p->N * (p->M / p->Q) * sizeof(float) : (size_t)p->N * lbf::kP * p->M * sizeof(float2);
  unsigned char *dst = static_cast<unsigned char *>(h_out) + (size_t)first_subband * sub_bytes;
  return cuda_status(cudaMemcpy2DAsync(dst, (size_t)n_subbands_full * sub_bytes, d_out, (size_t)p->F * sub_bytes,
                                       (size_t)p->F * sub_bytes, rows, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
}

lbf_status lbf_dedisperse(lbf_plan_t p, double dm, int32_t fft_len, const void *d_vol_in, void *d_vol_out,
                          void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (fft_len < 2 || fft_len > 4096 || (fft_len & (fft_len - 1)) != 0 || !std::isfinite(dm)) return LBF_EINVAL;
  if (p->M % fft_len != 0) return LBF_EINVAL;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_vol_in, 16) || !device_ptr(d_vol_out, 16)) return LBF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const lbf::Geometry g = p->geometry();
  return cuda_status(traced(p, K_DEDISP, st, [&] {
    return lbf::launch_dedisperse(g, dm, fft_len, static_cast<const float2 *>(d_vol_in), static_cast<float2 *>(d_vol_out), st); }));
}

lbf_status lbf_debug_stall_next(lbf_plan_t p, int64_t item) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (item < 0) return LBF_EINVAL;
  p->stall_item = item;
  return LBF_OK;
}

lbf_status lbf_device_status(lbf_plan_t p, int32_t *code) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (code) *code = h;
  if (h != 0) {
    e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e);
    return h == lbf::DERR_PPF_ALIGN ? LBF_ECUDA : LBF_ETIMEOUT;
  }
  return LBF_OK;
}

lbf_status lbf_superstation(lbf_plan_t p, const int32_t *group_of_station, int32_t n_groups, const void *d_ct,
                            void *d_ss, void *stream) {
  lbf_status s = check_call(p);
  if (s != LBF_OK) return s;
  if (!group_of_station || n_groups < 1 || n_groups > p->S) return LBF_EINVAL;
  for (int i = 0; i < p->S; ++i)
    if (group_of_station[i] < 0 || group_of_station[i] >= n_groups) return LBF_EINVAL;
  if (p->M == 0) return LBF_OK;
  if (!device_ptr(d_ct, 8) || !device_ptr(d_ss, 8)) return LBF_EINVAL;
  // stations listed group by group, in station order within a group
  std::vector<int> members, offs(n_groups + 1, 0);
  for (int g = 0; g < n_groups; ++g) {
    offs[g] = (int)members.size();
    for (int i = 0; i < p->S; ++i)
      if (group_of_station[i] == g) members.push_back(i);
  }
  offs[n_groups] = (int)members.size();
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(p->ss_members, members.data(), sizeof(int) * members.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->ss_offs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice, st);
  // the host vectors must outlive the copies: pageable copies are staged before the call returns
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  const lbf::Geometry g = p->geometry();
  return cuda_status(traced(p, K_SS, st, [&] {
    return lbf::launch_superstation(g, (const float2 *)d_ct, (float2 *)d_ss, p->ss_members, p->ss_offs, n_groups, st); }));
}

lbf_status lbf_trace_begin(lbf_plan_t p, int32_t max_launches) {
  if (!valid_plan(p)) return LBF_ESTATE;
  if (max_launches < 1 || max_launches > (1 << 20)) return LBF_EINVAL;
  trace_free(p);
  p->trace.resize((size_t)max_launches);
  for (auto &slot : p->trace) {
    slot.kernel = -1;
    if (cudaEventCreate(&slot.a) != cudaSuccess || cudaEventCreate(&slot.b) != cudaSuccess) {
      cudaGetLastError();
      p->trace.clear();
      return LBF_ECUDA;
    }
  }
  p->tracing = true;
  return LBF_OK;
}

lbf_status lbf_trace_end(lbf_plan_t p, lbf_trace *out) {
  if (!valid_plan(p)) return LBF_ESTATE;
  if (!p->tracing) return LBF_ESTATE;
  lbf_trace t;
  std::memset(&t, 0, sizeof(t));
  t.n_kernels = K_COUNT;
  for (int k = 0; k < K_COUNT; ++k) std::strncpy(t.names[k], kKernelNames[k], sizeof(t.names[k]) - 1);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < p->trace_used && e == cudaSuccess; ++i) {
    auto &slot = p->trace[i];
    e = cudaEventSynchronize(slot.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, slot.a, slot.b);
    if (e == cudaSuccess && slot.kernel >= 0) {
      t.launches[slot.kernel] += 1;
      t.total_ms[slot.kernel] += ms;
    }
  }
  t.dropped = p->trace_dropped;
  trace_free(p);
  if (out) *out = t;
  return cuda_status(e);
}

}  // extern "C"
