// lbf_run_block_static: the fused FP32 path for one block without any device allocation.
//
// Some callers cannot allocate device memory: a process whose device-memory budget is handed out
// by a host framework that forbids its plugins to call cudaMalloc, or an ingest thread that must
// not take the allocator's locks or latency in the middle of an observation.  This entry point
// serves them: every byte it needs beyond the caller's input and output lives in one file-scope
// device array of fixed size, reached through its device address obtained once per device.
//
// The array is shared by every call on a device and keeps the previous call's contents; the parts
// that must start at zero are cleared on each call.  Calls whose device work overlaps (two streams,
// two host threads) race on it.  The host side -- the per-device address cache and the host
// staging area of the tables -- is process-wide too, so a lock serialises it: two host threads may
// call at once (on the same or different devices) without corrupting each other's tables.
#include <cmath>
#include <cstring>
#include <mutex>

#include "lbf.h"
#include "lbf_internal.cuh"

namespace {

constexpr size_t kScratchBytes = 32u << 20;       // the whole static scratch: 32 MiB
constexpr size_t kCtBytes = 24u << 20;            // corner-turned block (cf32)
constexpr size_t kHistBytes = 4u << 20;           // zero history (samples before the stream)
constexpr size_t kTableBytes = kScratchBytes - kCtBytes - kHistBytes;   // 4 MiB of tables
constexpr int kMaxDevices = 64;
constexpr double kC = 299792458.0;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Host-side state, guarded by g_lock: the device address of the array per device ordinal (looked
// up once per device and process), and the staging area the tables are built in before upload.
std::mutex g_lock;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};
unsigned char g_host_tables[kTableBytes];

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

double delay_of(const double *xyz, double l, double m) {
  double nn = 1.0 - l * l - m * m;
  const double n = std::sqrt(nn > 0.0 ? nn : 0.0);
  const double dot = xyz[0] * l + xyz[1] * m + xyz[2] * n;
  return -dot / kC;
}

double half_away(double x) {
  const double a = std::floor(std::fabs(x) + 0.5);
  return x < 0 ? -a : (x > 0 ? a : 0.0);
}

bool on_device(const void *p, size_t align) {
  if (!p || (reinterpret_cast<uintptr_t>(p) % align) != 0) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Offsets of the tables inside the table region (host staging and device copy use the same map).
struct TableMap {
  size_t err, taps, tw, bp, dshift, tau, resid, f0, dtau, phase0, step, total;
};

TableMap table_map(int S, int F, int B) {
  TableMap m;
  size_t o = 0;
  m.err = o;    o += align256(sizeof(int));   // device error word of bounded waits (cleared per call)
  m.taps = o;   o += align256(sizeof(float) * lbf::kL * lbf::kN);
  m.tw = o;     o += align256(sizeof(float2) * lbf::kN);
  m.bp = o;     o += align256(sizeof(float) * lbf::kN);
  m.dshift = o; o += align256(sizeof(int) * (size_t)S);
  m.tau = o;    o += align256(sizeof(double) * (size_t)S);
  m.resid = o;  o += align256(sizeof(double) * (size_t)S);
  m.f0 = o;     o += align256(sizeof(double) * (size_t)F);
  m.dtau = o;   o += align256(sizeof(double) * (size_t)B * S);
  m.phase0 = o; o += align256(sizeof(float) * (size_t)F * B * S);
  m.step = o;   o += align256(sizeof(float) * (size_t)B * S);
  m.total = o;
  return m;
}

}  // namespace

extern "C" lbf_status lbf_run_block_static(const lbf_config *c, const void *d_in, void *d_out, void *stream) {
  // ---- validation, all on the host, before any device work
  if (!c || c->n_stations < 1 || c->n_subbands < 1 || c->n_beams < 1 || c->block_samples < 0) return LBF_EINVAL;
  if (c->n_channels != lbf::kN || c->n_taps != lbf::kL) return LBF_EUNSUPPORTED;
  if (c->block_samples % lbf::kN != 0) return LBF_EINVAL;
  if (c->sample_bits != 16 && c->sample_bits != 8) return LBF_EINVAL;
  if (c->output != LBF_STOKES_I && c->output != LBF_STOKES_IQUV && c->output != LBF_VOLTAGES) return LBF_EINVAL;
  if (c->precision != LBF_FP32 || c->flags != 0) return LBF_EUNSUPPORTED;
  const int q = c->int_factor;
  if (!(q == 1 || q == 2 || q == 4 || q == 8 || q == 16 || q == 32)) return LBF_EINVAL;
  const int S = c->n_stations, F = c->n_subbands, B = c->n_beams, T = c->block_samples, M = T / lbf::kN;
  if (c->output != LBF_VOLTAGES && M % q != 0) return LBF_EINVAL;
  if (!c->station_xyz_m || !c->subband_centre_hz || !c->beam_dlm || !c->fir_taps) return LBF_EINVAL;
  if (!(c->sample_rate_hz > 0.0)) return LBF_EINVAL;
  if (M == 0) return LBF_OK;
  const size_t word = c->sample_bits == 16 ? 8 : 4;
  const double ts = 1.0 / c->sample_rate_hz;
  const double l0 = c->phase_centre_l, m0 = c->phase_centre_m;
  long long nmax = 0;
  for (int s = 0; s < S; ++s) {
    const double n = half_away(delay_of(c->station_xyz_m + 3 * s, l0, m0) / ts);
    if (!(std::fabs(n) < 1e6)) return LBF_EUNSUPPORTED;
    nmax = (s == 0 || (long long)n > nmax) ? (long long)n : nmax;
  }
  long long dmax = 0;
  for (int s = 0; s < S; ++s) {
    const long long d = nmax - (long long)half_away(delay_of(c->station_xyz_m + 3 * s, l0, m0) / ts);
    dmax = d > dmax ? d : dmax;
  }
  const long long H = (long long)(lbf::kL - 1) * lbf::kN + dmax;
  const TableMap tm = table_map(S, F, B);
  if ((size_t)S * F * lbf::kP * (size_t)T * sizeof(float2) > kCtBytes) return LBF_ETOOBIG;
  if ((size_t)S * F * (size_t)H * word > kHistBytes) return LBF_ETOOBIG;
  if (tm.total > kTableBytes) return LBF_ETOOBIG;
  if (c->bf_variant < LBF_BF_AUTO || c->bf_variant > LBF_BF_MANY64) return LBF_EINVAL;
  if ((c->bf_variant == LBF_BF_MANY || c->bf_variant == LBF_BF_MANY64) && S > lbf::many_beam_max_stations())
    return LBF_EUNSUPPORTED;
  const int variant = c->bf_variant == LBF_BF_AUTO ? lbf::auto_bf_variant(B, S) : c->bf_variant;
  if (!on_device(d_in, word) || !on_device(d_out, c->output == LBF_VOLTAGES ? 8 : 4)) return LBF_EINVAL;

  // From here to the last enqueue the host-side state is in use: one caller at a time.  The lock
  // is held until cudaMemcpyAsync has returned, by which time the pageable staging area has been
  // copied out by the runtime and may be rebuilt by the next caller.
  std::lock_guard<std::mutex> hold(g_lock);

  // ---- once per device: the device address of the static array (host code only sees a stand-in)
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBF_ECUDA;
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) { cudaGetLastError(); return LBF_ECUDA; }
    g_scratch_addr[dev] = static_cast<unsigned char *>(ptr);
  }
  unsigned char *base = g_scratch_addr[dev];
  float2 *ct = reinterpret_cast<float2 *>(base);
  unsigned char *hist = base + kCtBytes;
  unsigned char *tab = base + kCtBytes + kHistBytes;

  // ---- host FP64 geometry into the static host staging area
  unsigned char *h = g_host_tables;
  *reinterpret_cast<int *>(h + tm.err) = 0;
  std::memcpy(h + tm.taps, c->fir_taps, sizeof(float) * lbf::kL * lbf::kN);
  for (int n = 0; n < lbf::kN; ++n) {
    const double a = 2.0 * M_PI * (double)n / (double)lbf::kN;
    reinterpret_cast<float2 *>(h + tm.tw)[n] = make_float2((float)std::cos(a), (float)-std::sin(a));
    reinterpret_cast<float *>(h + tm.bp)[n] = c->bandpass ? c->bandpass[n] : 1.0f;
  }
  for (int s = 0; s < S; ++s) {
    const double tau = delay_of(c->station_xyz_m + 3 * s, l0, m0);
    const double n = half_away(tau / ts);
    reinterpret_cast<int *>(h + tm.dshift)[s] = (int)(nmax - (long long)n);
    reinterpret_cast<double *>(h + tm.tau)[s] = tau;
    reinterpret_cast<double *>(h + tm.resid)[s] = tau - n * ts;
  }
  std::memcpy(h + tm.f0, c->subband_centre_hz, sizeof(double) * F);
  for (int b = 0; b < B; ++b)
    for (int s = 0; s < S; ++s)
      reinterpret_cast<double *>(h + tm.dtau)[(size_t)b * S + s] =
          delay_of(c->station_xyz_m + 3 * s, l0 + c->beam_dlm[2 * b], m0 + c->beam_dlm[2 * b + 1]) -
          reinterpret_cast<double *>(h + tm.tau)[s];

  cudaStream_t st = (cudaStream_t)stream;
  const size_t upload = tm.phase0;   // everything before the device-computed phase tables
  cudaError_t e = cudaMemcpyAsync(tab, h, upload, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, (size_t)S * F * (size_t)H * word, st);   // zero history

  lbf::Geometry g;
  g.S = S; g.F = F; g.B = B; g.T = T; g.M = M; g.Q = q;
  g.nS = c->output == LBF_STOKES_I ? 1 : c->output == LBF_STOKES_IQUV ? 4 : 0;
  g.H = (int)H; g.fs = c->sample_rate_hz;
  g.taps = reinterpret_cast<const float *>(tab + tm.taps);
  g.twiddle = reinterpret_cast<const float2 *>(tab + tm.tw);
  g.bandpass = reinterpret_cast<const float *>(tab + tm.bp);
  g.dshift = reinterpret_cast<const int *>(tab + tm.dshift);
  g.tau = reinterpret_cast<const double *>(tab + tm.tau);
  g.resid = reinterpret_cast<const double *>(tab + tm.resid);
  g.f0 = reinterpret_cast<const double *>(tab + tm.f0);
  g.dtau = reinterpret_cast<const double *>(tab + tm.dtau);
  g.phase0 = reinterpret_cast<const float *>(tab + tm.phase0);
  g.step = reinterpret_cast<const float *>(tab + tm.step);
  g.err = reinterpret_cast<int *>(tab + tm.err);
  const int out_kind = c->output == LBF_STOKES_I ? lbf::OUT_STOKES_I
                     : c->output == LBF_STOKES_IQUV ? lbf::OUT_STOKES_IQUV : lbf::OUT_VOLTAGES;
  if (e == cudaSuccess)
    e = lbf::launch_phase_tables(F, B, S, g.fs, g.f0, g.dtau, reinterpret_cast<float *>(tab + tm.phase0),
                                 reinterpret_cast<float *>(tab + tm.step), st);
  if (e == cudaSuccess) e = lbf::launch_ppf(g, c->sample_bits, d_in, hist, nullptr, ct, st);
  if (e == cudaSuccess) e = lbf::launch_beamform(g, variant, out_kind, ct, d_out, st);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LBF_ENOMEM : LBF_ECUDA;
  return LBF_OK;
}
