// Stand-alone sub-sample delay compensation + bandpass + corner turn (Sections 3 and 4.3):
//   ct[f][c][s][pol][m] = chan[f][s][pol][m][c] * bp[c] * exp(+2 pi i (f0_f tau_s + df_c (tau_s - n_s Ts)))
// The phase is formed in FP64 cycles per (s, f, c) and reduced before the FP32 sine/cosine; the
// transpose goes through an XOR-swizzled shared-memory tile so that both the 2 KB channel rows read
// and the 128-byte spectrum runs written are coalesced and bank-conflict free.
#include <cuda_fp16.h>

#include "lbf_internal.cuh"

namespace lbf {
namespace {

constexpr int kTile = 16;   // spectra per CTA

__global__ void __launch_bounds__(256)
delay_ct_kernel(Geometry g, const float2 *__restrict__ chan, float2 *__restrict__ ct, int tiles) {
  __shared__ __align__(16) float2 stage[kN * kTile];
  const int tid = threadIdx.x;
  long long idx = blockIdx.x;
  const int tile = (int)(idx % tiles);
  idx /= tiles;
  const int pol = (int)(idx % kP);
  idx /= kP;
  const int s = (int)(idx % g.S);
  const int f = (int)(idx / g.S);
  const int m0 = tile * kTile;

  const int c = tid;
  const double df = (double)(c - kN / 2) * (g.fs / kN);
  const double phi = g.f0[f] * g.tau[s] + df * g.resid[s];
  const float2 ph = unit_phasor_cycles(phi);
  const float b = g.bandpass[c];
  const float2 gain = make_float2(b * ph.x, b * ph.y);

  const float2 *src = chan + (((long long)f * g.S + s) * kP + pol) * g.M * kN;
#pragma unroll 4
  for (int q = 0; q < kTile; ++q) {
    const int m = m0 + q;
    if (m < g.M) stage[c * kTile + (q ^ (c & 15))] = cmul(src[(long long)m * kN + c], gain);
  }
  __syncthreads();
  const int q = tid & 15;
  if (m0 + q < g.M) {
#pragma unroll 4
    for (int pass = 0; pass < kN / 16; ++pass) {
      const int cc = pass * 16 + (tid >> 4);
      ct[((((long long)f * kN + cc) * g.S + s) * kP + pol) * g.M + m0 + q] =
          stage[cc * kTile + (q ^ (cc & 15))];
    }
  }
}

// ct [F][N][S][P][M] cf32 -> FP16 planes [F*N][Mt][kpad][P][32] (rows k = 2s re, 2s+1 im): an
// elementwise split, both sides spectrum-fastest, so reads and writes are coalesced as they are.
__global__ void __launch_bounds__(256)
ct_to_ct16_kernel(Geometry g, const float2 *__restrict__ ct, Ct16Out o, long long n) {
  __half *hi = reinterpret_cast<__half *>(o.hi);
  __half *lo = reinterpret_cast<__half *>(o.lo);
  const int mb = tc_tiles(g.M);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i % g.M);
    const long long r = i / g.M;                             // (fc * S + s) * P + pol
    const int pol = (int)(r % kP);
    const long long fcs = r / kP;
    const long long fc = fcs / g.S;
    const int s = (int)(fcs - fc * g.S);
    const float2 v = ct[i];
    const long long re = (((fc * mb + (m >> 5)) * o.kpad + 2 * s) * 64) + pol * 32 + (m & 31);
    const long long im = re + 64;
    const __half hr = __float2half_rn(v.x), hm = __float2half_rn(v.y);
    hi[re] = hr;
    hi[im] = hm;
    if (lo) {
      lo[re] = __float2half_rn(v.x - __half2float(hr));
      lo[im] = __float2half_rn(v.y - __half2float(hm));
    }
  }
}

// Incoherent beam of a tensor-core plan (Section 3) from its FP16 planes [F*N][Mt][kpad][P][32]:
// thread per (subband-channel, spectrum), summing over stations the Stokes parameters of
// Y = hi (+ lo); writes beam index B of the Stokes output.  Planes written before the delay phase
// and bandpass (g.ct16_raw) get the bandpass here: the unit delay phasor leaves the powers alone,
// the bandpass scales every Stokes parameter by bp[c]^2.  Lane l of a warp holds spectrum
// 32 w + l, so the integration over Q <= 32 spectra is a warp-shuffle reduction.
template <int NS>
__global__ void __launch_bounds__(256)
incoherent_ct16_kernel(Geometry g, Ct16Out o, float *__restrict__ out) {
  const __half *hi = reinterpret_cast<const __half *>(o.hi);
  const __half *lo = reinterpret_cast<const __half *>(o.lo);
  const int mb = tc_tiles(g.M);
  const int mspan = (g.M + 31) & ~31;
  const long long fc = blockIdx.x;
  const int f = (int)(fc / kN), c = (int)(fc - (long long)f * kN);
  const int Mq = g.M / g.Q;
  for (int m0 = 0; m0 < mspan; m0 += blockDim.x) {
    const int m = m0 + threadIdx.x;
    const bool active = m < g.M;
    float xx = 0.f, yy = 0.f, re = 0.f, im = 0.f;
    if (active) {
      const long long blk = (fc * mb + (m >> 5)) * o.kpad;
      for (int s = 0; s < g.S; ++s) {
        const long long r0 = (blk + 2 * s) * 64 + (m & 31);            // k = 2s (re)
        const long long r1 = r0 + 64;                                   // k = 2s+1 (im)
        float xr = __half2float(hi[r0]), xi = __half2float(hi[r1]);
        float yr = __half2float(hi[r0 + 32]), yi = __half2float(hi[r1 + 32]);
        if (lo) {
          xr += __half2float(lo[r0]); xi += __half2float(lo[r1]);
          yr += __half2float(lo[r0 + 32]); yi += __half2float(lo[r1 + 32]);
        }
        xx = fmaf(xr, xr, fmaf(xi, xi, xx));
        yy = fmaf(yr, yr, fmaf(yi, yi, yy));
        re = fmaf(xr, yr, fmaf(xi, yi, re));
        im = fmaf(xi, yr, fmaf(-xr, yi, im));
      }
    }
    const float b2 = g.ct16_raw ? g.bandpass[c] * g.bandpass[c] : 1.f;
#pragma unroll
    for (int st = 0; st < NS; ++st) {
      float v = b2 * (st == 0 ? xx + yy : st == 1 ? xx - yy : st == 2 ? 2.f * re : 2.f * im);
      for (int o2 = 1; o2 < g.Q; o2 <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
      if (active && (m & (g.Q - 1)) == 0)
        out[((((long long)g.B * NS + st) * g.F + f) * kN + c) * Mq + m / g.Q] = v;
    }
  }
}

// Superstation beam former (Section 4.2): ss[f][c][g][pol][m] = sum of ct[f][c][s][pol][m] over the
// stations s of group g (unit weights: the stations are already delay-compensated to the phase
// centre).  members[] lists the stations group by group, offs[g]..offs[g+1] those of group g; a
// thread owns one spectrum of one (subband-channel, group, pol) row, so reads and writes are
// coalesced along the spectra.
__global__ void __launch_bounds__(256)
superstation_kernel(Geometry g, const float2 *__restrict__ ct, float2 *__restrict__ ss, const int *__restrict__ members,
                    const int *__restrict__ offs, int ngroups, long long rows) {
  for (long long r = blockIdx.y; r < rows; r += gridDim.y) {          // r = (fc * G + grp) * P + pol
    const int pol = (int)(r % kP);
    const long long fg = r / kP;
    const int grp = (int)(fg % ngroups);
    const long long fc = fg / ngroups;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < g.M; m += gridDim.x * blockDim.x) {
      float2 acc = make_float2(0.f, 0.f);
      for (int i = offs[grp]; i < offs[grp + 1]; ++i) {
        const float2 v = ct[((fc * g.S + members[i]) * kP + pol) * g.M + m];
        acc.x += v.x;
        acc.y += v.y;
      }
      ss[r * g.M + m] = acc;
    }
  }
}

// The same with two spectra per thread (M even, 16-byte aligned buffers): 16-byte loads and
// stores, and the loads of all members of the group issued before they are summed.
__global__ void __launch_bounds__(256)
superstation2_kernel(Geometry g, const float4 *__restrict__ ct, float4 *__restrict__ ss,
                     const int *__restrict__ members, const int *__restrict__ offs, int ngroups, long long rows) {
  const int M2 = g.M >> 1;
  for (long long r = blockIdx.y; r < rows; r += gridDim.y) {          // r = (fc * G + grp) * P + pol
    const int pol = (int)(r % kP);
    const long long fg = r / kP;
    const int grp = (int)(fg % ngroups);
    const long long fc = fg / ngroups;
    const int i0 = offs[grp], i1 = offs[grp + 1];
    for (int m2 = blockIdx.x * blockDim.x + threadIdx.x; m2 < M2; m2 += gridDim.x * blockDim.x) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      int i = i0;
      for (; i + 4 <= i1; i += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = ct[((fc * g.S + members[i + u]) * kP + pol) * M2 + m2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc.x += v[u].x; acc.y += v[u].y; acc.z += v[u].z; acc.w += v[u].w;
        }
      }
      for (; i < i1; ++i) {
        const float4 v = ct[((fc * g.S + members[i]) * kP + pol) * M2 + m2];
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
      }
      ss[r * M2 + m2] = acc;
    }
  }
}

}  // namespace

cudaError_t launch_superstation(const Geometry &g, const float2 *ct, float2 *ss, const int *members, const int *offs,
                                int ngroups, cudaStream_t st) {
  const long long rows = (long long)g.F * kN * ngroups * kP;
  if (rows == 0 || g.M == 0) return cudaSuccess;
  const unsigned by = (unsigned)(rows < 65535 ? rows : 65535);
  if ((g.M & 1) == 0 && (reinterpret_cast<uintptr_t>(ct) & 15) == 0 && (reinterpret_cast<uintptr_t>(ss) & 15) == 0) {
    const int m2 = g.M / 2;
    const unsigned bx = (unsigned)((m2 + 255) / 256 < 4 ? (m2 + 255) / 256 : 4);
    superstation2_kernel<<<dim3(bx, by), 256, 0, st>>>(g, reinterpret_cast<const float4 *>(ct),
                                                       reinterpret_cast<float4 *>(ss), members, offs, ngroups, rows);
    return cudaGetLastError();
  }
  const unsigned bx = (unsigned)((g.M + 255) / 256 < 4 ? (g.M + 255) / 256 : 4);
  superstation_kernel<<<dim3(bx, by), 256, 0, st>>>(g, ct, ss, members, offs, ngroups, rows);
  return cudaGetLastError();
}

cudaError_t launch_incoherent_ct16(const Geometry &g, int out_kind, const Ct16Out &o, float *out, cudaStream_t st) {
  const long long fcs = (long long)g.F * kN;
  if (fcs == 0 || g.M == 0) return cudaSuccess;
  if (out_kind == OUT_STOKES_IQUV)
    incoherent_ct16_kernel<4><<<(unsigned)fcs, 256, 0, st>>>(g, o, out);
  else
    incoherent_ct16_kernel<1><<<(unsigned)fcs, 256, 0, st>>>(g, o, out);
  return cudaGetLastError();
}

cudaError_t launch_ct_to_ct16(const Geometry &g, const float2 *ct, const Ct16Out &o, cudaStream_t st) {
  const long long n = (long long)g.F * kN * g.S * kP * g.M;
  if (n == 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  ct_to_ct16_kernel<<<(unsigned)(want < 152LL * 64 ? want : 152LL * 64), 256, 0, st>>>(g, ct, o, n);
  return cudaGetLastError();
}

cudaError_t launch_delay_ct(const Geometry &g, const float2 *chan, float2 *ct, cudaStream_t st) {
  const int tiles = (g.M + kTile - 1) / kTile;
  const long long ctas = (long long)g.F * g.S * kP * tiles;
  if (ctas == 0) return cudaSuccess;
  delay_ct_kernel<<<(unsigned)ctas, 256, 0, st>>>(g, chan, ct, tiles);
  return cudaGetLastError();
}

}  // namespace lbf
