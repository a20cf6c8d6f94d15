// Batches: several observations (plans) processed together, one block each, by persistent grouped
// kernels instead of three launches per observation.  Uneven observations share the GPU through
// work counters: CTAs take (observation, stream, spectrum chunk) and (observation, subband-channel,
// beam group) items until all are done, so small observations do not leave the GPU idle and large
// ones do not serialise the batch.  There is one launch per class of plans whose bodies need the
// same registers and shared memory, so that each body runs as it does alone: the filter bank per
// (sample width, FP32 or FP16-plane output, tensor-store output or not -- each observation's
// tensor maps sit in a device array its table entry points at), one history launch, the FP32 beam former per
// (kernel variant, output kind, CTAs per SM), and one tensor-core launch per (output kind,
// integration length), whose work items number the class's plans one after the other.
//
// A batch can be captured as CUDA graphs (one per history parity: each block flips every plan's
// history ping-pong) and replayed with a single graph launch per block.  Its shapes -- spectra per
// filter-bank item, for observations with 9..64 beams the few- or many-beam beam former, and the
// many-beam tile (128 or 64 beams per CTA) -- and its mode are tuned by timing the candidates on
// the batch itself.  The per-plan mode runs each stage as the plan's own kernel, as separate
// launches would (still one graph launch per block); it wins where the observations are large
// enough to fill the GPU alone.
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "lbf.h"
#include "lbf_internal.cuh"
#include "plan.h"

namespace {

constexpr uint32_t kBatchMagic = 0x4c424642u;   // "LBFB"
// work counters, one per grouped launch: at most one filter-bank and one beam-former launch per
// plan, plus the partly filled launches of each class
int max_counters(int n) { return 2 * n + 64; }

bool plan_ok(lbf_plan_t p) { return p && p->magic == lbf::kPlanMagic; }

bool dev_ptr(const void *p, size_t align) {
  if (!p || (reinterpret_cast<uintptr_t>(p) % align) != 0) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

lbf_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return LBF_OK;
  return e == cudaErrorMemoryAllocation ? LBF_ENOMEM : LBF_ECUDA;
}

}  // namespace

struct lbf_batch_s {
  uint32_t magic = kBatchMagic;
  int device = 0;
  std::vector<lbf_plan_t> plans;
  int spc = 256;                       // spectra per filter-bank item (tuned: 64, 256 or 1024)
  bool per_plan = false;               // every stage as each plan's own kernels (tuned)
  std::vector<int> variant;            // beam-former kernel per plan
  // group tables: [parity][plan]; parity p describes the plans' history state after p blocks
  lbf::PpfGroup *h_ppf = nullptr, *d_ppf = nullptr;   // pinned host / device, 2 * n
  unsigned char *h_maps = nullptr, *d_maps = nullptr; // their tensor maps (2 * n entries of
                                                      // ppf_group_maps_bytes()), pinned host / device
  lbf::BfGroup *h_bf = nullptr;                      // pinned host, 2 * n: FP32 plans, class by class
  unsigned long long *d_counter = nullptr;            // [max_counters(n)] work counters, one per launch
  long long hist_items = 0;
  // launch classes: filter bank per (sample width, FP32 or FP16 output); FP32 beam former per
  // (variant, output kind, CTAs per SM) -- each class one persistent launch over its groups
  struct PpfClass { int bits, tc, tma, first, n; long long items; };
  struct BfClass { int variant, out_kind, per_sm, first, n; long long items; size_t smem; };
  std::vector<PpfClass> ppf_cls;
  std::vector<BfClass> bf_cls;
  int ppf_ctas = 0, sms = 0;
  std::vector<void *> tc_out;          // output of each plan's block
  std::vector<const void *> d_in_cur;  // input of each plan's block (per-plan mode)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_parity = 0;                // which graph describes the current state
};

namespace {

void free_graphs(lbf_batch_t b) {
  for (auto &g : b->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

// Fill the group tables of parity `par` (par = 1: every plan's history one block ahead) for the
// given block buffers: filter-bank groups class by class (work items numbered from 0 within a
// class; history elements numbered over the whole table), then the FP32 beam-former groups class
// by class.
void fill_tables(lbf_batch_t b, int par, const void *const *d_in, void *const *d_out) {
  const int n = (int)b->plans.size();
  long long hi = 0;
  int slot = 0;
  b->ppf_cls.clear();
  const size_t mb = lbf::ppf_group_maps_bytes();
  for (int bits : {16, 8})
    for (int tc = 0; tc < 2; ++tc)
    for (int tma = 1; tma >= 0; --tma) {   // tensor-store output (FP16 planes; FP32 with even M) or not
      lbf_batch_s::PpfClass cls{bits, tc, tma, slot, 0, 0};
      for (int i = 0; i < n; ++i) {
        lbf_plan_t p = b->plans[i];
        if (p->bits != bits || (p->tc ? 1 : 0) != tc) continue;
        lbf::PpfGroup probe;
        probe.g = p->geometry();
        probe.tc = tc;
        probe.ct = p->ws;
        if ((lbf::ppf_group_tma(probe) ? 1 : 0) != tma) continue;
        if (cls.n == lbf::kMaxGroups) {   // one launch holds at most kMaxGroups groups
          b->ppf_cls.push_back(cls);
          cls = lbf_batch_s::PpfClass{bits, tc, tma, slot, 0, 0};
        }
        const int cur = p->cur ^ par;
        const int at = par * n + slot;
        lbf::PpfGroup &G = b->h_ppf[par * n + slot++];
        G.g = p->geometry();
        G.in = d_in[i];
        G.hist = p->hist[cur];
        G.new_hist = p->hist[cur ^ 1];
        G.ct = p->ws;
        G.tc = tc;
        G.ct16.hi = p->ct16[0];
        G.ct16.lo = p->tc ? static_cast<unsigned char *>(p->ct16[0]) + p->ct16_bytes : nullptr;
        G.ct16.kpad = p->kpad;
        G.bits = p->bits;
        G.spc = b->spc;
        G.chunks = lbf::ppf_items_per_stream(p->M, b->spc);
        G.first_item = cls.items;
        G.first_hist = hi;
        G.maps = nullptr;
        if (tma && lbf::ppf_group_maps(G, b->h_maps + (size_t)at * mb) == cudaSuccess)
          G.maps = b->d_maps + (size_t)at * mb;
        cls.items += (long long)p->S * p->F * G.chunks;   // one item: both polarisations of a chunk
        hi += (long long)p->S * p->F * p->H;
        ++cls.n;
      }
      if (cls.n) b->ppf_cls.push_back(cls);
    }
  b->hist_items = hi;
  b->tc_out.assign(d_out, d_out + n);
  b->d_in_cur.assign(d_in, d_in + n);
  // FP32 beam former: plans of the same variant, output kind and residency share a launch
  std::vector<int> per_sm(n, 0);
  std::vector<size_t> smem_of(n, 0);
  for (int i = 0; i < n; ++i) {
    lbf_plan_t p = b->plans[i];
    if (p->tc) continue;
    smem_of[i] = lbf::bf_smem_bytes(b->variant[i], p->S);
    per_sm[i] = lbf::bf_group_residency(b->variant[i], p->out_kind, smem_of[i]);
  }
  b->bf_cls.clear();
  slot = 0;
  std::vector<bool> placed(n, false);
  for (int i = 0; i < n; ++i) {
    lbf_plan_t pi = b->plans[i];
    if (pi->tc || placed[i]) continue;
    lbf_batch_s::BfClass cls{b->variant[i], pi->out_kind, per_sm[i], slot, 0, 0, 0};
    for (int j = i; j < n; ++j) {
      lbf_plan_t p = b->plans[j];
      if (p->tc || placed[j] || b->variant[j] != cls.variant || p->out_kind != cls.out_kind ||
          per_sm[j] != cls.per_sm || cls.n == lbf::kMaxGroups)
        continue;
      placed[j] = true;
      lbf::BfGroup &Bg = b->h_bf[par * n + slot++];
      Bg.g = p->geometry();
      Bg.ct = p->ws;
      Bg.out = d_out[j];
      Bg.variant = b->variant[j];
      Bg.out_kind = p->out_kind;
      const int per = b->variant[j] == 1 ? lbf::few_beams_per_item() : lbf::many_beams_per_item(b->variant[j]);
      Bg.per_fc = (p->B + per - 1) / per;
      Bg.first_item = cls.items;
      cls.items += (long long)p->F * lbf::kN * Bg.per_fc;
      cls.smem = smem_of[j] > cls.smem ? smem_of[j] : cls.smem;
      ++cls.n;
    }
    b->bf_cls.push_back(cls);
  }
}

// Enqueue one batch block with the tables of parity `par` (already filled).
cudaError_t enqueue(lbf_batch_t b, int par, cudaStream_t st) {
  const int n = (int)b->plans.size();
  // the history update reads the filter-bank table from device memory; the grouped filter bank
  // and beam former take theirs as kernel parameters
  cudaError_t e = cudaMemcpyAsync(b->d_ppf + par * n, b->h_ppf + par * n, sizeof(lbf::PpfGroup) * n,
                                  cudaMemcpyHostToDevice, st);
  const size_t mb = lbf::ppf_group_maps_bytes();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_maps + (size_t)par * n * mb, b->h_maps + (size_t)par * n * mb, mb * n,
                        cudaMemcpyHostToDevice, st);
  if (b->per_plan) {
    // each plan's own filter bank, history update and FP32 beam former (the hardware schedules
    // their CTAs; large observations each fill the GPU); the tensor-core plans follow, one
    // launch each
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
      lbf_plan_t p = b->plans[i];
      if (p->M == 0) continue;
      const int cur = p->cur ^ par;
      const lbf::Geometry g = p->geometry();
      const void *din = b->d_in_cur[i];
      if (p->tc) {
        lbf::Ct16Out o;
        o.hi = p->ct16[0];
        o.lo = static_cast<unsigned char *>(p->ct16[0]) + p->ct16_bytes;
        o.kpad = p->kpad;
        e = lbf::launch_ppf(g, p->bits, din, p->hist[cur], nullptr, nullptr, st, &o);
      } else {
        e = lbf::launch_ppf(g, p->bits, din, p->hist[cur], nullptr, p->ws, st);
      }
      if (e == cudaSuccess) e = lbf::launch_hist_update(g, p->bits, din, p->hist[cur], p->hist[cur ^ 1], st);
      if (e == cudaSuccess && !p->tc) e = lbf::launch_beamform(g, b->variant[i], p->out_kind, p->ws, b->tc_out[i], st);
    }
  } else {
    int counter = 0;
    if ((int)(b->ppf_cls.size() + b->bf_cls.size()) > max_counters(n)) return cudaErrorInvalidValue;
    for (const auto &c : b->ppf_cls)
      if (e == cudaSuccess)
        e = lbf::launch_ppf_group(c.bits, c.tc, c.tma, b->h_ppf + par * n + c.first, c.n, c.items,
                                  b->d_counter + counter++, b->ppf_ctas, st);
    if (e == cudaSuccess) e = lbf::launch_hist_group(b->d_ppf + par * n, n, b->hist_items, st);
    for (const auto &c : b->bf_cls)
      if (e == cudaSuccess)
        e = lbf::launch_bf_group(c.variant, c.out_kind, b->h_bf + par * n + c.first, c.n, c.items,
                                 b->d_counter + counter++, c.smem, st);
  }
  // tensor-core plans: their incoherent beams, then ONE persistent tcgen05 launch per class of
  // output kind and integration length (up to tc_max_plans_per_launch() plans each), whose CTAs
  // walk the work items of all the class's plans
  std::vector<std::pair<long long, lbf::TcPlanRef>> refs;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    lbf_plan_t p = b->plans[i];
    if (!p->tc || p->M == 0) continue;
    lbf::Geometry g = p->geometry();
    g.ct16_raw = 1;   // planes from the grouped filter bank: delay and bandpass go with the weights
    if (p->inc) {
      lbf::Ct16Out o;
      o.hi = p->ct16[0];
      o.lo = static_cast<unsigned char *>(p->ct16[0]) + p->ct16_bytes;
      o.kpad = p->kpad;
      e = lbf::launch_incoherent_ct16(g, p->out_kind, o, static_cast<float *>(b->tc_out[i]), st);
    }
    const long long cls = (long long)p->out_kind * 64 + (p->out_kind == lbf::OUT_VOLTAGES ? 1 : p->Q);
    refs.push_back({cls, lbf::TcPlanRef{g, &p->tmap[0], &p->tmap[1], static_cast<float *>(b->tc_out[i]), p->d_err}});
  }
  std::vector<bool> done(refs.size(), false);
  // per-plan mode: each tensor-core plan in its own launch (the single-plan kernel, with the plan
  // and its product count compiled in); grouped mode: one launch per class
  const int cap = b->per_plan ? 1 : lbf::tc_max_plans_per_launch();
  for (size_t i = 0; i < refs.size() && e == cudaSuccess; ++i) {
    if (done[i]) continue;
    std::vector<lbf::TcPlanRef> cls;
    for (size_t j = i; j < refs.size() && (int)cls.size() < cap; ++j)
      if (!done[j] && refs[j].first == refs[i].first) { cls.push_back(refs[j].second); done[j] = true; }
    const int out_kind = (int)(refs[i].first / 64);
    const int q = (int)(refs[i].first % 64);
    // (a class of more than `cap` plans continues at its first plan not yet launched)
    e = lbf::launch_bf_tc_group(cls.data(), (int)cls.size(), out_kind, q, st);
  }
  return e;
}

void advance(lbf_batch_t b) {
  for (lbf_plan_t p : b->plans) p->cur ^= 1;
}

lbf_status check_buffers(lbf_batch_t b, const void *const *d_in, void *const *d_out) {
  if (!d_in || !d_out) return LBF_EINVAL;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    lbf_plan_t p = b->plans[i];
    if (!dev_ptr(d_in[i], p->word) || !dev_ptr(d_out[i], p->nS ? 4 : 8)) return LBF_EINVAL;
  }
  return LBF_OK;
}

}  // namespace

extern "C" {

lbf_status lbf_batch_create(const lbf_plan_t *plans, int32_t n, lbf_batch_t *out) {
  if (!out) return LBF_EINVAL;
  *out = nullptr;
  if (!plans || n < 1 || n > 4096) return LBF_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBF_ECUDA;
  for (int i = 0; i < n; ++i) {
    lbf_plan_t p = plans[i];
    if (!plan_ok(p)) return LBF_ESTATE;
    if (p->device != dev) return LBF_ESTATE;
    if (p->external_ws) return LBF_EUNSUPPORTED;   // batches use each plan's own scratch
    for (int j = 0; j < i; ++j)
      if (plans[j] == p) return LBF_EINVAL;
  }
  lbf_batch_s *b = new (std::nothrow) lbf_batch_s();
  if (!b) return LBF_ENOMEM;
  b->device = dev;
  b->plans.assign(plans, plans + n);
  b->variant.resize(n);
  for (int i = 0; i < n; ++i) b->variant[i] = plans[i]->variant;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->sms = sms > 0 ? sms : 152;
  b->ppf_ctas = lbf::ppf_ctas_per_sm() * b->sms;   // persistent filter-bank CTAs
  cudaError_t e = cudaMallocHost((void **)&b->h_ppf, sizeof(lbf::PpfGroup) * 2 * n);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_bf, sizeof(lbf::BfGroup) * 2 * n);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_maps, lbf::ppf_group_maps_bytes() * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_ppf, sizeof(lbf::PpfGroup) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_maps, lbf::ppf_group_maps_bytes() * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_counter, max_counters(n) * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFreeHost(b->h_ppf); cudaFreeHost(b->h_bf); cudaFreeHost(b->h_maps);
    cudaFree(b->d_ppf); cudaFree(b->d_maps); cudaFree(b->d_counter);
    delete b;
    cudaGetLastError();
    return status_of(e);
  }
  *out = b;
  return LBF_OK;
}

lbf_status lbf_batch_destroy(lbf_batch_t b) {
  if (!b) return LBF_OK;
  if (b->magic != kBatchMagic) return LBF_ESTATE;
  cudaDeviceSynchronize();
  free_graphs(b);
  cudaFreeHost(b->h_ppf); cudaFreeHost(b->h_bf); cudaFreeHost(b->h_maps);
  cudaFree(b->d_ppf); cudaFree(b->d_maps); cudaFree(b->d_counter);
  b->magic = 0;
  delete b;
  return LBF_OK;
}

lbf_status lbf_batch_run(lbf_batch_t b, const void *const *d_in, void *const *d_out, void *stream) {
  if (!b || b->magic != kBatchMagic) return LBF_ESTATE;
  lbf_status s = check_buffers(b, d_in, d_out);
  if (s != LBF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // the pinned tables of parity 0 may still be read by an earlier copy on this stream
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return status_of(e);
  fill_tables(b, 0, d_in, d_out);
  e = enqueue(b, 0, st);
  if (e != cudaSuccess) return status_of(e);
  advance(b);
  free_graphs(b);   // captured graphs described the previous state
  return LBF_OK;
}

lbf_status lbf_batch_capture(lbf_batch_t b, const void *const *d_in, void *const *d_out, void *stream) {
  if (!b || b->magic != kBatchMagic) return LBF_ESTATE;
  lbf_status s = check_buffers(b, d_in, d_out);
  if (s != LBF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return status_of(e);
  free_graphs(b);
  for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
    fill_tables(b, par, d_in, d_out);
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = enqueue(b, par, cs);
      e = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[par], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
  }
  if (e != cudaSuccess) {
    free_graphs(b);
    cudaGetLastError();
    return status_of(e);
  }
  b->graph_parity = 0;
  return LBF_OK;
}

lbf_status lbf_batch_launches(lbf_batch_t b, int32_t *n_launches) {
  if (!b || b->magic != kBatchMagic) return LBF_ESTATE;
  if (!n_launches) return LBF_EINVAL;
  // classes of the tables last filled (lbf_batch_run, lbf_batch_capture or lbf_batch_tune)
  if (b->per_plan) {   // per plan: filter bank, history and beam former (+ incoherent beam) each
    int k = 0;
    for (lbf_plan_t p : b->plans) k += p->M ? 3 + (p->tc && p->inc ? 1 : 0) : 0;
    *n_launches = k;
    return LBF_OK;
  }
  int tc_classes = 0;
  std::vector<long long> seen;
  for (lbf_plan_t p : b->plans) {
    if (!p->tc || p->M == 0) continue;
    const long long cls = (long long)p->out_kind * 64 + (p->out_kind == lbf::OUT_VOLTAGES ? 1 : p->Q);
    int same = 0;
    for (long long c : seen) same += c == cls;
    if (same % lbf::tc_max_plans_per_launch() == 0) ++tc_classes;
    seen.push_back(cls);
    if (p->inc) ++tc_classes;   // its incoherent-beam kernel
  }
  *n_launches = (int32_t)(b->ppf_cls.size() + 1 + b->bf_cls.size()) + tc_classes;
  return LBF_OK;
}

lbf_status lbf_batch_launch(lbf_batch_t b, void *stream) {
  if (!b || b->magic != kBatchMagic) return LBF_ESTATE;
  if (!b->graph[0] || !b->graph[1]) return LBF_ESTATE;
  cudaError_t e = cudaGraphLaunch(b->graph[b->graph_parity], (cudaStream_t)stream);
  if (e != cudaSuccess) return status_of(e);
  b->graph_parity ^= 1;
  advance(b);
  return LBF_OK;
}

lbf_status lbf_batch_tune(lbf_batch_t b, const void *const *d_in, void *const *d_out, void *stream, int32_t reps,
                          lbf_batch_tuning *out) {
  if (!b || b->magic != kBatchMagic) return LBF_ESTATE;
  if (reps < 1 || reps > 1000) return LBF_EINVAL;
  lbf_status s = check_buffers(b, d_in, d_out);
  if (s != LBF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = (int)b->plans.size();
  // spectra per filter-bank item: a quarter, half, or all of a stream's block (1024 >= M here)
  const int spcs[3] = {64, 256, 1024};
  // beam-former choices: 0 each plan's own; 1 plans with 9..64 beams switched between the few- and
  // many-beam kernels; 2 plans with more than 8 beams switched between the 128- and 64-beam tiles
  std::vector<int> choice[3];
  bool has[3] = {true, false, false};
  for (int k = 0; k < 3; ++k) choice[k].resize(n);
  for (int i = 0; i < n; ++i) {
    lbf_plan_t p = b->plans[i];
    const int v = p->variant;
    choice[0][i] = v;
    const bool fp32_many_ok = !p->tc && p->B > 8 && p->S <= lbf::many_beam_max_stations();
    const bool mid = fp32_many_ok && p->B <= 64;
    choice[1][i] = mid ? (v == 1 ? 2 : 1) : v;
    choice[2][i] = fp32_many_ok ? (v == 3 ? 2 : 3) : v;
    has[1] = has[1] || mid;
    has[2] = has[2] || fp32_many_ok;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_spc = b->spc, best_v = 0;
  lbf_batch_tuning t;
  std::memset(&t, 0, sizeof(t));
  cudaError_t e = cudaSuccess;
  int idx = 0;
  for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
    if (!has[v]) continue;
    b->variant = choice[v];
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      b->spc = spcs[k];
      e = cudaStreamSynchronize(st);
      fill_tables(b, 0, d_in, d_out);
      if (e == cudaSuccess) e = enqueue(b, 0, st);   // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue(b, 0, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      t.ms[idx] = ms;
      t.spc[idx] = spcs[k];
      t.mid_variant[idx] = v;
      ++idx;
      if (e == cudaSuccess && ms < best) { best = ms; best_spc = spcs[k]; best_v = v; }
    }
  }
  // the per-plan mode (each plan's own kernels in the graph), with the best beam-former choice
  bool best_pp = false;
  if (e == cudaSuccess) {
    b->variant = choice[best_v];
    b->per_plan = true;
    e = cudaStreamSynchronize(st);
    fill_tables(b, 0, d_in, d_out);
    if (e == cudaSuccess) e = enqueue(b, 0, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue(b, 0, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    t.ms[idx] = ms;
    t.spc[idx] = 0;
    t.mid_variant[idx] = best_v;
    ++idx;
    if (e == cudaSuccess && ms < best) { best = ms; best_pp = true; }
    b->per_plan = false;
  }
  t.n_candidates = idx;
  t.best_spc = best_pp ? 0 : best_spc;
  t.best_mid_variant = best_v;
  t.best_ms = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->spc = best_spc;
  b->variant = choice[best_v];
  b->per_plan = best_pp;
  // the candidate runs advanced nothing (parity-0 tables, histories untouched by design of the
  // tables: each run read hist[cur] and wrote hist[cur^1]); restart every stream cleanly
  for (lbf_plan_t p : b->plans) {
    if (e == cudaSuccess) e = cudaMemsetAsync(p->hist[0], 0, p->hist_bytes ? p->hist_bytes : 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->hist[1], 0, p->hist_bytes ? p->hist_bytes : 16, st);
    p->cur = 0;
  }
  free_graphs(b);
  if (out) *out = t;
  return status_of(e);
}

}  // extern "C"
