// capi.cu -- the C ABI of include/tersoff.h: context, neighbour build, batch planning and the
// stream-ordered evaluation calls. Host code only; kernels live in the other translation units.
#include <algorithm>
#include <atomic>
#include <iterator>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ctx.hpp"

using tsf::Ctx;

namespace tsf {
namespace {
std::atomic<long long> g_launches{0};
}
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
namespace {
std::atomic<uint64_t> g_buf_gen{0}, g_plan_gen{0};
}
uint64_t buffer_generation() { return g_buf_gen.load(); }
void bump_buffer_generation() { g_buf_gen.fetch_add(1); }
}  // namespace tsf

namespace {

int fail(tersoff_ctx *ctx, int code, const char *fmt, const char *detail = "") {
  if (ctx) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), fmt, detail);
    ctx->c.err = buf;
  }
  return code;
}

#define TSF_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(ctx, TERSOFF_E_CUDA, "CUDA error: %s", cudaGetErrorString(e_)); \
  } while (0)

inline cudaStream_t S(tersoff_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// The cluster size and kernel variant of every configuration for one precision, and one record per
// (configuration, cluster rank) of every launch bucket, longest configurations first. The plan does
// not depend on the number of parameter sets: a launch covers nconf x ntiles x cluster CTAs.
int build_plan(tersoff_ctx *ctx, int precision) {
  Ctx &c = ctx->c;
  tsf::BatchPlan &plan = precision == 64 ? c.plan64 : c.plan32;
  if (plan.precision == precision && !plan.buckets.empty()) return TERSOFF_OK;
  const int optin = tsf::batch_max_smem_optin();
  const size_t soft = std::min<size_t>((size_t)optin, 112 * 1024);  // two CTAs per SM
  struct Key {
    int mmax, cl;
    bool operator<(const Key &o) const { return mmax != o.mmax ? mmax < o.mmax : cl < o.cl; }
  };
  std::map<Key, std::vector<int>> groups;
  std::map<Key, size_t> smem, adj_smem, smem16, smem12;
  // bonds and pair slots of the atoms s0 .. s1-1 of one configuration (a0 <= s0 <= s1 <= a1), and where
  // they start (for an empty slice at the end: where the configuration's bonds end)
  auto bstart = [&](int s, int a1) { return s < a1 ? c.h_boff[s] : c.h_boff[a1 - 1] + c.h_m[a1 - 1]; };
  auto qstart = [&](int s, int a1) { return s < a1 ? c.h_poff[s] : c.h_poff[a1 - 1] + tsf::pair_slots(c.h_m[a1 - 1]); };
  for (int cf = 0; cf < c.C; ++cf) {
    const int a0 = c.h_atom_off[cf], a1 = c.h_atom_off[cf + 1], nat = a1 - a0;
    // the smallest cluster whose CTAs fit two per SM; failing that, the smallest of 8 or 16 CTAs that
    // fits at all (one CTA per SM). FP64 variants run one CTA per SM whatever their shared memory
    // (registers), so there clusters of 8 or more take the whole opt-in limit from the first pass.
    const bool one_per_sm = precision == 64;
    int chosen = 0;
    size_t need = 0;
    for (int pass = 0; pass < 2 && !chosen; ++pass) {
      for (int cl = pass == 0 ? 1 : 8; cl <= 16 && !chosen; cl *= 2) {
        if (cl > 1 && (cl / 2) >= nat) break;
        const int per = (nat + cl - 1) / cl;
        size_t mx = 0;
        for (int r = 0; r < cl; ++r) {
          const int s0 = a0 + std::min(nat, r * per), s1 = a0 + std::min(nat, (r + 1) * per);
          const int nb = bstart(s1, a1) - bstart(s0, a1), nq = qstart(s1, a1) - qstart(s0, a1);
          mx = std::max(mx, tsf::batch_smem_bytes_pt(precision, nb, nq, s1 - s0, cl));
        }
        if (mx <= (pass == 0 && !(one_per_sm && cl >= 8) ? soft : (size_t)optin)) {
          chosen = cl;
          need = mx;
        }
      }
    }
    if (!chosen) return fail(ctx, TERSOFF_E_UNSUPPORTED, "configuration too large for the batched kernels%s");
    const int mm = c.h_cfg_maxm[cf];
    int mmax = precision == 64 ? 8 : (mm <= 4 ? 4 : (mm <= 6 ? 6 : 8));
    Key k{mmax, chosen};
    groups[k].push_back(cf);
    smem[k] = std::max(smem[k], need);
    if (chosen == 1) {
      const int nb = bstart(a1, a1) - bstart(a0, a1), nq = qstart(a1, a1) - qstart(a0, a1);
      adj_smem[k] = std::max(adj_smem[k], tsf::adjoint_smem_bytes(nb, nq, nat));
      if (precision == 32 && mmax == 4) {
        smem16[k] = std::max(smem16[k], tsf::batch_smem_bytes_pt16(nb, nq, nat));
        smem12[k] = std::max(smem12[k], tsf::batch_smem_bytes_nw12(nb, nq, nat));
      }
    }
  }
  std::vector<tsf::CtaRec> recs;
  plan.buckets.clear();
  // largest clusters (longest items) first so that they start early
  std::vector<Key> keys;
  for (auto &g : groups) keys.push_back(g.first);
  std::sort(keys.begin(), keys.end(), [](const Key &x, const Key &y) {
    return x.cl != y.cl ? x.cl > y.cl : x.mmax > y.mmax;
  });
  for (const Key &k : keys) {
    std::vector<int> &cfgs = groups[k];
    auto cfg_bonds = [&](int x) {
      const int x0 = c.h_atom_off[x], x1 = c.h_atom_off[x + 1];
      return bstart(x1, x1) - bstart(x0, x1);
    };
    std::stable_sort(cfgs.begin(), cfgs.end(), [&](int x, int y) { return cfg_bonds(x) > cfg_bonds(y); });
    tsf::Bucket b;
    b.mmax = k.mmax;
    b.cluster = k.cl;
    b.precision = precision;
    b.smem = smem[k];
    b.adj_smem = adj_smem[k];
    // the gradient of configurations spread over a cluster, or beyond the adjoint kernel's shared
    // memory, takes the split path (evaluation, weights, tangent passes per atom slice)
    b.adj_split = k.cl > 1 || adj_smem[k] > (size_t)optin;
    b.smem16 = (k.cl == 1 && k.mmax == 4 && precision == 32) ? smem16[k] : 0;
    b.smem12 = (k.cl == 1 && k.mmax == 4 && precision == 32) ? smem12[k] : 0;
    b.item_off = (int)recs.size();
    b.uniform = true;
    for (int cf : cfgs) {
      const int f0 = cfgs.front();
      const int na = c.h_atom_off[cf + 1] - c.h_atom_off[cf], nf = c.h_atom_off[f0 + 1] - c.h_atom_off[f0];
      const int ba = cfg_bonds(cf), bf = cfg_bonds(f0);
      if (na != nf || ba != bf) b.uniform = false;
    }
    for (int cf : cfgs) {
      const int a0 = c.h_atom_off[cf], a1 = c.h_atom_off[cf + 1], nat = a1 - a0;
      const int per = (nat + k.cl - 1) / k.cl;
      for (int r = 0; r < k.cl; ++r) {
        const int s0 = a0 + std::min(nat, r * per), s1 = a0 + std::min(nat, (r + 1) * per);
        tsf::CtaRec q;
        q.c = cf;
        q.s0 = s0;
        q.ns = s1 - s0;
        q.B0 = bstart(s0, a1);
        q.nb = bstart(s1, a1) - q.B0;
        q.Q0 = qstart(s0, a1);
        q.nq = qstart(s1, a1) - q.Q0;
        q.cb0 = c.h_boff[a0];
        q.nat = nat;
        q.pad = 0;
        q.inv_nat = 1.0 / (double)nat;
        recs.push_back(q);
        if (b.adj_split)
          b.adj_split_smem = std::max(b.adj_split_smem, tsf::adjoint_split_smem_bytes(q.nb, q.nq, q.ns));
      }
    }
    b.nitems = ((int)recs.size() - b.item_off) / k.cl;   // configurations in the bucket
    plan.buckets.push_back(b);
  }
  TSF_CUDA(plan.items.ensure(std::max<size_t>(1, recs.size()) * sizeof(tsf::CtaRec)));
  TSF_CUDA(cudaMemcpy(plan.items.p, recs.data(), recs.size() * sizeof(tsf::CtaRec), cudaMemcpyHostToDevice));
  plan.precision = precision;
  plan.gen = ++tsf::g_plan_gen;
  return TERSOFF_OK;
}

uint64_t bits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, sizeof(u));
  return u;
}

// Run a per-call launch sequence through a CUDA graph: captured on the context's private stream the
// first time (or whenever the key changed), then replayed on `s` with one graph launch. Direct
// launches while kernel timing is on, while graphs are off, or when `s` is itself being captured.
template <typename Issue>
int run_graphed(tersoff_ctx *ctx, tsf::GraphCache &g, std::vector<uint64_t> key, cudaStream_t s, Issue &&issue) {
  Ctx &c = ctx->c;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TSF_CUDA(cudaStreamIsCapturing(s, &cs));
  if (!c.graphs || c.timer.on || cs != cudaStreamCaptureStatusNone) {
    TSF_CUDA(issue(s));
    return TERSOFF_OK;
  }
  key.push_back(tsf::buffer_generation());
  key.push_back((uint64_t)c.device);
  key.push_back((uint64_t)c.form);
  if (!g.exec || g.key != key) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    if (!c.cap_stream) TSF_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    const int64_t n0 = tersoff_kernel_launches();
    TSF_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t ei = issue(c.cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c.cap_stream, &graph);
    const int kernels = (int)(tersoff_kernel_launches() - n0);
    tsf::count_launches(-kernels);   // captured, not executed
    if (ei != cudaSuccess || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(ctx, TERSOFF_E_CUDA, "CUDA error while capturing: %s",
                  cudaGetErrorString(ei != cudaSuccess ? ei : ec));
    }
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return fail(ctx, TERSOFF_E_CUDA, "CUDA error: %s", cudaGetErrorString(e));
    }
    g.key = std::move(key);
    g.kernels = kernels;
  }
  TSF_CUDA(cudaGraphLaunch(g.exec, s));
  tsf::count_launches(g.kernels);
  return TERSOFF_OK;
}

// Queue the fitness launch sequence of tersoff_fitness on the current schedule (arguments checked).
int queue_fitness(tersoff_ctx *ctx, const double *params, int32_t P, const tersoff_targets *tg, const double *w,
                  int32_t precision, double *Z, double *Zq, double *Sq, tersoff_stream stream) {
  Ctx &c = ctx->c;
  cudaSetDevice(c.device);
  int rc = build_plan(ctx, precision);
  if (rc) return rc;
  if (precision == 64 && (rc = tsf::ensure_geom64(ctx, S(stream)))) return rc;
  TSF_CUDA(c.part.ensure((size_t)P * c.C * tsf::kResidualTerms * sizeof(double)));
  TSF_CUDA(c.dpart.ensure((size_t)c.C * 3 * sizeof(double)));
  TSF_CUDA(c.work.ensure((size_t)P * (c.form ? 16 : 8) * sizeof(double)));
  TSF_CUDA(c.counters.ensure(64 * sizeof(int)));
  tsf::BatchOut o = {};
  o.form = c.form;
  o.counters = c.counters.as<int>();
  o.consts = c.work.p;
  o.tE = tg->E;
  o.tW = tg->W;
  o.tF = tg->F;
  o.tmask = tg->mask;
  o.part = c.part.as<double>();
  o.dpart = c.dpart.as<double>();
  o.pdl = c.pdl;
  const tsf::BatchPlan &plan = precision == 64 ? c.plan64 : c.plan32;
  const double w0 = w[0], w1 = w[1], w2 = w[2];
  const tersoff_targets t = *tg;
  std::vector<uint64_t> key = {(uint64_t)precision, (uint64_t)P, (uint64_t)(uintptr_t)params,
                               (uint64_t)(uintptr_t)t.E, (uint64_t)(uintptr_t)t.W, (uint64_t)(uintptr_t)t.F,
                               (uint64_t)(uintptr_t)t.mask, bits(w0), bits(w1), bits(w2), (uint64_t)(uintptr_t)Z,
                               (uint64_t)(uintptr_t)Zq, (uint64_t)(uintptr_t)Sq, plan.gen, (uint64_t)c.C,
                               (uint64_t)c.Ntot, (uint64_t)c.pdl, (uint64_t)c.wait_spins};
  return run_graphed(ctx, c.g_fitness, std::move(key), S(stream), [&](cudaStream_t s) {
    cudaError_t e = tsf::launch_batch(c, plan, params, P, tsf::kModeFitness, o, s);
    if (e == cudaSuccess)
      e = tsf::launch_fitness_finalize(P, c.C, o.part, o.dpart, w0, w1, w2, Z, Zq, Sq, o.pdl, s);
    return e;
  });
}

}  // namespace

namespace tsf {
// Host side of a neighbour build whose kernel is queued: wait for its counts and status (copied to
// pinned memory by the build), report its errors, and build or keep the work schedules.
int finish_build(tersoff_ctx *ctx) {
  Ctx &c = ctx->c;
  if (!c.pending) return c.built ? TERSOFF_OK : fail(ctx, TERSOFF_E_STATE, "call tersoff_build_neighbors first%s");
  c.pending = false;
  TSF_CUDA(cudaSetDevice(c.device));
  TSF_CUDA(cudaEventSynchronize(c.stage_event));
  const int64_t N = c.Ntot;
  const int C = c.C;
  const int *h_cnt = c.hp_stage.as<int>();
  const unsigned hst = *reinterpret_cast<const unsigned *>(h_cnt + N);   // the build's own status bits
  if (hst & TERSOFF_STATUS_NONFINITE) return fail(ctx, TERSOFF_E_NONFINITE, "non-finite positions or box%s");
  if (hst & TERSOFF_STATUS_NBR_OVERFLOW) return fail(ctx, TERSOFF_E_NBR_OVERFLOW, "an atom has more than max_nbr neighbours%s");
  const bool same_counts = c.pending_same_layout && (int64_t)c.h_cnt.size() == N &&
                           std::equal(c.h_cnt.begin(), c.h_cnt.end(), h_cnt);
  if (!same_counts) {
    // new schedules overwrite the record buffers of the old ones: queued launches (a fitness call
    // queued ahead of this check among them) must be done with them first
    TSF_CUDA(cudaDeviceSynchronize());
    // host copy of the CSR the device built (same prefix sums over the configurations in order)
    c.h_cnt.assign(h_cnt, h_cnt + N);
    for (BatchPlan *pl : {&c.plan32, &c.plan64}) {
      pl->precision = 0;
      pl->gen = 0;
      pl->buckets.clear();
    }
    // host copy of the bond and pair-slot offsets the device built: per configuration from its fixed
    // base (atom_off[c] * M and atom_off[c] * pair_slots(M)), prefix sums over its atoms
    c.h_m.assign(N, 0);
    c.h_boff.assign(N, 0);
    c.h_poff.assign(N, 0);
    c.h_cfg_maxm.assign(C, 0);
    int maxm = 0;
    int64_t nbonds = 0;
    for (int k = 0; k < C; ++k) {
      int b = c.h_atom_off[k] * c.M, q = c.h_atom_off[k] * pair_slots(c.M);
      for (int i = c.h_atom_off[k]; i < c.h_atom_off[k + 1]; ++i) {
        const int m = std::min(c.h_cnt[i], c.M);
        c.h_m[i] = m;
        c.h_boff[i] = b;
        c.h_poff[i] = q;
        b += m;
        q += pair_slots(m);
        nbonds += m;
        maxm = std::max(maxm, c.h_cnt[i]);
        c.h_cfg_maxm[k] = std::max(c.h_cfg_maxm[k], c.h_cnt[i]);
      }
    }
    c.max_m = maxm;
    c.nbonds = nbonds;
    c.Btot = N * c.M;
    c.Qtot = N * pair_slots(c.M);
  }
  if (c.max_m <= 8) {
    int rc = build_plan(ctx, 32);
    if (rc) return rc;
    rc = build_plan(ctx, 64);
    if (rc) return rc;
  }
  c.built = true;
  return TERSOFF_OK;
}

// FP64 geometry records, built on the first FP64 evaluation after a neighbour build (stream-ordered).
int ensure_geom64(tersoff_ctx *ctx, cudaStream_t s) {
  Ctx &c = ctx->c;
  if (c.geom64) return TERSOFF_OK;
  // the buffers were allocated by the neighbour build with the capacity of full lists
  const size_t B = std::max<int64_t>(1, c.Btot), Q = std::max<int64_t>(1, c.Qtot);
  TSF_CUDA(c.gA64.ensure(B * sizeof(tsf::dvec4)));
  TSF_CUDA(c.gB64.ensure(B * sizeof(tsf::dvec4)));
  TSF_CUDA(c.gcos64.ensure(Q * sizeof(double)));
  TSF_CUDA(launch_geometry64(c.Ntot, c.M, c.atom_cfg.as<int>(), c.atom_off.as<int>(), c.brev.as<int>(),
                             c.pos.as<double>(), c.box.as<double>(), c.cnt.as<int>(), c.nbr.as<int>(),
                             c.shift.as<char4>(), c.boff.as<int>(), c.poff.as<int>(), c.R1, c.R2, c.gA64.p,
                             c.gB64.p, c.gcos64.p, pair_slots(std::min(c.max_m, c.M)), s));
  c.geom64 = true;
  return TERSOFF_OK;
}
}  // namespace tsf

extern "C" {

int tersoff_create(tersoff_ctx **out, int device) {
  if (!out) return TERSOFF_E_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TERSOFF_E_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return TERSOFF_E_CUDA;
  tersoff_ctx *ctx = new tersoff_ctx();
  ctx->c.device = device;
  // two words: the context's status, then the last neighbour build's own
  if (ctx->c.status.ensure(2 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(ctx->c.status.p, 0, 2 * sizeof(unsigned)) != cudaSuccess) {
    delete ctx;
    return TERSOFF_E_CUDA;
  }
  // set-up of the allocation-free fitness call on this device: the device address of its scratch array
  // (loads the array's module, which holds it); a failure here is reported by that call
  void *scratch = nullptr;
  (void)tsf::static_scratch_address(device, &scratch);
  *out = ctx;
  return TERSOFF_OK;
}

void tersoff_destroy(tersoff_ctx *ctx) {
  if (!ctx) return;
  Ctx &c = ctx->c;
  cudaSetDevice(c.device);
  cudaDeviceSynchronize();
  tsf::DevBuf *bufs[] = {&c.status, &c.atom_off, &c.atom_cfg, &c.pos, &c.box, &c.counters,
                         &c.cnt, &c.nbr, &c.shift, &c.boff, &c.poff, &c.brev, &c.gA32, &c.gB32,
                         &c.gcos32, &c.gA64, &c.gB64, &c.gcos64, &c.ameta, &c.arev, &c.part, &c.dpart, &c.work,
                         &c.tf4, &c.gpart, &c.adj_v, &c.adj_ew, &c.adj_aw, &c.adj_gsplit,
                         &c.plan32.items, &c.plan64.items, &c.md_pos, &c.md_cnt, &c.md_nbr,
                         &c.md_shift, &c.md_cells, &c.md_cellcnt, &c.md_Pij, &c.md_red,
                         &c.md_keys, &c.md_ke, &c.md_boxd};
  for (auto *b : bufs) b->release();
  c.hp_stage.release();
  if (c.stage_event) cudaEventDestroy(c.stage_event);
  if (c.build_done) cudaEventDestroy(c.build_done);
  if (c.copy_stream) cudaStreamDestroy(c.copy_stream);
  for (cudaEvent_t ev : c.timer.ev) cudaEventDestroy(ev);
  if (c.g_fitness.exec) cudaGraphExecDestroy(c.g_fitness.exec);
  for (cudaStream_t st : c.side) cudaStreamDestroy(st);
  for (cudaEvent_t ev : c.side_ev) cudaEventDestroy(ev);
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  delete ctx;
}

int64_t tersoff_kernel_launches(void) { return (int64_t)tsf::g_launches.load(); }

int tersoff_set_form(tersoff_ctx *ctx, int32_t form) {
  if (!ctx) return TERSOFF_E_ARG;
  if (form != TERSOFF_FORM_MINIMAL && form != TERSOFF_FORM_TERSOFF) return fail(ctx, TERSOFF_E_ARG, "unknown form%s");
  ctx->c.form = form;
  return TERSOFF_OK;
}

int tersoff_set_wait_limit(tersoff_ctx *ctx, int64_t spins) {
  if (!ctx) return TERSOFF_E_ARG;
  if (spins > 0xffffffffll) return fail(ctx, TERSOFF_E_ARG, "spins must be below 2^32%s");
  ctx->c.wait_spins = spins < 0 ? -1 : spins;
  return TERSOFF_OK;
}

int tersoff_set_launch_mode(tersoff_ctx *ctx, int32_t mode) {
  if (!ctx) return TERSOFF_E_ARG;
  if (mode & ~(TERSOFF_LAUNCH_GRAPHS | TERSOFF_LAUNCH_PDL)) return fail(ctx, TERSOFF_E_ARG, "unknown launch mode bits%s");
  ctx->c.graphs = (mode & TERSOFF_LAUNCH_GRAPHS) != 0;
  ctx->c.pdl = (mode & TERSOFF_LAUNCH_PDL) != 0;
  return TERSOFF_OK;
}

int tersoff_profile(tersoff_ctx *ctx, int32_t enable) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  TSF_CUDA(cudaSetDevice(c.device));
  c.timer.on = false;
  c.timer.n = 0;
  if (!enable) return TERSOFF_OK;
  while (c.timer.ev.size() < 2 * (size_t)tsf::KernelTimer::kCap) {
    cudaEvent_t ev = nullptr;
    TSF_CUDA(cudaEventCreate(&ev));
    c.timer.ev.push_back(ev);
  }
  c.timer.on = true;
  return TERSOFF_OK;
}

int tersoff_profile_read(tersoff_ctx *ctx, int64_t *count, double *ms) {
  if (!ctx || !count || !ms) return fail(ctx, TERSOFF_E_ARG, "null argument%s");
  Ctx &c = ctx->c;
  TSF_CUDA(cudaSetDevice(c.device));
  double total = 0.0;
  for (int i = 0; i < c.timer.n; ++i) {
    float t = 0.f;
    TSF_CUDA(cudaEventSynchronize(c.timer.ev[2 * i + 1]));
    TSF_CUDA(cudaEventElapsedTime(&t, c.timer.ev[2 * i], c.timer.ev[2 * i + 1]));
    total += t;
  }
  *count = c.timer.n;
  *ms = total;
  c.timer.n = 0;
  return TERSOFF_OK;
}

const char *tersoff_last_error(const tersoff_ctx *ctx) { return ctx ? ctx->c.err.c_str() : ""; }

int tersoff_get_status(tersoff_ctx *ctx, tersoff_stream stream) {
  if (!ctx) return -1;
  cudaSetDevice(ctx->c.device);
  unsigned v = 0;
  if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return -1;
  if (cudaMemcpy(&v, ctx->c.status.p, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (cudaMemset(ctx->c.status.p, 0, sizeof(unsigned)) != cudaSuccess) return -1;
  return (int)v;
}

int tersoff_build_neighbors(tersoff_ctx *ctx, const tersoff_configs *cfg, double R1, double R2,
                            int32_t max_nbr, tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (c.pending) tsf::finish_build(ctx);   // a previous build still unchecked: settle it (errors dropped)
  const bool was_built = c.built;
  c.built = false;
  if (!cfg || !cfg->atom_off || !cfg->pos || !cfg->box) return fail(ctx, TERSOFF_E_ARG, "null configuration pointer%s");
  if (cfg->C < 1) return fail(ctx, TERSOFF_E_ARG, "C must be >= 1%s");
  if (!(R1 > 0.0 && R2 > R1 && std::isfinite(R2))) return fail(ctx, TERSOFF_E_ARG, "need 0 < R1 < R2%s");
  if (max_nbr < 1 || max_nbr > 32) return fail(ctx, TERSOFF_E_ARG, "max_nbr must be in [1, 32]%s");
  const int C = cfg->C;
  if (cfg->atom_off[0] != 0) return fail(ctx, TERSOFF_E_ARG, "atom_off[0] must be 0%s");
  for (int k = 0; k < C; ++k) {
    const int n = cfg->atom_off[k + 1] - cfg->atom_off[k];
    if (n < 1 || n > 1024) return fail(ctx, TERSOFF_E_ARG, "every configuration needs 1..1024 atoms%s");
  }
  cudaSetDevice(c.device);
  cudaStream_t s = S(stream);
  const int64_t N = cfg->atom_off[C];
  const int M = max_nbr;
  // the atom table (and the plans, if every neighbour count turns out unchanged) of the previous
  // build are reused when this build has the same configuration sizes, cutoffs and list width
  const bool same_layout = was_built && c.C == C && c.M == M && c.R1 == R1 && c.R2 == R2 &&
                           (int64_t)c.h_atom_off.size() == C + 1 &&
                           std::equal(c.h_atom_off.begin(), c.h_atom_off.end(), cfg->atom_off);
  // the pinned staging buffer is reused: wait for the uploads of the previous build to finish
  if (c.stage_event) TSF_CUDA(cudaEventSynchronize(c.stage_event));
  else TSF_CUDA(cudaEventCreateWithFlags(&c.stage_event, cudaEventDisableTiming));
  c.C = C;
  c.Ntot = N;
  c.M = M;
  c.R1 = R1;
  c.R2 = R2;
  TSF_CUDA(c.hp_stage.ensure((size_t)(2 * N + C + 8) * sizeof(int)));
  int *hp = c.hp_stage.as<int>();
  if (!same_layout) {
    c.h_atom_off.assign(cfg->atom_off, cfg->atom_off + C + 1);
    // the schedules are rebuilt into the same record buffers once the counts are known: queued
    // launches must be done with the old records first
    TSF_CUDA(cudaDeviceSynchronize());
    for (tsf::BatchPlan *pl : {&c.plan32, &c.plan64}) {
      pl->precision = 0;
      pl->gen = 0;
      pl->buckets.clear();
    }
    TSF_CUDA(c.atom_off.ensure((C + 1) * sizeof(int)));
    TSF_CUDA(c.atom_cfg.ensure(N * sizeof(int)));
    int *h_off = hp, *h_cfg = hp + (C + 1);
    std::copy(cfg->atom_off, cfg->atom_off + C + 1, h_off);
    for (int k = 0; k < C; ++k)
      for (int i = cfg->atom_off[k]; i < cfg->atom_off[k + 1]; ++i) h_cfg[i] = k;
    TSF_CUDA(cudaMemcpyAsync(c.atom_off.p, h_off, (C + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    TSF_CUDA(cudaMemcpyAsync(c.atom_cfg.p, h_cfg, N * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  // bond and pair-slot arrays are written by the device before the host knows the counts: they get
  // the capacity of full lists (M bonds and pair_slots(M) slots per atom)
  const int64_t bond_cap = std::max<int64_t>(1, N * M), slot_cap = std::max<int64_t>(1, N * tsf::pair_slots(M));
  TSF_CUDA(c.pos.ensure(N * 3 * sizeof(double)));
  TSF_CUDA(c.box.ensure((size_t)C * 9 * sizeof(double)));
  TSF_CUDA(c.cnt.ensure(N * sizeof(int)));
  TSF_CUDA(c.nbr.ensure(N * M * sizeof(int)));
  TSF_CUDA(c.shift.ensure(N * M * sizeof(char4)));
  TSF_CUDA(c.boff.ensure((N + 1) * sizeof(int)));
  TSF_CUDA(c.poff.ensure((N + 1) * sizeof(int)));
  TSF_CUDA(c.brev.ensure(bond_cap * sizeof(int)));
  TSF_CUDA(c.ameta.ensure(std::max<int64_t>(1, N) * sizeof(int)));
  TSF_CUDA(c.arev.ensure(std::max<int64_t>(1, N) * sizeof(int4)));
  TSF_CUDA(c.gA32.ensure(bond_cap * sizeof(float4)));
  TSF_CUDA(c.gB32.ensure(bond_cap * sizeof(float4)));
  TSF_CUDA(c.gcos32.ensure(slot_cap * sizeof(float)));
  // everything the later calls of this build need is allocated here, so that those calls (the
  // allocation-free fitness among them) allocate nothing: the FP64 geometry records (computed on the
  // first FP64 use), the work-schedule records of both precisions, the side streams, and the code of
  // the fitness kernels (loaded up front instead of lazily on their first launch)
  TSF_CUDA(c.gA64.ensure(bond_cap * sizeof(tsf::dvec4)));
  TSF_CUDA(c.gB64.ensure(bond_cap * sizeof(tsf::dvec4)));
  TSF_CUDA(c.gcos64.ensure(slot_cap * sizeof(double)));
  TSF_CUDA(c.plan32.items.ensure((size_t)C * tsf::kMaxClusterCtas * sizeof(tsf::CtaRec)));
  TSF_CUDA(c.plan64.items.ensure((size_t)C * tsf::kMaxClusterCtas * sizeof(tsf::CtaRec)));
  TSF_CUDA(tsf::ensure_side_streams(c));
  if (!c.preloaded) {
    TSF_CUDA(tsf::preload_fitness_kernels());
    c.preloaded = true;
  }
  if (!c.copy_stream) TSF_CUDA(cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking));
  if (!c.build_done) TSF_CUDA(cudaEventCreateWithFlags(&c.build_done, cudaEventDisableTiming));
  int nat_max = 1;
  for (int k = 0; k < C; ++k) nat_max = std::max(nat_max, cfg->atom_off[k + 1] - cfg->atom_off[k]);
  TSF_CUDA(cudaMemsetAsync(c.status.p, 0, 2 * sizeof(unsigned), s));   // status and build status
  unsigned *st = c.status.as<unsigned>();
  tsf::BuildLaunch L = {};
  L.C = C;
  L.M = M;
  L.Ntot = N;
  L.R1 = R1;
  L.R2 = R2;
  L.atom_off = c.atom_off.as<int>();
  L.pos_in = cfg->pos;
  L.box_in = cfg->box;
  L.pos = c.pos.as<double>();
  L.box = c.box.as<double>();
  L.cnt = c.cnt.as<int>();
  L.nbr = c.nbr.as<int>();
  L.shift = c.shift.as<char4>();
  L.boff = c.boff.as<int>();
  L.poff = c.poff.as<int>();
  L.brev = c.brev.as<int>();
  L.gA = c.gA32.as<float4>();
  L.gB = c.gB32.as<float4>();
  L.gcos = c.gcos32.as<float>();
  L.ameta = c.ameta.as<int>();
  L.arev = c.arev.as<int4>();
  L.status = st;
  L.build_status = c.status.as<unsigned>() + 1;
  L.nat_max = nat_max;
  TSF_CUDA(tsf::launch_build_batch(L, s));
  // neighbour counts and the build's status go back to pinned host memory on a side stream, beside
  // whatever the caller queues next on `stream`; the host reads them (and builds or keeps the work
  // schedule) when the next call needs the build
  TSF_CUDA(cudaEventRecord(c.build_done, s));
  TSF_CUDA(cudaStreamWaitEvent(c.copy_stream, c.build_done, 0));
  TSF_CUDA(cudaMemcpyAsync(hp, c.cnt.p, N * sizeof(int), cudaMemcpyDeviceToHost, c.copy_stream));
  TSF_CUDA(cudaMemcpyAsync(hp + N, c.status.as<unsigned>() + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           c.copy_stream));
  TSF_CUDA(cudaEventRecord(c.stage_event, c.copy_stream));
  c.geom64 = false;
  c.pending = true;
  c.pending_same_layout = same_layout;
  return TERSOFF_OK;
}

int tersoff_export_neighbors(tersoff_ctx *ctx, int32_t *cnt, int32_t *nbr, int8_t *shift) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (int rc = tsf::finish_build(ctx)) return rc;
  cudaSetDevice(c.device);
  const int64_t N = c.Ntot, M = c.M;
  if (cnt) TSF_CUDA(cudaMemcpy(cnt, c.cnt.p, N * sizeof(int), cudaMemcpyDeviceToHost));
  if (nbr) TSF_CUDA(cudaMemcpy(nbr, c.nbr.p, N * M * sizeof(int), cudaMemcpyDeviceToHost));
  if (shift) {
    std::vector<char4> tmp(N * M);
    TSF_CUDA(cudaMemcpy(tmp.data(), c.shift.p, N * M * sizeof(char4), cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < N * M; ++k) {
      shift[3 * k] = tmp[k].x;
      shift[3 * k + 1] = tmp[k].y;
      shift[3 * k + 2] = tmp[k].z;
    }
  }
  return TERSOFF_OK;
}

int tersoff_build_info(tersoff_ctx *ctx, int64_t *ntot, int64_t *nbonds, int32_t *max_m) {
  if (!ctx) return TERSOFF_E_ARG;
  if (int rc = tsf::finish_build(ctx)) return rc;
  if (ntot) *ntot = ctx->c.Ntot;
  if (nbonds) *nbonds = ctx->c.nbonds;
  if (max_m) *max_m = ctx->c.max_m;
  return TERSOFF_OK;
}

int tersoff_eval(tersoff_ctx *ctx, const double *params, int32_t P, int32_t precision, double *E,
                 void *F, double *W, tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (int rc = tsf::finish_build(ctx)) return rc;
  if (!params || P < 1) return fail(ctx, TERSOFF_E_ARG, "need params and P >= 1%s");
  if (precision != 32 && precision != 64) return fail(ctx, TERSOFF_E_ARG, "precision must be 32 or 64%s");
  if (c.max_m > 8) return fail(ctx, TERSOFF_E_UNSUPPORTED, "an atom has more than 8 neighbours%s");
  cudaSetDevice(c.device);
  int rc = build_plan(ctx, precision);
  if (rc) return rc;
  if (precision == 64 && (rc = tsf::ensure_geom64(ctx, S(stream)))) return rc;
  TSF_CUDA(c.work.ensure((size_t)P * (c.form ? 16 : 8) * sizeof(double)));
  TSF_CUDA(c.counters.ensure(64 * sizeof(int)));
  tsf::BatchOut o = {};
  o.form = c.form;
  o.counters = c.counters.as<int>();
  o.E = E;
  o.F = F;
  o.W = W;
  o.consts = c.work.p;
  TSF_CUDA(tsf::launch_batch(c, precision == 64 ? c.plan64 : c.plan32, params, P, tsf::kModeEval, o, S(stream)));
  return TERSOFF_OK;
}

int tersoff_fitness(tersoff_ctx *ctx, const double *params, int32_t P, const tersoff_targets *tg,
                    const double *w, int32_t precision, double *Z, double *Zq, double *Sq,
                    tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (!params || P < 1 || !tg || !w || !Z) return fail(ctx, TERSOFF_E_ARG, "null argument or P < 1%s");
  if (!tg->E || !tg->W || !tg->F || !tg->mask) return fail(ctx, TERSOFF_E_ARG, "null target pointer%s");
  if (precision != 32 && precision != 64) return fail(ctx, TERSOFF_E_ARG, "precision must be 32 or 64%s");
  // After a rebuild of the same layout whose neighbour counts the host has not checked yet, the
  // launch is queued on the previous schedule before the host waits for the counts, so the GPU goes
  // from the build straight to the fitness. The batched kernel skips every work item whose record
  // no longer matches the device's bond CSR; if the counts did change, the host (which then drains
  // the device before rebuilding the schedule) clears the status bits of that launch and queues the
  // call again on the new schedule.
  const bool speculate = c.pending && c.pending_same_layout && precision == 32 && c.plan32.precision == 32 &&
                         !c.plan32.buckets.empty() && c.max_m <= 8;
  if (speculate) {
    const uint64_t gen = c.plan32.gen;
    if (int rc = queue_fitness(ctx, params, P, tg, w, precision, Z, Zq, Sq, stream)) return rc;
    if (int rc = tsf::finish_build(ctx)) return rc;
    if (c.plan32.gen == gen && !c.plan32.buckets.empty()) return TERSOFF_OK;
    TSF_CUDA(cudaMemsetAsync(c.status.p, 0, sizeof(unsigned), S(stream)));
  } else if (int rc = tsf::finish_build(ctx)) {
    return rc;
  }
  if (c.max_m > 8) return fail(ctx, TERSOFF_E_UNSUPPORTED, "an atom has more than 8 neighbours%s");
  return queue_fitness(ctx, params, P, tg, w, precision, Z, Zq, Sq, stream);
}

int tersoff_autotune(tersoff_ctx *ctx, const double *params, int32_t P, const tersoff_targets *tg,
                     int32_t precision, int32_t reps, double *best_ms, int32_t *tried, tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (c.form != 0) return fail(ctx, TERSOFF_E_UNSUPPORTED, "only the batched evaluation and fitness take the Tersoff form%s");
  if (int rc = tsf::finish_build(ctx)) return rc;
  if (!params || P < 1 || !tg) return fail(ctx, TERSOFF_E_ARG, "null argument or P < 1%s");
  if (!tg->E || !tg->W || !tg->F || !tg->mask) return fail(ctx, TERSOFF_E_ARG, "null target pointer%s");
  if (precision != 32 && precision != 64) return fail(ctx, TERSOFF_E_ARG, "precision must be 32 or 64%s");
  if (reps < 1 || reps > 100) return fail(ctx, TERSOFF_E_ARG, "reps must be in [1, 100]%s");
  if (c.max_m > 8) return fail(ctx, TERSOFF_E_UNSUPPORTED, "an atom has more than 8 neighbours%s");
  cudaSetDevice(c.device);
  int rc = build_plan(ctx, precision);
  if (rc) return rc;
  if (precision == 64 && (rc = tsf::ensure_geom64(ctx, S(stream)))) return rc;
  TSF_CUDA(c.part.ensure((size_t)P * c.C * tsf::kResidualTerms * sizeof(double)));
  TSF_CUDA(c.dpart.ensure((size_t)c.C * 3 * sizeof(double)));
  TSF_CUDA(c.work.ensure((size_t)P * (c.form ? 16 : 8) * sizeof(double)));
  TSF_CUDA(c.counters.ensure(64 * sizeof(int)));
  tsf::BatchOut o = {};
  o.form = c.form;
  o.counters = c.counters.as<int>();
  o.consts = c.work.p;
  o.tE = tg->E;
  o.tW = tg->W;
  o.tF = tg->F;
  o.tmask = tg->mask;
  o.part = c.part.as<double>();
  o.dpart = c.dpart.as<double>();
  o.pdl = c.pdl;
  tsf::BatchPlan &plan = precision == 64 ? c.plan64 : c.plan32;
  float ms = 0.f;
  int n = 0;
  TSF_CUDA(tsf::autotune_batch(c, plan, params, P, tsf::kModeFitness, o, reps, S(stream), &ms, &n));
  plan.gen = ++tsf::g_plan_gen;   // captured launch sequences of the old schedule are stale
  if (best_ms) *best_ms = ms;
  if (tried) *tried = n;
  return TERSOFF_OK;
}

int tersoff_set_schedule(tersoff_ctx *ctx, int32_t precision, int32_t P, int32_t tile, int32_t warps,
                         int32_t items_per_config, int32_t narrow) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (int rc = tsf::finish_build(ctx)) return rc;
  if (precision != 32 && precision != 64) return fail(ctx, TERSOFF_E_ARG, "precision must be 32 or 64%s");
  if (P < 1 || items_per_config < 1 || (tile != 32 && tile != 16) || (warps != 8 && warps != 12) ||
      (narrow != 0 && narrow != 1))
    return fail(ctx, TERSOFF_E_ARG, "need P >= 1, tile 32 or 16, warps 8 or 12, items_per_config >= 1, narrow 0 or 1%s");
  if (c.max_m > 8) return fail(ctx, TERSOFF_E_UNSUPPORTED, "an atom has more than 8 neighbours%s");
  int rc = build_plan(ctx, precision);
  if (rc) return rc;
  tsf::BatchPlan &plan = precision == 64 ? c.plan64 : c.plan32;
  for (tsf::Bucket &b : plan.buckets) {
    b.tune_P = P;
    b.tune_mode = tsf::kModeFitness;
    b.tune_pt = (tile == 16 && b.smem16 > 0) ? 16 : 32;
    b.tune_nw = (b.tune_pt == 32 && warps == 12 && b.smem12 > 0) ? 12 : 8;
    b.tune_per_conf = items_per_config;
    b.tune_narrow = narrow;
  }
  plan.gen = ++tsf::g_plan_gen;
  return TERSOFF_OK;
}

int tersoff_schedule_info(tersoff_ctx *ctx, int32_t precision, int32_t bucket, int32_t *info) {
  if (!ctx || !info) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (int rc = tsf::finish_build(ctx)) return rc;
  if (precision != 32 && precision != 64) return fail(ctx, TERSOFF_E_ARG, "precision must be 32 or 64%s");
  if (c.max_m > 8) return fail(ctx, TERSOFF_E_UNSUPPORTED, "an atom has more than 8 neighbours%s");
  int rc = build_plan(ctx, precision);
  if (rc) return rc;
  const tsf::BatchPlan &plan = precision == 64 ? c.plan64 : c.plan32;
  if (bucket < 0) {
    info[0] = (int32_t)plan.buckets.size();
    return TERSOFF_OK;
  }
  if (bucket >= (int)plan.buckets.size()) return fail(ctx, TERSOFF_E_ARG, "bucket index out of range%s");
  const tsf::Bucket &b = plan.buckets[bucket];
  const bool tuned = b.tune_mode >= 0;
  info[0] = b.mmax;
  info[1] = b.cluster;
  info[2] = b.nitems;
  info[3] = tuned ? b.tune_P : 0;
  info[4] = tuned ? b.tune_pt : 32;
  info[5] = tuned ? b.tune_per_conf : 0;
  info[6] = tuned ? b.tune_narrow : 1;
  info[7] = tuned ? b.tune_nw : 8;
  return TERSOFF_OK;
}

int tersoff_param_grad(tersoff_ctx *ctx, const double *params, int32_t P, const tersoff_targets *tg,
                       const double *w, int32_t loss, double *L, double *dL, tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (int rc = tsf::finish_build(ctx)) return rc;
  if (!params || P < 1 || !tg || !w || !L || !dL) return fail(ctx, TERSOFF_E_ARG, "null argument or P < 1%s");
  if (!tg->E || !tg->W || !tg->F || !tg->mask) return fail(ctx, TERSOFF_E_ARG, "null target pointer%s");
  if (loss != TERSOFF_LOSS_SQ && loss != TERSOFF_LOSS_Z) return fail(ctx, TERSOFF_E_ARG, "unknown loss%s");
  if (c.max_m > 8) return fail(ctx, TERSOFF_E_UNSUPPORTED, "an atom has more than 8 neighbours%s");
  if (int rc = build_plan(ctx, 32)) return rc;
  cudaSetDevice(c.device);
  const int NG = c.form ? 27 : 18;
  TSF_CUDA(c.part.ensure((size_t)P * c.C * 3 * sizeof(double)));
  TSF_CUDA(c.dpart.ensure((size_t)c.C * 3 * sizeof(double)));
  TSF_CUDA(c.gpart.ensure((size_t)P * c.C * NG * sizeof(double)));
  TSF_CUDA(c.work.ensure((size_t)P * 16 * sizeof(double)));
  TSF_CUDA(c.tf4.ensure((size_t)c.Ntot * sizeof(tsf::dvec4)));
  TSF_CUDA(c.counters.ensure(64 * sizeof(int)));
  {
    // split-path workspaces: v = 2 (F - F*) [Ntot][3][ldP], E and W [P][C](1 + 6), the weights
    // [C][7][ldP], the tangent sums of every atom slice [P][slices][NG]
    const int64_t ldP = ((int64_t)P + 31) / 32 * 32;
    int64_t slices = 0;
    for (const tsf::Bucket &b : c.plan32.buckets)
      if (b.adj_split) slices += (int64_t)b.nitems * b.cluster;
    if (slices > 0) {
      TSF_CUDA(c.adj_v.ensure((size_t)c.Ntot * 3 * ldP * sizeof(float)));
      TSF_CUDA(c.adj_ew.ensure((size_t)P * c.C * 7 * sizeof(double)));
      TSF_CUDA(c.adj_aw.ensure((size_t)c.C * 7 * ldP * sizeof(float)));
      TSF_CUDA(c.adj_gsplit.ensure((size_t)P * slices * NG * sizeof(double)));
    }
  }
  TSF_CUDA(tsf::launch_param_grad(c, params, P, tg->E, tg->W, tg->F, tg->mask, w, loss, L, dL, c.work.p, c.tf4.p,
                                  c.part.as<double>(), c.dpart.as<double>(), c.gpart.as<double>(), S(stream)));
  return TERSOFF_OK;
}

int tersoff_eval_plain(tersoff_ctx *ctx, const double *params, int32_t P, double *E, double *F,
                       double *W, tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (c.form != 0) return fail(ctx, TERSOFF_E_UNSUPPORTED, "only the batched evaluation and fitness take the Tersoff form%s");
  if (int rc = tsf::finish_build(ctx)) return rc;
  if (!params || P < 1 || !E || !F || !W) return fail(ctx, TERSOFF_E_ARG, "null argument or P < 1%s");
  if (c.max_m > 8) return fail(ctx, TERSOFF_E_UNSUPPORTED, "an atom has more than 8 neighbours%s");
  cudaSetDevice(c.device);
  TSF_CUDA(tsf::launch_plain(c, params, P, E, F, W, S(stream)));
  return TERSOFF_OK;
}

int tersoff_md_force(tersoff_ctx *ctx, int32_t N, const double *pos, const double *box,
                     const double *params, double R1, double R2, int32_t max_nbr, int32_t precision,
                     double *E, void *F, double *W, tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (c.form != 0) return fail(ctx, TERSOFF_E_UNSUPPORTED, "only the batched evaluation and fitness take the Tersoff form%s");
  if (N < 1 || N > (1 << 24) || !pos || !box || !params || !E || !F || !W)
    return fail(ctx, TERSOFF_E_ARG, "need 1 <= N <= 2^24 and non-null pointers%s");
  if (!(R1 > 0.0 && R2 > R1 && std::isfinite(R2))) return fail(ctx, TERSOFF_E_ARG, "need 0 < R1 < R2%s");
  if (max_nbr < 1 || max_nbr > 32) return fail(ctx, TERSOFF_E_ARG, "max_nbr must be in [1, 32]%s");
  if (precision != 32 && precision != 64) return fail(ctx, TERSOFF_E_ARG, "precision must be 32 or 64%s");
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(params[k])) return fail(ctx, TERSOFF_E_ARG, "non-finite parameters%s");
  cudaSetDevice(c.device);
  std::string err;
  const int rc = tsf::md_force(c, N, pos, box, params, R1, R2, max_nbr, precision, E, F, W, S(stream), err);
  if (rc != TERSOFF_OK) return fail(ctx, rc, "%s", err.c_str());
  return TERSOFF_OK;
}

int tersoff_md_nve(tersoff_ctx *ctx, int32_t N, double *pos, double *vel, const double *mass, const double *box,
                   const double *params, double R1, double R2, int32_t max_nbr, int32_t precision, double dt,
                   int32_t nsteps, double *Epot, double *Ekin, void *F, double *W, tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (c.form != 0) return fail(ctx, TERSOFF_E_UNSUPPORTED, "only the batched evaluation and fitness take the Tersoff form%s");
  if (N < 1 || N > (1 << 24) || !pos || !vel || !mass || !box || !params || !Epot || !Ekin || !F || !W)
    return fail(ctx, TERSOFF_E_ARG, "need 1 <= N <= 2^24 and non-null pointers%s");
  if (pos == vel) return fail(ctx, TERSOFF_E_ARG, "pos and vel must be distinct arrays%s");
  if (!(R1 > 0.0 && R2 > R1 && std::isfinite(R2))) return fail(ctx, TERSOFF_E_ARG, "need 0 < R1 < R2%s");
  if (max_nbr < 1 || max_nbr > 32) return fail(ctx, TERSOFF_E_ARG, "max_nbr must be in [1, 32]%s");
  if (precision != 32 && precision != 64) return fail(ctx, TERSOFF_E_ARG, "precision must be 32 or 64%s");
  if (!(dt > 0.0 && std::isfinite(dt)) || nsteps < 0) return fail(ctx, TERSOFF_E_ARG, "need dt > 0 and nsteps >= 0%s");
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(params[k])) return fail(ctx, TERSOFF_E_ARG, "non-finite parameters%s");
  cudaSetDevice(c.device);
  std::string err;
  const int rc = tsf::md_nve(c, N, pos, vel, mass, box, params, R1, R2, max_nbr, precision, dt, nsteps, Epot, Ekin,
                             F, W, S(stream), err);
  if (rc != TERSOFF_OK) return fail(ctx, rc, "%s", err.c_str());
  return TERSOFF_OK;
}

int tersoff_md_export_neighbors(tersoff_ctx *ctx, int32_t *cnt, int32_t *nbr, int8_t *shift) {
  if (!ctx) return TERSOFF_E_ARG;
  Ctx &c = ctx->c;
  if (c.md_N < 1) return fail(ctx, TERSOFF_E_STATE, "no MD force call yet%s");
  cudaSetDevice(c.device);
  const int64_t N = c.md_N, M = c.md_M;
  TSF_CUDA(cudaDeviceSynchronize());
  // the device list is slot-major ([max_nbr][N]) and holds the first min(count, max_nbr) entries of
  // each atom; the transpose and the padding are done here
  std::vector<int> count(N);
  TSF_CUDA(cudaMemcpy(count.data(), c.md_cnt.p, N * sizeof(int), cudaMemcpyDeviceToHost));
  if (cnt) std::memcpy(cnt, count.data(), N * sizeof(int));
  if (nbr) {
    std::vector<int> tmp(N * M);
    TSF_CUDA(cudaMemcpy(tmp.data(), c.md_nbr.p, N * M * sizeof(int), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < N; ++i)
      for (int64_t e = 0; e < M; ++e) nbr[i * M + e] = e < count[i] ? tmp[e * N + i] : -1;
  }
  if (shift) {
    std::vector<char4> tmp(N * M);
    TSF_CUDA(cudaMemcpy(tmp.data(), c.md_shift.p, N * M * sizeof(char4), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < N; ++i)
      for (int64_t e = 0; e < M; ++e) {
        const int64_t k = i * M + e;
        const bool kept = e < count[i];
        const char4 v = tmp[e * N + i];
        shift[3 * k] = kept ? v.x : 0;
        shift[3 * k + 1] = kept ? v.y : 0;
        shift[3 * k + 2] = kept ? v.z : 0;
      }
  }
  return TERSOFF_OK;
}

}  // extern "C"
