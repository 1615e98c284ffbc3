// batch.cu -- launchers of the batched evaluation kernel and the fitness finalisation
// (Eq. 15, 17-19 of arXiv:1909.11474).
#include <math.h>

#include <algorithm>
#include <vector>

#include "batch_launch.cuh"

namespace tsf {

size_t batch_smem_bytes_pt(int precision, int nb, int nq, int nat, int ncta) {
  const bool cl = ncta > 1;
  if (precision == 64)
    return cl ? batch_smem<kPT, true, double>(nb, nq, nat, ncta) : batch_smem<kPT, false, double>(nb, nq, nat, 1);
  return cl ? batch_smem<kPT, true, float>(nb, nq, nat, ncta) : batch_smem<kPT, false, float>(nb, nq, nat, 1);
}

int batch_param_tile() { return kPT; }

size_t batch_smem_bytes_pt16(int nb, int nq, int nat) { return batch_smem<16, false, float>(nb, nq, nat, 1); }
size_t batch_smem_bytes_nw12(int nb, int nq, int nat) { return batch_smem<kPT, false, float, 12>(nb, nq, nat, 1); }

static int precision_of(const BatchPlan &plan) { return plan.precision; }

int batch_max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Side streams (at most kSide) and their events, created on first use.
constexpr int kSide = 4;
static cudaError_t ensure_side(const Ctx &ctx, int nbuckets) {
  const size_t want = (size_t)std::min(kSide, nbuckets);
  while (ctx.side.size() < want) {
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    ctx.side.push_back(st);
  }
  while (ctx.side_ev.size() < 1 + ctx.side.size()) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    ctx.side_ev.push_back(ev);
  }
  return cudaSuccess;
}

cudaError_t ensure_side_streams(const Ctx &ctx) { return ensure_side(ctx, kSide); }

cudaError_t launch_batch(const Ctx &ctx, const BatchPlan &plan, const double *params, int P,
                         int mode, const BatchOut &out, cudaStream_t s) {
  const bool f64 = plan.precision == 64;
  // per-call preparation: per-parameter-set constants, and the launches' work counters set to zero
  // (the batched kernel claims its first item without the counter and waits for this kernel before
  // its first claim from it)
  {
    const int ncounters = (int)plan.buckets.size();
    const unsigned blocks = (unsigned)((std::max(P, ncounters) + 255) / 256);
    if (f64)
      prep_kernel<double><<<blocks, 256, 0, s>>>(P, params, reinterpret_cast<double *>(out.consts), out.form,
                                                 ctx.Ntot, nullptr, nullptr, out.counters, ncounters);
    else
      prep_kernel<float><<<blocks, 256, 0, s>>>(P, params, reinterpret_cast<float *>(out.consts), out.form,
                                                ctx.Ntot, nullptr, nullptr, out.counters, ncounters);
    cudaError_t e = launched(1);
    if (e != cudaSuccess) return e;
  }
  BatchParams bp = {};
  bp.P = P;
  bp.C = ctx.C;
  bp.Ntot = ctx.Ntot;
  bp.consts = out.consts;
  bp.atom_off = ctx.atom_off.as<int>();
  bp.boff = ctx.boff.as<int>();
  bp.poff = ctx.poff.as<int>();
  bp.ameta = ctx.ameta.as<int>();
  bp.arev = ctx.arev.as<int4>();
  bp.gA = f64 ? ctx.gA64.p : ctx.gA32.p;
  bp.gB = f64 ? ctx.gB64.p : ctx.gB32.p;
  bp.gcos = f64 ? ctx.gcos64.p : ctx.gcos32.p;
  bp.ntiles = (P + kPT - 1) / kPT;
  bp.mode = mode;
  bp.E = out.E;
  bp.F = out.F;
  bp.f_ld = out.f_ld;
  bp.W = out.W;
  bp.tE = out.tE;
  bp.tW = out.tW;
  bp.tF = out.tF;
  bp.tmask = out.tmask;
  bp.part = out.part;
  bp.dpart = out.dpart;
  bp.status = ctx.status.as<unsigned>();
  bp.wait_spins = ctx.wait_spins < 0 ? kMbarSpins : (unsigned)std::min<int64_t>(ctx.wait_spins, 0xffffffffll);
  const bool timed = ctx.timer.begin(s);
  // several buckets run side by side on the context's side streams (forked from and joined back into
  // `s` by events), so one bucket's last items overlap the next bucket's first ones
  auto runs = [&](const Bucket &b) { return b.nitems > 0 && (!out.split_only || b.adj_split); };
  int nlaunch = 0;
  for (const Bucket &b : plan.buckets) nlaunch += runs(b);
  const bool fork = nlaunch > 1 && ensure_side(ctx, (int)plan.buckets.size()) == cudaSuccess;
  if (fork) {
    cudaError_t e = cudaEventRecord(ctx.side_ev[0], s);
    for (size_t k = 0; e == cudaSuccess && k < ctx.side.size(); ++k) e = cudaStreamWaitEvent(ctx.side[k], ctx.side_ev[0], 0);
    if (e != cudaSuccess) return e;
  }
  int bi = 0;
  for (const Bucket &b : plan.buckets) {
    const int k = bi;
    bp.counter = out.counters + bi++;
    if (!runs(b)) continue;
    bp.recs = plan.items.as<CtaRec>() + b.item_off;
    cudaError_t e = cudaSuccess;
    const cudaStream_t bs = s;
    cudaStream_t s = fork ? ctx.side[k % ctx.side.size()] : bs;
    const bool cl = b.cluster > 1;
    if (out.form == kFormTersoff) {
      e = launch_bucket_tersoff_form(bp, b, f64, out.pdl, s);
    } else if (!f64) {
      const bool tuned = b.tune_P == P && b.tune_mode == mode;
      if (!cl && b.mmax <= 4 && tuned && b.tune_pt == 16 && b.smem16 > 0)
        e = launch_variant<16, 4, false, 3, float>(bp, b, out.pdl, s);
      else if (!cl && b.mmax <= 4 && tuned && b.tune_nw == 12 && b.smem12 > 0)
        e = launch_variant<kPT, 4, false, 2, float, 12>(bp, b, out.pdl, s);
      else if (!cl && b.mmax <= 4) e = launch_variant<kPT, 4, false, 2, float>(bp, b, out.pdl, s);
      else if (!cl && b.mmax <= 6) e = launch_variant<kPT, 6, false, 2, float>(bp, b, out.pdl, s);
      else if (!cl) e = launch_variant<kPT, 8, false, 2, float>(bp, b, out.pdl, s);
      else if (b.mmax <= 4) e = launch_variant<kPT, 4, true, 2, float>(bp, b, out.pdl, s);
      else if (b.mmax <= 6) e = launch_variant<kPT, 6, true, 2, float>(bp, b, out.pdl, s);
      else e = launch_variant<kPT, 8, true, 2, float>(bp, b, out.pdl, s);
    } else {
      if (!cl) e = launch_variant<kPT, 8, false, 1, double>(bp, b, out.pdl, s);
      else e = launch_variant<kPT, 8, true, 1, double>(bp, b, out.pdl, s);
    }
    if (e != cudaSuccess) return e;
  }
  if (fork) {
    for (size_t k = 0; k < ctx.side.size(); ++k) {
      cudaError_t e = cudaEventRecord(ctx.side_ev[1 + k], ctx.side[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx.side_ev[1 + k], 0);
      if (e != cudaSuccess) return e;
    }
  }
  if (timed) ctx.timer.end(s);
  return cudaSuccess;
}

// Autotuner of the batched launch: for each bucket in turn, times every candidate schedule (work
// items per configuration, and 2-or-4-atoms-per-warp last tiles on or off where the variant has
// them) over whole launches with CUDA events on `s`, keeps the fastest, and leaves the choices in the
// plan for this (P, mode). Synchronises `s`.
cudaError_t autotune_batch(const Ctx &ctx, BatchPlan &plan, const double *params, int P, int mode,
                           const BatchOut &out, int reps, cudaStream_t s, float *best_ms, int *tried) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const bool timer_on = ctx.timer.on;
  ctx.timer.on = false;   // the tuner's launches are not measurements
  auto time_launch = [&](float &best) -> cudaError_t {
    best = 3.4e38f;
    for (int r = 0; r < reps + 1; ++r) {   // the first launch warms up
      cudaError_t er = cudaEventRecord(e0, s);
      if (er == cudaSuccess) er = launch_batch(ctx, plan, params, P, mode, out, s);
      if (er == cudaSuccess) er = cudaEventRecord(e1, s);
      if (er == cudaSuccess) er = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (er == cudaSuccess) er = cudaEventElapsedTime(&ms, e0, e1);
      if (er != cudaSuccess) return er;
      if (r > 0) best = std::min(best, ms);
    }
    return cudaSuccess;
  };
  int count = 0;
  float best = 0.f;
  for (size_t bi = 0; e == cudaSuccess && bi < plan.buckets.size(); ++bi) {
    Bucket &b = plan.buckets[bi];
    if (b.nitems == 0) continue;
    b.tune_P = P;
    b.tune_mode = mode;
    int best_pc = 0, best_nw = 1, best_pt = kPT, best_warps = kNW;
    float bt = 3.4e38f;
    // variants: 32-wide tiles with 8 or 12 warps per CTA, 16-wide tiles with 8 (where they exist)
    for (int var = 0; var < 3; ++var) {
      const int pt = var == 2 ? 16 : kPT, warps = var == 1 ? 12 : kNW;
      if ((var == 1 && b.smem12 == 0) || (var == 2 && b.smem16 == 0)) continue;
      const int ntiles = (P + pt - 1) / pt;
      std::vector<int> cands;
      for (int v : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64})
        if (v <= ntiles) cands.push_back(v);
      if (cands.empty() || cands.back() != ntiles) cands.push_back(ntiles);
      const bool narrow_capable = precision_of(plan) == 32 && b.cluster == 1 && b.mmax <= 4 && P % pt != 0 &&
                                  P % pt <= pt / 2;
      for (int pc : cands)
        for (int nw = 1; nw >= (narrow_capable ? 0 : 1) && e == cudaSuccess; --nw) {
          b.tune_pt = pt;
          b.tune_nw = warps;
          b.tune_per_conf = pc;
          b.tune_narrow = nw;
          float t = 0.f;
          e = time_launch(t);
          ++count;
          // a later candidate must be more than 1 % faster: the first (the built-in schedule) wins
          // a tie within the timing noise
          if (e == cudaSuccess && t < 0.99f * bt) {
            bt = t;
            best_pc = pc;
            best_nw = nw;
            best_pt = pt;
            best_warps = warps;
          }
        }
    }
    b.tune_pt = best_pt;
    b.tune_nw = best_warps;
    b.tune_per_conf = best_pc;
    b.tune_narrow = best_nw;
  }
  if (e == cudaSuccess) e = time_launch(best);
  ctx.timer.on = timer_on;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (best_ms) *best_ms = best;
  if (tried) *tried = count;
  return e;
}

// Fitness of every parameter set from the per-(p, c) residual terms of the batched kernel
// (Eq. 15-19): S_q[p] = sum_c part[p][c][q] and D_q = sum_c dpart[c][q], all in FP64 in a fixed order
// (threads strided over c, a fixed xor-shuffle tree per warp, then the warps in order). Zq =
// sqrt(S_q/D_q) (0 where D_q = 0), Z = sum_q w_q Zq, and Z = +inf when any residual sum of p is not
// finite. One block of kFinWarps warps per parameter set, so that each thread sums only a few
// configurations; every block forms D_q alongside.
constexpr int kFinWarps = 4;

__global__ void __launch_bounds__(kFinWarps * 32) fitness_finalize_kernel(
    int P, int C, const double *__restrict__ part, const double *__restrict__ dpart, double we, double wv,
    double wf, double *__restrict__ Z, double *__restrict__ Zq, double *__restrict__ S) {
  __shared__ double s_red[kFinWarps][6];
  pdl_wait();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p = blockIdx.x;
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // S_e, S_v, S_f, D_e, D_v, D_f
  const double *pp = part + (size_t)p * C * kResidualTerms;
#pragma unroll 2
  for (int c = tid; c < C; c += kFinWarps * 32)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      v[q] += pp[(size_t)c * kResidualTerms + q];
      v[3 + q] += dpart[3 * c + q];
    }
#pragma unroll
  for (int k = 0; k < 6; ++k)
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) s_red[warp][k] = v[k];
  __syncthreads();
  if (warp == 0) {
    // lane k < 6 sums quantity k over the warps in order; lane q < 3 forms Zq of its quantity (the
    // three divisions and square roots side by side), lane 0 sums w_q Zq in the order q = 0, 1, 2
    double t = 0.0;
    if (lane < 6) {
      t = s_red[0][lane];
      for (int w = 1; w < kFinWarps; ++w) t += s_red[w][lane];
    }
    const double d = __shfl_down_sync(0xffffffffu, t, 3);   // lane q < 3: D_q
    double zq = 0.0, z = 0.0;
    bool finite = true;
    if (lane < 3) {
      finite = isfinite(t);
      zq = d > 0.0 ? sqrt(t / d) : 0.0;
      z = (lane == 0 ? we : lane == 1 ? wv : wf) * zq;
    }
    const double z1 = __shfl_sync(0xffffffffu, z, 1), z2 = __shfl_sync(0xffffffffu, z, 2);
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) Z[p] = finite ? (z + z1) + z2 : INFINITY;
    if (Zq && lane < 3) Zq[(size_t)p * 3 + lane] = zq;
    if (S && lane < 3) S[(size_t)p * 3 + lane] = t;
  }
}

cudaError_t launch_fitness_finalize(int P, int C, const double *part, const double *dpart,
                                    double we, double wv, double wf, double *Z, double *Zq, double *S, bool pdl,
                                    cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)P);
  cfg.blockDim = dim3(kFinWarps * 32);
  cfg.stream = s;
  // the batched kernel gives no early trigger, so this launch starts when it completes; the attribute
  // only shortens the hand-over
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fitness_finalize_kernel, P, C, part, dpart, we, wv, wf, Z, Zq, S);
  if (e == cudaSuccess) count_launches(1);
  return e;
}

// Force the module loading of every kernel the minimal-form fitness path launches (with lazy loading the
// driver would otherwise load each on its first launch, allocating device memory for its code then).
template <int PTV, int MMAX, bool CLUSTER, int MINB, typename R, int NW = kNW>
static cudaError_t touch_variant() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, batch_kernel<PTV, MMAX, CLUSTER, MINB, R, NW, false>);
}
cudaError_t preload_fitness_kernels() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, prep_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, prep_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fitness_finalize_kernel);
  if (e == cudaSuccess) e = touch_variant<16, 4, false, 3, float>();
  if (e == cudaSuccess) e = touch_variant<kPT, 4, false, 2, float, 12>();
  if (e == cudaSuccess) e = touch_variant<kPT, 4, false, 2, float>();
  if (e == cudaSuccess) e = touch_variant<kPT, 6, false, 2, float>();
  if (e == cudaSuccess) e = touch_variant<kPT, 8, false, 2, float>();
  if (e == cudaSuccess) e = touch_variant<kPT, 4, true, 2, float>();
  if (e == cudaSuccess) e = touch_variant<kPT, 6, true, 2, float>();
  if (e == cudaSuccess) e = touch_variant<kPT, 8, true, 2, float>();
  if (e == cudaSuccess) e = touch_variant<kPT, 8, false, 1, double>();
  if (e == cudaSuccess) e = touch_variant<kPT, 8, true, 1, double>();
  if (e == cudaSuccess) e = preload_geometry64_kernels();
  return e;
}

}  // namespace tsf

// Debug builds (TSF_DEBUG_BOUNDS): the first out-of-range or misaligned shared-memory access of the
// batched kernel, as {flag, site, byte offset, window size}; zeros otherwise. Clears the record.
extern "C" int tersoff_debug_bounds(unsigned *out4) {
#ifdef TSF_DEBUG_BOUNDS
  cudaError_t e = cudaMemcpyFromSymbol(out4, tsf::tsf_dbg, 4 * sizeof(unsigned));
  unsigned z[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(tsf::tsf_dbg, z, sizeof(z));
  return e == cudaSuccess ? 0 : 3;
#else
  for (int k = 0; k < 4; ++k) out4[k] = 0;
  return 0;
#endif
}
