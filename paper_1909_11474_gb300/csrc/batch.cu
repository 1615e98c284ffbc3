// batch.cu -- launchers of the batched evaluation kernel and the fitness finalisation
// (Eq. 15, 17-19 of arXiv:1909.11474).
#include <math.h>

#include <algorithm>

#include "batch_kernel.cuh"

namespace tsf {

constexpr int kPT = 32;   // parameter sets per warp: one atom per warp

size_t batch_smem_bytes_pt(int precision, int nb, int nq, int nat, bool cluster) {
  if (precision == 64)
    return cluster ? batch_smem<kPT, true, double>(nb, nq, nat) : batch_smem<kPT, false, double>(nb, nq, nat);
  return cluster ? batch_smem<kPT, true, float>(nb, nq, nat) : batch_smem<kPT, false, float>(nb, nq, nat);
}

int batch_param_tile() { return kPT; }

int batch_max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

template <int MMAX, bool CLUSTER, int MINB, typename R>
static cudaError_t launch_variant(BatchParams bp, int nconf, int cluster, size_t smem, bool uniform,
                                  cudaStream_t s) {
  auto kern = batch_kernel<kPT, MMAX, CLUSTER, MINB, R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ncta = CLUSTER ? cluster : 1;
  // resident CTAs of this variant, rounded down to whole clusters
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  const int slots = std::max(1, per_sm * nsm / ncta);
  // work items: whole configurations when they are all alike and fit in one wave of CTAs (the
  // geometry is then staged once per configuration); otherwise each configuration's tiles are split
  // into chunks so that about four items per CTA slot balance the dynamically claimed work
  int per_conf = 1;
  if (!(uniform && nconf <= slots)) per_conf = std::min(bp.ntiles, std::max(1, (4 * slots + nconf - 1) / nconf));
  bp.nconf = nconf;
  bp.chunk_tiles = (bp.ntiles + per_conf - 1) / per_conf;
  bp.nchunks = (bp.ntiles + bp.chunk_tiles - 1) / bp.chunk_tiles;
  const int nitems = nconf * bp.nchunks;
  const int grid_clusters = std::min(nitems, slots);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(grid_clusters * ncta));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if constexpr (CLUSTER) {
    if (cluster > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  const cudaError_t el = cudaLaunchKernelEx(&cfg, kern, bp);
  if (el == cudaSuccess) count_launches(1);
  return el;
}

cudaError_t launch_batch(const Ctx &ctx, const BatchPlan &plan, const double *params, int P,
                         int mode, const BatchOut &out, cudaStream_t s) {
  const bool f64 = plan.precision == 64;
  // per-call preparation: per-parameter-set constants and the target forces in the working precision
  {
    const int64_t n = std::max<int64_t>(std::max<int64_t>(P, ctx.C), out.tF ? ctx.Ntot : 0);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const bool tew = mode == kModeFitness && out.tEW;
    if (f64)
      prep_kernel<double><<<blocks, 256, 0, s>>>(P, params, reinterpret_cast<double *>(out.consts),
                                                 ctx.Ntot, out.tF, reinterpret_cast<dvec4 *>(out.tF4), ctx.C,
                                                 ctx.atom_off.as<int>(), out.tE, out.tW,
                                                 tew ? reinterpret_cast<double *>(out.tEW) : nullptr);
    else
      prep_kernel<float><<<blocks, 256, 0, s>>>(P, params, reinterpret_cast<float *>(out.consts),
                                                ctx.Ntot, out.tF, reinterpret_cast<float4 *>(out.tF4), ctx.C,
                                                ctx.atom_off.as<int>(), out.tE, out.tW,
                                                tew ? reinterpret_cast<float *>(out.tEW) : nullptr);
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
  bp.outer = ctx.outer.as<int>();
  bp.gA = f64 ? ctx.gA64.p : ctx.gA32.p;
  bp.gB = f64 ? ctx.gB64.p : ctx.gB32.p;
  bp.gcos = f64 ? ctx.gcos64.p : ctx.gcos32.p;
  bp.ntiles = (P + kPT - 1) / kPT;
  bp.mode = mode;
  bp.E = out.E;
  bp.F = out.F;
  bp.W = out.W;
  bp.tE = out.tE;
  bp.tW = out.tW;
  bp.tF4 = out.tF4;
  bp.tmask = out.tmask;
  bp.tEW = out.tEW;
  bp.part = out.part;
  bp.dpart = out.dpart;
  bp.status = ctx.status.as<unsigned>();
  cudaError_t ez = cudaMemsetAsync(out.counters, 0, plan.buckets.size() * sizeof(int), s);
  if (ez != cudaSuccess) return ez;
  const bool timed = ctx.timer.begin(s);
  int bi = 0;
  for (const Bucket &b : plan.buckets) {
    bp.counter = out.counters + bi++;
    if (b.nitems == 0) continue;
    bp.recs = plan.items.as<CtaRec>() + b.item_off;
    cudaError_t e = cudaSuccess;
    const bool cl = b.cluster > 1;
    if (!f64) {
      if (!cl && b.mmax <= 4) e = launch_variant<4, false, 2, float>(bp, b.nitems, 1, b.smem, b.uniform, s);
      else if (!cl && b.mmax <= 6) e = launch_variant<6, false, 1, float>(bp, b.nitems, 1, b.smem, b.uniform, s);
      else if (!cl) e = launch_variant<8, false, 1, float>(bp, b.nitems, 1, b.smem, b.uniform, s);
      else if (b.mmax <= 6) e = launch_variant<6, true, 1, float>(bp, b.nitems, b.cluster, b.smem, b.uniform, s);
      else e = launch_variant<8, true, 1, float>(bp, b.nitems, b.cluster, b.smem, b.uniform, s);
    } else {
      if (!cl) e = launch_variant<8, false, 1, double>(bp, b.nitems, 1, b.smem, b.uniform, s);
      else e = launch_variant<8, true, 1, double>(bp, b.nitems, b.cluster, b.smem, b.uniform, s);
    }
    if (e != cudaSuccess) return e;
  }
  if (timed) ctx.timer.end(s);
  return cudaSuccess;
}

// Fitness of every parameter set from the per-(p, c) residual terms of the batched kernel
// (Eq. 15-19): S_q[p] = sum_c part[p][c][q]; D_e = sum_c E*_c^2 and D_v = sum_c |W*_c|^2 over the
// configurations whose mask has the quantity; D_f = sum_c of the per-configuration |F*|^2 sums.
// All sums in FP64 in a fixed order (threads strided over c, then a fixed xor-shuffle tree and the
// warps in index order). Zq = sqrt(S_q/D_q) (0 where D_q = 0), Z = sum_q w_q Zq, and Z = +inf when
// any residual sum of p is not finite. One block per kFinPB parameter sets.
constexpr int kFinPB = 4;
constexpr int kFinThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kFinThreads) fitness_finalize_kernel(
    int P, int C, const R *__restrict__ part, const R *__restrict__ dpart, const double *__restrict__ tE,
    const double *__restrict__ tW, const uint8_t *__restrict__ tmask, double we, double wv, double wf,
    double *__restrict__ Z, double *__restrict__ Zq, double *__restrict__ S) {
  constexpr int NV = 3 * kFinPB + 3;   // S_q of the block's parameter sets, then D_q
  constexpr int NWARP = kFinThreads / 32;
  __shared__ double red[NWARP][NV];
  const int p0 = blockIdx.x * kFinPB;
  const int np = min(kFinPB, P - p0);
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int c = threadIdx.x; c < C; c += kFinThreads) {
    const uint8_t m = tmask[c];
    if (m & 1) v[3 * kFinPB] += tE[c] * tE[c];
    if (m & 2)
      for (int k = 0; k < 6; ++k) v[3 * kFinPB + 1] += tW[6 * c + k] * tW[6 * c + k];
    if (m & 4) v[3 * kFinPB + 2] += (double)dpart[c];
#pragma unroll
    for (int j = 0; j < kFinPB; ++j)
      if (j < np)
        for (int q = 0; q < 3; ++q) v[3 * j + q] += (double)part[((size_t)(p0 + j) * C + c) * 3 + q];
  }
#pragma unroll
  for (int k = 0; k < NV; ++k)
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x < np) {
    const int j = threadIdx.x;
    double s[3], d[3];
    for (int q = 0; q < 3; ++q) {
      s[q] = 0.0;
      d[q] = 0.0;
      for (int w = 0; w < NWARP; ++w) {
        s[q] += red[w][3 * j + q];
        d[q] += red[w][3 * kFinPB + q];
      }
    }
    const double wq[3] = {we, wv, wf};
    double z = 0.0, zq[3];
    bool finite = true;
    for (int q = 0; q < 3; ++q) {
      finite = finite && isfinite(s[q]);
      zq[q] = d[q] > 0.0 ? sqrt(s[q] / d[q]) : 0.0;
      z += wq[q] * zq[q];
    }
    const int p = p0 + j;
    Z[p] = finite ? z : INFINITY;
    if (Zq)
      for (int q = 0; q < 3; ++q) Zq[(size_t)p * 3 + q] = zq[q];
    if (S)
      for (int q = 0; q < 3; ++q) S[(size_t)p * 3 + q] = s[q];
  }
}

cudaError_t launch_fitness_finalize(int precision, int P, int C, const void *part, const void *dpart,
                                    const double *tE, const double *tW, const uint8_t *tmask,
                                    double we, double wv, double wf, double *Z, double *Zq,
                                    double *S, cudaStream_t s) {
  const unsigned blocks = (unsigned)((P + kFinPB - 1) / kFinPB);
  if (precision == 64)
    fitness_finalize_kernel<double><<<blocks, kFinThreads, 0, s>>>(
        P, C, static_cast<const double *>(part), static_cast<const double *>(dpart), tE, tW, tmask, we, wv,
        wf, Z, Zq, S);
  else
    fitness_finalize_kernel<float><<<blocks, kFinThreads, 0, s>>>(
        P, C, static_cast<const float *>(part), static_cast<const float *>(dpart), tE, tW, tmask, we, wv,
        wf, Z, Zq, S);
  return launched(1);
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
