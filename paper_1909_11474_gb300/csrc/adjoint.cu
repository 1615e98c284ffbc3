// adjoint.cu -- gradient of the fitness loss with respect to the parameters, x = [D0, alpha, r0,
// beta, n, h] (Eq. 16) of the minimal potential or x = [D0, alpha, r0, S, n, h, gamma, c, d] of the
// Tersoff form (Eq. 8, free S), for many parameter sets at once.
//
// For one parameter set the loss terms are S_e = sum_c (E_c/N_c - E*_c)^2,
// S_v = sum_c sum_k (W_ck/N_c - W*_ck)^2 and S_f = sum_i |F_i - F*_i|^2 (Eq. 17-19 before the square
// root). Their gradients, per configuration, are
//   dS_e/dx = a_e dE/dx,                     a_e = 2 (E/N - E*) / N,
//   dS_v/dx = sum_k a_k dW_k/dx = -d/dx sum_ij P_ij . (B d_ij),   a_k = 2 (W_k/N - W*_k) / N,
//   dS_f/dx = sum_i v_i . dF_i/dx = -d/dx sum_ij P_ij . (v_j - v_i),   v_i = 2 (F_i - F*_i),
// with P_ij = dU_i/dd_ij and (B d)_nu = sum_{k = (mu, nu)} a_k d_mu: the virial and force terms are
// directional derivatives of the site energies along fixed bond directions, which keeps the work
// atom-local. One CTA evaluates a configuration for 32 parameter sets (the forward passes of the
// batched kernel give F, E, W and the weights), then re-runs the per-atom core in forward-mode dual
// arithmetic carrying K parameter tangents at a time. Configurations that the batched schedule
// spreads over a cluster of CTAs (or that exceed the adjoint kernel's shared memory) take the split
// path: the batched kernel's evaluation mode gives their F, E and W, a weights kernel forms the
// residuals, a_e, a_k and v, and the tangent passes run per atom slice (each needs only its own bonds
// and the v of the neighbours, read from global memory). FP32 arithmetic, FP64 accumulation across
// warps, slices and configurations.
#include <math.h>

#include <algorithm>

#include "adjoint_kernel.cuh"

namespace tsf {

// the kernel variants are compiled in adjoint_m*.cu
extern template cudaError_t launch_adjoint_variant<4, false>(const AdjParams &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_adjoint_variant<4, true>(const AdjParams &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_adjoint_variant<6, false>(const AdjParams &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_adjoint_variant<6, true>(const AdjParams &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_adjoint_variant<8, false>(const AdjParams &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_adjoint_variant<8, true>(const AdjParams &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_tangent_split<4, false>(const AdjParams &, const AdjSplit &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_tangent_split<4, true>(const AdjParams &, const AdjSplit &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_tangent_split<6, false>(const AdjParams &, const AdjSplit &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_tangent_split<6, true>(const AdjParams &, const AdjSplit &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_tangent_split<8, false>(const AdjParams &, const AdjSplit &, size_t, unsigned, cudaStream_t);
extern template cudaError_t launch_tangent_split<8, true>(const AdjParams &, const AdjSplit &, size_t, unsigned, cudaStream_t);

size_t adjoint_split_smem_bytes(int nb, int nq, int ns) { return adj_split_smem_bytes(nb, nq, ns); }

size_t adjoint_smem_bytes(int nb, int nq, int nat) {
  size_t b = adj_region0(nb) * sizeof(float) + (size_t)nb * 2 * sizeof(float4);
  b += ((size_t)nq * sizeof(float) + 31) / 32 * 32;
  b += (size_t)nat * sizeof(int4) + (size_t)nat * sizeof(float4);
  b += (size_t)nat * 3 * kAdjPT * sizeof(float) + 7 * kAdjPT * sizeof(float);
  return b;
}

// One warp per parameter set: S_q, D_q and G_q = dS_q/dx summed over configurations (FP64, fixed
// order); L and dL/dx for the squared loss (w_q S_q / D_q) or Z (w_q sqrt(S_q / D_q)).
template <int NX>
__global__ void grad_finalize_kernel(int P, int C, const double *__restrict__ part,
                                     const double *__restrict__ dpart, const double *__restrict__ gpart,
                                     double we, double wv, double wf, int loss, double *__restrict__ L,
                                     double *__restrict__ dL) {
  constexpr int NG = 3 * NX;
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= P) return;
  double s[3] = {0, 0, 0}, d[3] = {0, 0, 0}, g[NG];
  for (int k = 0; k < NG; ++k) g[k] = 0.0;
  for (int c = lane; c < C; c += 32) {
    for (int q = 0; q < 3; ++q) {
      s[q] += part[((size_t)p * C + c) * 3 + q];
      d[q] += dpart[(size_t)c * 3 + q];
    }
    for (int k = 0; k < NG; ++k) g[k] += gpart[((size_t)p * C + c) * NG + k];
  }
  for (int off = 16; off > 0; off >>= 1) {
    for (int q = 0; q < 3; ++q) {
      s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
      d[q] += __shfl_xor_sync(0xffffffffu, d[q], off);
    }
    for (int k = 0; k < NG; ++k) g[k] += __shfl_xor_sync(0xffffffffu, g[k], off);
  }
  if (lane == 0) {
    const double w[3] = {we, wv, wf};
    double l = 0.0, cq[3];
    bool finite = true;
    for (int q = 0; q < 3; ++q) {
      finite = finite && isfinite(s[q]);
      cq[q] = 0.0;
      if (d[q] > 0.0) {
        if (loss == TERSOFF_LOSS_SQ) {
          l += w[q] * s[q] / d[q];
          cq[q] = w[q] / d[q];
        } else {
          l += w[q] * sqrt(s[q] / d[q]);
          cq[q] = s[q] > 0.0 ? w[q] / (2.0 * sqrt(s[q] * d[q])) : 0.0;
        }
      }
    }
    L[p] = finite ? l : INFINITY;
    for (int x = 0; x < NX; ++x) {
      double gx = 0.0;
      for (int q = 0; q < 3; ++q) gx += cq[q] * g[q * NX + x];
      dL[(size_t)p * NX + x] = finite ? gx : __longlong_as_double(0x7ff8000000000000ll);
    }
  }
}

// One CTA per (configuration, parameter tile): FP32 sums over the configuration's atoms per warp,
// FP64 across warps, as the batched kernel.
__global__ void __launch_bounds__(kThreads) adj_weights_kernel(const AdjSplit a) {
  __shared__ float red[kNW][3][kAdjPT];
  const int tid = threadIdx.x, warp = tid >> 5, pl = tid & 31;
  const int ci = blockIdx.x / a.ntiles, tile = blockIdx.x % a.ntiles;
  const CtaRec rec = a.recs[(size_t)ci * a.cl];
  const int c = rec.c, nat = rec.nat;
  const int64_t a0 = a.atom_off[c];
  const int64_t p = (int64_t)tile * kAdjPT + pl;
  const uint8_t mask = a.tmask[c];
  float sf = 0.f, sF2 = 0.f;
  for (int li = warp; li < nat; li += kNW) {
    const int64_t i = a0 + li;
    float *vp = a.v + i * 3 * a.ldP + p;
    const float Fx = vp[0], Fy = vp[a.ldP], Fz = vp[2 * a.ldP];
    sF2 += Fx * Fx + Fy * Fy + Fz * Fz;
    float vx = 0.f, vy = 0.f, vz = 0.f;
    if (mask & 4) {
      const float4 t = a.tF4[i];
      const float ex = Fx - t.x, ey = Fy - t.y, ez = Fz - t.z;
      sf += ex * ex + ey * ey + ez * ez;
      vx = 2.f * ex;
      vy = 2.f * ey;
      vz = 2.f * ez;
    }
    vp[0] = vx;
    vp[a.ldP] = vy;
    vp[2 * a.ldP] = vz;
  }
  red[warp][0][pl] = sf;
  red[warp][1][pl] = sF2;
  __syncthreads();
  if (tid < kAdjPT) {
    double q7 = 0.0, q8 = 0.0;
    for (int w = 0; w < kNW; ++w) {
      q7 += widen(red[w][0][tid]);
      q8 += widen(red[w][1][tid]);
    }
    const int64_t pp = (int64_t)tile * kAdjPT + tid;
    const bool active = pp < a.P;
    const double invN = 1.0 / (double)nat;
    double se = 0.0, sv = 0.0, sfv = 0.0, ae = 0.0, ak[6] = {0, 0, 0, 0, 0, 0};
    if (active) {
      const double E = a.E[pp * a.C + c];
      double Wk[6];
      bool finite = isfinite(E) && isfinite(q8);
      for (int k = 0; k < 6; ++k) {
        Wk[k] = a.W[(pp * a.C + c) * 6 + k];
        finite = finite && isfinite(Wk[k]);
      }
      if (mask & 1) {
        const double d = E * invN - a.tE[c];
        se = d * d;
        ae = 2.0 * d * invN;
      }
      if (mask & 2)
        for (int k = 0; k < 6; ++k) {
          const double d = Wk[k] * invN - a.tW[(size_t)c * 6 + k];
          sv += d * d;
          ak[k] = 2.0 * d * invN;
        }
      if (mask & 4) sfv = q7;
      if (!finite) se = sv = sfv = __longlong_as_double(0x7ff8000000000000ll);
      double *o = a.part + ((size_t)pp * a.C + c) * 3;
      o[0] = se;
      o[1] = sv;
      o[2] = sfv;
    }
    float *w = a.aw + (size_t)c * 7 * a.ldP + pp;
    w[0] = (float)ae;
    for (int k = 0; k < 6; ++k) w[(1 + k) * a.ldP] = (float)ak[k];
    if (tile == 0 && tid == 0) {   // target norms of Eq. 17-19 in FP64
      double de = 0.0, dv = 0.0, df = 0.0;
      if (mask & 1) de = a.tE[c] * a.tE[c];
      if (mask & 2)
        for (int k = 0; k < 6; ++k) dv += a.tW[(size_t)c * 6 + k] * a.tW[(size_t)c * 6 + k];
      if (mask & 4)
        for (int li = 0; li < nat; ++li) {
          const double *f = a.tF + 3 * (a0 + li);
          df += (f[0] * f[0] + f[1] * f[1]) + f[2] * f[2];
        }
      a.dpart[(size_t)c * 3 + 0] = de;
      a.dpart[(size_t)c * 3 + 1] = dv;
      a.dpart[(size_t)c * 3 + 2] = df;
    }
  }
}

// gpart[p][c][k] = sum of the configuration's slices (in slice order), one thread per (item, p, k).
__global__ void adj_gsum_kernel(const AdjSplit a, int NG) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = (int)(t % NG);
  const int64_t rest = t / NG;
  const int p = (int)(rest % a.P);
  const int64_t ci = rest / a.P;
  if (ci >= a.nitems) return;
  const int c = a.recs[ci * a.cl].c;
  double s = 0.0;
  for (int r = 0; r < a.cl; ++r) s += a.gsplit[((size_t)p * a.nslices + a.slice0 + ci * a.cl + r) * NG + k];
  a.gpart[((size_t)p * a.C + c) * NG + k] = s;
}

cudaError_t launch_param_grad(const Ctx &ctx, const double *params, int P, const double *tE, const double *tW,
                              const double *tF, const uint8_t *tmask, const double *w, int loss, double *L,
                              double *dL, void *consts, void *tf4, double *part, double *dpart, double *gpart,
                              cudaStream_t s) {
  const BatchPlan &plan = ctx.plan32;
  const bool gen = ctx.form == kFormTersoff;
  {
    const int64_t n = std::max<int64_t>(P, ctx.Ntot);
    prep_kernel<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, params, reinterpret_cast<float *>(consts),
                                                                   ctx.form, ctx.Ntot, tF,
                                                                   reinterpret_cast<float4 *>(tf4));
    cudaError_t e = launched(1);
    if (e != cudaSuccess) return e;
  }
  AdjParams ap = {};
  ap.P = P;
  ap.C = ctx.C;
  ap.Ntot = ctx.Ntot;
  ap.consts = reinterpret_cast<const float *>(consts);
  ap.params = params;
  ap.boff = ctx.boff.as<int>();
  ap.poff = ctx.poff.as<int>();
  ap.ameta = ctx.ameta.as<int>();
  ap.gA = ctx.gA32.as<float4>();
  ap.gB = ctx.gB32.as<float4>();
  ap.gcos = ctx.gcos32.as<float>();
  ap.ntiles = (P + kAdjPT - 1) / kAdjPT;
  ap.tE = tE;
  ap.tW = tW;
  ap.tF4 = reinterpret_cast<const float4 *>(tf4);
  ap.tmask = tmask;
  ap.part = part;
  ap.dpart = dpart;
  ap.gpart = gpart;
  ap.status = ctx.status.as<unsigned>();
  // split path (configurations over several CTAs): evaluation of those buckets, then the weights, the
  // tangent passes per atom slice and the slice sums
  int64_t nslices = 0;
  for (const Bucket &b : plan.buckets)
    if (b.adj_split) nslices += (int64_t)b.nitems * b.cluster;
  if (nslices > 0) {
    const int64_t ldP = (int64_t)ap.ntiles * kAdjPT;
    BatchOut o = {};
    o.E = ctx.adj_ew.as<double>();
    o.W = o.E + (size_t)P * ctx.C;
    o.F = ctx.adj_v.p;
    o.f_ld = ldP;
    o.split_only = true;
    o.consts = consts;
    o.counters = ctx.counters.as<int>();
    o.form = ctx.form;
    cudaError_t e = launch_batch(ctx, plan, params, P, kModeEval, o, s);
    if (e != cudaSuccess) return e;
    AdjSplit as = {};
    as.P = P;
    as.C = ctx.C;
    as.ntiles = ap.ntiles;
    as.ldP = ldP;
    as.atom_off = ctx.atom_off.as<int>();
    as.E = o.E;
    as.W = o.W;
    as.v = ctx.adj_v.as<float>();
    as.tF4 = ap.tF4;
    as.tE = tE;
    as.tW = tW;
    as.tF = tF;
    as.tmask = tmask;
    as.aw = ctx.adj_aw.as<float>();
    as.part = part;
    as.dpart = dpart;
    as.gsplit = ctx.adj_gsplit.as<double>();
    as.nslices = nslices;
    as.gpart = gpart;
    const int NG = gen ? 27 : 18;
    for (const Bucket &b : plan.buckets) {
      if (!b.adj_split || b.nitems == 0) continue;
      as.recs = plan.items.as<CtaRec>() + b.item_off;
      as.cl = b.cluster;
      as.nitems = b.nitems;
      adj_weights_kernel<<<(unsigned)(b.nitems * ap.ntiles), kThreads, 0, s>>>(as);
      const unsigned grid = (unsigned)((int64_t)b.nitems * b.cluster * ap.ntiles);
      const size_t smem = b.adj_split_smem;
      if (gen)
        e = b.mmax <= 4 ? launch_tangent_split<4, true>(ap, as, smem, grid, s)
                        : (b.mmax <= 6 ? launch_tangent_split<6, true>(ap, as, smem, grid, s)
                                       : launch_tangent_split<8, true>(ap, as, smem, grid, s));
      else
        e = b.mmax <= 4 ? launch_tangent_split<4, false>(ap, as, smem, grid, s)
                        : (b.mmax <= 6 ? launch_tangent_split<6, false>(ap, as, smem, grid, s)
                                       : launch_tangent_split<8, false>(ap, as, smem, grid, s));
      if (e != cudaSuccess) return e;
      const int64_t nt = (int64_t)b.nitems * P * NG;
      adj_gsum_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(as, NG);
      e = launched(3);
      if (e != cudaSuccess) return e;
      as.slice0 += (int64_t)b.nitems * b.cluster;
    }
  }
  for (const Bucket &b : plan.buckets) {
    if (b.nitems == 0 || b.adj_split) continue;
    const size_t smem = b.adj_smem;
    ap.recs = plan.items.as<CtaRec>() + b.item_off;
    const unsigned grid = (unsigned)(b.nitems * ap.ntiles);
    cudaError_t e;
    if (gen)
      e = b.mmax <= 4 ? launch_adjoint_variant<4, true>(ap, smem, grid, s)
                      : (b.mmax <= 6 ? launch_adjoint_variant<6, true>(ap, smem, grid, s)
                                     : launch_adjoint_variant<8, true>(ap, smem, grid, s));
    else
      e = b.mmax <= 4 ? launch_adjoint_variant<4, false>(ap, smem, grid, s)
                      : (b.mmax <= 6 ? launch_adjoint_variant<6, false>(ap, smem, grid, s)
                                     : launch_adjoint_variant<8, false>(ap, smem, grid, s));
    if (e != cudaSuccess) return e;
    e = launched(1);
    if (e != cudaSuccess) return e;
  }
  if (gen)
    grad_finalize_kernel<9><<<(P + 7) / 8, 256, 0, s>>>(P, ctx.C, part, dpart, gpart, w[0], w[1], w[2], loss, L, dL);
  else
    grad_finalize_kernel<6><<<(P + 7) / 8, 256, 0, s>>>(P, ctx.C, part, dpart, gpart, w[0], w[1], w[2], loss, L, dL);
  return launched(1);
}

}  // namespace tsf
