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
// arithmetic carrying K parameter tangents at a time. FP32 arithmetic, FP64 accumulation across
// atoms-of-a-CTA totals and configurations.
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
  for (const Bucket &b : plan.buckets) {
    if (b.nitems == 0) continue;
    if (b.cluster != 1) return cudaErrorNotSupported;   // the host rejects such builds first
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
