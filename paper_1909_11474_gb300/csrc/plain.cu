// plain.cu -- the plain FP64 path: energy, forces and virial of one configuration under one
// parameter set per kernel launch, one thread per atom, every bond quantity recomputed from the
// positions and the neighbour list (no batching over parameter sets, no geometry cache). It is the
// comparison baseline of the batched path and computes Eq. 1-14 of arXiv:1909.11474 with the force
// and virial derivation of the batched kernel (P_ij = dU_i/dd_ij, F_i = sum_j (P_ij - P_ji)).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "ctx.hpp"

namespace tsf {

constexpr int kPlainMaxM = 8;

__device__ __forceinline__ void plain_cutoff(double r, double R1, double R2, double &fc, double &fcp) {
  if (r <= R1) {
    fc = 1.0;
    fcp = 0.0;
  } else if (r >= R2) {
    fc = 0.0;
    fcp = 0.0;
  } else {
    const double w = (r - R1) / (R2 - R1);
    fc = 0.5 * (1.0 + cospi(w));
    fcp = -0.5 * M_PI / (R2 - R1) * sinpi(w);
  }
}

// One block per (p, c); thread t = atom a0 + t. Shared memory: P_ij [nat][mcap][3] doubles, then
// 7 doubles per warp for the energy/virial block reduction.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) plain_kernel(const double *__restrict__ x, int a0, int nat, int mcap,
                             const double *__restrict__ pos, const double *__restrict__ box,
                             const int *__restrict__ cnt, const int *__restrict__ nbr,
                             const char4 *__restrict__ shift, int M, double R1, double R2,
                             double *__restrict__ E, double *__restrict__ F, double *__restrict__ W) {
  extern __shared__ double psm[];
  double *Pst = psm;                                  // [nat][mcap][3]
  double *red = psm + (size_t)nat * mcap * 3;         // [warps][7]
  const int t = threadIdx.x;
  const double D0 = x[0], al = x[1], r0 = x[2], be = x[3], n = x[4], h = x[5];
  double U = 0.0, Wv[6] = {0, 0, 0, 0, 0, 0};
  const double *H = box;
  if (t < nat) {
    const int i = a0 + t;
    const int m = min(cnt[i], kPlainMaxM);
    double dx[kPlainMaxM], dy[kPlainMaxM], dz[kPlainMaxM], r[kPlainMaxM], fc[kPlainMaxM], fcp[kPlainMaxM];
    for (int e = 0; e < m; ++e) {
      const int j = nbr[(size_t)i * M + e];
      const char4 s = shift[(size_t)i * M + e];
      dx[e] = (pos[3 * j] - pos[3 * i]) + (s.x * H[0] + s.y * H[3] + s.z * H[6]);
      dy[e] = (pos[3 * j + 1] - pos[3 * i + 1]) + (s.x * H[1] + s.y * H[4] + s.z * H[7]);
      dz[e] = (pos[3 * j + 2] - pos[3 * i + 2]) + (s.x * H[2] + s.y * H[5] + s.z * H[8]);
      r[e] = sqrt(dx[e] * dx[e] + dy[e] * dy[e] + dz[e] * dz[e]);
      plain_cutoff(r[e], R1, R2, fc[e], fcp[e]);
    }
    double fR[kPlainMaxM], fA[kPlainMaxM], cc[kPlainMaxM], rad[kPlainMaxM];
    for (int j = 0; j < m; ++j) {
      // Eq. 4-5 with Eq. 11-14 at S = 2
      const double xx = exp(-al * (r[j] - r0));
      fR[j] = D0 * xx * xx;
      fA[j] = 2.0 * D0 * xx;
      // Eq. 7, 10
      double zeta = 0.0;
      for (int k = 0; k < m; ++k) {
        if (k == j) continue;
        const double cs = (dx[j] * dx[k] + dy[j] * dy[k] + dz[j] * dz[k]) / (r[j] * r[k]);
        zeta += fc[k] * be * (cs - h) * (cs - h);
      }
      // Eq. 6; b = 1, b' = 0 at zeta = 0
      double b = 1.0, bp = 0.0;
      if (zeta > 0.0) {
        const double zn = pow(zeta, n);
        b = pow(1.0 + zn, -0.5 / n);
        bp = -0.5 * b * zn / (zeta * (1.0 + zn));
      }
      const double e = fR[j] - b * fA[j];
      U += 0.5 * fc[j] * e;
      cc[j] = -0.5 * fc[j] * fA[j] * bp;
      rad[j] = 0.5 * (fcp[j] * e - al * fc[j] * (2.0 * fR[j] - b * fA[j]));
    }
    for (int j = 0; j < m; ++j) {
      const double uxj = dx[j] / r[j], uyj = dy[j] / r[j], uzj = dz[j] / r[j];
      double Px = rad[j] * uxj, Py = rad[j] * uyj, Pz = rad[j] * uzj;
      for (int k = 0; k < m; ++k) {
        if (k == j) continue;
        const double uxk = dx[k] / r[k], uyk = dy[k] / r[k], uzk = dz[k] / r[k];
        const double cs = uxj * uxk + uyj * uyk + uzj * uzk;
        const double g = be * (cs - h) * (cs - h), gp = 2.0 * be * (cs - h);
        const double w = (cc[j] * fc[k] + cc[k] * fc[j]) * gp / r[j];
        Px += w * (uxk - cs * uxj) + cc[k] * fcp[j] * g * uxj;
        Py += w * (uyk - cs * uyj) + cc[k] * fcp[j] * g * uyj;
        Pz += w * (uzk - cs * uzj) + cc[k] * fcp[j] * g * uzj;
      }
      double *o = Pst + ((size_t)t * mcap + j) * 3;
      o[0] = Px;
      o[1] = Py;
      o[2] = Pz;
      Wv[0] -= dx[j] * Px; Wv[1] -= dy[j] * Py; Wv[2] -= dz[j] * Pz;
      Wv[3] -= dx[j] * Py; Wv[4] -= dy[j] * Pz; Wv[5] -= dz[j] * Px;
    }
  }
  __syncthreads();
  if (t < nat) {
    const int i = a0 + t;
    const int m = min(cnt[i], kPlainMaxM);
    double Fx = 0.0, Fy = 0.0, Fz = 0.0;
    for (int e = 0; e < m; ++e) {
      const double *o = Pst + ((size_t)t * mcap + e) * 3;
      Fx += o[0];
      Fy += o[1];
      Fz += o[2];
      // reverse entry (j; i, -n), searched in j's list
      const int j = nbr[(size_t)i * M + e];
      const char4 s = shift[(size_t)i * M + e];
      const int mj = min(cnt[j], kPlainMaxM);
      for (int f = 0; f < mj; ++f) {
        const char4 q = shift[(size_t)j * M + f];
        if (nbr[(size_t)j * M + f] == i && q.x == -s.x && q.y == -s.y && q.z == -s.z) {
          const double *pr = Pst + ((size_t)(j - a0) * mcap + f) * 3;
          Fx -= pr[0];
          Fy -= pr[1];
          Fz -= pr[2];
          break;
        }
      }
    }
    F[3 * (size_t)i] = Fx;
    F[3 * (size_t)i + 1] = Fy;
    F[3 * (size_t)i + 2] = Fz;
  }
  // block reduction of U and W (FP64, fixed order)
  double v[7] = {U, Wv[0], Wv[1], Wv[2], Wv[3], Wv[4], Wv[5]};
  for (int k = 0; k < 7; ++k)
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  const int warp = t >> 5, nw = (blockDim.x + 31) >> 5;
  if ((t & 31) == 0)
    for (int k = 0; k < 7; ++k) red[warp * 7 + k] = v[k];
  __syncthreads();
  if (t < 7) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * 7 + t];
    if (t == 0) *E = s;
    else W[t - 1] = s;
  }
}

cudaError_t launch_plain(const Ctx &ctx, const double *params, int P, double *E, double *F, double *W,
                         cudaStream_t s) {
  for (int c = 0; c < ctx.C; ++c) {
    const int a0 = ctx.h_atom_off[c], nat = ctx.h_atom_off[c + 1] - a0;
    const int mcap = std::max(1, std::min(ctx.h_cfg_maxm[c], kPlainMaxM));
    const int threads = ((nat + 31) / 32) * 32;
    const size_t smem = ((size_t)nat * mcap * 3 + (size_t)(threads / 32) * 7) * sizeof(double);
    // blocks of up to 256 threads get the registers they need; larger ones are capped at 64
    auto kern = threads <= 256 ? plain_kernel<256> : plain_kernel<1024>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    for (int p = 0; p < P; ++p) {
      kern<<<1, threads, smem, s>>>(params + 6 * (size_t)p, a0, nat, mcap, ctx.pos.as<double>(),
                                            ctx.box.as<double>() + 9 * (size_t)c, ctx.cnt.as<int>(),
                                            ctx.nbr.as<int>(), ctx.shift.as<char4>(), ctx.M, ctx.R1,
                                            ctx.R2, E + (size_t)p * ctx.C + c, F + (size_t)p * ctx.Ntot * 3,
                                            W + ((size_t)p * ctx.C + c) * 6);
    }
  }
  return launched(ctx.C * P);
}

}  // namespace tsf
