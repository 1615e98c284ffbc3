// batch_kernel.cuh -- batched evaluation of the minimal Tersoff potential (arXiv:1909.11474,
// Eq. 1-14) for many parameter sets x many small periodic configurations, with the fitness
// residuals of Eq. 15-19.
//
// Work decomposition (one CTA, or one thread-block cluster, per (configuration c, parameter tile)):
//  * a warp's 32 lanes are APW = 32/PT atom slots x PT parameter sets; lane = slot * PT + pl.
//    All lanes of a slot read the same bond geometry (shared-memory broadcast) and run the same
//    control flow; the warp processes max(m) bonds, absent bonds of shorter lists are phantom
//    bonds with f_C = f_C' = 0, which contribute exactly zero to every sum below.
//  * pass 1 (per atom i, per parameter set): f_R, f_A per bond, zeta_ij over the bond pairs,
//    b_ij and b'_ij, U_i, and per bond c_ij = dU_i/dzeta_ij = -1/2 f_C f_A b'_ij.
//  * pass 2: the partial derivative P_ij = dU_i/dd_ij of the site energy with respect to each of
//    its bond vectors,
//        P_ij = [rad_ij - s_ij/r_ij + f_C'(r_ij) R_ij] u_ij + A_ij / r_ij,
//        rad_ij = 1/2 [f_C'(f_R - b f_A) + f_C (f_R' - b f_A')],
//        A_ij  = sum_k w_jk u_ik,  s_ij = sum_k w_jk cos_jk,  R_ij = sum_k c_ik g(cos_jk),
//        w_jk  = (c_ij f_C(r_ik) + c_ik f_C(r_ij)) g'(cos_jk)   (symmetric in j, k),
//    staged in shared memory, and the atom's virial -sum_j d_ij (x) P_ij.
//  * pass 3 (after a CTA / cluster barrier): F_i = sum_j (P_ij - P_ji), reading P_ji through the
//    reverse-bond index (from a peer CTA's shared memory when the configuration spans a cluster).
//  * per-lane FP32 partial sums over a lane's atoms, converted once to FP64 and reduced across
//    atom slots, warps and cluster ranks in a fixed order.
#pragma once

#include "common.cuh"
#include "ctx.hpp"

namespace tsf {

constexpr int kNW = 8;           // warps per CTA
constexpr int kThreads = kNW * kWarp;
constexpr int kNRed = 10;        // reduced quantities: U, W[6], S_f, sum|F|^2, sum|F*|^2

template <typename R>
struct PConsts {
  R D0, k1, k0, alpha, beta, h, n, inv2n;
};

template <typename R>
__device__ __forceinline__ PConsts<R> load_consts(const double *__restrict__ params, int p) {
  const double *x = params + 6 * p;
  const double D0 = x[0], al = x[1], r0 = x[2], be = x[3], n = x[4], h = x[5];
  const double log2e = 1.4426950408889634;
  PConsts<R> K;
  K.D0 = (R)D0;
  K.k1 = (R)(-al * log2e);          // x = exp(-alpha (r - r0)) = 2^(k1 r + k0)
  K.k0 = (R)(al * r0 * log2e);
  K.alpha = (R)al;
  K.beta = (R)be;
  K.h = (R)h;
  K.n = (R)n;
  K.inv2n = (R)(-0.5 / n);
  return K;
}

// b = (1 + zeta^n)^(-1/(2n)) and b' = db/dzeta = -1/2 b zeta^(n-1) / (1 + zeta^n)   (Eq. 6);
// zeta = 0 gives b = 1, b' = 0 without evaluating 0^n.
template <typename R>
__device__ __forceinline__ void bond_order(R zeta, const PConsts<R> &K, R &b, R &bp) {
  const bool pos = zeta > R(0);
  const R z = pos ? zeta : R(1);
  const R zn = ex2(K.n * lg2(z));
  const R u = R(1) + zn;
  const R bb = ex2(K.inv2n * lg2(u));
  const R bbp = R(-0.5) * bb * zn * rcp(z * u);
  b = pos ? bb : R(1);
  bp = pos ? bbp : R(0);
}

template <typename R>
struct AtomAcc {
  R U, W[6];
};

// Passes 1 and 2 for one atom per atom slot, M = the warp's largest neighbour count.
// sA/sB: bond records (u_x, u_y, u_z, r), (1/r, f_C, f_C', rev); sC: pair cosines; lb/lq: this
// atom's first bond / pair in shared memory; m: its neighbour count (<= M).
template <int M, int PT, typename R>
__device__ __forceinline__ void atom_forward(const typename Vec4<R>::T *__restrict__ sA,
                                             const typename Vec4<R>::T *__restrict__ sB,
                                             const R *__restrict__ sC, R *__restrict__ stage,
                                             int lb, int lq, int m, bool store, int pl,
                                             const PConsts<R> &K, AtomAcc<R> &acc) {
  R ux[M], uy[M], uz[M], r[M], ir[M], fc[M], fcp[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    if (j < m) {
      const auto A = sA[lb + j];
      const auto B = sB[lb + j];
      ux[j] = A.x; uy[j] = A.y; uz[j] = A.z; r[j] = A.w;
      ir[j] = B.x; fc[j] = B.y; fcp[j] = B.z;
    } else {
      ux[j] = R(0); uy[j] = R(0); uz[j] = R(0); r[j] = R(1);
      ir[j] = R(0); fc[j] = R(0); fcp[j] = R(0);
    }
  }
  constexpr int NP = M * (M - 1) / 2;
  R cs[NP > 0 ? NP : 1];
  {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const int rowbase = lq + j * m - (j * (j + 1)) / 2 - j - 1;
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        cs[q] = R(0);
        if (k < m) cs[q] = sC[rowbase + k];
        ++q;
      }
    }
  }

  // ---- pass 1: pair functions (Eq. 4-5 with Eq. 11-14 at S = 2) and zeta (Eq. 7, 10)
  R fR[M], fA[M], zeta[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const R x = ex2(r[j] * K.k1 + K.k0);
    const R Dx = K.D0 * x;
    fR[j] = Dx * x;
    fA[j] = Dx + Dx;
    zeta[j] = R(0);
  }
  {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const R u = cs[q] - K.h;
        const R t = K.beta * u;
        const R g = t * u;
        zeta[j] += fc[k] * g;
        zeta[k] += fc[j] * g;
        ++q;
      }
    }
  }
  R cc[M], rad[M];
  R U = R(0);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    R b, bp;
    bond_order(zeta[j], K, b, bp);
    const R e = fR[j] - b * fA[j];                 // f_R - b f_A
    U += fc[j] * e;                                // Eq. 3 (the 1/2 of Eq. 2 is applied below)
    cc[j] = R(-0.5) * fc[j] * fA[j] * bp;          // dU_i / dzeta_ij
    const R de = -K.alpha * (fR[j] + e);           // f_R' - b f_A' = -alpha (2 f_R - b f_A)
    rad[j] = R(0.5) * (fcp[j] * e + fc[j] * de);
  }

  // ---- pass 2: dU_i/dd_ij
  R Ax[M], Ay[M], Az[M], s[M], Rg[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    Ax[j] = R(0); Ay[j] = R(0); Az[j] = R(0); s[j] = R(0); Rg[j] = R(0);
  }
  {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const R u = cs[q] - K.h;
        const R t = K.beta * u;
        const R gp = t + t;                         // g' = 2 beta (cos - h)
        const R w = (cc[j] * fc[k] + cc[k] * fc[j]) * gp;
        Ax[j] += w * ux[k]; Ay[j] += w * uy[k]; Az[j] += w * uz[k];
        Ax[k] += w * ux[j]; Ay[k] += w * uy[j]; Az[k] += w * uz[j];
        const R wc = w * cs[q];
        s[j] += wc;
        s[k] += wc;
        ++q;
      }
    }
  }
  // bonds inside the switching region (R1 < r < R2) carry the f_C'(r_ij) g term; the vote keeps
  // this loop off the common path where no bond of the warp is in that region
  bool sw = false;
#pragma unroll
  for (int j = 0; j < M; ++j) sw |= (fcp[j] != R(0));
  if (__any_sync(0xffffffffu, sw)) {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const R u = cs[q] - K.h;
        const R g = K.beta * u * u;
        Rg[j] += cc[k] * g;
        Rg[k] += cc[j] * g;
        ++q;
      }
    }
  }
  R W0 = R(0), W1 = R(0), W2 = R(0), W3 = R(0), W4 = R(0), W5 = R(0);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const R coef = rad[j] + fcp[j] * Rg[j] - s[j] * ir[j];
    const R Px = coef * ux[j] + ir[j] * Ax[j];
    const R Py = coef * uy[j] + ir[j] * Ay[j];
    const R Pz = coef * uz[j] + ir[j] * Az[j];
    if (store && j < m) {
      R *st = stage + (size_t)(lb + j) * 3 * PT + pl;
      st[0] = Px;
      st[PT] = Py;
      st[2 * PT] = Pz;
    }
    const R dx = r[j] * ux[j], dy = r[j] * uy[j], dz = r[j] * uz[j];
    W0 -= dx * Px; W1 -= dy * Py; W2 -= dz * Pz;
    W3 -= dx * Py; W4 -= dy * Pz; W5 -= dz * Px;
  }
  if (store) {
    acc.U += R(0.5) * U;
    acc.W[0] += W0; acc.W[1] += W1; acc.W[2] += W2;
    acc.W[3] += W3; acc.W[4] += W4; acc.W[5] += W5;
  }
}

template <int PT, int MMAX, typename R>
__device__ __forceinline__ void atom_forward_dispatch(int Mw, const typename Vec4<R>::T *sA,
                                                      const typename Vec4<R>::T *sB, const R *sC,
                                                      R *stage, int lb, int lq, int m, bool store,
                                                      int pl, const PConsts<R> &K, AtomAcc<R> &acc) {
  switch (Mw) {
    case 0:
      break;
    case 1: atom_forward<1, PT, R>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); break;
    case 2: atom_forward<2, PT, R>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); break;
    case 3: atom_forward<3, PT, R>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); break;
    case 4: atom_forward<4, PT, R>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); break;
    case 5: if constexpr (MMAX >= 5) atom_forward<5, PT, R>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); break;
    case 6: if constexpr (MMAX >= 6) atom_forward<6, PT, R>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); break;
    case 7: if constexpr (MMAX >= 7) atom_forward<7, PT, R>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); break;
    case 8: if constexpr (MMAX >= 8) atom_forward<8, PT, R>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); break;
    default: break;
  }
}

// ---- cluster helpers (distributed shared memory) ----
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned map_to_rank(unsigned saddr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ float ld_cluster(unsigned addr, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ double ld_cluster(unsigned addr, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void st_cluster(unsigned addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

struct BatchParams {
  int P, C;
  int64_t Ntot;
  const double *params;
  const int *atom_off, *boff, *poff;
  const void *gA, *gB, *gcos;
  const int2 *items;
  int mode;
  double *E;
  void *F;
  double *W;
  const double *tE, *tW, *tF;
  const uint8_t *tmask;
  double *part, *dpart;
  unsigned *status;
};

// Shared memory layout (bytes): [red: kNW*kNRed*PT doubles][cred: 16*kNRed*PT doubles]
// [stage: nb*3*PT R][sA: nb R4][sB: nb R4][sC: nq R] (cred only in cluster launches, <= 16 ranks). The fixed-size head puts every CTA's stage
// at the same offset, so a peer's stage is addressed by mapping this CTA's own stage address.
template <int PT, bool CLUSTER>
__host__ __device__ constexpr size_t smem_head_bytes() {
  return (size_t)(kNW + (CLUSTER ? 16 : 0)) * kNRed * PT * sizeof(double);
}

template <int PT, int MMAX, bool CLUSTER, int MINB, typename R>
__global__ void __launch_bounds__(kThreads, MINB) batch_kernel(const BatchParams a) {
  using R4 = typename Vec4<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  double *red = reinterpret_cast<double *>(smem);
  double *cred = red + kNW * kNRed * PT;
  R *stage = reinterpret_cast<R *>(smem + smem_head_bytes<PT, CLUSTER>());

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = lane / PT, pl = lane % PT;
  constexpr int APW = kWarp / PT;

  unsigned rank = 0, ncta = 1;
  int item_idx = blockIdx.x;
  if constexpr (CLUSTER) {
    rank = cluster_ctarank();
    ncta = cluster_nctarank();
    item_idx = blockIdx.x / ncta;
  }
  const int2 item = a.items[item_idx];
  const int c = item.x;
  const int p = item.y * PT + pl;
  const bool active = p < a.P;
  const PConsts<R> K = load_consts<R>(a.params, active ? p : a.P - 1);

  // atom slice of this CTA
  const int ca0 = a.atom_off[c], ca1 = a.atom_off[c + 1];
  const int nat = ca1 - ca0;
  const int per = (nat + (int)ncta - 1) / (int)ncta;
  const int s0 = ca0 + min(nat, (int)rank * per);
  const int s1 = ca0 + min(nat, ((int)rank + 1) * per);
  const int cb0 = a.boff[ca0];           // first bond of the configuration
  const int B0 = a.boff[s0], B1 = a.boff[s1];
  const int Q0 = a.poff[s0], Q1 = a.poff[s1];
  const int nb = B1 - B0, nq = Q1 - Q0;
  R4 *sA = reinterpret_cast<R4 *>(stage + (size_t)nb * 3 * PT);
  R4 *sB = sA + nb;
  R *sC = reinterpret_cast<R *>(sB + nb);

  // stage this slice's geometry in shared memory
  {
    const R4 *gA = reinterpret_cast<const R4 *>(a.gA) + B0;
    const R4 *gB = reinterpret_cast<const R4 *>(a.gB) + B0;
    const R *gC = reinterpret_cast<const R *>(a.gcos) + Q0;
    for (int t = tid; t < nb; t += kThreads) {
      sA[t] = gA[t];
      sB[t] = gB[t];
    }
    for (int t = tid; t < nq; t += kThreads) sC[t] = gC[t];
  }
  __syncthreads();

  AtomAcc<R> acc;
  acc.U = R(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) acc.W[k] = R(0);

  // ---- passes 1-2
  for (int base = s0 + warp * APW; base < s1; base += kNW * APW) {
    const int i = base + slot;
    const bool valid = i < s1;
    const int m = valid ? a.boff[i + 1] - a.boff[i] : 0;
    const int lb = valid ? a.boff[i] - B0 : 0;
    const int lq = valid ? a.poff[i] - Q0 : 0;
    const int Mw = __reduce_max_sync(0xffffffffu, (unsigned)m);
    if (Mw > MMAX) {
      if (lane == 0) set_status(a.status, TERSOFF_STATUS_MANY_NBRS);
      continue;
    }
    atom_forward_dispatch<PT, MMAX, R>(Mw, sA, sB, sC, stage, lb, lq, m, valid, pl, K, acc);
  }
  if constexpr (CLUSTER) cluster_sync_all(); else __syncthreads();

  // ---- pass 3: F_i = sum_j (P_ij - P_ji)
  R sf = R(0), sF2 = R(0), sT = R(0);
  const uint8_t mask = (a.mode == kModeFitness) ? a.tmask[c] : 0;
  unsigned peer_stage[16];
  int peer_b0[17];
  if constexpr (CLUSTER) {
    const unsigned own = smem_addr(stage);
    for (unsigned r = 0; r < ncta; ++r) {
      peer_stage[r] = map_to_rank(own, r);
      peer_b0[r] = a.boff[ca0 + min(nat, (int)r * per)] - cb0;
    }
    peer_b0[ncta] = a.boff[ca1] - cb0;
  }
  for (int base = s0 + warp * APW; base < s1; base += kNW * APW) {
    const int i = base + slot;
    if (i >= s1) continue;
    const int m = a.boff[i + 1] - a.boff[i];
    const int lb = a.boff[i] - B0;
    R Fx = R(0), Fy = R(0), Fz = R(0);
    for (int e = 0; e < m; ++e) {
      const R *st = stage + (size_t)(lb + e) * 3 * PT + pl;
      Fx += st[0];
      Fy += st[PT];
      Fz += st[2 * PT];
      int rb;  // configuration-local bond index of the reverse entry
      if constexpr (sizeof(R) == 4) rb = __float_as_int((float)sB[lb + e].w);
      else rb = (int)sB[lb + e].w;
      if constexpr (CLUSTER) {
        unsigned r = 0;
        while (r + 1 < ncta && rb >= peer_b0[r + 1]) ++r;
        const unsigned addr = peer_stage[r] + (unsigned)(((rb - peer_b0[r]) * 3 * PT + pl) * sizeof(R));
        Fx -= ld_cluster(addr, R(0));
        Fy -= ld_cluster(addr + PT * sizeof(R), R(0));
        Fz -= ld_cluster(addr + 2 * PT * sizeof(R), R(0));
      } else {
        const R *sr = stage + (size_t)(rb + cb0 - B0) * 3 * PT + pl;
        Fx -= sr[0];
        Fy -= sr[PT];
        Fz -= sr[2 * PT];
      }
    }
    sF2 += Fx * Fx + Fy * Fy + Fz * Fz;
    if (a.mode == kModeEval) {
      if (active && a.F) {
        const size_t o = ((size_t)p * a.Ntot + i) * 3;
        R *F = reinterpret_cast<R *>(a.F);
        F[o] = Fx;
        F[o + 1] = Fy;
        F[o + 2] = Fz;
      }
    } else if (mask & 4) {
      const double *t = a.tF + (size_t)i * 3;
      const R tx = (R)t[0], ty = (R)t[1], tz = (R)t[2];
      const R ex = Fx - tx, ey = Fy - ty, ez = Fz - tz;
      sf += ex * ex + ey * ey + ez * ez;
      sT += tx * tx + ty * ty + tz * tz;
    }
  }

  // ---- reductions: FP32 per lane -> FP64 across atom slots, warps and cluster ranks
  double v[kNRed];
  v[0] = (double)acc.U;
#pragma unroll
  for (int k = 0; k < 6; ++k) v[1 + k] = (double)acc.W[k];
  v[7] = (double)sf;
  v[8] = (double)sF2;
  v[9] = (double)sT;
#pragma unroll
  for (int k = 0; k < kNRed; ++k) v[k] = sum_over_atom_slots<PT>(v[k]);
  if (slot == 0) {
#pragma unroll
    for (int k = 0; k < kNRed; ++k) red[(warp * kNRed + k) * PT + pl] = v[k];
  }
  __syncthreads();
  double tot = 0.0;
  const int k_of = tid / PT, pl_of = tid % PT;   // thread -> (quantity, parameter lane)
  if (tid < kNRed * PT) {
    for (int w = 0; w < kNW; ++w) tot += red[(w * kNRed + k_of) * PT + pl_of];
  }
  if constexpr (CLUSTER) {
    if (tid < kNRed * PT) {
      const unsigned dst = map_to_rank(smem_addr(cred + (rank * kNRed + k_of) * PT + pl_of), 0);
      st_cluster(dst, tot);
    }
    cluster_sync_all();
    if (rank != 0) return;
    tot = 0.0;
    if (tid < kNRed * PT)
      for (unsigned r = 0; r < ncta; ++r) tot += cred[(r * kNRed + k_of) * PT + pl_of];
  }
  __syncthreads();
  if (tid < kNRed * PT) red[k_of * PT + pl_of] = tot;   // totals, [quantity][lane]
  __syncthreads();

  if (tid < PT) {
    const int pp = item.y * PT + tid;
    if (pp < a.P) {
      const double U = red[0 * PT + tid];
      double Wt[6];
      for (int k = 0; k < 6; ++k) Wt[k] = red[(1 + k) * PT + tid];
      if (a.mode == kModeEval) {
        if (a.E) a.E[(size_t)pp * a.C + c] = U;
        if (a.W)
          for (int k = 0; k < 6; ++k) a.W[((size_t)pp * a.C + c) * 6 + k] = Wt[k];
      } else {
        const double N = (double)nat;
        bool finite = isfinite(U) && isfinite(red[8 * PT + tid]);
        for (int k = 0; k < 6; ++k) finite = finite && isfinite(Wt[k]);
        double se = 0.0, sv = 0.0, sfv = 0.0;
        if (mask & 1) {
          const double d = U / N - a.tE[c];
          se = d * d;
        }
        if (mask & 2)
          for (int k = 0; k < 6; ++k) {
            const double d = Wt[k] / N - a.tW[c * 6 + k];
            sv += d * d;
          }
        if (mask & 4) sfv = red[7 * PT + tid];
        if (!finite) se = sv = sfv = __longlong_as_double(0x7ff8000000000000ll);
        double *o = a.part + ((size_t)pp * a.C + c) * 3;
        o[0] = se;
        o[1] = sv;
        o[2] = sfv;
      }
    }
    if (a.mode == kModeFitness && item.y == 0 && tid == 0) {
      double de = 0.0, dv = 0.0;
      if (mask & 1) de = a.tE[c] * a.tE[c];
      if (mask & 2)
        for (int k = 0; k < 6; ++k) dv += a.tW[c * 6 + k] * a.tW[c * 6 + k];
      a.dpart[c * 3 + 0] = de;
      a.dpart[c * 3 + 1] = dv;
      a.dpart[c * 3 + 2] = (mask & 4) ? red[9 * PT + 0] : 0.0;
    }
  }
}

}  // namespace tsf
