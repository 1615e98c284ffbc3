// adjoint_kernel.cuh -- the per-CTA kernel of the parameter gradient (see adjoint.cu for the method)
// and its launcher. Each (largest neighbour count, form) variant is instantiated in a translation unit
// of its own (adjoint_m*.cu), so that the variants compile in parallel.
#pragma once
#include <math.h>

#include <algorithm>

#include "batch_kernel.cuh"

namespace tsf {

constexpr int kAdjPT = 32;
constexpr int kAdjK = 2;          // parameter tangents carried per pass (3 passes for 6 parameters, 5 for 9)
constexpr int kAdjGMax = 27;      // accumulated gradient terms per lane: 3 loss terms x up to 9 parameters

struct AdjParams {
  int P, C;
  int64_t Ntot;
  const float *consts;            // [P][8] PConsts<float> ([P][16] in the Tersoff form)
  const double *params;           // [P][9] raw parameters of the Tersoff form (its tangent seeds)
  const int *boff, *poff;
  const int *ameta;               // [Ntot]: bonds kept | (some bond beyond R1) << 16
  const float4 *gA, *gB;
  const float *gcos;
  const CtaRec *recs;
  int ntiles;
  const double *tE, *tW;
  const float4 *tF4;
  const uint8_t *tmask;
  double *part, *dpart, *gpart;   // [P][C][3], [C][3], [P][C][3][NX]
  unsigned *status;
};

__host__ __device__ inline size_t adj_region0(int nb) {
  const size_t st = (size_t)nb * 3 * kAdjPT;
  const size_t rd = std::max<size_t>((size_t)(kNW + 2) * kNRed * kAdjPT, (size_t)kNW * kAdjGMax * kAdjPT);
  return ((st > rd ? st : rd) * sizeof(float) + 31) / 32 * 32 / sizeof(float);
}

// Dual constants for tangents of parameters q0 .. q0+K-1 (order D0, alpha, r0, beta, n, h).
template <int K>
__device__ __forceinline__ PConsts<Dual<K, float>> seed_consts_minimal(const PConsts<float> &k, int q0) {
  PConsts<Dual<K, float>> D;
  D.D0 = Dual<K, float>(k.D0);
  D.k1 = Dual<K, float>(k.k1);
  D.k0 = Dual<K, float>(k.k0);
  D.mha = Dual<K, float>(k.mha);
  D.beta = Dual<K, float>(k.beta);
  D.h = Dual<K, float>(k.h);
  D.n = Dual<K, float>(k.n);
  D.inv2n = Dual<K, float>(k.inv2n);
  const float log2e = 1.4426950408889634f;
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const int q = q0 + t;
    if (q == 0) D.D0.d[t] = 1.f;
    if (q == 1) {                                  // k1 = -alpha log2e, mha = -alpha/2
      D.k1.d[t] = -log2e;
      D.mha.d[t] = -0.5f;
    }
    if (q == 2) D.k0.d[t] = 1.f;                   // k0 = r0
    if (q == 3) D.beta.d[t] = 1.f;
    if (q == 4) {                                  // inv2n = -1/(2n): d/dn = 1/(2 n^2)
      D.n.d[t] = 1.f;
      D.inv2n.d[t] = 2.f * k.inv2n * k.inv2n;
    }
    if (q == 5) D.h.d[t] = 1.f;
  }
  return D;
}

// Dual constants of the Tersoff form for tangents of parameters q0 .. q0+K-1 (order D0, alpha, r0, S,
// n, h, gamma, c, d; tangents of q >= 9 stay zero). The constants (see PConsts) depend on them as
// f_A/2 = D0 S/(2(S-1)) 2^(k1 (r - r0)), f_R = D0/(S-1) 2^(kR1 (r - r0)), k1 = -mu log2e,
// kR1 = -lambda log2e, mu = alpha sqrt(2/S), lambda = alpha sqrt(2S), mha = mu, hl = -lambda/2,
// g0 = gamma, gc2 = gamma c^2, d2 = d^2, gcd = gamma c^2 / d^2. x: the raw parameters.
template <int K>
__device__ __forceinline__ PConsts<Dual<K, float>> seed_consts_tersoff(const PConsts<float> &k, const float (&x)[9],
                                                                      int q0) {
  using DK = Dual<K, float>;
  PConsts<DK> D;
  D.D0 = DK(k.D0); D.k1 = DK(k.k1); D.k0 = DK(k.k0); D.mha = DK(k.mha);
  D.beta = DK(k.beta); D.h = DK(k.h); D.n = DK(k.n); D.inv2n = DK(k.inv2n);
  D.cR = DK(k.cR); D.kR1 = DK(k.kR1); D.kR0 = DK(k.kR0); D.hl = DK(k.hl);
  D.g0 = DK(k.g0); D.gc2 = DK(k.gc2); D.d2 = DK(k.d2); D.gcd = DK(k.gcd);
  const float D0 = x[0], alpha = x[1], S = x[3], ga = x[6], c = x[7], d = x[8];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const int q = q0 + t;
    if (q == 0) {                                  // f_A and f_R prefactors are proportional to D0
      D.D0.d[t] = k.D0 / D0;
      D.cR.d[t] = k.cR / D0;
    }
    if (q == 1) {                                  // mu and lambda are proportional to alpha
      D.k1.d[t] = k.k1 / alpha;
      D.mha.d[t] = k.mha / alpha;
      D.kR1.d[t] = k.kR1 / alpha;
      D.hl.d[t] = k.hl / alpha;
    }
    if (q == 2) D.k0.d[t] = 1.f;                   // the r0 slot
    if (q == 3) {                                  // S: prefactors, mu ~ S^-1/2, lambda ~ S^1/2
      D.D0.d[t] = -k.D0 / (S * (S - 1.f));
      D.cR.d[t] = -k.cR / (S - 1.f);
      D.k1.d[t] = -0.5f * k.k1 / S;
      D.mha.d[t] = -0.5f * k.mha / S;
      D.kR1.d[t] = 0.5f * k.kR1 / S;
      D.hl.d[t] = 0.5f * k.hl / S;
    }
    if (q == 4) {
      D.n.d[t] = 1.f;
      D.inv2n.d[t] = 2.f * k.inv2n * k.inv2n;
    }
    if (q == 5) D.h.d[t] = 1.f;
    if (q == 6) {                                  // gamma
      D.g0.d[t] = 1.f;
      D.gc2.d[t] = c * c;
      D.gcd.d[t] = c * c / (d * d);
    }
    if (q == 7) {                                  // c
      D.gc2.d[t] = 2.f * ga * c;
      D.gcd.d[t] = 2.f * ga * c / (d * d);
    }
    if (q == 8) {                                  // d
      D.d2.d[t] = 2.f * d;
      D.gcd.d[t] = -2.f * ga * c * c / (d * d * d);
    }
  }
  return D;
}

template <int K, bool GEN>
__device__ __forceinline__ PConsts<Dual<K, float>> seed_consts(const PConsts<float> &k, const float (&x)[9], int q0) {
  if constexpr (GEN) return seed_consts_tersoff<K>(k, x, q0);
  else return seed_consts_minimal<K>(k, q0);
}

// One atom's tangent contribution for parameters q0.. (q0+K-1): accumulates dS_q/dx into G[q][x].
// gT[q][t] receives the tangent t of loss term q (e, v, f) for parameter q0 + t; q0 is a runtime value,
// so one copy of the dual core per neighbour count serves every pass.
// v_j of neighbour j (configuration-local index jl) is vb[jl * vsa + k * vsk] (vb: this lane's first
// element; shared memory in the single-CTA kernel, global memory in the split path).
template <int M, int K, bool GEN>
__device__ __forceinline__ void atom_tangent(const float4 *sA, const float4 *sB, const float *sC, int lb,
                                             int lq, const float *vi, const float *vb, int64_t vsa, int64_t vsk,
                                             int pl, const float *aw, const PConsts<float> &Kf,
                                             const float (&xr)[9], int q0, float (&gT)[3][K]) {
  float ux[M], uy[M], uz[M], r[M], ir2[M], fc[M], fcp[M];
  int jl[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float4 A = sld(&sA[lb + j], 31);
    const float4 B = sld(&sB[lb + j], 32);
    ux[j] = A.x; uy[j] = A.y; uz[j] = A.z; r[j] = A.w;
    ir2[j] = B.x; fc[j] = B.y; fcp[j] = B.z;
    jl[j] = __float_as_int(B.w) >> 16;
  }
  constexpr int NP = M * (M - 1) / 2;
  constexpr int NP4 = (NP + 3) / 4;
  float cs[NP4 > 0 ? 4 * NP4 : 4];
  {
    const float4 *c4 = reinterpret_cast<const float4 *>(sC + lq);
#pragma unroll
    for (int q = 0; q < NP4; ++q) {
      const float4 v = sld(&c4[q], 33);
      cs[4 * q] = v.x; cs[4 * q + 1] = v.y; cs[4 * q + 2] = v.z; cs[4 * q + 3] = v.w;
    }
  }
  using D = Dual<K, float>;
  const PConsts<D> KD = seed_consts<K, GEN>(Kf, xr, q0);
  D U, Px[M], Py[M], Pz[M];
  atom_core<M, false, D, float, GEN>(ux, uy, uz, r, ir2, fc, fcp, cs, KD, U, Px, Py, Pz);
  const float ae = aw[0 * kAdjPT + pl];
  const float a0 = aw[1 * kAdjPT + pl], a1 = aw[2 * kAdjPT + pl], a2 = aw[3 * kAdjPT + pl];
  const float a3 = aw[4 * kAdjPT + pl], a4 = aw[5 * kAdjPT + pl], a5 = aw[6 * kAdjPT + pl];
#pragma unroll
  for (int t = 0; t < K; ++t) gT[0][t] = 0.5f * ae * U.d[t];
#pragma unroll
  for (int t = 0; t < K; ++t) gT[1][t] = gT[2][t] = 0.f;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float dx = r[j] * ux[j], dy = r[j] * uy[j], dz = r[j] * uz[j];
    // virial direction B d: W_xx, W_yy, W_zz, W_xy, W_yz, W_zx = -sum d_mu P_nu
    const float bx = a0 * dx + a5 * dz, by = a1 * dy + a3 * dx, bz = a2 * dz + a4 * dy;
    const float *vj = vb + jl[j] * vsa;
    const float fx = vj[0] - vi[0], fy = vj[vsk] - vi[1], fz = vj[2 * vsk] - vi[2];
#pragma unroll
    for (int t = 0; t < K; ++t) {
      gT[1][t] -= Px[j].d[t] * bx + Py[j].d[t] * by + Pz[j].d[t] * bz;
      gT[2][t] -= Px[j].d[t] * fx + Py[j].d[t] * fy + Pz[j].d[t] * fz;
    }
  }
}

// G[q][x] += gT[q][x - q0] for the parameters q0 .. q0+K-1 that exist (static indices into G).
template <int NX, int K>
__device__ __forceinline__ void add_tangents(float (&G)[3 * NX], int q0, const float (&gT)[3][K]) {
#pragma unroll
  for (int b = 0; b < NX; b += K)
    if (b == q0) {
#pragma unroll
      for (int t = 0; t < K; ++t)
        if (b + t < NX)
#pragma unroll
          for (int q = 0; q < 3; ++q) G[q * NX + b + t] += gT[q][t];
    }
}

template <int MMAX, bool GEN = false>
__global__ void __launch_bounds__(kThreads, 1) adjoint_kernel(const AdjParams a) {
  constexpr int PT = kAdjPT, NX = GEN ? 9 : 6, NG = 3 * NX;
  extern __shared__ __align__(32) unsigned char smem[];
  float *stage = reinterpret_cast<float *>(smem);
  const int tid = threadIdx.x, warp = tid >> 5, pl = tid & 31;
  const int item = blockIdx.x;
  const int tile = item % a.ntiles;
  const CtaRec rec = a.recs[item / a.ntiles];
  const int c = rec.c;
  const int p = tile * PT + pl;
  const bool active = p < a.P;
  PConsts<float> K;
  {
    const float4 *kc = reinterpret_cast<const float4 *>(a.consts) + (GEN ? 4 : 2) * (active ? p : a.P - 1);
    const float4 k0 = kc[0], k1 = kc[1];
    K.D0 = k0.x; K.k1 = k0.y; K.k0 = k0.z; K.mha = k0.w;
    K.beta = k1.x; K.h = k1.y; K.n = k1.z; K.inv2n = k1.w;
    if constexpr (GEN) {
      const float4 k2 = kc[2], k3 = kc[3];
      K.cR = k2.x; K.kR1 = k2.y; K.kR0 = k2.z; K.hl = k2.w;
      K.g0 = k3.x; K.gc2 = k3.y; K.d2 = k3.z; K.gcd = k3.w;
    }
  }
  float xr[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if constexpr (GEN)
#pragma unroll
    for (int q = 0; q < 9; ++q) xr[q] = (float)a.params[9 * (size_t)(active ? p : a.P - 1) + q];
  const int nat = rec.nat, s0 = rec.s0, ns = rec.ns;
  const int B0 = rec.B0, nb = rec.nb, Q0 = rec.Q0, nq = rec.nq;
  float4 *sA = reinterpret_cast<float4 *>(stage + adj_region0(nb));
  float4 *sB = sA + nb;
  float *sC = reinterpret_cast<float *>(sB + nb);
  int4 *satom = reinterpret_cast<int4 *>(reinterpret_cast<unsigned char *>(sC) + ((size_t)nq * 4 + 31) / 32 * 32);
  float4 *stF = reinterpret_cast<float4 *>(satom + ns);
  float *vsm = reinterpret_cast<float *>(stF + ns);          // [ns][3][PT]: v_i = 2 (F_i - F*_i)
  float *aw = vsm + (size_t)ns * 3 * PT;                     // [7][PT]: a_e, a_k (k = xx..zx)
  {
    for (int t = tid; t < nb; t += kThreads) {
      sst(&sA[t], a.gA[B0 + t], 6);
      sst(&sB[t], a.gB[B0 + t], 7);
    }
    for (int t = tid; t < nq; t += kThreads) sst(&sC[t], a.gcos[Q0 + t], 8);
    for (int t = tid; t < ns; t += kThreads) {
      sst(&satom[t], make_int4(a.boff[s0 + t] - B0, a.poff[s0 + t] - Q0, a.ameta[s0 + t] & 0xffff, 0), 9);
      sst(&stF[t], a.tF4[s0 + t], 10);
    }
  }
  __syncthreads();

  // ---- forward passes 1-2 (the batched kernel's atom code)
  AtomAcc<float> acc;
  acc.U = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) acc.W[k] = 0.f;
  for (int li = warp; li < ns; li += kNW) {
    const int4 at = sld(&satom[li], 11);
    const int m = at.z;
    if (m > MMAX) {
      if (pl == 0) set_status(a.status, TERSOFF_STATUS_MANY_NBRS);
      continue;
    }
    atom_forward_dispatch<PT, MMAX, true, false, float, GEN>(m, sA, sB, sC, stage, at.x, at.y, m, true, pl, K, acc);
  }
  __syncthreads();

  // ---- pass 3: forces, residuals and v_i
  const uint8_t mask = a.tmask[c];
  float sf = 0.f, sF2 = 0.f, sT = 0.f;
  for (int li = warp; li < ns; li += kNW) {
    const int4 at = sld(&satom[li], 12);
    const int m = at.z, lb = at.x;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    for (int e = 0; e < m; ++e) {   // the stage rows written by atom_forward (its layout: stage_store)
      float x, y, z;
      stage_load<PT, float>(stage, lb + e, pl, x, y, z, 13);
      Fx += x;
      Fy += y;
      Fz += z;
      const int rb = __float_as_int(sld(&sB[lb + e].w, 14)) & 0xffff;
      stage_load<PT, float>(stage, rb + rec.cb0 - B0, pl, x, y, z, 15);
      Fx -= x;
      Fy -= y;
      Fz -= z;
    }
    sF2 += Fx * Fx + Fy * Fy + Fz * Fz;
    float vx = 0.f, vy = 0.f, vz = 0.f;
    if (mask & 4) {
      const float4 t = sld(&stF[li], 16);
      const float ex = Fx - t.x, ey = Fy - t.y, ez = Fz - t.z;
      sf += ex * ex + ey * ey + ez * ez;
      sT += t.w;
      vx = 2.f * ex;
      vy = 2.f * ey;
      vz = 2.f * ez;
    }
    float *vv = vsm + (size_t)li * 3 * PT + pl;
    sst(&vv[0], vx, 35);
    sst(&vv[PT], vy, 35);
    sst(&vv[2 * PT], vz, 35);
  }

  // ---- forward reductions (as the batched kernel) and the per-parameter-set weights
  float v[kNRed];
  v[0] = acc.U;
#pragma unroll
  for (int k = 0; k < 6; ++k) v[1 + k] = acc.W[k];
  v[7] = sf;
  v[8] = sF2;
  v[9] = sT;
  __syncthreads();
  float *red = stage;
  double *tot = reinterpret_cast<double *>(stage + kNW * kNRed * PT);   // sums over warps, FP64
#pragma unroll
  for (int k = 0; k < kNRed; ++k) sst(&red[(warp * kNRed + k) * PT + pl], v[k], 17);
  __syncthreads();
  for (int idx = tid; idx < kNRed * PT; idx += kThreads) {
    float xw[kNW];
#pragma unroll
    for (int w = 0; w < kNW; ++w) xw[w] = sld(&red[w * kNRed * PT + idx], 18);
    sst(&tot[idx], exact_sum<kNW>(xw), 19);
  }
  __syncthreads();
  if (tid < PT) {
    double q[kNRed];
#pragma unroll
    for (int k = 0; k < kNRed; ++k) q[k] = sld(&tot[k * PT + tid], 20);
    const double invN = 1.0 / (double)nat;
    bool finite = isfinite(q[0]) && isfinite(q[8]);
    for (int k = 0; k < 6; ++k) finite = finite && isfinite(q[1 + k]);
    double se = 0.0, sv = 0.0, sfv = 0.0, ae = 0.0, ak[6] = {0, 0, 0, 0, 0, 0};
    if (mask & 1) {
      const double d = q[0] * invN - a.tE[c];
      se = d * d;
      ae = 2.0 * d * invN;
    }
    if (mask & 2)
      for (int k = 0; k < 6; ++k) {
        const double d = q[1 + k] * invN - a.tW[c * 6 + k];
        sv += d * d;
        ak[k] = 2.0 * d * invN;
      }
    if (mask & 4) sfv = q[7];
    if (!finite) se = sv = sfv = __longlong_as_double(0x7ff8000000000000ll);
    const int pp = tile * PT + tid;
    if (pp < a.P) {
      double *o = a.part + ((size_t)pp * a.C + c) * 3;
      o[0] = se;
      o[1] = sv;
      o[2] = sfv;
    }
    sst(&aw[0 * PT + tid], (float)ae, 36);
    for (int k = 0; k < 6; ++k) sst(&aw[(1 + k) * PT + tid], (float)ak[k], 36);
    if (tile == 0 && tid == 0) {
      double de = 0.0, dv = 0.0;
      if (mask & 1) de = a.tE[c] * a.tE[c];
      if (mask & 2)
        for (int k = 0; k < 6; ++k) dv += a.tW[c * 6 + k] * a.tW[c * 6 + k];
      a.dpart[c * 3 + 0] = de;
      a.dpart[c * 3 + 1] = dv;
      a.dpart[c * 3 + 2] = (mask & 4) ? q[9] : 0.0;
    }
  }
  __syncthreads();

  // ---- tangent passes: K parameters at a time
  float G[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) G[k] = 0.f;
  for (int li = warp; li < ns; li += kNW) {
    const int4 at = sld(&satom[li], 21);
    const int m = at.z;
    if (m > MMAX) continue;
    const float *vp = vsm + (size_t)li * 3 * PT + pl;
    const float vi[3] = {sld(&vp[0], 22), sld(&vp[PT], 22), sld(&vp[2 * PT], 22)};
#define TSF_TAN(MM)                                                                           \
  case MM:                                                                                    \
    if constexpr (MMAX >= MM) {                                                               \
      _Pragma("unroll 1") for (int q0 = 0; q0 < NX; q0 += kAdjK) {                            \
        float gT[3][kAdjK];                                                                   \
        atom_tangent<MM, kAdjK, GEN>(sA, sB, sC, at.x, at.y, vi, vsm + pl, 3 * PT, PT, pl, aw, K, xr, q0, gT); \
        add_tangents<NX, kAdjK>(G, q0, gT);                                                   \
      }                                                                                       \
    }                                                                                         \
    break;
    switch (m) {
      TSF_TAN(1) TSF_TAN(2) TSF_TAN(3) TSF_TAN(4) TSF_TAN(5) TSF_TAN(6) TSF_TAN(7) TSF_TAN(8)
      default: break;
    }
#undef TSF_TAN
  }
  // reduce G over warps (region0 is free again) and write the per-(p, c) gradient partial sums
  __syncthreads();
  float *gred = stage;                                       // [kNW][NG][PT]
#pragma unroll
  for (int k = 0; k < NG; ++k) sst(&gred[(warp * NG + k) * PT + pl], G[k], 23);
  __syncthreads();
  for (int idx = tid; idx < NG * PT; idx += kThreads) {
    const int k = idx / PT, lp = idx % PT;
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kNW; ++w) t += (double)sld(&gred[(w * NG + k) * PT + lp], 24);
    const int pp = tile * PT + lp;
    if (pp < a.P) a.gpart[((size_t)pp * a.C + c) * NG + k] = t;
  }
}

// ---- split path: configurations spread over a cluster of CTAs by the batched schedule, or beyond the
// adjoint kernel's shared memory. The batched kernel in evaluation mode gives E, W and F (F laid out
// [Ntot][3][ldP]); adj_weights_kernel turns F into v = 2 (F - F*) in place and forms the residual
// terms and the weights a_e, a_k of every (p, c); adj_tangent_split_kernel runs the dual passes of
// one atom slice of the schedule per CTA (the tangents need only the slice's own bonds; v_j of a
// neighbour in another slice is read from global memory); adj_gsum_kernel adds the slices of each
// configuration in a fixed order.
struct AdjSplit {
  int P, C, ntiles;
  int64_t ldP;                    // parameter-set stride of v and aw (ntiles * 32)
  const CtaRec *recs;             // the bucket's records: configuration ci, slice r at ci * cl + r
  int cl;                         // slices per configuration
  int nitems;                     // configurations of the bucket
  const int *atom_off;
  const double *E, *W;            // [P][C], [P][C][6] from the evaluation
  float *v;                       // [Ntot][3][ldP]: F on entry to the weights kernel, then v
  const float4 *tF4;              // target forces in FP32 (x, y, z, |F*|^2)
  const double *tE, *tW, *tF;
  const uint8_t *tmask;
  float *aw;                      // [C][7][ldP]: a_e, a_k (k = xx .. zx)
  double *part, *dpart;           // [P][C][3], [C][3]
  double *gsplit;                 // [P][nslices][NG]: tangent sums of every slice
  int64_t nslices, slice0;        // split slices of all buckets; this bucket's first
  double *gpart;                  // [P][C][NG]
};

__host__ __device__ inline size_t adj_split_smem_bytes(int nb, int nq, int ns) {
  size_t b = (size_t)kNW * kAdjGMax * kAdjPT * sizeof(float);   // per-warp gradient sums
  b += (size_t)nb * 2 * sizeof(float4) + ((size_t)nq * sizeof(float) + 31) / 32 * 32;
  b += (size_t)ns * sizeof(int4) + 7 * kAdjPT * sizeof(float);
  return b;
}

// One CTA per (atom slice, parameter tile): the tangent passes of the slice's atoms.
template <int MMAX, bool GEN>
__global__ void __launch_bounds__(kThreads, 1) adj_tangent_split_kernel(const AdjParams ap, const AdjSplit a) {
  constexpr int PT = kAdjPT, NX = GEN ? 9 : 6, NG = 3 * NX;
  extern __shared__ __align__(32) unsigned char smem[];
  float *gred = reinterpret_cast<float *>(smem);              // [kNW][NG][PT]
  const int tid = threadIdx.x, warp = tid >> 5, pl = tid & 31;
  const int slice = blockIdx.x / a.ntiles, tile = blockIdx.x % a.ntiles;
  const CtaRec rec = a.recs[slice];
  const int c = rec.c;
  const int p = tile * PT + pl;
  const bool active = p < a.P;
  PConsts<float> K;
  {
    const float4 *kc = reinterpret_cast<const float4 *>(ap.consts) + (GEN ? 4 : 2) * (active ? p : a.P - 1);
    const float4 k0 = kc[0], k1 = kc[1];
    K.D0 = k0.x; K.k1 = k0.y; K.k0 = k0.z; K.mha = k0.w;
    K.beta = k1.x; K.h = k1.y; K.n = k1.z; K.inv2n = k1.w;
    if constexpr (GEN) {
      const float4 k2 = kc[2], k3 = kc[3];
      K.cR = k2.x; K.kR1 = k2.y; K.kR0 = k2.z; K.hl = k2.w;
      K.g0 = k3.x; K.gc2 = k3.y; K.d2 = k3.z; K.gcd = k3.w;
    }
  }
  float xr[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if constexpr (GEN)
#pragma unroll
    for (int q = 0; q < 9; ++q) xr[q] = (float)ap.params[9 * (size_t)(active ? p : a.P - 1) + q];
  const int s0 = rec.s0, ns = rec.ns, B0 = rec.B0, nb = rec.nb, Q0 = rec.Q0, nq = rec.nq;
  float4 *sA = reinterpret_cast<float4 *>(gred + (size_t)kNW * kAdjGMax * PT);
  float4 *sB = sA + nb;
  float *sC = reinterpret_cast<float *>(sB + nb);
  int4 *satom = reinterpret_cast<int4 *>(reinterpret_cast<unsigned char *>(sC) + ((size_t)nq * 4 + 31) / 32 * 32);
  float *aw = reinterpret_cast<float *>(satom + ns);          // [7][PT]
  for (int t = tid; t < nb; t += kThreads) {
    sA[t] = ap.gA[B0 + t];
    sB[t] = ap.gB[B0 + t];
  }
  for (int t = tid; t < nq; t += kThreads) sC[t] = ap.gcos[Q0 + t];
  for (int t = tid; t < ns; t += kThreads)
    satom[t] = make_int4(ap.boff[s0 + t] - B0, ap.poff[s0 + t] - Q0, ap.ameta[s0 + t] & 0xffff, 0);
  for (int t = tid; t < 7 * PT; t += kThreads)
    aw[t] = a.aw[((size_t)c * 7 + t / PT) * a.ldP + (size_t)tile * PT + t % PT];
  __syncthreads();
  const int64_t a0c = a.atom_off[c];
  const float *vb = a.v + a0c * 3 * a.ldP + (int64_t)tile * PT + pl;
  float G[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) G[k] = 0.f;
  for (int li = warp; li < ns; li += kNW) {
    const int4 at = satom[li];
    const int m = at.z;
    if (m > MMAX) continue;                        // flagged by the evaluation
    const float *vp = vb + (int64_t)(s0 - a0c + li) * 3 * a.ldP;
    const float vi[3] = {vp[0], vp[a.ldP], vp[2 * a.ldP]};
#define TSF_TAN_SPLIT(MM)                                                                                 \
  case MM:                                                                                                \
    if constexpr (MMAX >= MM) {                                                                           \
      _Pragma("unroll 1") for (int q0 = 0; q0 < NX; q0 += kAdjK) {                                        \
        float gT[3][kAdjK];                                                                               \
        atom_tangent<MM, kAdjK, GEN>(sA, sB, sC, at.x, at.y, vi, vb, 3 * a.ldP, a.ldP, pl, aw, K, xr, q0, gT); \
        add_tangents<NX, kAdjK>(G, q0, gT);                                                               \
      }                                                                                                   \
    }                                                                                                     \
    break;
    switch (m) {
      TSF_TAN_SPLIT(1) TSF_TAN_SPLIT(2) TSF_TAN_SPLIT(3) TSF_TAN_SPLIT(4)
      TSF_TAN_SPLIT(5) TSF_TAN_SPLIT(6) TSF_TAN_SPLIT(7) TSF_TAN_SPLIT(8)
      default: break;
    }
#undef TSF_TAN_SPLIT
  }
#pragma unroll
  for (int k = 0; k < NG; ++k) gred[(warp * NG + k) * PT + pl] = G[k];
  __syncthreads();
  for (int idx = tid; idx < NG * PT; idx += kThreads) {
    const int k = idx / PT, lp = idx % PT;
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kNW; ++w) t += widen(gred[(w * NG + k) * PT + lp]);
    const int pp = tile * PT + lp;
    if (pp < a.P) a.gsplit[((size_t)pp * a.nslices + a.slice0 + slice) * NG + k] = t;
  }
}

template <int MMAX, bool GEN>
cudaError_t launch_tangent_split(const AdjParams &ap, const AdjSplit &as, size_t smem, unsigned grid,
                                 cudaStream_t s) {
  auto kern = adj_tangent_split_kernel<MMAX, GEN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(ap, as);   // the caller checks the launch
  return cudaSuccess;
}

// Launch of one bucket's adjoint kernel (grid = configurations x parameter tiles, one CTA each).
template <int MMAX, bool GEN>
cudaError_t launch_adjoint_variant(const AdjParams &ap, size_t smem, unsigned grid, cudaStream_t s) {
  auto kern = adjoint_kernel<MMAX, GEN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(ap);   // the caller checks the launch
  return cudaSuccess;
}

}  // namespace tsf
