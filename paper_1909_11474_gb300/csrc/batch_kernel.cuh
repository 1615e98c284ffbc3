// batch_kernel.cuh -- batched evaluation of the minimal Tersoff potential (arXiv:1909.11474,
// Eq. 1-14) for many parameter sets x many small periodic configurations, with the fitness
// residuals of Eq. 15-19.
//
// Work decomposition (one CTA, or one thread-block cluster, per (configuration c, parameter tile)):
//  * a warp's 32 lanes are APW = 32/PT atom slots x PT parameter sets; lane = slot * PT + pl. With
//    PT = 32 a warp evaluates one atom for 32 parameter sets: every lane reads the same bond geometry
//    (shared-memory broadcast) and runs the same control flow, specialised at compile time for the
//    atom's neighbour count. With PT < 32 the warp runs max(m) bonds and the missing bonds of shorter
//    lists are phantom bonds with f_C = f_C' = 0, which contribute exactly zero to every sum below.
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
//  * per-lane partial sums over a lane's atoms, reduced over atom slots and warps in a fixed order;
//    the per-(parameter set, configuration) totals and residuals are formed in FP64.
#pragma once

#include "common.cuh"
#include "ctx.hpp"
#include "dual.cuh"

namespace tsf {

constexpr int kNW = 8;           // warps per CTA
constexpr int kThreads = kNW * kWarp;
constexpr int kNRed = 10;        // quantities of the adjoint kernel's forward reductions (adjoint.cu)
// Quantities the batched kernel reduces per (parameter set, configuration): U, W[6] and the force sum
// (sum |F - F*|^2, or sum |F|^2 where the configuration has no force target, to test finiteness).
// Per-warp partials are FP32 sums over the warp's atoms; sums over warps and cluster ranks are FP64.
constexpr int kNSum = 8;
constexpr int kMaxCluster = kMaxClusterCtas;

// ---- checked shared-memory access (TSF_DEBUG_BOUNDS builds) ----
// In a debug build every shared-memory access of the batched kernel checks that it lies inside the
// dynamic shared-memory window and is aligned for its type; a violation records (site, byte offset,
// window size) in tsf_dbg, the first one only, and the access is skipped (loads return zero).
// Release builds compile these helpers to plain accesses.
#ifdef TSF_DEBUG_BOUNDS
static __device__ unsigned tsf_dbg[4];
#endif
template <typename T>
__device__ __forceinline__ bool smem_ok(const T *p, int site) {
#ifdef TSF_DEBUG_BOUNDS
  extern __shared__ __align__(32) unsigned char smem[];
  unsigned dsz;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsz));
  const long off = reinterpret_cast<const unsigned char *>(p) - smem;
  const bool ok = off >= 0 && off + (long)sizeof(T) <= (long)dsz && (off % (long)alignof(T)) == 0;
  if (!ok && atomicCAS(&tsf_dbg[0], 0u, 1u) == 0u) {
    tsf_dbg[1] = (unsigned)site;
    tsf_dbg[2] = (unsigned)off;
    tsf_dbg[3] = dsz;
  }
  return ok;
#else
  (void)p;
  (void)site;
  return true;
#endif
}
template <typename T>
__device__ __forceinline__ T sld(const T *p, int site) {
  if (smem_ok(p, site)) return *p;
  return T{};
}
template <typename T>
__device__ __forceinline__ void sst(T *p, const T &v, int site) {
  if (smem_ok(p, site)) *p = v;
}

// Per-parameter-set constants (prepared once per call by prep_kernel from the FP64 parameters).
// Minimal form: x = exp(-alpha (r - r0)) = 2^(k1 (r - k0)) with k1 = -alpha log2(e), k0 = r0 (r - r0 is
// exact in FP32 near r0, where k1 r and k1 r0 would cancel), f_R = D0 x^2, f_A = 2 D0 x (Eq. 4-5,
// 11-14 at S = 2); mha = -alpha/2; inv2n = -1/(2n).
// Tersoff form (Eq. 8, free S): f_A / 2 = D0 2^(k1 (r - k0)) with D0 = D0 S / (2 (S - 1)),
// k1 = -mu log2(e), mu = alpha sqrt(2/S), k0 = r0; f_R = cR 2^(kR1 (r - k0)) with cR = D0 / (S - 1),
// kR1 = -lambda log2(e), lambda = alpha sqrt(2 S); mha = mu, hl = -lambda / 2. The angular function of Eq. 8,
// gamma (1 + c^2/d^2 - c^2/(d^2 + u^2)) with u = cos - h, is evaluated as the equal
// g = g0 + gcd u^2 / (d2 + u^2) (g0 = gamma, gcd = gamma c^2/d^2, d2 = d^2), which has no cancellation
// of its large terms; g'/2 = gc2 u / (d2 + u^2)^2 with gc2 = gamma c^2.
template <typename R>
struct PConsts {
  R D0, k1, k0, mha, beta, h, n, inv2n;
  R cR, kR1, kR0, hl, g0, gc2, d2, gcd;
};
constexpr int kFormMinimal = 0, kFormTersoff = 1;

// b = (1 + zeta^n)^(-1/(2n)) and b' = db/dzeta = -1/2 b zeta^(n-1) / (1 + zeta^n)   (Eq. 6).
// zeta is clamped to 1e-30 from below: at zeta = 0 this gives b = 1 to working precision, and b'
// stays finite; it then only ever multiplies g or g' of the same (vanishing) pairs, so every
// contribution of a zeta = 0 bond to the forces is exactly zero, as with b' = 0.
template <typename T>
__device__ __forceinline__ void bond_order(T zeta, const PConsts<T> &K, T &b, T &bp) {
  const T z = zeta > T(1e-30f) ? zeta : T(1e-30f);
  const T zn = ex2(K.n * lg2(z));
  const T u = T(1.0f) + zn;
  b = ex2(K.inv2n * lg2(u));
  bp = T(-0.5f) * b * zn * rcp(z * u);
}

template <typename R>
struct AtomAcc {
  R U, W[6];
};

// Row stride of the P_ij stage [bond][3][PT] (elements). With 2 or 4 atoms in a warp (PT = 16, 8) the
// atoms' rows start m bonds apart; the padding puts the rows of consecutive 4-neighbour atoms on
// disjoint bank groups (4 S = PT mod 32), so the stage accesses are conflict-free.
template <int PT>
__host__ __device__ constexpr int stage_stride() {
  return PT == 8 ? 26 : PT == 16 ? 52 : 3 * PT;
}

// Layout of one stage row (bond b, PT parameter sets). FP32 rows of 32 parameter sets hold the (x, y)
// components as 32 float2 followed by the 32 z components, so that a warp stores and loads a row with
// one 64-bit and one 32-bit access (each conflict-free); other rows hold x, y and z as three runs of PT.
template <int PT, typename R>
__host__ __device__ constexpr bool stage_packed() {
  return PT == 32 && sizeof(R) == 4;
}
template <int PT, typename R>
__device__ __forceinline__ void stage_store(R *stage, int row, int pl, R x, R y, R z) {
  R *st = stage + (size_t)row * stage_stride<PT>();
  if constexpr (stage_packed<PT, R>()) {
    sst(reinterpret_cast<float2 *>(st) + pl, make_float2(x, y), 5);
    sst(&st[2 * PT + pl], z, 5);
  } else {
    sst(&st[pl], x, 5);
    sst(&st[PT + pl], y, 5);
    sst(&st[2 * PT + pl], z, 5);
  }
}
template <int PT, typename R>
__device__ __forceinline__ void stage_load_row(const R *st, int pl, R &x, R &y, R &z, int site) {
  if constexpr (stage_packed<PT, R>()) {
    const float2 v = sld(reinterpret_cast<const float2 *>(st) + pl, site);
    x = v.x;
    y = v.y;
    z = sld(&st[2 * PT + pl], site);
  } else {
    x = sld(&st[pl], site);
    y = sld(&st[PT + pl], site);
    z = sld(&st[2 * PT + pl], site);
  }
}
template <int PT, typename R>
__device__ __forceinline__ void stage_load(const R *stage, int row, int pl, R &x, R &y, R &z, int site) {
  stage_load_row<PT, R>(stage + (size_t)row * stage_stride<PT>(), pl, x, y, z, site);
}

// The per-atom core of passes 1 and 2: from the bond geometry (unit vectors, r, 2/r, f_C, f_C', the
// cosines of the bond pairs; R) and the parameter constants (T: R itself, or a dual number carrying
// parameter tangents), U = sum_j f_C (f_R - b f_A), which is twice the site energy U_i of Eq. 2,
// and P_ij = dU_i/dd_ij of every bond (the derivative of U_i itself, 1/2 included). INNER: every bond
// is inside R1 (callers pass f_C = 1 and f_C' = 0 as constants, which the compiler folds away).
//
// Per bond, with h_A = f_A/2 = D0 x and u2 = 2 (1 + zeta^n):
//   b = 2^(-(log2 u2 - 1)/(2n)),   f_R - b f_A = f_R - 2 b h_A,
//   c_ij = dU_i/dzeta_ij = -1/2 f_C f_A b' = f_C (b h_A) zeta^n / (zeta u2),
//   rad_ij = 1/2 [f_C' (f_R - b f_A) + f_C (f_R' - b f_A')],   f_R' - b f_A' = -alpha (2 f_R - b f_A),
// the same quantities as Eq. 3-6 and their derivatives, with the constant factors folded.
template <int M, bool INNER, typename T, typename R, bool GEN = false>
__device__ __forceinline__ void atom_core(const R (&ux)[M], const R (&uy)[M], const R (&uz)[M],
                                          const R (&r)[M], const R (&ir2)[M], const R (&fc)[M],
                                          const R (&fcp)[M], const R *cs, const PConsts<T> &K, T &U,
                                          T (&Px)[M], T (&Py)[M], T (&Pz)[M]) {
  // ---- pass 1: pair functions (Eq. 4-5 with Eq. 11-14 at S = 2) and zeta (Eq. 7, 10)
  constexpr int NP = M * (M - 1) / 2;
  T fR[M], hA[M], zeta[M], tq[NP > 0 ? NP : 1];
  T gq[GEN && NP > 0 ? NP : 1];                    // g itself (Tersoff form; the minimal form has g = t u)
#pragma unroll
  for (int j = 0; j < M; ++j) {
    if constexpr (GEN) {                           // exponents of r - r0 (exact in FP32 near r0)
      const T dr = r[j] - K.k0;
      hA[j] = K.D0 * ex2(dr * K.k1);               // f_A / 2
      fR[j] = K.cR * ex2(dr * K.kR1);
    } else {                                       // x = e^{-alpha (r - r0)}; r - r0 is exact in FP32 near r0
      const T x = ex2((r[j] - K.k0) * K.k1);
      hA[j] = K.D0 * x;                            // f_A / 2
      fR[j] = hA[j] * x;
    }
    zeta[j] = T(0.0f);
  }
  {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const T u = cs[q] - K.h;
        T g;
        if constexpr (GEN) {                       // Eq. 8, in the form without cancellation
          const T u2 = u * u;
          const T iv = rcp(u2 + K.d2);
          g = K.g0 + K.gcd * u2 * iv;
          tq[q] = K.gc2 * u * iv * iv;                // g' / 2
          gq[q] = g;
        } else {
          const T t = K.beta * u;                   // g = t u, g' = 2 t
          g = t * u;
          tq[q] = t;
        }
        zeta[j] += fc[k] * g;
        zeta[k] += fc[j] * g;
        ++q;
      }
    }
  }
  T cc[M], rad[M];
  U = T(0.0f);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const T z = zeta[j] > T(1e-30f) ? zeta[j] : T(1e-30f);   // see bond_order
    const T zn = ex2(K.n * lg2(z));                // zeta^n
    const T u2 = zn * R(2) + R(2);
    const T b = ex2(K.inv2n * lg2(u2) - K.inv2n);  // (1 + zeta^n)^(-1/(2n))
    const T bh = b * hA[j];                        // b f_A / 2
    const T e = bh * R(-2) + fR[j];                // f_R - b f_A
    U += fc[j] * e;                                // Eq. 3 (the 1/2 of Eq. 2 is applied by callers)
    cc[j] = fc[j] * bh * zn * rcp(z * u2);         // dU_i / dzeta_ij
    T mde;                                         // (f_R' - b f_A') / 2
    if constexpr (GEN) mde = K.hl * fR[j] + K.mha * bh;   // (-lambda f_R + mu b f_A) / 2
    else mde = K.mha * (fR[j] + e);
    rad[j] = R(0.5) * fcp[j] * e + fc[j] * mde;
  }

  // ---- pass 2: dU_i/dd_ij
  T Ax[M], Ay[M], Az[M], Rg[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    Ax[j] = T(0.0f); Ay[j] = T(0.0f); Az[j] = T(0.0f); Rg[j] = T(0.0f);
  }
  {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const T w = (cc[j] * fc[k] + cc[k] * fc[j]) * tq[q];   // half of the w of the header
        Ax[j] += w * ux[k]; Ay[j] += w * uy[k]; Az[j] += w * uz[k];
        Ax[k] += w * ux[j]; Ay[k] += w * uy[j]; Az[k] += w * uz[j];
        ++q;
      }
    }
  }
  // bonds inside the switching region (R1 < r < R2) carry the f_C'(r_ij) g term; the vote keeps
  // this loop off the common path where no bond of the warp is in that region
  bool sw = false;
  if constexpr (!INNER) {
#pragma unroll
    for (int j = 0; j < M; ++j) sw |= (fcp[j] != R(0));
    sw = __any_sync(0xffffffffu, sw);
  }
  if (sw) {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        T g;
        if constexpr (GEN) g = gq[q];
        else g = tq[q] * (cs[q] - K.h);
        Rg[j] += cc[k] * g;
        Rg[k] += cc[j] * g;
        ++q;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    // 2/r restores the factor 2 of g' = 2 t; s_ij = sum_k w_jk cos_jk = u_ij . A_ij, since
    // cos_jk = u_ij . u_ik
    const T sj = ux[j] * Ax[j] + uy[j] * Ay[j] + uz[j] * Az[j];
    const T coef = rad[j] + fcp[j] * Rg[j] - sj * ir2[j];
    Px[j] = coef * ux[j] + ir2[j] * Ax[j];
    Py[j] = coef * uy[j] + ir2[j] * Ay[j];
    Pz[j] = coef * uz[j] + ir2[j] * Az[j];
  }
}

// atom_core for FP32 and the minimal form with an even neighbour bound M: the per-bond work of pass 1
// and of the bond-order loop runs on bond pairs (2e, 2e+1) in packed FP32 pairs (two lanes of the
// pair per instruction; the SFU operations stay scalar), the x and y components of the pass-2 sums
// A_ij likewise; the pair loops and the final per-bond step are those of atom_core. Each packed
// operation rounds as its scalar counterpart; only the energy sum runs in two partial sums.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

template <int M, bool INNER>
__device__ __forceinline__ void atom_core_x2(const float (&ux)[M], const float (&uy)[M], const float (&uz)[M],
                                             const float (&r)[M], const float (&ir2)[M], const float (&fc)[M],
                                             const float (&fcp)[M], const float *cs, const PConsts<float> &K,
                                             float &U, float (&Px)[M], float (&Py)[M], float (&Pz)[M]) {
  static_assert(M % 2 == 0, "bond pairs");
  constexpr int H = M / 2, NP = M * (M - 1) / 2;
  // ---- pass 1: pair functions on bond pairs, then zeta (Eq. 7, 10) as atom_core
  float2 fR[H], hA[H];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const float2 t = __fmul2_rn(__fadd2_rn(make_float2(r[2 * h], r[2 * h + 1]), f2(-K.k0)), f2(K.k1));
    const float2 x = make_float2(ex2(t.x), ex2(t.y));
    hA[h] = __fmul2_rn(f2(K.D0), x);               // f_A / 2
    fR[h] = __fmul2_rn(hA[h], x);
  }
  float zeta[M], tq[NP > 0 ? NP : 1];
#pragma unroll
  for (int j = 0; j < M; ++j) zeta[j] = 0.0f;
  {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const float u = cs[q] - K.h;
        const float t = K.beta * u;                 // g = t u, g' = 2 t
        const float g = t * u;
        tq[q] = t;
        zeta[j] += fc[k] * g;
        zeta[k] += fc[j] * g;
        ++q;
      }
  }
  // ---- bond order and its derivative on bond pairs
  float cc[M], rad[M];
  float2 Uh = make_float2(0.f, 0.f);
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const float z0 = zeta[2 * h] > 1e-30f ? zeta[2 * h] : 1e-30f;
    const float z1 = zeta[2 * h + 1] > 1e-30f ? zeta[2 * h + 1] : 1e-30f;
    const float2 z = make_float2(z0, z1);
    const float2 a = __fmul2_rn(f2(K.n), make_float2(lg2(z0), lg2(z1)));
    const float2 zn = make_float2(ex2(a.x), ex2(a.y));               // zeta^n
    const float2 u2 = __ffma2_rn(zn, f2(2.f), f2(2.f));
    const float2 bl = __ffma2_rn(f2(K.inv2n), make_float2(lg2(u2.x), lg2(u2.y)), f2(-K.inv2n));
    const float2 b = make_float2(ex2(bl.x), ex2(bl.y));              // (1 + zeta^n)^(-1/(2n))
    const float2 bh = __fmul2_rn(b, hA[h]);
    const float2 e = __ffma2_rn(bh, f2(-2.f), fR[h]);                // f_R - b f_A
    const float2 zu = __fmul2_rn(z, u2);
    float2 c = __fmul2_rn(__fmul2_rn(bh, zn), make_float2(rcp(zu.x), rcp(zu.y)));
    const float2 mde = __fmul2_rn(f2(K.mha), __fadd2_rn(fR[h], e));
    float2 rd;
    if constexpr (INNER) {
      Uh = __fadd2_rn(Uh, e);
      rd = mde;
    } else {
      const float2 fch = make_float2(fc[2 * h], fc[2 * h + 1]);
      Uh = __ffma2_rn(fch, e, Uh);
      c = __fmul2_rn(fch, c);
      rd = __ffma2_rn(__fmul2_rn(f2(0.5f), make_float2(fcp[2 * h], fcp[2 * h + 1])), e, __fmul2_rn(fch, mde));
    }
    cc[2 * h] = c.x;
    cc[2 * h + 1] = c.y;
    rad[2 * h] = rd.x;
    rad[2 * h + 1] = rd.y;
  }
  U = Uh.x + Uh.y;

  // ---- pass 2: dU_i/dd_ij (atom_core's loops, the x and y sums packed)
  float2 Axy[M];
  float Az[M], Rg[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    Axy[j] = make_float2(0.f, 0.f);
    Az[j] = 0.f;
    Rg[j] = 0.f;
  }
  {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const float w = (cc[j] * fc[k] + cc[k] * fc[j]) * tq[q];
        const float2 ww = f2(w);
        Axy[j] = __ffma2_rn(ww, make_float2(ux[k], uy[k]), Axy[j]);
        Az[j] = __fmaf_rn(w, uz[k], Az[j]);
        Axy[k] = __ffma2_rn(ww, make_float2(ux[j], uy[j]), Axy[k]);
        Az[k] = __fmaf_rn(w, uz[j], Az[k]);
        ++q;
      }
  }
  bool sw = false;
  if constexpr (!INNER) {
#pragma unroll
    for (int j = 0; j < M; ++j) sw |= (fcp[j] != 0.f);
    sw = __any_sync(0xffffffffu, sw);
  }
  if (sw) {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const float g = tq[q] * (cs[q] - K.h);
        Rg[j] += cc[k] * g;
        Rg[k] += cc[j] * g;
        ++q;
      }
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float sj = ux[j] * Axy[j].x + uy[j] * Axy[j].y + uz[j] * Az[j];
    const float coef = rad[j] + fcp[j] * Rg[j] - sj * ir2[j];
    Px[j] = coef * ux[j] + ir2[j] * Axy[j].x;
    Py[j] = coef * uy[j] + ir2[j] * Axy[j].y;
    Pz[j] = coef * uz[j] + ir2[j] * Az[j];
  }
}

// Passes 1 and 2 for one atom per atom slot, M = the warp's largest neighbour count.
// sA/sB: bond records (u_x, u_y, u_z, r), (2/r, f_C, f_C', rev | j << 16); sC: pair cosines; lb/lq: this
// atom's first bond / pair in shared memory; m: its neighbour count (<= M). EXACT: every slot has
// m == M, so no bond is a phantom.
template <int M, int PT, bool EXACT, bool INNER, typename R, bool GEN = false>
__device__ __forceinline__ void atom_forward(const typename Vec4<R>::T *__restrict__ sA,
                                             const typename Vec4<R>::T *__restrict__ sB,
                                             const R *__restrict__ sC, R *__restrict__ stage,
                                             int lb, int lq, int m, bool store, int pl,
                                             const PConsts<R> &K, AtomAcc<R> &acc) {
  R ux[M], uy[M], uz[M], r[M], ir2[M], fc[M], fcp[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    if (EXACT || j < m) {
      const auto A = sld(&sA[lb + j], 1);
      const auto B = sld(&sB[lb + j], 2);
      ux[j] = A.x; uy[j] = A.y; uz[j] = A.z; r[j] = A.w;
      ir2[j] = B.x;
      if constexpr (INNER) {
        fc[j] = R(1);
        fcp[j] = R(0);
      } else {
        fc[j] = B.y;
        fcp[j] = B.z;
      }
    } else {
      ux[j] = R(0); uy[j] = R(0); uz[j] = R(0); r[j] = R(1);
      ir2[j] = R(0); fc[j] = R(0); fcp[j] = R(0);
    }
  }
  constexpr int NP = M * (M - 1) / 2;
  constexpr int NP4 = (NP + 3) / 4;     // 16-byte (float) / 32-byte (double) pair-row vectors
  R cs[NP4 > 0 ? 4 * NP4 : 4];
  if constexpr (EXACT) {
    const typename Vec4<R>::T *c4 = reinterpret_cast<const typename Vec4<R>::T *>(sC + lq);
#pragma unroll
    for (int q = 0; q < NP4; ++q) {
      const auto v = sld(&c4[q], 3);
      cs[4 * q] = v.x; cs[4 * q + 1] = v.y; cs[4 * q + 2] = v.z; cs[4 * q + 3] = v.w;
    }
  } else {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const int rowbase = lq + j * m - (j * (j + 1)) / 2 - j - 1;
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        cs[q] = R(0);
        if (k < m) cs[q] = sld(&sC[rowbase + k], 4);
        ++q;
      }
    }
  }

  R U, Px[M], Py[M], Pz[M];
  if constexpr (sizeof(R) == 4 && !GEN && M % 2 == 0)
    atom_core_x2<M, INNER>(ux, uy, uz, r, ir2, fc, fcp, cs, K, U, Px, Py, Pz);
  else
    atom_core<M, INNER, R, R, GEN>(ux, uy, uz, r, ir2, fc, fcp, cs, K, U, Px, Py, Pz);
  // the stage rows of this atom's bonds, and its terms of the virial -sum_j d_ij (x) P_ij added to the
  // lane's running sums (a phantom bond has P = 0)
#pragma unroll
  for (int j = 0; j < M; ++j) {
    if (store && (EXACT || j < m)) stage_store<PT, R>(stage, lb + j, pl, Px[j], Py[j], Pz[j]);
    if (store) {
      const R dx = r[j] * ux[j], dy = r[j] * uy[j], dz = r[j] * uz[j];
      acc.W[0] -= dx * Px[j]; acc.W[1] -= dy * Py[j]; acc.W[2] -= dz * Pz[j];
      acc.W[3] -= dx * Py[j]; acc.W[4] -= dy * Pz[j]; acc.W[5] -= dz * Px[j];
    }
  }
  if (store) acc.U += R(0.5) * U;
}

template <int PT, int MMAX, bool EXACT, bool INNER, typename R, bool GEN = false>
__device__ __forceinline__ void atom_forward_dispatch(int Mw, const typename Vec4<R>::T *sA,
                                                      const typename Vec4<R>::T *sB, const R *sC,
                                                      R *stage, int lb, int lq, int m, bool store,
                                                      int pl, const PConsts<R> &K, AtomAcc<R> &acc) {
#define TSF_CASE(MM)                                                                          \
  case MM:                                                                                    \
    if constexpr (MMAX >= MM)                                                                 \
      atom_forward<MM, PT, EXACT, INNER, R, GEN>(sA, sB, sC, stage, lb, lq, m, store, pl, K, acc); \
    break;
  switch (Mw) {
    TSF_CASE(1) TSF_CASE(2) TSF_CASE(3) TSF_CASE(4) TSF_CASE(5) TSF_CASE(6) TSF_CASE(7) TSF_CASE(8)
    default:
      break;
  }
#undef TSF_CASE
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
__device__ __forceinline__ float2 ld_cluster2(unsigned addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ double ld_cluster(unsigned addr, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void st_cluster(unsigned addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(unsigned addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(unsigned addr, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

struct BatchParams {
  int P, C;
  int64_t Ntot;
  const void *consts;              // R [P][8]: PConsts of every parameter set
  const int *atom_off, *boff, *poff;
  const int *ameta;                // [Ntot]: bonds kept | (some bond beyond R1) << 16
  const int4 *arev;                // [Ntot]: reverse bonds of the atom's first 8 bonds, configuration-local,
                                   // 16 bits each (bond e in bits 16 (e % 2) of component e / 2)
  const void *gA, *gB, *gcos;
  const CtaRec *recs;
  int ntiles;                      // parameter tiles: ceil(P / PT)
  int nconf, nchunks, chunk_tiles; // work items: nconf configurations x nchunks chunks of tiles
  int narrow;                      // run a partly filled last tile with 2 or 4 atoms per warp
  int *counter;                    // work-claiming counter of the launch, zero at launch
  unsigned wait_spins;             // polls of the staging wait before it gives up (a timeout)
  int mode;
  double *E;
  void *F;                         // [P][Ntot][3], or [Ntot][3][f_ld] when f_ld > 0
  int64_t f_ld;
  double *W;
  const double *tE, *tW;
  const double *tF;                // [Ntot][3]: target forces (fitness)
  const uint8_t *tmask;
  double *part;                    // [P][C][3]: FP64 residual terms e, v, f of every (p, c) (fitness)
  double *dpart;                   // [C][3]: FP64 target-norm terms of every configuration (fitness)
  unsigned *status;
};

// Shared memory of one CTA (R = float or double, R4 its 4-vector):
//   [region0: max(nb*stride(PT) R, (NW + (cluster ? ncta : 0)) * PT * kNSum double)]  stage of P_ij,
//    later the per-warp FP64 partial sums and, in rank 0 of a cluster, the totals of every rank
//   [sA: nb R4][sB: nb R4][sC: nq R][satom: natoms int4][stF: natoms R4 (fitness only)][srev: natoms int4]
// region0 sits at offset 0 in every CTA, so a peer's stage is addressed by mapping this CTA's own
// stage address to the peer rank.
template <int PT, bool CLUSTER, typename R, int NW = kNW>
__host__ __device__ inline size_t region0_bytes(int nb, int ncta) {
  const size_t st = (size_t)nb * stage_stride<PT>() * sizeof(R);
  const size_t rd = (size_t)(NW + (CLUSTER ? ncta : 0)) * kNSum * PT * sizeof(double);
  const size_t e = st > rd ? st : rd;
  return (e + 31) / 32 * 32;
}
template <int PT, bool CLUSTER, typename R, int NW = kNW>
__host__ __device__ inline size_t batch_smem(int nb, int nq, int nat, int ncta) {
  using R4 = typename Vec4<R>::T;
  size_t b = region0_bytes<PT, CLUSTER, R, NW>(nb, ncta) + (size_t)nb * 2 * sizeof(R4);
  b += ((size_t)nq * sizeof(R) + 31) / 32 * 32;
  b += (size_t)nat * sizeof(int4);
  b += (size_t)nat * sizeof(R4);
  b += (size_t)nat * sizeof(int4);
  return b;
}

// ---- TMA bulk copies into shared memory, completed on an mbarrier ----
__device__ __forceinline__ void mbar_init(unsigned long long *mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1D bulk copy global -> shared (both addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(mbar))
      : "memory");
}
constexpr unsigned kMbarSpins = 1u << 22;   // bound of a wait for one configuration's copies

// Single-CTA kernels of up to four neighbours with one atom per warp keep each atom's reverse rows as
// byte offsets in the stage (set when the item is staged), so the gather adds them to its base.
template <int PTT, int MMAX, bool CLUSTER, typename R>
__host__ __device__ constexpr bool kRevBytes() {
  return PTT == 32 && MMAX <= 4 && !CLUSTER;
}

// Pass 3 of one atom with a compile-time neighbour count M from a single-CTA stage: F_i = sum_j P_ij
// over the atom's own rows minus sum_j P_ji over the rows of the reverse bonds. rv: the reverse bonds'
// configuration-local indices, 16 bits each (roff maps them to stage rows). Every gather forms the two
// sums separately, each over its rows in order, and subtracts them once (F = Fo - Fr), so that an
// atom's force has the same rounding on every path; the rows are loaded before any is summed.
template <int M, int PTT, typename R>
struct GatherRows {
  R o[M][3], r[M][3];
};
// REVB: rv holds the reverse rows' byte offsets in the stage (first four bonds; kernels of up to four
// neighbours), otherwise their configuration-local indices, 16 bits each (roff maps them to stage rows).
template <int M, int PTT, typename R, bool REVB>
__device__ __forceinline__ void gather_load(const R *__restrict__ stage, int4 rv, int lb, int roff, int pl,
                                            GatherRows<M, PTT, R> &g) {
  const int rw[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
  for (int e = 0; e < M; ++e) stage_load<PTT, R>(stage, lb + e, pl, g.o[e][0], g.o[e][1], g.o[e][2], 13);
#pragma unroll
  for (int e = 0; e < M; ++e) {
    if constexpr (REVB) {
      static_assert(M <= 4, "byte offsets of the first four reverse rows");
      const R *st = reinterpret_cast<const R *>(reinterpret_cast<const unsigned char *>(stage) + rw[e]);
      stage_load_row<PTT, R>(st, pl, g.r[e][0], g.r[e][1], g.r[e][2], 15);
    } else {
      const int rb = (rw[e >> 1] >> (16 * (e & 1))) & 0xffff;
      stage_load<PTT, R>(stage, rb + roff, pl, g.r[e][0], g.r[e][1], g.r[e][2], 15);
    }
  }
}
template <int M, int PTT, typename R>
__device__ __forceinline__ void gather_sum(const GatherRows<M, PTT, R> &g, R &Fx, R &Fy, R &Fz) {
  R o[3] = {g.o[0][0], g.o[0][1], g.o[0][2]}, r[3] = {g.r[0][0], g.r[0][1], g.r[0][2]};
#pragma unroll
  for (int e = 1; e < M; ++e)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k] += g.o[e][k];
      r[k] += g.r[e][k];
    }
  Fx = o[0] - r[0];
  Fy = o[1] - r[1];
  Fz = o[2] - r[2];
}
template <int M, int PTT, typename R, bool REVB>
__device__ __forceinline__ void gather_atom(const R *__restrict__ stage, int4 rv, int lb, int roff, int pl,
                                            R &Fx, R &Fy, R &Fz) {
  GatherRows<M, PTT, R> g;
  gather_load<M, PTT, R, REVB>(stage, rv, lb, roff, pl, g);
  gather_sum<M, PTT, R>(g, Fx, Fy, Fz);
}
// Two atoms of the same neighbour count M, their loads issued together (one warp keeps both atoms'
// rows in flight); each atom's arithmetic is that of gather_atom.
template <int M, int PTT, typename R, bool REVB>
__device__ __forceinline__ void gather_atom_pair(const R *__restrict__ stage, int4 rv0, int lb0, int4 rv1, int lb1,
                                                 int roff, int pl, R (&F0)[3], R (&F1)[3]) {
  GatherRows<M, PTT, R> g0, g1;
  gather_load<M, PTT, R, REVB>(stage, rv0, lb0, roff, pl, g0);
  gather_load<M, PTT, R, REVB>(stage, rv1, lb1, roff, pl, g1);
  gather_sum<M, PTT, R>(g0, F0[0], F0[1], F0[2]);
  gather_sum<M, PTT, R>(g1, F1[0], F1[1], F1[2]);
}
// Dispatch on the atom's neighbour count; false when it exceeds MMAX (the caller's loop handles it).
template <int PTT, int MMAX, typename R, bool REVB>
__device__ __forceinline__ bool gather_dispatch(int m, const R *stage, int4 rv, int lb, int roff, int pl, R &Fx,
                                                R &Fy, R &Fz) {
#define TSF_GCASE(MM)                                                              \
  case MM:                                                                         \
    if constexpr (MMAX >= MM) {                                                    \
      gather_atom<MM, PTT, R, REVB>(stage, rv, lb, roff, pl, Fx, Fy, Fz);          \
      return true;                                                                 \
    }                                                                              \
    return false;
  switch (m) {
    case 0:
      return true;
    TSF_GCASE(1) TSF_GCASE(2) TSF_GCASE(3) TSF_GCASE(4) TSF_GCASE(5) TSF_GCASE(6) TSF_GCASE(7) TSF_GCASE(8)
    default:
      return false;
  }
#undef TSF_GCASE
}
// Both atoms with neighbour count m; false when m is not a count with a pair variant.
template <int PTT, int MMAX, typename R, bool REVB>
__device__ __forceinline__ bool gather_pair_dispatch(int m, const R *stage, int4 rv0, int lb0, int4 rv1, int lb1,
                                                     int roff, int pl, R (&F0)[3], R (&F1)[3]) {
#define TSF_PCASE(MM)                                                                    \
  case MM:                                                                               \
    if constexpr (MMAX >= MM) {                                                          \
      gather_atom_pair<MM, PTT, R, REVB>(stage, rv0, lb0, rv1, lb1, roff, pl, F0, F1);   \
      return true;                                                                       \
    }                                                                                    \
    return false;
  switch (m) {
    TSF_PCASE(3) TSF_PCASE(4)
    default:
      return false;
  }
#undef TSF_PCASE
}

// One parameter tile of PTT parameter sets (PTT = 32: one atom per warp; 16 or 8: 2 or 4 atoms per
// warp, used for the last, partly filled tile) of the item staged in shared memory: passes 1-3, the
// reductions and the per-(parameter set, configuration) outputs. `tile` counts tiles of the launch's
// full width PTW, so the tile's parameter sets are tile * PTW + (0 .. PTT-1).
template <typename R>
struct TileEnv {
  R *stage;
  const typename Vec4<R>::T *sA, *sB;
  const R *sC;
  const int4 *satom;
  const int4 *srev;                // per atom: the reverse bonds' configuration-local indices, 16 bits each
  const typename Vec4<R>::T *stF;
  int ns, s0, nat, c, cb0, B0;
  double inv_nat;
  const double *tgt;               // fitness: the configuration's targets E*, W*_1..6 (shared memory)
  uint8_t mask;
  bool fit;
  unsigned rank, ncta;
  const unsigned *peer_stage;
  const int *peer_b0;
};

template <int PTT, int PTW, int MMAX, bool CLUSTER, typename R, int NW, bool GEN = false>
__device__ __forceinline__ void tile_pass(const BatchParams &a, const TileEnv<R> &env, int tile) {
  using R4 = typename Vec4<R>::T;
  constexpr int APW = kWarp / PTT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = lane / PTT, pl = lane % PTT;
  R *stage = env.stage;
  const R4 *sA = env.sA, *sB = env.sB, *stF = env.stF;
  const R *sC = env.sC;
  const int4 *satom = env.satom;
  const int ns = env.ns, s0 = env.s0, nat = env.nat, c = env.c, cb0 = env.cb0, B0 = env.B0;
  const uint8_t mask = env.mask;
  const bool fit = env.fit;
  const unsigned rank = env.rank, ncta = env.ncta;
  const int per = (nat + (int)ncta - 1) / (int)ncta;   // atoms per cluster rank (the schedule's split)
  (void)per;
  const unsigned *peer_stage = env.peer_stage;
  const int *peer_b0 = env.peer_b0;
  (void)B0;
  (void)peer_stage;
  (void)peer_b0;
  (void)rank;
  (void)ncta;
  const int p = tile * PTW + pl;
  const bool active = p < a.P;
  PConsts<R> K;
  {
    constexpr int kStride = GEN ? 4 : 2;          // R4 records of constants per parameter set
    const R4 *kc = reinterpret_cast<const R4 *>(a.consts) + kStride * (active ? p : a.P - 1);
    const R4 k0 = kc[0], k1 = kc[1];
    K.D0 = k0.x; K.k1 = k0.y; K.k0 = k0.z; K.mha = k0.w;
    K.beta = k1.x; K.h = k1.y; K.n = k1.z; K.inv2n = k1.w;
    if constexpr (GEN) {
      const R4 k2 = kc[2], k3 = kc[3];
      K.cR = k2.x; K.kR1 = k2.y; K.kR0 = k2.z; K.hl = k2.w;
      K.g0 = k3.x; K.gc2 = k3.y; K.d2 = k3.z; K.gcd = k3.w;
    }
  }
  AtomAcc<R> acc;
  acc.U = R(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) acc.W[k] = R(0);

  // ---- passes 1-2
  for (int base = warp * APW; base < ns; base += NW * APW) {
    const int li = base + slot;
    const bool valid = li < ns;
    int4 at = make_int4(0, 0, 0, 0);
    if (valid) at = sld(&satom[li], 11);
    const int m = at.z;
    if constexpr (APW == 1) {
      if (m > MMAX) {
        if (lane == 0) set_status(a.status, TERSOFF_STATUS_MANY_NBRS);
        continue;
      }
      if (sizeof(R) == 4 && at.w == 0)
        atom_forward_dispatch<PTT, MMAX, true, sizeof(R) == 4, R, GEN>(m, sA, sB, sC, stage, at.x, at.y, m, true, pl, K, acc);
      else
        atom_forward_dispatch<PTT, MMAX, true, false, R, GEN>(m, sA, sB, sC, stage, at.x, at.y, m, true, pl, K, acc);
    } else {
      const int Mw = __reduce_max_sync(0xffffffffu, (unsigned)m);
      const bool uniform = __all_sync(0xffffffffu, m == Mw);
      if (Mw > MMAX) {
        if (lane == 0) set_status(a.status, TERSOFF_STATUS_MANY_NBRS);
        continue;
      }
      if (uniform && sizeof(R) == 4 && __all_sync(0xffffffffu, at.w == 0))
        atom_forward_dispatch<PTT, MMAX, true, sizeof(R) == 4, R, GEN>(Mw, sA, sB, sC, stage, at.x, at.y, m, valid, pl, K, acc);
      else if (uniform)
        atom_forward_dispatch<PTT, MMAX, true, false, R, GEN>(Mw, sA, sB, sC, stage, at.x, at.y, m, valid, pl, K, acc);
      else
        atom_forward_dispatch<PTT, MMAX, false, false, R, GEN>(Mw, sA, sB, sC, stage, at.x, at.y, m, valid, pl, K, acc);
    }
  }
  if constexpr (CLUSTER) cluster_sync_all(); else __syncthreads();

  // ---- pass 3: F_i = sum_j (P_ij - P_ji)
  R sf = R(0);   // sum |F - F*|^2 over the warp's atoms, or sum |F|^2 without a force target
  // F of atom li with a neighbour count beyond the compile-time gathers (and in the cluster and
  // several-atoms-per-warp variants): the own and the reverse rows summed in order, as in gather_sum
  auto gather_loop = [&](int li, const int4 &at, R (&F)[3]) {
    const int m = at.z, lb = at.x;
    R o[3] = {R(0), R(0), R(0)}, r[3] = {R(0), R(0), R(0)};
    for (int e = 0; e < m; ++e) {
      {
        R x, y, z;
        stage_load<PTT, R>(stage, lb + e, pl, x, y, z, 13);
        o[0] += x;
        o[1] += y;
        o[2] += z;
      }
      int packed;  // configuration-local indices of the reverse entry (bits 0-15) and of atom j (16-31)
      if constexpr (sizeof(R) == 4) packed = __float_as_int((float)sld(&sB[lb + e].w, 14));
      else packed = (int)sld(&sB[lb + e].w, 14);
      const int rb = packed & 0xffff;
      if constexpr (CLUSTER) {
        // the reverse entry belongs to atom j, whose rank is its slice of the configuration's atoms
        const unsigned rk = min((unsigned)(packed >> 16) / (unsigned)per, ncta - 1);
        // a reverse bond outside the configuration's bond range is an inconsistent schedule:
        // flag it and skip the peer read rather than touch another CTA's shared memory
        if (rb < peer_b0[rk] || rb >= peer_b0[rk + 1]) {
          set_status(a.status, TERSOFF_STATUS_NBR_OVERFLOW);
#ifdef TSF_DEBUG_BOUNDS
          if (atomicCAS(&tsf_dbg[0], 0u, 1u) == 0u) {
            tsf_dbg[1] = 21;
            tsf_dbg[2] = (unsigned)rb;
            tsf_dbg[3] = (unsigned)peer_b0[ncta];
          }
#endif
          continue;
        }
        const unsigned row = peer_stage[rk] + (unsigned)((rb - peer_b0[rk]) * stage_stride<PTT>() * sizeof(R));
        if constexpr (stage_packed<PTT, R>()) {
          const float2 xy = ld_cluster2(row + pl * sizeof(float2));
          r[0] += xy.x;
          r[1] += xy.y;
          r[2] += ld_cluster(row + (2 * PTT + pl) * sizeof(R), R(0));
        } else {
          r[0] += ld_cluster(row + pl * sizeof(R), R(0));
          r[1] += ld_cluster(row + (PTT + pl) * sizeof(R), R(0));
          r[2] += ld_cluster(row + (2 * PTT + pl) * sizeof(R), R(0));
        }
      } else {
        R x, y, z;
        stage_load<PTT, R>(stage, rb + cb0 - B0, pl, x, y, z, 15);
        r[0] += x;
        r[1] += y;
        r[2] += z;
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] = o[k] - r[k];
  };
  // the force of atom li: stored (evaluation) or its residual added to sf (fitness)
  auto finish = [&](int li, const R (&F)[3]) {
    const int i = s0 + li;
    if (a.mode == kModeEval) {
      if (active && a.F) {
        R *Fo = reinterpret_cast<R *>(a.F);
        if (a.f_ld > 0) {
          const size_t o = (size_t)i * 3 * a.f_ld + p;
          Fo[o] = F[0];
          Fo[o + a.f_ld] = F[1];
          Fo[o + 2 * a.f_ld] = F[2];
        } else {
          const size_t o = ((size_t)p * a.Ntot + i) * 3;
          Fo[o] = F[0];
          Fo[o + 1] = F[1];
          Fo[o + 2] = F[2];
        }
      }
    } else if (mask & 4) {
      const R4 t = sld(&stF[li], 16);
      const R ex = F[0] - t.x, ey = F[1] - t.y, ez = F[2] - t.z;
      sf += ex * ex + ey * ey + ez * ez;
    } else {
      sf += F[0] * F[0] + F[1] * F[1] + F[2] * F[2];   // finiteness of F where no residual checks it
    }
  };
  if constexpr (APW == 1 && !CLUSTER) {
    // one atom per warp: two atoms (li and li + NW) per iteration, whose row loads are issued together;
    // sf still takes the warp's atoms in ascending order
    const int roff = cb0 - B0;
    for (int l0 = warp; l0 < ns; l0 += 2 * NW) {
      const int l1 = l0 + NW;
      const int4 at0 = sld(&satom[l0], 12), rv0 = sld(&env.srev[l0], 12);
      R F0[3] = {R(0), R(0), R(0)}, F1[3] = {R(0), R(0), R(0)};   // an atom without bonds keeps F = 0
      if (l1 < ns) {
        const int4 at1 = sld(&satom[l1], 12), rv1 = sld(&env.srev[l1], 12);
        if (!(at0.z == at1.z &&
              gather_pair_dispatch<PTT, MMAX, R, kRevBytes<PTT, MMAX, CLUSTER, R>()>(at0.z, stage, rv0, at0.x, rv1, at1.x, roff, pl, F0, F1))) {
          if (!gather_dispatch<PTT, MMAX, R, kRevBytes<PTT, MMAX, CLUSTER, R>()>(at0.z, stage, rv0, at0.x, roff, pl, F0[0], F0[1], F0[2]))
            gather_loop(l0, at0, F0);
          if (!gather_dispatch<PTT, MMAX, R, kRevBytes<PTT, MMAX, CLUSTER, R>()>(at1.z, stage, rv1, at1.x, roff, pl, F1[0], F1[1], F1[2]))
            gather_loop(l1, at1, F1);
        }
        finish(l0, F0);
        finish(l1, F1);
      } else {
        if (!gather_dispatch<PTT, MMAX, R, kRevBytes<PTT, MMAX, CLUSTER, R>()>(at0.z, stage, rv0, at0.x, roff, pl, F0[0], F0[1], F0[2]))
          gather_loop(l0, at0, F0);
        finish(l0, F0);
      }
    }
  } else {
    for (int base = warp * APW; base < ns; base += NW * APW) {
      const int li = base + slot;
      if (li >= ns) continue;
      R F[3];
      gather_loop(li, sld(&satom[li], 12), F);   // F = 0 for an atom without bonds
      finish(li, F);
    }
  }

  // ---- reductions: over atom slots (FP32 shuffles), then over warps and cluster ranks in FP64, each in
  // a fixed order. Thread (lp, k) = (tid / 8, tid % 8) of the first kNSum * PTT threads forms quantity k
  // of parameter set lp; the partials are stored [warp][lp][k ^ (lp % 8)] (the xor spreads a warp's
  // stores of one k over the banks; the reads of a row are a permutation of it).
  static_assert(kNSum == 8, "the reduction maps eight quantities onto eight lanes");
  R v[kNSum];
  v[0] = acc.U;
#pragma unroll
  for (int k = 0; k < 6; ++k) v[1 + k] = acc.W[k];
  v[7] = sf;
#pragma unroll
  for (int k = 0; k < kNSum; ++k) v[k] = sum_over_atom_slots<PTT>(v[k]);
  if constexpr (CLUSTER) cluster_sync_all(); else __syncthreads();   // stages no longer read
  double *red = reinterpret_cast<double *>(stage);            // [NW][PTT][kNSum] per-warp partials
  double *tot = red + NW * PTT * kNSum;                       // [ncta][PTT][kNSum] rank totals (rank 0)
  if (slot == 0) {
#pragma unroll
    for (int k = 0; k < kNSum; ++k) {
      // FP32 partials are stored as they are (summed exactly below), FP64 ones as doubles
      if constexpr (sizeof(R) == 4) sst(&reinterpret_cast<float *>(red)[(warp * PTT + pl) * kNSum + (k ^ (pl & 7))], v[k], 17);
      else sst(&red[(warp * PTT + pl) * kNSum + (k ^ (pl & 7))], widen(v[k]), 17);
    }
  }
  __syncthreads();
  const bool red_thread = tid < kNSum * PTT;
  const int rl = tid >> 3, rk = tid & 7, rx = rk ^ (rl & 7);
  double T = 0.0;
  if (red_thread) {
    if constexpr (sizeof(R) == 4) {   // the FP32 partials' exact sum, rounded once to FP64
      float xw[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) xw[w] = sld(&reinterpret_cast<const float *>(red)[(w * PTT + rl) * kNSum + rx], 18);
      T = exact_sum<NW>(xw);
    } else {                          // FP64 partials: a pairwise tree in a fixed order
      double sw[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) sw[w] = sld(&red[(w * PTT + rl) * kNSum + rx], 18);
#pragma unroll
      for (int h = 1; h < NW; h <<= 1)
#pragma unroll
        for (int w = 0; w + h < NW; w += 2 * h) sw[w] += sw[w + h];
      T = sw[0];
    }
  }
  if constexpr (CLUSTER) {
    if (red_thread) st_cluster(map_to_rank(smem_addr(tot + ((int)rank * PTT + rl) * kNSum + rx), 0), T);
    cluster_sync_all();
    if (rank == 0 && red_thread) {
      T = 0.0;
      for (unsigned r = 0; r < ncta; ++r) T += sld(&tot[((int)r * PTT + rl) * kNSum + rx], 20);
    }
  }
  if (rank == 0 && red_thread) {   // whole warps: kNSum * PTT is a multiple of 32
    const int pp = tile * PTW + rl;
    const size_t pc = (size_t)pp * a.C + c;
    if (a.mode == kModeEval) {
      if (pp < a.P) {
        if (rk == 0 && a.E) a.E[pc] = T;
        if (rk >= 1 && rk <= 6 && a.W) a.W[pc * 6 + (rk - 1)] = T;
      }
    } else {
      // residual terms of Eq. 17-19 in FP64: (E/N - E*)^2, sum_k (W_k/N - W*_k)^2 and the force sum;
      // a quantity without a target contributes 0 when finite and NaN otherwise, so that any
      // non-finite prediction makes Z infinite
      const int bit = rk == 0 ? 1 : (rk <= 6 ? 2 : 4);
      double term = T;
      if (rk <= 6) {
        const double d = T * env.inv_nat - env.tgt[rk];
        term = d * d;
      }
      if (!(mask & bit)) term = isfinite(T) ? 0.0 : T - T;
      // the six virial terms of a parameter set sit in lanes 8g+1 .. 8g+6 of one warp: a fixed xor tree
      double tv = (rk >= 1 && rk <= 6) ? term : 0.0;
      tv += __shfl_xor_sync(0xffffffffu, tv, 1);
      tv += __shfl_xor_sync(0xffffffffu, tv, 2);
      tv += __shfl_xor_sync(0xffffffffu, tv, 4);
      const int g0 = lane & ~7;
      const double te = __shfl_sync(0xffffffffu, term, g0);
      const double tf = __shfl_sync(0xffffffffu, term, g0 + 7);
      if (pp < a.P && rk < kResidualTerms) a.part[pc * kResidualTerms + rk] = rk == 0 ? te : (rk == 1 ? tv : tf);
    }
  }
  // the next tile (or item) reuses the stage, where the partial sums live. A CTA barrier suffices in
  // a cluster too: peers touch a CTA's stage, and rank 0's totals, only after the next tile's first
  // cluster barrier, which this CTA reaches after the barrier below
  __syncthreads();
}

// Persistent work loop. The launch covers nconf configurations of one bucket (longest first), each
// split into nchunks chunks of chunk_tiles parameter tiles; a CTA (or cluster) claims the next item
// from an atomic counter, stages the configuration's geometry once (single-CTA launches: one TMA
// bulk copy per array, completed on an mbarrier) and runs the chunk's tiles.
template <int PT, int MMAX, bool CLUSTER, int MINB, typename R, int NW = kNW, bool GEN = false>
__global__ void __launch_bounds__(NW * kWarp, MINB) batch_kernel(const BatchParams a) {
  using R4 = typename Vec4<R>::T;
  extern __shared__ __align__(32) unsigned char smem[];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ int abort_flag;
  __shared__ int s_item;
  __shared__ double s_fn[NW];            // per-warp FP64 sums of |F*|^2 (target norm, first chunk)
  __shared__ double s_fr[kMaxCluster];   // rank 0 of a cluster: the ranks' sums
  __shared__ double s_tgt[7];            // fitness: targets E*, W*_1..6 of the item's configuration
  R *stage = reinterpret_cast<R *>(smem);
  constexpr int APW = kWarp / PT;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = lane / PT, pl = lane % PT;

  unsigned rank = 0, ncta = 1;
  if constexpr (CLUSTER) {
    rank = cluster_ctarank();
    ncta = cluster_nctarank();
  }
  const bool fit = a.mode == kModeFitness;
  if constexpr (!CLUSTER) {
    if (tid == 0) {
      mbar_init(&mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  unsigned phase = 0;
  const int nitems = a.nconf * a.nchunks;
  // the first item of a CTA (cluster) is its index in the grid; later ones are claimed from the
  // counter, which the preparation kernel zeroes: the claiming thread waits for it first
  const int nclusters = (int)(gridDim.x / ncta);
  bool first = true;
  for (;;) {
    if constexpr (CLUSTER) {
      if (rank == 0 && tid == 0) {
        int v = (int)(blockIdx.x / ncta);
        if (!first) {
          pdl_wait();
          v = nclusters + atomicAdd(a.counter, 1);
        }
        for (unsigned r = 0; r < ncta; ++r) st_cluster(map_to_rank(smem_addr(&s_item), r), v);
      }
      cluster_sync_all();
    } else {
      if (tid == 0) {
        int v = (int)blockIdx.x;
        if (!first) {
          pdl_wait();
          v = nclusters + atomicAdd(a.counter, 1);
        }
        s_item = v;
      }
      __syncthreads();
    }
    first = false;
    const int it = s_item;
    if (it >= nitems) break;
    const int ci = it / a.nchunks, chunk = it % a.nchunks;
    const int tile0 = chunk * a.chunk_tiles;
    const int tile1 = min(a.ntiles, tile0 + a.chunk_tiles);
    const int rec0 = ci * (int)ncta;
    const CtaRec rec = a.recs[rec0 + rank];
    const int c = rec.c;
    // the schedule record must match the device's bond CSR: a fitness launch may be queued on the
    // previous schedule before the host has checked a rebuild's neighbour counts, and then every
    // item whose configuration changed is skipped (the host launches again on the new schedule).
    // Every rank checks the records of all ranks of the item, so a cluster decides alike.
    {
      bool match = true;
      for (unsigned r = 0; r < ncta; ++r) {
        const CtaRec q = r == rank ? rec : a.recs[rec0 + r];
        if (q.ns == 0) continue;
        const int l = q.s0 + q.ns - 1, ml = a.ameta[l] & 0xffff;
        match = match && a.boff[q.s0] == q.B0 && a.boff[l] + ml == q.B0 + q.nb && a.poff[q.s0] == q.Q0 &&
                a.poff[l] + pair_slots(ml) == q.Q0 + q.nq;
      }
      if (!match) continue;
    }

    // atom slice of this CTA
    const int nat = rec.nat, s0 = rec.s0, ns = rec.ns, cb0 = rec.cb0;
    const int B0 = rec.B0, nb = rec.nb, Q0 = rec.Q0, nq = rec.nq;
    R4 *sA = reinterpret_cast<R4 *>(smem + region0_bytes<PT, CLUSTER, R, NW>(nb, (int)ncta));
    R4 *sB = sA + nb;
    R *sC = reinterpret_cast<R *>(sB + nb);
    int4 *satom = reinterpret_cast<int4 *>(reinterpret_cast<unsigned char *>(sC) +
                                           ((size_t)nq * sizeof(R) + 31) / 32 * 32);
    R4 *stF = reinterpret_cast<R4 *>(satom + ns);
    int4 *srev = reinterpret_cast<int4 *>(stF + ns);

    // stage this slice's geometry, atom table and target forces in shared memory
    {
      const R4 *gA = reinterpret_cast<const R4 *>(a.gA) + B0;
      const R4 *gB = reinterpret_cast<const R4 *>(a.gB) + B0;
      const R *gC = reinterpret_cast<const R *>(a.gcos) + Q0;
      if constexpr (!CLUSTER) {
        if (tid == 0) {
          const unsigned bA = (unsigned)(nb * sizeof(R4)), bC = (unsigned)(nq * sizeof(R));
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(&mbar, 2 * bA + bC);
          if (bA) {
            bulk_g2s(sA, gA, bA, &mbar);
            bulk_g2s(sB, gB, bA, &mbar);
          }
          if (bC) bulk_g2s(sC, gC, bC, &mbar);
        }
      } else {
        for (int t = tid; t < nb; t += (NW * kWarp)) {
          sst(&sA[t], gA[t], 6);
          sst(&sB[t], gB[t], 7);
        }
        for (int t = tid; t < nq; t += (NW * kWarp)) sst(&sC[t], gC[t], 8);
      }
      if (fit && tid < 7) s_tgt[tid] = tid == 0 ? a.tE[c] : a.tW[6 * (size_t)c + (tid - 1)];
      double f2 = 0.0;   // FP64 sum of |F*|^2 over this thread's atoms (target norm D_f of Eq. 19)
      for (int t = tid; t < ns; t += (NW * kWarp)) {
        const int am = a.ameta[s0 + t];
        sst(&satom[t], make_int4(a.boff[s0 + t] - B0, a.poff[s0 + t] - Q0, am & 0xffff, am >> 16), 9);
        int4 rv = a.arev[s0 + t];
        if constexpr (kRevBytes<PT, MMAX, CLUSTER, R>()) {   // rows of the full-width stage, in bytes
          const int rw[2] = {rv.x, rv.y};
          int off[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            off[e] = (((rw[e >> 1] >> (16 * (e & 1))) & 0xffff) + cb0 - B0) * (int)(stage_stride<PT>() * sizeof(R));
          rv = make_int4(off[0], off[1], off[2], off[3]);
        }
        sst(&srev[t], rv, 9);
        if (fit) {   // target force in the working precision
          const double *f = a.tF + 3 * (int64_t)(s0 + t);
          const double fx = f[0], fy = f[1], fz = f[2];
          R4 v;
          v.x = (R)fx;
          v.y = (R)fy;
          v.z = (R)fz;
          v.w = R(0);
          sst(&stF[t], v, 10);
          f2 += (fx * fx + fy * fy) + fz * fz;
        }
      }
      if (fit && chunk == 0) {   // the configuration's target norms are formed once, by its first chunk
        for (int off = 16; off > 0; off >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, off);
        if (lane == 0) s_fn[warp] = f2;
      }
      if constexpr (!CLUSTER) {
        // thread 0 waits (at most wait_spins polls) for the bulk copies; the barrier below publishes
        // them. A wait that gives up reports a timeout, and the CTA stops after a second wait (with
        // the built-in bound) for the copies still in flight, so that none lands after it exits
        if (tid == 0) {
          bool done = false;
          for (unsigned k = 0; k < a.wait_spins && !done; ++k) done = mbar_try_wait(&mbar, phase);
          abort_flag = done ? 0 : 1;
          if (!done) {
            set_status(a.status, TERSOFF_STATUS_TIMEOUT);
            for (unsigned k = 0; k < kMbarSpins && !done; ++k) done = mbar_try_wait(&mbar, phase);
          }
        }
        phase ^= 1u;
        __syncthreads();
        if (abort_flag) return;
      } else {
        __syncthreads();
      }
    }
    const uint8_t mask = fit ? a.tmask[c] : 0;
    if (fit && chunk == 0) {
      // target-norm terms of Eq. 17-19 in FP64: E*^2, |W*|^2 and sum_i |F*_i|^2 (0 without the target)
      double fsum = 0.0;
      if (tid == 0) {
        for (int w = 0; w < NW; ++w) fsum += s_fn[w];
        if constexpr (CLUSTER) st_cluster(map_to_rank(smem_addr(&s_fr[rank]), 0), fsum);
      }
      if constexpr (CLUSTER) {
        cluster_sync_all();
        if (rank == 0 && tid == 0) {
          fsum = 0.0;
          for (unsigned r = 0; r < ncta; ++r) fsum += s_fr[r];
        }
      }
      if (rank == 0 && tid == 0) {
        double dv = 0.0;
        for (int k = 0; k < 6; ++k) dv += a.tW[6 * (size_t)c + k] * a.tW[6 * (size_t)c + k];
        a.dpart[3 * c] = (mask & 1) ? a.tE[c] * a.tE[c] : 0.0;
        a.dpart[3 * c + 1] = (mask & 2) ? dv : 0.0;
        a.dpart[3 * c + 2] = (mask & 4) ? fsum : 0.0;
      }
    }
    unsigned peer_stage[kMaxCluster];
    int peer_b0[kMaxCluster + 1];
    if constexpr (CLUSTER) {
      const unsigned own = smem_addr(stage);
      for (unsigned r = 0; r < ncta; ++r) {
        peer_stage[r] = map_to_rank(own, r);
        peer_b0[r] = a.recs[rec0 + r].B0 - cb0;
      }
      peer_b0[ncta] = a.recs[rec0 + ncta - 1].B0 + a.recs[rec0 + ncta - 1].nb - cb0;
    }

    const TileEnv<R> env = {stage, sA, sB, sC, satom, srev, stF, ns, s0, nat, c, cb0, B0, rec.inv_nat, s_tgt, mask, fit,
                             rank, ncta, peer_stage, peer_b0};
    pdl_wait();   // per-call constants of the preparation kernel (a no-op after the first item)
    // the last tile may hold fewer parameter sets: the FP32 single-CTA variants for up to 4 neighbours
    // run it with more atoms in a warp (tiles of 16 or 8 parameter sets); other variants keep the
    // full width
    constexpr bool kNarrow = !CLUSTER && MMAX <= 4 && sizeof(R) == 4 && PT >= 16;
    for (int tile = tile0; tile < tile1; ++tile) {
      const int width = min(PT, a.P - tile * PT);
      if (kNarrow && a.narrow && width <= 8) tile_pass<(kNarrow ? 8 : PT), PT, MMAX, CLUSTER, R, NW, GEN>(a, env, tile);
      else if (kNarrow && PT > 16 && a.narrow && width <= 16)
        tile_pass<(kNarrow ? 16 : PT), PT, MMAX, CLUSTER, R, NW, GEN>(a, env, tile);
      else tile_pass<PT, PT, MMAX, CLUSTER, R, NW, GEN>(a, env, tile);
    }
  }
}

// Per call, one thread per parameter set: the FP32/FP64 constants of every parameter set (PConsts).
// When tF4 is given (the adjoint kernel), also one thread per atom: the target forces in the working
// precision as R4 (x, y, z, |F|^2).
template <typename R>
__global__ void prep_kernel(int P, const double *__restrict__ params, R *__restrict__ consts, int form,
                            int64_t Ntot, const double *__restrict__ tF, typename Vec4<R>::T *__restrict__ tF4,
                            int *__restrict__ counters = nullptr, int ncounters = 0) {
  pdl_trigger();   // the batched kernel may start staging geometry; it waits before reading our output
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ncounters) counters[t] = 0;   // the work counters of the batched launches that follow
  if (t < P && form == kFormMinimal) {
    const double *x = params + 6 * t;
    const double D0 = x[0], al = x[1], r0 = x[2], be = x[3], n = x[4], h = x[5];
    const double log2e = 1.4426950408889634;
    R *o = consts + 8 * t;
    o[0] = (R)D0;
    o[1] = (R)(-al * log2e);
    o[2] = (R)r0;
    o[3] = (R)(-0.5 * al);
    o[4] = (R)be;
    o[5] = (R)h;
    o[6] = (R)n;
    o[7] = (R)(-0.5 / n);
  } else if (t < P) {                              // Tersoff form: [D0, alpha, r0, S, n, h, gamma, c, d]
    const double *x = params + 9 * t;
    const double D0 = x[0], al = x[1], r0 = x[2], S = x[3], n = x[4], h = x[5], ga = x[6], c = x[7], d = x[8];
    const double log2e = 1.4426950408889634;
    const double lam = al * sqrt(2.0 * S), mu = al * sqrt(2.0 / S);   // Eq. 13-14
    R *o = consts + 16 * t;
    o[0] = (R)(0.5 * D0 * S / (S - 1.0));          // f_A / 2 prefactor (Eq. 12)
    o[1] = (R)(-mu * log2e);
    o[2] = (R)r0;
    o[3] = (R)mu;
    o[4] = (R)0.0;
    o[5] = (R)h;
    o[6] = (R)n;
    o[7] = (R)(-0.5 / n);
    o[8] = (R)(D0 / (S - 1.0));                    // f_R prefactor (Eq. 11)
    o[9] = (R)(-lam * log2e);
    o[10] = (R)0.0;
    o[11] = (R)(-0.5 * lam);
    o[12] = (R)ga;                                 // Eq. 8: g = gamma + gamma c^2/d^2 u^2 / (d^2 + u^2)
    o[13] = (R)(ga * c * c);
    o[14] = (R)(d * d);
    o[15] = (R)(ga * c * c / (d * d));
  }
  if (tF4 && t < Ntot) {
    const double fx = tF[3 * t], fy = tF[3 * t + 1], fz = tF[3 * t + 2];
    typename Vec4<R>::T v;
    v.x = (R)fx;
    v.y = (R)fy;
    v.z = (R)fz;
    v.w = (R)(fx * fx + fy * fy + fz * fz);
    tF4[t] = v;
  }
}

}  // namespace tsf
