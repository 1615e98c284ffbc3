// md.cu -- MD-scale force call: one large periodic cell, one parameter set, neighbour rebuild by a
// cell list plus energy, forces and virial (Eq. 1-14 of arXiv:1909.11474), every call.
//
// Coordinates. Every atom's fractional coordinate s = x H^-1 is split, in FP64, into an integer
// wrap m = floor(s), a cell index c = floor((s - m) nc) and an in-cell coordinate u = (s - m) nc - c
// in [0, 1), stored in FP32. A bond to an atom of a neighbouring cell (offset o in {-1,0,1}^3) is then
// d = sum_k (o_k + u_j,k - u_i,k) E_k with the cell edge vectors E_k = H_k / nc_k, all in FP32 and
// accurate to ~1e-6 A whatever the box size; its image shift is n = kw + m_i - m_j (kw = the
// periodic wrap of the neighbouring cell). Neighbour membership uses this FP32 distance where it is
// farther than a rounding margin from R2, and the exact FP64 test of the batched build otherwise, so
// the lists equal the batched build's bit for bit; they are sorted to the same (j, n) order.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "batch_kernel.cuh"
#include "common.cuh"
#include "ctx.hpp"

namespace tsf {

constexpr int kMdCap = 16;    // atom slots per cell
constexpr int kMdMaxM = 8;    // neighbours per atom handled by the force kernel
constexpr int kMdThreads = 128;

struct MdGeom {
  double H[9], Hinv[9];
  int nc[3];
  float E[9];                 // cell edge vectors, row k = H_k / nc_k
  float cut2_lo, cut2_hi;     // FP32 decision band around R2^2
  double R1, R2, R2sq;
};

__global__ void md_cells_kernel(int N, const double *__restrict__ pos, const MdGeom G,
                                int *__restrict__ cellcnt, int *__restrict__ cellatoms,
                                float4 *__restrict__ u4, int4 *__restrict__ m4, unsigned *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
    set_status(status, TERSOFF_STATUS_NONFINITE);
    m4[i] = make_int4(0, 0, 0, -1);
    return;
  }
  int mm[3], cc[3];
  float uu[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double s = x * G.Hinv[k] + y * G.Hinv[3 + k] + z * G.Hinv[6 + k];
    const double f = floor(s);
    const double w = (s - f) * (double)G.nc[k];
    int c = (int)floor(w);
    c = c < 0 ? 0 : (c >= G.nc[k] ? G.nc[k] - 1 : c);
    mm[k] = (int)f;
    cc[k] = c;
    uu[k] = (float)(w - (double)c);
  }
  const int cell = (cc[0] * G.nc[1] + cc[1]) * G.nc[2] + cc[2];
  u4[i] = make_float4(uu[0], uu[1], uu[2], 0.f);
  m4[i] = make_int4(mm[0], mm[1], mm[2], cell);
  const int slot = atomicAdd(&cellcnt[cell], 1);
  if (slot < kMdCap) cellatoms[cell * kMdCap + slot] = i;
  else set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
}

__global__ void __launch_bounds__(kMdThreads) md_neighbors_kernel(
    int N, const double *__restrict__ pos, const MdGeom G, const float4 *__restrict__ u4,
    const int4 *__restrict__ m4, const int *__restrict__ cellcnt, const int *__restrict__ cellatoms,
    int M, int *__restrict__ cnt_out, int *__restrict__ nbr, char4 *__restrict__ shift,
    unsigned *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int4 mi = m4[i];
  if (mi.w < 0) {
    cnt_out[i] = 0;
    return;
  }
  const float4 ui = u4[i];
  const int ci2 = mi.w % G.nc[2], ci1 = (mi.w / G.nc[2]) % G.nc[1], ci0 = mi.w / (G.nc[2] * G.nc[1]);
  int ej[32];
  int en[32];    // packed shift: (n0+128) << 16 | (n1+128) << 8 | (n2+128)
  int count = 0;
  const double xix = pos[3 * i], xiy = pos[3 * i + 1], xiz = pos[3 * i + 2];
  for (int o0 = -1; o0 <= 1; ++o0) {
    int a0 = ci0 + o0, w0 = 0;
    if (a0 < 0) { a0 += G.nc[0]; w0 = -1; } else if (a0 >= G.nc[0]) { a0 -= G.nc[0]; w0 = 1; }
    for (int o1 = -1; o1 <= 1; ++o1) {
      int a1 = ci1 + o1, w1 = 0;
      if (a1 < 0) { a1 += G.nc[1]; w1 = -1; } else if (a1 >= G.nc[1]) { a1 -= G.nc[1]; w1 = 1; }
      for (int o2 = -1; o2 <= 1; ++o2) {
        int a2 = ci2 + o2, w2 = 0;
        if (a2 < 0) { a2 += G.nc[2]; w2 = -1; } else if (a2 >= G.nc[2]) { a2 -= G.nc[2]; w2 = 1; }
        const int cell = (a0 * G.nc[1] + a1) * G.nc[2] + a2;
        const int ncell = min(cellcnt[cell], kMdCap);
        for (int q = 0; q < ncell; ++q) {
          const int j = cellatoms[cell * kMdCap + q];
          if (j == i && o0 == 0 && o1 == 0 && o2 == 0) continue;
          const float4 uj = u4[j];
          const float v0 = (float)o0 + (uj.x - ui.x), v1 = (float)o1 + (uj.y - ui.y), v2 = (float)o2 + (uj.z - ui.z);
          const float dx = v0 * G.E[0] + v1 * G.E[3] + v2 * G.E[6];
          const float dy = v0 * G.E[1] + v1 * G.E[4] + v2 * G.E[7];
          const float dz = v0 * G.E[2] + v1 * G.E[5] + v2 * G.E[8];
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 > G.cut2_hi) continue;
          const int4 mj = m4[j];
          const int n0 = w0 + mi.x - mj.x, n1 = w1 + mi.y - mj.y, n2 = w2 + mi.z - mj.z;
          bool in = r2 < G.cut2_lo;
          if (!in) {
            const ExactPair e = exact_pair(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], xix, xiy, xiz, G.H, n0, n1, n2);
            in = e.r2 < G.R2sq;
          }
          if (!in) continue;
          if (count < 32) {
            ej[count] = j;
            en[count] = ((n0 + 128) << 16) | ((n1 + 128) << 8) | (n2 + 128);
          }
          ++count;
        }
      }
    }
  }
  cnt_out[i] = count;
  if (count > M) {
    set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
    count = M;
  }
  // canonical order: ascending (j, n0, n1, n2); the packed shift sorts like (n0, n1, n2)
  for (int a = 1; a < count; ++a) {
    const int kj = ej[a], kn = en[a];
    int b = a - 1;
    while (b >= 0 && (ej[b] > kj || (ej[b] == kj && en[b] > kn))) {
      ej[b + 1] = ej[b];
      en[b + 1] = en[b];
      --b;
    }
    ej[b + 1] = kj;
    en[b + 1] = kn;
  }
  for (int e = 0; e < M; ++e) {
    if (e < count) {
      nbr[(size_t)i * M + e] = ej[e];
      shift[(size_t)i * M + e] = make_char4((signed char)(((en[e] >> 16) & 255) - 128),
                                            (signed char)(((en[e] >> 8) & 255) - 128),
                                            (signed char)((en[e] & 255) - 128), 0);
    } else {
      nbr[(size_t)i * M + e] = -1;
      shift[(size_t)i * M + e] = make_char4(0, 0, 0, 0);
    }
  }
}

// Reverse entry of every bond as a slot of the [N][kMdMaxM] partial-force array.
__global__ void md_reverse_kernel(int N, int M, const int *__restrict__ cnt, const int *__restrict__ nbr,
                                  const char4 *__restrict__ shift, int *__restrict__ rev, unsigned *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int m = min(cnt[i], M);
  for (int e = 0; e < m && e < kMdMaxM; ++e) {
    const int j = nbr[(size_t)i * M + e];
    const char4 n = shift[(size_t)i * M + e];
    const int mj = min(cnt[j], M);
    int found = -1;
    for (int f = 0; f < mj; ++f) {
      const char4 q = shift[(size_t)j * M + f];
      if (nbr[(size_t)j * M + f] == i && q.x == -n.x && q.y == -n.y && q.z == -n.z) {
        found = f;
        break;
      }
    }
    if (found < 0 || found >= kMdMaxM) {
      set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
      found = 0;
    }
    rev[(size_t)i * kMdMaxM + e] = j * kMdMaxM + found;
  }
}

// Passes 1-2 of one atom per thread, M = the warp's largest neighbour count; bonds e >= m of this
// thread are phantoms (f_C = f_C' = 0, unit vector 0), which contribute exactly zero.
template <int M, typename R>
__device__ __forceinline__ void md_atom(const R (&ux)[kMdMaxM], const R (&uy)[kMdMaxM],
                                        const R (&uz)[kMdMaxM], const R (&r)[kMdMaxM],
                                        const R (&ir)[kMdMaxM], const R (&fc)[kMdMaxM],
                                        const R (&fcp)[kMdMaxM], const PConsts<R> &K, R &U,
                                        R (&Wv)[6], R (&Px)[kMdMaxM], R (&Py)[kMdMaxM], R (&Pz)[kMdMaxM]) {
  constexpr int NP = M * (M - 1) / 2;
  R cs[NP > 0 ? NP : 1], tq[NP > 0 ? NP : 1];
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
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        cs[q] = ux[j] * ux[k] + uy[j] * uy[k] + uz[j] * uz[k];
        const R u = cs[q] - K.h;
        const R t = K.beta * u;
        const R g = t * u;
        tq[q] = t;
        zeta[j] += fc[k] * g;
        zeta[k] += fc[j] * g;
        ++q;
      }
  }
  R cc[M], rad[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    R b, bp;
    bond_order(zeta[j], K, b, bp);
    const R e = fR[j] - b * fA[j];
    U += R(0.5) * fc[j] * e;
    cc[j] = R(-0.5) * fc[j] * fA[j] * bp;
    const R de = R(2) * K.mha * (fR[j] + e);    // f_R' - b f_A' = -alpha (f_R + e)
    rad[j] = R(0.5) * (fcp[j] * e + fc[j] * de);
  }
  R Ax[M], Ay[M], Az[M], s[M], Rg[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    Ax[j] = R(0); Ay[j] = R(0); Az[j] = R(0); s[j] = R(0); Rg[j] = R(0);
  }
  {
    int q = 0;
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int k = j + 1; k < M; ++k) {
        const R w = (cc[j] * fc[k] + cc[k] * fc[j]) * tq[q];
        Ax[j] += w * ux[k]; Ay[j] += w * uy[k]; Az[j] += w * uz[k];
        Ax[k] += w * ux[j]; Ay[k] += w * uy[j]; Az[k] += w * uz[j];
        const R wc = w * cs[q];
        s[j] += wc;
        s[k] += wc;
        const R g = tq[q] * (cs[q] - K.h);
        Rg[j] += cc[k] * g;
        Rg[k] += cc[j] * g;
        ++q;
      }
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const R ir2 = ir[j] + ir[j];
    const R coef = rad[j] + fcp[j] * Rg[j] - s[j] * ir2;
    Px[j] = coef * ux[j] + ir2 * Ax[j];
    Py[j] = coef * uy[j] + ir2 * Ay[j];
    Pz[j] = coef * uz[j] + ir2 * Az[j];
    const R dx = r[j] * ux[j], dy = r[j] * uy[j], dz = r[j] * uz[j];
    Wv[0] -= dx * Px[j]; Wv[1] -= dy * Py[j]; Wv[2] -= dz * Pz[j];
    Wv[3] -= dx * Py[j]; Wv[4] -= dy * Pz[j]; Wv[5] -= dz * Px[j];
  }
}

template <typename R>
__global__ void __launch_bounds__(kMdThreads) md_force_kernel(
    int N, int M, const MdGeom G, const PConsts<R> K, const double *__restrict__ pos,
    const float4 *__restrict__ u4, const int4 *__restrict__ m4, const int *__restrict__ cnt,
    const int *__restrict__ nbr, const char4 *__restrict__ shift, typename Vec4<R>::T *__restrict__ Pst,
    double *__restrict__ partial, unsigned *status) {
  using R4 = typename Vec4<R>::T;
  __shared__ double red[kMdThreads / 32][7];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < N;
  int m = valid ? cnt[i] : 0;
  if (m > kMdMaxM) {
    set_status(status, TERSOFF_STATUS_MANY_NBRS);
    m = 0;
  }
  R ux[kMdMaxM], uy[kMdMaxM], uz[kMdMaxM], r[kMdMaxM], ir[kMdMaxM], fc[kMdMaxM], fcp[kMdMaxM];
  float4 ui = make_float4(0.f, 0.f, 0.f, 0.f);
  int4 mi = make_int4(0, 0, 0, 0);
  if (valid) {
    ui = u4[i];
    mi = m4[i];
  }
  const int ci2 = mi.w % G.nc[2], ci1 = (mi.w / G.nc[2]) % G.nc[1], ci0 = mi.w / (G.nc[2] * G.nc[1]);
#pragma unroll
  for (int e = 0; e < kMdMaxM; ++e) {
    ux[e] = R(0); uy[e] = R(0); uz[e] = R(0); r[e] = R(1); ir[e] = R(0); fc[e] = R(0); fcp[e] = R(0);
    if (e < m) {
      const int j = nbr[(size_t)i * M + e];
      const char4 n = shift[(size_t)i * M + e];
      R dx, dy, dz;
      if constexpr (sizeof(R) == 4) {
        // cell offset of j's image relative to i's cell, then the in-cell FP32 construction
        const float4 uj = u4[j];
        const int4 mj = m4[j];
        const int cj2 = mj.w % G.nc[2], cj1 = (mj.w / G.nc[2]) % G.nc[1], cj0 = mj.w / (G.nc[2] * G.nc[1]);
        const float v0 = (float)(cj0 - ci0 + G.nc[0] * (n.x + mj.x - mi.x)) + (uj.x - ui.x);
        const float v1 = (float)(cj1 - ci1 + G.nc[1] * (n.y + mj.y - mi.y)) + (uj.y - ui.y);
        const float v2 = (float)(cj2 - ci2 + G.nc[2] * (n.z + mj.z - mi.z)) + (uj.z - ui.z);
        dx = v0 * G.E[0] + v1 * G.E[3] + v2 * G.E[6];
        dy = v0 * G.E[1] + v1 * G.E[4] + v2 * G.E[7];
        dz = v0 * G.E[2] + v1 * G.E[5] + v2 * G.E[8];
      } else {
        const ExactPair p = exact_pair(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], pos[3 * i], pos[3 * i + 1],
                                       pos[3 * i + 2], G.H, n.x, n.y, n.z);
        dx = p.dx;
        dy = p.dy;
        dz = p.dz;
      }
      const R rr = sqrt(dx * dx + dy * dy + dz * dz);
      r[e] = rr;
      ir[e] = R(1) / rr;
      ux[e] = dx * ir[e];
      uy[e] = dy * ir[e];
      uz[e] = dz * ir[e];
      if (rr <= (R)G.R1) {
        fc[e] = R(1);
      } else if (rr < (R)G.R2) {
        const R w = (rr - (R)G.R1) / (R)(G.R2 - G.R1);
        if constexpr (sizeof(R) == 4) {
          fc[e] = 0.5f * (1.f + cospif(w));
          fcp[e] = (float)(-0.5 * M_PI / (G.R2 - G.R1)) * sinpif(w);
        } else {
          fc[e] = 0.5 * (1.0 + cospi(w));
          fcp[e] = -0.5 * M_PI / (G.R2 - G.R1) * sinpi(w);
        }
      } else {
        fc[e] = R(0);
      }
    }
  }
  R U = R(0), Wv[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  R Px[kMdMaxM], Py[kMdMaxM], Pz[kMdMaxM];
  const int Mw = __reduce_max_sync(0xffffffffu, (unsigned)m);
  switch (Mw) {
    case 1: md_atom<1, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz); break;
    case 2: md_atom<2, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz); break;
    case 3: md_atom<3, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz); break;
    case 4: md_atom<4, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz); break;
    case 5: md_atom<5, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz); break;
    case 6: md_atom<6, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz); break;
    case 7: md_atom<7, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz); break;
    case 8: md_atom<8, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz); break;
    default: break;
  }
#pragma unroll
  for (int e = 0; e < kMdMaxM; ++e)
    if (e < m) {
      R4 v;
      v.x = Px[e];
      v.y = Py[e];
      v.z = Pz[e];
      v.w = R(0);
      Pst[(size_t)i * kMdMaxM + e] = v;
    }
  // per-block FP64 partial sums of U and W
  double v[7] = {(double)U, (double)Wv[0], (double)Wv[1], (double)Wv[2], (double)Wv[3], (double)Wv[4], (double)Wv[5]};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    float f = (float)v[k];
    if constexpr (sizeof(R) == 8) {
      double d = v[k];
      for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
      v[k] = d;
    } else {
      for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
      v[k] = (double)f;
    }
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 7; ++k) red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x < 7) {
    double s = 0.0;
    for (int w = 0; w < kMdThreads / 32; ++w) s += red[w][threadIdx.x];
    partial[(size_t)blockIdx.x * 7 + threadIdx.x] = s;
  }
}

template <typename R>
__global__ void md_gather_kernel(int N, int M, const int *__restrict__ cnt, const int *__restrict__ rev,
                                 const typename Vec4<R>::T *__restrict__ Pst, R *__restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int m = min(min(cnt[i], M), kMdMaxM);
  R Fx = R(0), Fy = R(0), Fz = R(0);
  for (int e = 0; e < m; ++e) {
    const auto a = Pst[(size_t)i * kMdMaxM + e];
    const auto b = Pst[rev[(size_t)i * kMdMaxM + e]];
    Fx += a.x - b.x;
    Fy += a.y - b.y;
    Fz += a.z - b.z;
  }
  F[3 * (size_t)i] = Fx;
  F[3 * (size_t)i + 1] = Fy;
  F[3 * (size_t)i + 2] = Fz;
}

// Sum of the per-block partials in a fixed order (one warp per quantity).
__global__ void md_reduce_kernel(int nblocks, const double *__restrict__ partial, double *E, double *W) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= 7) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(size_t)b * 7 + k];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    if (k == 0) *E = s;
    else W[k - 1] = s;
  }
}

// ---------------------------------------------------------------------------------------------
int md_force(Ctx &c, int N, const double *pos, const double *boxh, const double *x, double R1, double R2,
             int M, int precision, double *E, void *F, double *W, cudaStream_t s, std::string &err) {
  MdGeom G;
  for (int k = 0; k < 9; ++k) G.H[k] = boxh[k];
  const double *H = G.H;
  const double bxc[3] = {H[4] * H[8] - H[5] * H[7], H[5] * H[6] - H[3] * H[8], H[3] * H[7] - H[4] * H[6]};
  const double cxa[3] = {H[7] * H[2] - H[8] * H[1], H[8] * H[0] - H[6] * H[2], H[6] * H[1] - H[7] * H[0]};
  const double axb[3] = {H[1] * H[5] - H[2] * H[4], H[2] * H[3] - H[0] * H[5], H[0] * H[4] - H[1] * H[3]};
  const double det = H[0] * bxc[0] + H[1] * bxc[1] + H[2] * bxc[2];
  if (!std::isfinite(det) || det == 0.0) {
    err = "singular or non-finite box";
    return TERSOFF_E_ARG;
  }
  for (int mu = 0; mu < 3; ++mu) {
    G.Hinv[3 * mu + 0] = bxc[mu] / det;
    G.Hinv[3 * mu + 1] = cxa[mu] / det;
    G.Hinv[3 * mu + 2] = axb[mu] / det;
  }
  const double vol = std::fabs(det);
  const double gap[3] = {vol / std::sqrt(bxc[0] * bxc[0] + bxc[1] * bxc[1] + bxc[2] * bxc[2]),
                         vol / std::sqrt(cxa[0] * cxa[0] + cxa[1] * cxa[1] + cxa[2] * cxa[2]),
                         vol / std::sqrt(axb[0] * axb[0] + axb[1] * axb[1] + axb[2] * axb[2])};
  double esum = 0.0;
  for (int k = 0; k < 3; ++k) {
    G.nc[k] = (int)std::floor(gap[k] / R2);
    if (G.nc[k] < 3) {
      err = "every plane spacing of the box must be at least 3*R2";
      return TERSOFF_E_ARG;
    }
    double en = 0.0;
    for (int mu = 0; mu < 3; ++mu) {
      G.E[3 * k + mu] = (float)(H[3 * k + mu] / G.nc[k]);
      en += G.E[3 * k + mu] * (double)G.E[3 * k + mu];
    }
    esum += std::sqrt(en);
  }
  // FP32 distance error <= a few ulp of the cell edge lengths; the band is 64x wider
  const double margin = 64.0 * 1.2e-7 * esum * 2.0 * R2 + 1e-6;
  G.R1 = R1;
  G.R2 = R2;
  G.R2sq = R2 * R2;
  G.cut2_lo = (float)(R2 * R2 - margin);
  G.cut2_hi = (float)(R2 * R2 + margin);
  const long ncells = (long)G.nc[0] * G.nc[1] * G.nc[2];
  if (ncells > (1L << 26)) {
    err = "too many cells";
    return TERSOFF_E_ARG;
  }
  const int nblk = (N + kMdThreads - 1) / kMdThreads;
  const size_t rs = precision == 64 ? 8 : 4;
  if (c.md_cellcnt.ensure(ncells * sizeof(int)) || c.md_cells.ensure(ncells * kMdCap * sizeof(int)) ||
      c.md_pos.ensure((size_t)N * (sizeof(float4) + sizeof(int4))) || c.md_cnt.ensure((size_t)N * sizeof(int)) ||
      c.md_nbr.ensure((size_t)N * M * sizeof(int)) || c.md_shift.ensure((size_t)N * M * sizeof(char4)) ||
      c.md_rev.ensure((size_t)N * kMdMaxM * sizeof(int)) || c.md_Pij.ensure((size_t)N * kMdMaxM * 4 * rs) ||
      c.md_red.ensure((size_t)nblk * 7 * sizeof(double))) {
    err = "device allocation failed";
    return TERSOFF_E_CUDA;
  }
  c.md_N = N;
  c.md_M = M;
  float4 *u4 = reinterpret_cast<float4 *>(c.md_pos.p);
  int4 *m4 = reinterpret_cast<int4 *>(u4 + N);
  unsigned *st = c.status.as<unsigned>();
  cudaMemsetAsync(c.md_cellcnt.p, 0, ncells * sizeof(int), s);
  md_cells_kernel<<<nblk, kMdThreads, 0, s>>>(N, pos, G, c.md_cellcnt.as<int>(), c.md_cells.as<int>(), u4, m4, st);
  md_neighbors_kernel<<<nblk, kMdThreads, 0, s>>>(N, pos, G, u4, m4, c.md_cellcnt.as<int>(), c.md_cells.as<int>(),
                                                  M, c.md_cnt.as<int>(), c.md_nbr.as<int>(),
                                                  c.md_shift.as<char4>(), st);
  md_reverse_kernel<<<nblk, kMdThreads, 0, s>>>(N, M, c.md_cnt.as<int>(), c.md_nbr.as<int>(),
                                                c.md_shift.as<char4>(), c.md_rev.as<int>(), st);
  const double D0 = x[0], al = x[1], r0 = x[2], be = x[3], n = x[4], h = x[5];
  const double log2e = 1.4426950408889634;
  if (precision == 64) {
    PConsts<double> K{D0, -al * log2e, al * r0 * log2e, -0.5 * al, be, h, n, -0.5 / n};
    md_force_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, M, G, K, pos, u4, m4, c.md_cnt.as<int>(),
                                                        c.md_nbr.as<int>(), c.md_shift.as<char4>(),
                                                        c.md_Pij.as<dvec4>(), c.md_red.as<double>(), st);
    md_gather_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, M, c.md_cnt.as<int>(), c.md_rev.as<int>(),
                                                         c.md_Pij.as<dvec4>(), reinterpret_cast<double *>(F));
  } else {
    PConsts<float> K{(float)D0, (float)(-al * log2e), (float)(al * r0 * log2e), (float)(-0.5 * al), (float)be, (float)h,
                     (float)n, (float)(-0.5 / n)};
    md_force_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, M, G, K, pos, u4, m4, c.md_cnt.as<int>(),
                                                       c.md_nbr.as<int>(), c.md_shift.as<char4>(),
                                                       c.md_Pij.as<float4>(), c.md_red.as<double>(), st);
    md_gather_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, M, c.md_cnt.as<int>(), c.md_rev.as<int>(),
                                                        c.md_Pij.as<float4>(), reinterpret_cast<float *>(F));
  }
  md_reduce_kernel<<<1, 7 * 32, 0, s>>>(nblk, c.md_red.as<double>(), E, W);
  cudaError_t e = launched(6);   // cells, neighbours, reverse, force, gather, reduce
  if (e != cudaSuccess) {
    err = std::string("CUDA error: ") + cudaGetErrorString(e);
    return TERSOFF_E_CUDA;
  }
  return TERSOFF_OK;
}

}  // namespace tsf
