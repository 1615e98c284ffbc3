// md.cu -- MD-scale force call: one large periodic cell, one parameter set, neighbour rebuild by a
// cell list plus energy, forces and virial (Eq. 1-14 of arXiv:1909.11474), every call.
//
// Coordinates. Every atom's cell coordinate w = x H^-1 nc is split, in FP64, into its floor C and an
// in-cell coordinate u = w - C in [0, 1), stored in FP32, and C into an integer wrap m and a cell
// index c (C = m nc + c). The force kernel builds a bond to an atom of a neighbouring cell (offset o
// in {-1,0,1}^3) as d = sum_k (o_k + u_j,k - u_i,k) E_k with the cell edge vectors E_k = H_k / nc_k,
// all in FP32 and accurate to ~1e-6 A whatever the box size; its image shift is n = kw + m_i - m_j
// (kw = the periodic wrap of the neighbouring cell). The pair search works in Cartesian coordinates
// relative to a brick of cells (a few cell edges long, so equally accurate). Membership uses the FP32
// distance where it is farther than a rounding margin from R2, and the exact FP64 test of the batched
// build otherwise, so the lists equal the batched build's bit for bit; they are sorted to the same
// (j, n) order.
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
constexpr int kBrick = 4;                                      // interior cells per brick edge
constexpr int kHaloEdge = kBrick + 2;                          // brick plus one cell on each side
constexpr int kHaloCells = kHaloEdge * kHaloEdge * kHaloEdge;  // 216
constexpr int kBrickCells = kBrick * kBrick * kBrick;          // 64
constexpr int kStageCap = 1024;                                // halo atoms staged in shared memory

struct MdGeom {
  double H[9], Hinv[9];
  int nc[3];
  int diag;                   // H (and so H^-1) diagonal: cell coordinates need 3 products, not 9
  double Hn[9];               // H^-1 with column k scaled by nc_k: x Hn = cell coordinates
  float Hnh[9], Hnl[9];       // Hn as FP32 head + tail (Hn = Hnh + Hnl to ~2^-48 relative)
  float E[9];                 // cell edge vectors, row k = H_k / nc_k
  float cut2_lo, cut2_hi;     // FP32 decision band around R2^2
  double R1, R2, R2sq;
  double inv_w, fcp_k;        // 1 / (R2 - R1) and -pi / (2 (R2 - R1)) (Eq. 9)
  float R1f, R2f, inv_wf, fcp_kf;
};

// Cell of every atom; the cell's slots hold (u, atom index) so the pair search reads one record per
// candidate. Every atom's neighbour count starts at zero here; an atom that gets no slot (non-finite
// position, full cell) keeps an empty list and the call is flagged.
//
// The cell coordinates w = x Hn are formed in FP32 head + tail arithmetic (products split exactly by
// FMA, sums by two-sum), accurate to ~2^-44 |w|; below |w| = 2^16 cells that is under the FP32 rounding
// of u itself. Other positions take FP64 arithmetic. The floor C is then that of head + tail, and
// u = w - C is rounded once to FP32: any consistent (C, u) serves the search and the bond vectors.
__global__ void md_cells_kernel(int N, const double *__restrict__ pos, const MdGeom G,
                                int *__restrict__ cellcnt, float4 *__restrict__ cellu,
                                float4 *__restrict__ u4, int4 *__restrict__ m4, int *__restrict__ cnt,
                                unsigned *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  cnt[i] = 0;
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  float xh[3], xl[3];
  bool fast = split_f64(x, xh[0], xl[0]);
  fast = split_f64(y, xh[1], xl[1]) && fast;
  fast = split_f64(z, xh[2], xl[2]) && fast;
  int Ci[3];
  float uu[3];
  if (fast) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float wh, wl;
      if (G.diag) {
        const float a = G.Hnh[4 * k], b = G.Hnl[4 * k];
        const float p = xh[k] * a;
        wl = __fmaf_rn(xh[k], a, -p) + __fmaf_rn(xh[k], b, xl[k] * a);
        wh = p;
      } else {
        float p[3], q = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float h = G.Hnh[3 * a + k], l = G.Hnl[3 * a + k];
          p[a] = xh[a] * h;
          q += __fmaf_rn(xh[a], h, -p[a]) + __fmaf_rn(xh[a], l, xl[a] * h);
        }
        float s1, t1, s2, t2;
        two_sum(p[0], p[1], s1, t1);
        two_sum(s1, p[2], s2, t2);
        wh = s2;
        wl = q + t1 + t2;
      }
      // normalise (|wl| <= ulp(wh) / 2), then C = floor(wh) + floor(frac(wh) + wl)
      float h2, t2;
      two_sum(wh, wl, h2, t2);
      wh = h2;
      wl = t2;
      fast = fast && fabsf(wh) < 65536.f;
      const float ch = floorf(wh);
      const float s = (wh - ch) + wl;
      const float cl = floorf(s);
      uu[k] = s - cl;
      Ci[k] = (int)ch + (int)cl;
    }
  }
  if (!fast) {
    // FP64 cell coordinates: w = s nc (nc folded into the inverse box), its floor C, u = w - C
    double w[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      w[k] = G.diag ? (k == 0 ? x : (k == 1 ? y : z)) * G.Hn[4 * k]
                    : x * G.Hn[k] + y * G.Hn[3 + k] + z * G.Hn[6 + k];
      ok = ok && fabs(w[k]) < 1e9;                 // false for NaN and inf
    }
    if (!ok) {
      set_status(status, TERSOFF_STATUS_NONFINITE);
      u4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      m4[i] = make_int4(0, 0, 0, 0);
      return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double C = floor(w[k]);
      uu[k] = (float)(w[k] - C);
      Ci[k] = (int)C;
    }
  }
  int mm[3], cc[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {   // the integer split C = m nc + c
    const int n = G.nc[k];
    const int m = Ci[k] >= 0 ? Ci[k] / n : -((n - 1 - Ci[k]) / n);
    mm[k] = m;
    cc[k] = Ci[k] - m * n;
  }
  const int cell = (cc[0] * G.nc[1] + cc[1]) * G.nc[2] + cc[2];
  u4[i] = make_float4(uu[0], uu[1], uu[2], 0.f);
  m4[i] = make_int4(mm[0], mm[1], mm[2], cell);
  const int slot = atomicAdd(&cellcnt[cell], 1);
  if (slot < kMdCap) cellu[cell * kMdCap + slot] = make_float4(uu[0], uu[1], uu[2], __int_as_float(i));
  else set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
}

// Code of the periodic wrap of cell coordinates c (each in [-1, nc]): (w0+1) << 4 | (w1+1) << 2 | (w2+1).
// The code of the opposite wrap is 42 - code.
__device__ __forceinline__ unsigned wrap_code(const MdGeom &G, int c0, int c1, int c2) {
  const int w0 = c0 < 0 ? 0 : (c0 >= G.nc[0] ? 2 : 1), w1 = c1 < 0 ? 0 : (c1 >= G.nc[1] ? 2 : 1),
            w2 = c2 < 0 ? 0 : (c2 >= G.nc[2] ? 2 : 1);
  return (unsigned)((w0 << 4) | (w1 << 2) | w2);
}
constexpr unsigned kWrapNeg = 42u;

// One candidate pair at Cartesian separation d (FP32): the FP32 distance decides outside the
// rounding band, the exact FP64 test inside it. The test is symmetric (the FP64 separation of
// (j, i, -n) is exactly the negated one of (i, j, n)), so deciding a pair once decides both entries.
__device__ __forceinline__ bool md_pair_in(const MdGeom &G, const double *__restrict__ pos,
                                           const int4 *__restrict__ m4, int i, int j, unsigned code,
                                           float dx, float dy, float dz) {
  const float r2 = dx * dx + dy * dy + dz * dz;
  if (r2 > G.cut2_hi) return false;
  if (r2 < G.cut2_lo) return true;
  const int4 mi = m4[i], mj = m4[j];
  const ExactPair e = exact_pair(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], pos[3 * i], pos[3 * i + 1],
                                 pos[3 * i + 2], G.H, (int)(code >> 4) - 1 + mi.x - mj.x,
                                 (int)((code >> 2) & 3) - 1 + mi.y - mj.y, (int)(code & 3) - 1 + mi.z - mj.z);
  return e.r2 < G.R2sq;
}

// Cartesian vector of a separation v in cell units: v0 E_0 + v1 E_1 + v2 E_2.
__device__ __forceinline__ float3 md_cart(const MdGeom &G, float v0, float v1, float v2) {
  return make_float3(v0 * G.E[0] + v1 * G.E[3] + v2 * G.E[6], v0 * G.E[1] + v1 * G.E[4] + v2 * G.E[7],
                     v0 * G.E[2] + v1 * G.E[5] + v2 * G.E[8]);
}

// The entries of the pairs one thread accepted, keys (partner << 6 | wrap code) in slot-major
// [M][N] rows: the thread's own nf entries take one atomic on its count, each partner's entry one on
// the partner's; all are issued after the search so that their round trips overlap. The order of
// appends is undone by the sort of the rows kernel. A thread keeps at most kFwdCap pairs: more means
// more than max_nbr (<= 32) neighbours, which the count records and the rows kernel flags.
constexpr int kFwdCap = 32;
__device__ __forceinline__ void md_flush_pairs(int i, int N, int M, const unsigned *list, int nf,
                                               int *__restrict__ cnt, unsigned *__restrict__ keys) {
  if (nf == 0) return;
  const int kept = min(nf, kFwdCap);
  const int p0 = atomicAdd(&cnt[i], nf);
  for (int e = 0; e < kept && p0 + e < M; ++e) keys[(size_t)(p0 + e) * N + i] = list[e * kMdThreads];
#pragma unroll 4
  for (int e = 0; e < kept; ++e) {
    const unsigned key = list[e * kMdThreads];
    const int j = (int)(key >> 6);
    const int q = atomicAdd(&cnt[j], 1);
    if (q < M) keys[(size_t)q * N + j] = ((unsigned)i << 6) | (kWrapNeg - (key & 63u));
  }
}

// Neighbour pairs by bricks of 4x4x4 cells: a CTA stages the records of its brick and of the cells
// around it (6x6x6) in shared memory, as Cartesian brick coordinates X = (u + halo cell - 1) E with
// the halo cell's periodic wrap packed above the atom index. One thread per atom of the brick tests the half
// shell: the 13 forward cells (offset d0 = 1; d0 = 0, d1 = 1; d0 = d1 = 0, d2 = 1) and the records
// after its own in its cell, each pair once. In the stage the three cells along z of one (d0, d1) are
// consecutive, so the half shell is 5 runs of records. A brick whose surroundings hold more than
// kStageCap atoms reads the records from global memory, cell by cell.
__global__ void __launch_bounds__(kMdThreads) md_pairs_kernel(
    int N, const double *__restrict__ pos, const MdGeom G, const int4 *__restrict__ m4,
    const int *__restrict__ cellcnt, const float4 *__restrict__ cellu, int M, int *__restrict__ cnt,
    unsigned *__restrict__ keys) {
  __shared__ float4 s_u[kStageCap];
  __shared__ unsigned s_list[kFwdCap * kMdThreads];
  __shared__ int s_cnt[kHaloCells], s_start[kHaloCells], s_gcell[kHaloCells], s_info[kHaloCells];
  __shared__ int s_ipre[kBrickCells + 1];
  __shared__ int s_total;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nb2 = (G.nc[2] + kBrick - 1) / kBrick, nb1 = (G.nc[1] + kBrick - 1) / kBrick;
  const int o0 = (blockIdx.x / (nb2 * nb1)) * kBrick, o1 = ((blockIdx.x / nb2) % nb1) * kBrick,
            o2 = (blockIdx.x % nb2) * kBrick;   // first interior cell of the brick
  // 1. counts of the halo cells; a halo cell beyond nc is next to no interior cell and stays empty
  for (int h = tid; h < kHaloCells; h += kMdThreads) {
    const int h0 = h / (kHaloEdge * kHaloEdge), h1 = (h / kHaloEdge) % kHaloEdge, h2 = h % kHaloEdge;
    const int c0 = o0 + h0 - 1, c1 = o1 + h1 - 1, c2 = o2 + h2 - 1;
    int n = 0, g = 0;
    if (c0 <= G.nc[0] && c1 <= G.nc[1] && c2 <= G.nc[2]) {
      const int g0 = c0 < 0 ? c0 + G.nc[0] : (c0 >= G.nc[0] ? c0 - G.nc[0] : c0);
      const int g1 = c1 < 0 ? c1 + G.nc[1] : (c1 >= G.nc[1] ? c1 - G.nc[1] : c1);
      const int g2 = c2 < 0 ? c2 + G.nc[2] : (c2 >= G.nc[2] ? c2 - G.nc[2] : c2);
      g = (g0 * G.nc[1] + g1) * G.nc[2] + g2;
      n = min(cellcnt[g], kMdCap);
    }
    s_cnt[h] = n;
    s_gcell[h] = g;
    s_info[h] = h0 | (h1 << 3) | (h2 << 6) | (int)(wrap_code(G, c0, c1, c2) << 9);
  }
  __syncthreads();
  // 2. warp 0: exclusive sums over the halo cells (7 per lane) and over the interior cells (2 per lane)
  if (tid < 32) {
    int a[7], tot = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const int h = 7 * lane + k;
      a[k] = h < kHaloCells ? s_cnt[h] : 0;
      tot += a[k];
    }
    int inc = tot;
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += v;
    }
    int run = inc - tot;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const int h = 7 * lane + k;
      if (h < kHaloCells) s_start[h] = run;
      run += a[k];
    }
    if (lane == 31) s_total = inc;
    int b[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int q = 2 * lane + k, q0 = q / (kBrick * kBrick), q1 = (q / kBrick) % kBrick, q2 = q % kBrick;
      const bool in = o0 + q0 < G.nc[0] && o1 + q1 < G.nc[1] && o2 + q2 < G.nc[2];
      b[k] = in ? s_cnt[((q0 + 1) * kHaloEdge + q1 + 1) * kHaloEdge + q2 + 1] : 0;
    }
    const int t2 = b[0] + b[1];
    int inc2 = t2;
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc2, off);
      if (lane >= off) inc2 += v;
    }
    s_ipre[2 * lane] = inc2 - t2;
    s_ipre[2 * lane + 1] = inc2 - t2 + b[0];
    if (lane == 31) s_ipre[kBrickCells] = inc2;
  }
  __syncthreads();
  // 3. stage the records, one thread per record (its cell by binary search over the starts)
  const int total = s_total;
  const bool staged = total <= kStageCap;
  if (staged) {
    for (int t = tid; t < total; t += kMdThreads) {
      int h = 0;
      for (int step = 128; step > 0; step >>= 1)
        if (h + step < kHaloCells && s_start[h + step] <= t) h += step;
      const int info = s_info[h];
      const float4 r = cellu[s_gcell[h] * kMdCap + (t - s_start[h])];
      const float3 X = md_cart(G, r.x + (float)((info & 7) - 1), r.y + (float)(((info >> 3) & 7) - 1),
                               r.z + (float)(((info >> 6) & 7) - 1));
      s_u[t] = make_float4(X.x, X.y, X.z, __int_as_float(__float_as_int(r.w) | ((info >> 9) << 24)));
    }
  } else {
    for (int h = tid; h < kHaloCells; h += kMdThreads) s_start[h] = s_gcell[h] * kMdCap;
  }
  __syncthreads();
  // 4. one thread per atom of the brick
  const int A = s_ipre[kBrickCells];
  unsigned *list = s_list + tid;
  for (int a = tid; a < A; a += kMdThreads) {
    int k = 0;                                     // interior cell of atom a
    for (int step = kBrickCells / 2; step > 0; step >>= 1)
      if (s_ipre[k + step] <= a) k += step;
    const int k0 = k / (kBrick * kBrick), k1 = (k / kBrick) % kBrick, k2 = k % kBrick;
    const int hi = ((k0 + 1) * kHaloEdge + k1 + 1) * kHaloEdge + k2 + 1;
    const int own = a - s_ipre[k];
    if (staged) {
      const int slot = s_start[hi] + own;
      const float4 ei = s_u[slot];
      const int i = __float_as_int(ei.w) & 0xffffff;
      int run = 0, p = 0, pend = 0, nf = 0;
      for (;;) {
        while (p >= pend && run < 5) {
          if (run < 4) {                           // (d0, d1) = (1,-1), (1,0), (1,1), (0,1)
            const int h = hi + (run < 3 ? (kHaloEdge + run - 1) : 1) * kHaloEdge;
            p = s_start[h - 1];
            pend = s_start[h + 1] + s_cnt[h + 1];
          } else {                                 // rest of the own cell, then (0, 0, 1)
            p = slot + 1;
            pend = s_start[hi + 1] + s_cnt[hi + 1];
          }
          ++run;
        }
        if (p >= pend) break;
        const float4 ej = s_u[p++];
        const unsigned tag = (unsigned)__float_as_int(ej.w);
        const int j = (int)(tag & 0xffffffu);
        if (md_pair_in(G, pos, m4, i, j, tag >> 24, ej.x - ei.x, ej.y - ei.y, ej.z - ei.z)) {
          if (nf < kFwdCap) list[nf * kMdThreads] = (tag & 0xffffffu) << 6 | (tag >> 24);
          ++nf;
        }
      }
      md_flush_pairs(i, N, M, list, nf, cnt, keys);
    } else {
      const float4 ei = cellu[s_start[hi] + own];
      const int i = __float_as_int(ei.w);
      int nf = 0;
      for (int l = 0; l < 14; ++l) {
        // l < 9: d0 = 1; l < 12: d0 = 0, d1 = 1; l = 12: (0, 0, 1); l = 13: own cell after own record
        const int d0 = l < 9 ? 1 : 0, d1 = l < 9 ? l / 3 - 1 : (l < 12 ? 1 : 0),
                  d2 = l < 9 ? l % 3 - 1 : (l < 12 ? l - 10 : (l == 12 ? 1 : 0));
        const int h = hi + (d0 * kHaloEdge + d1) * kHaloEdge + d2;
        const unsigned code = wrap_code(G, o0 + k0 + d0, o1 + k1 + d1, o2 + k2 + d2);
        const int n = s_cnt[h], st = s_start[h];
        for (int q = l == 13 ? own + 1 : 0; q < n; ++q) {
          const float4 ej = cellu[st + q];
          const int j = __float_as_int(ej.w);
          const float3 d = md_cart(G, (float)d0 + (ej.x - ei.x), (float)d1 + (ej.y - ei.y), (float)d2 + (ej.z - ei.z));
          if (md_pair_in(G, pos, m4, i, j, code, d.x, d.y, d.z)) {
            if (nf < kFwdCap) list[nf * kMdThreads] = ((unsigned)j << 6) | code;
            ++nf;
          }
        }
      }
      md_flush_pairs(i, N, M, list, nf, cnt, keys);
    }
  }
}

__device__ __forceinline__ void cas(unsigned &a, unsigned &b) {
  const unsigned lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// Entry (j, n) of a key (j << 6 | wrap code), n = wrap + m_i - m_j.
__device__ __forceinline__ void md_write_entry(const int4 *__restrict__ m4, int4 mi, unsigned key, size_t at,
                                               int *__restrict__ nbr, char4 *__restrict__ shift) {
  const int j = (int)(key >> 6);
  const int4 mj = m4[j];
  nbr[at] = j;
  shift[at] = make_char4((signed char)((int)((key >> 4) & 3) - 1 + mi.x - mj.x),
                         (signed char)((int)((key >> 2) & 3) - 1 + mi.y - mj.y),
                         (signed char)((int)(key & 3) - 1 + mi.z - mj.z), 0);
}

// One thread per atom: the appended keys in ascending (j, n) order (for one j the shift is the wrap
// plus a constant, so both orders agree) as the list (j, n); for an atom with at most kMdMaxM entries
// also the slot of each reverse bond in the partner's list, i.e. the rank of (i, -wrap) among the
// partner's keys.
__global__ void md_rows_kernel(int N, int M, const int4 *__restrict__ m4, const int *__restrict__ cnt,
                               const unsigned *__restrict__ keys, int *__restrict__ nbr,
                               char4 *__restrict__ shift, int *__restrict__ rev, unsigned *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int count = cnt[i];
  if (count > M) set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
  const int c = min(count, M);
  const int4 mi = m4[i];
  const unsigned *row = keys + i;                // entry e at row[e * N]
  if (c <= kMdMaxM) {
    unsigned k[kMdMaxM];
#pragma unroll
    for (int e = 0; e < kMdMaxM; ++e) k[e] = e < c ? row[(size_t)e * N] : 0xffffffffu;
    // Batcher's odd-even merge sort of 8 keys (19 compare-exchanges)
    cas(k[0], k[1]); cas(k[2], k[3]); cas(k[4], k[5]); cas(k[6], k[7]);
    cas(k[0], k[2]); cas(k[1], k[3]); cas(k[4], k[6]); cas(k[5], k[7]);
    cas(k[1], k[2]); cas(k[5], k[6]);
    cas(k[0], k[4]); cas(k[1], k[5]); cas(k[2], k[6]); cas(k[3], k[7]);
    cas(k[2], k[4]); cas(k[3], k[5]);
    cas(k[1], k[2]); cas(k[3], k[4]); cas(k[5], k[6]);
#pragma unroll
    for (int e = 0; e < kMdMaxM; ++e) {
      if (e < c) {
        md_write_entry(m4, mi, k[e], (size_t)e * N + i, nbr, shift);
        const int j = (int)(k[e] >> 6);
        const int cj = min(cnt[j], M);
        int slot = e * N + i;                      // partner beyond kMdMaxM: flagged by the force kernel
        if (cj <= kMdMaxM) {
          const unsigned want = ((unsigned)i << 6) | (kWrapNeg - (k[e] & 63u));
          const unsigned *rj = keys + j;
          int rank = 0;
          bool found = false;
#pragma unroll
          for (int f = 0; f < kMdMaxM; ++f) {
            if (f < cj) {
              const unsigned q = rj[(size_t)f * N];
              rank += q < want ? 1 : 0;
              found = found || q == want;
            }
          }
          if (!found) {
            set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
            rank = 0;
          }
          slot = rank * N + j;
        }
        rev[(size_t)e * N + i] = slot;
      }
    }
  } else {
    for (int e = 0; e < c; ++e) {                  // more than kMdMaxM entries: rank by counting
      const unsigned key = row[(size_t)e * N];
      int rank = 0;
      for (int f = 0; f < c; ++f) rank += row[(size_t)f * N] < key ? 1 : 0;
      md_write_entry(m4, mi, key, (size_t)rank * N + i, nbr, shift);
    }
#pragma unroll
    for (int e = 0; e < kMdMaxM; ++e) rev[(size_t)e * N + i] = e * N + i;
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
    const R x = ex2((r[j] - K.k0) * K.k1);   // r - r0 exact in FP32 near r0
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

// Fixed-order block sum of n values per quantity, src[k * stride + q] (q < n, k < K): a strided sum
// per thread (loads in flight together), a butterfly over each warp's lanes, then the warps in order
// (through `red`, [warps][>= K]); thread k < K returns quantity k.
template <int K>
__device__ __forceinline__ double md_block_sum(const double *src, size_t stride, int n, double (*red)[7]) {
  const int tid = threadIdx.x;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    acc[k] = 0.0;
#pragma unroll 4
    for (int q = tid; q < n; q += kMdThreads) acc[k] += __ldcg(&src[k * stride + q]);
    for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  }
  __syncthreads();                                 // earlier readers of red are done
  if ((tid & 31) == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[tid >> 5][k] = acc[k];
  __syncthreads();
  double s = 0.0;
  if (tid < K)
    for (int w = 0; w < kMdThreads / 32; ++w) s += red[w][tid];
  return s;
}

// Deterministic in-kernel sum of per-block partials [K][nblk] (FP64; blocks of kMdThreads threads):
// the last block of each group of kMdGroup blocks to finish sums its group into [K][ngroups], and
// the last group to finish sums the groups, both in a fixed order; quantity 0 goes to *out0 and
// quantity k >= 1 to out_rest[k - 1]. Counters [ngroups + 1] follow the group sums and are zeroed
// before the launch. The threads that wrote the block's partials have fenced before the call.
constexpr int kMdGroup = 64;
template <int K>
__device__ __forceinline__ void md_grouped_sum(double *partial, int nblk, int b, double *out0, double *out_rest,
                                               double (*red)[7]) {
  __shared__ int s_last;
  const int tid = threadIdx.x, ngroups = (nblk + kMdGroup - 1) / kMdGroup;
  double *gpart = partial + (size_t)K * nblk;
  unsigned *counter = reinterpret_cast<unsigned *>(gpart + (size_t)K * ngroups);
  const int g = b / kMdGroup, g0 = g * kMdGroup, gn = min(kMdGroup, nblk - g0);
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&counter[g], 1u) == (unsigned)(gn - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double t = md_block_sum<K>(partial + g0, (size_t)nblk, gn, red);
  if (tid < K) {
    gpart[(size_t)tid * ngroups + g] = t;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&counter[ngroups], 1u) == (unsigned)(ngroups - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double u = md_block_sum<K>(gpart, (size_t)ngroups, ngroups, red);
  if (tid == 0) *out0 = u;
  else if (tid < K) out_rest[tid - 1] = u;
}

// Bytes of the partial-sum area of K quantities over nblk blocks: partials, group sums, counters.
inline size_t md_sum_bytes(int K, int nblk) {
  const int ngroups = (nblk + kMdGroup - 1) / kMdGroup;
  return ((size_t)nblk + ngroups) * K * sizeof(double) + (ngroups + 1) * sizeof(unsigned);
}
inline size_t md_counter_offset(int K, int nblk) {
  const int ngroups = (nblk + kMdGroup - 1) / kMdGroup;
  return ((size_t)nblk + ngroups) * K * sizeof(double);
}

template <typename R>
__global__ void __launch_bounds__(kMdThreads, sizeof(R) == 4 ? 4 : 1) md_force_kernel(
    int N, int M, const MdGeom G, const PConsts<R> K, const double *__restrict__ pos,
    const float4 *__restrict__ u4, const int4 *__restrict__ m4, const int *__restrict__ cnt,
    const int *__restrict__ nbr, const char4 *__restrict__ shift, typename Vec4<R>::T *__restrict__ Pst,
    double *__restrict__ partial, double *__restrict__ E, double *__restrict__ W, unsigned *status) {
  using R4 = typename Vec4<R>::T;
  __shared__ double red[kMdThreads / 32][7];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < N;
  int m = valid ? min(cnt[i], M) : 0;   // a truncated list (count > M) is flagged; its row holds M entries
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
      const int j = nbr[(size_t)e * N + i];
      const char4 n = shift[(size_t)e * N + i];
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
      if constexpr (sizeof(R) == 4) {
        if (rr <= G.R1f) {
          fc[e] = 1.f;
        } else if (rr < G.R2f) {
          const float w = (rr - G.R1f) * G.inv_wf;
          fc[e] = 0.5f * (1.f + cospif(w));
          fcp[e] = G.fcp_kf * sinpif(w);
        }
      } else {
        if (rr <= G.R1) {
          fc[e] = 1.0;
        } else if (rr < G.R2) {
          const double w = (rr - G.R1) * G.inv_w;
          fc[e] = 0.5 * (1.0 + cospi(w));
          fcp[e] = G.fcp_k * sinpi(w);
        }
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
      Pst[(size_t)e * N + i] = v;
    }
  // per-warp sums in R, per-block FP64 partial sums of U and W, stored [7][blocks]
  R v[7] = {U, Wv[0], Wv[1], Wv[2], Wv[3], Wv[4], Wv[5]};
#pragma unroll
  for (int k = 0; k < 7; ++k)
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 7; ++k) red[warp][k] = (double)v[k];
  __syncthreads();
  const int nblk = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  if (tid < 7) {
    double s = 0.0;
    for (int w = 0; w < kMdThreads / 32; ++w) s += red[w][tid];
    partial[(size_t)tid * nblk + b] = s;
    __threadfence();                               // the partial before this block's count
  }
  md_grouped_sum<7>(partial, nblk, b, E, W, red);
}

template <typename R>
__global__ void md_gather_kernel(int N, int M, const int *__restrict__ cnt, const int *__restrict__ rev,
                                 const typename Vec4<R>::T *__restrict__ Pst, R *__restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int m = min(min(cnt[i], M), kMdMaxM);
  R Fx = R(0), Fy = R(0), Fz = R(0);
  for (int e = 0; e < m; ++e) {
    const auto a = Pst[(size_t)e * N + i];
    const auto b = Pst[rev[(size_t)e * N + i]];
    Fx += a.x - b.x;
    Fy += a.y - b.y;
    Fz += a.z - b.z;
  }
  F[3 * (size_t)i] = Fx;
  F[3 * (size_t)i + 1] = Fy;
  F[3 * (size_t)i + 2] = Fz;
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
  // FP32 distance error: brick coordinates of up to 6 cell edges, rounded once each and subtracted,
  // stay within ~12 ulp of the cell edge lengths; the band is 128 ulp wide
  const double margin = 128.0 * 1.2e-7 * esum * 2.0 * R2 + 1e-6;
  G.diag = 1;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (a != b && (H[3 * a + b] != 0.0 || G.Hinv[3 * a + b] != 0.0)) G.diag = 0;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) {
      G.Hn[3 * a + k] = G.Hinv[3 * a + k] * (double)G.nc[k];
      G.Hnh[3 * a + k] = (float)G.Hn[3 * a + k];
      G.Hnl[3 * a + k] = (float)(G.Hn[3 * a + k] - (double)G.Hnh[3 * a + k]);
    }
  G.R1 = R1;
  G.R2 = R2;
  G.R2sq = R2 * R2;
  G.inv_w = 1.0 / (R2 - R1);
  G.fcp_k = -0.5 * M_PI / (R2 - R1);
  G.R1f = (float)R1;
  G.R2f = (float)R2;
  G.inv_wf = (float)G.inv_w;
  G.fcp_kf = (float)G.fcp_k;
  G.cut2_lo = (float)(R2 * R2 - margin);
  G.cut2_hi = (float)(R2 * R2 + margin);
  const long ncells = (long)G.nc[0] * G.nc[1] * G.nc[2];
  if (ncells > (1L << 26)) {
    err = "too many cells";
    return TERSOFF_E_ARG;
  }
  const int nblk = (N + kMdThreads - 1) / kMdThreads;
  const int ngroups = (nblk + kMdGroup - 1) / kMdGroup;
  const size_t rs = precision == 64 ? 8 : 4;
  if (c.md_cellcnt.ensure(ncells * sizeof(int)) || c.md_cells.ensure(ncells * kMdCap * sizeof(float4)) ||
      c.md_pos.ensure((size_t)N * (sizeof(float4) + sizeof(int4))) || c.md_cnt.ensure((size_t)N * sizeof(int)) ||
      c.md_nbr.ensure((size_t)N * M * sizeof(int)) || c.md_shift.ensure((size_t)N * M * sizeof(char4)) ||
      c.md_keys.ensure((size_t)N * M * sizeof(unsigned)) ||
      c.md_rev.ensure((size_t)N * kMdMaxM * sizeof(int)) || c.md_Pij.ensure((size_t)N * kMdMaxM * 4 * rs) ||
      c.md_red.ensure(md_sum_bytes(7, nblk))) {
    err = "device allocation failed";
    return TERSOFF_E_CUDA;
  }
  c.md_N = N;
  c.md_M = M;
  float4 *u4 = reinterpret_cast<float4 *>(c.md_pos.p);
  int4 *m4 = reinterpret_cast<int4 *>(u4 + N);
  unsigned *st = c.status.as<unsigned>();
  cudaMemsetAsync(c.md_cellcnt.p, 0, ncells * sizeof(int), s);
  cudaMemsetAsync(static_cast<char *>(c.md_red.p) + md_counter_offset(7, nblk), 0, (ngroups + 1) * sizeof(unsigned), s);
  md_cells_kernel<<<nblk, kMdThreads, 0, s>>>(N, pos, G, c.md_cellcnt.as<int>(), c.md_cells.as<float4>(), u4, m4,
                                              c.md_cnt.as<int>(), st);
  const long nbricks = (long)((G.nc[0] + kBrick - 1) / kBrick) * ((G.nc[1] + kBrick - 1) / kBrick) *
                       ((G.nc[2] + kBrick - 1) / kBrick);
  md_pairs_kernel<<<(unsigned)nbricks, kMdThreads, 0, s>>>(N, pos, G, m4, c.md_cellcnt.as<int>(), c.md_cells.as<float4>(),
                                                           M, c.md_cnt.as<int>(), c.md_keys.as<unsigned>());
  md_rows_kernel<<<nblk, kMdThreads, 0, s>>>(N, M, m4, c.md_cnt.as<int>(), c.md_keys.as<unsigned>(),
                                             c.md_nbr.as<int>(), c.md_shift.as<char4>(), c.md_rev.as<int>(), st);
  const double D0 = x[0], al = x[1], r0 = x[2], be = x[3], n = x[4], h = x[5];
  const double log2e = 1.4426950408889634;
  if (precision == 64) {
    PConsts<double> K{D0, -al * log2e, r0, -0.5 * al, be, h, n, -0.5 / n};
    md_force_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, M, G, K, pos, u4, m4, c.md_cnt.as<int>(),
                                                        c.md_nbr.as<int>(), c.md_shift.as<char4>(),
                                                        c.md_Pij.as<dvec4>(), c.md_red.as<double>(), E, W, st);
    md_gather_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, M, c.md_cnt.as<int>(), c.md_rev.as<int>(),
                                                         c.md_Pij.as<dvec4>(), reinterpret_cast<double *>(F));
  } else {
    PConsts<float> K{(float)D0, (float)(-al * log2e), (float)r0, (float)(-0.5 * al), (float)be, (float)h,
                     (float)n, (float)(-0.5 / n)};
    md_force_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, M, G, K, pos, u4, m4, c.md_cnt.as<int>(),
                                                       c.md_nbr.as<int>(), c.md_shift.as<char4>(),
                                                       c.md_Pij.as<float4>(), c.md_red.as<double>(), E, W, st);
    md_gather_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, M, c.md_cnt.as<int>(), c.md_rev.as<int>(),
                                                        c.md_Pij.as<float4>(), reinterpret_cast<float *>(F));
  }
  cudaError_t e = launched(5);   // cells, pairs, rows, force (with the sums), gather
  if (e != cudaSuccess) {
    err = std::string("CUDA error: ") + cudaGetErrorString(e);
    return TERSOFF_E_CUDA;
  }
  return TERSOFF_OK;
}

// ---------------------------------------------------------------------------------------------
// Velocity-Verlet NVE on the MD-scale force call (units eV, A, amu, fs). The integrator is not part
// of the paper's method; it drives the force call the way an MD code does.
constexpr double kAccel = 9.648533215665e-3;      // 1 eV / (A amu) in A / fs^2 (CODATA 2018)
constexpr double kKinetic = 103.6426965268;       // 1 amu A^2 / fs^2 in eV

// a_i = (1 eV / (A amu)) / m_i in A / fs^2 per eV / A, once per run (the device's FP64 divide is slow).
__global__ void md_accel_kernel(int N, const double *__restrict__ mass, double *__restrict__ acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) acc[i] = kAccel / mass[i];
}

// v += a F dt / 2, then x += v dt (FP64 state, forces in R).
template <typename R>
__global__ void md_kick_drift_kernel(int N, double *__restrict__ pos, double *__restrict__ vel,
                                     const R *__restrict__ F, const double *__restrict__ acc, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double h = 0.5 * dt * acc[i];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double v = vel[3 * i + k] + h * (double)F[3 * i + k];
    vel[3 * i + k] = v;
    pos[3 * i + k] += v * dt;
  }
}

// v += a F dt / 2 (dt = 0: no kick) and the kinetic energy sum_i m v^2 / 2 into *Ekin, in a fixed
// order (per-block partials, then the grouped last-block sums).
template <typename R>
__global__ void __launch_bounds__(kMdThreads) md_kick_kernel(int N, double *__restrict__ vel,
                                                             const R *__restrict__ F, const double *__restrict__ mass,
                                                             const double *__restrict__ acc, double dt,
                                                             double *__restrict__ partial, double *__restrict__ Ekin) {
  __shared__ double red[kMdThreads / 32][7];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, tid = threadIdx.x;
  double ke = 0.0;
  if (i < N) {
    const double h = 0.5 * dt * acc[i];
    double v2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double v = vel[3 * i + k] + h * (double)F[3 * i + k];
      vel[3 * i + k] = v;
      v2 += v * v;
    }
    ke = (0.5 * kKinetic) * mass[i] * v2;
  }
  for (int off = 16; off > 0; off >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, off);
  if ((tid & 31) == 0) red[tid >> 5][0] = ke;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kMdThreads / 32; ++w) s += red[w][0];
    partial[blockIdx.x] = s;
    __threadfence();
  }
  md_grouped_sum<1>(partial, gridDim.x, blockIdx.x, Ekin, nullptr, red);
}

int md_nve(Ctx &c, int N, double *pos, double *vel, const double *mass, const double *boxh, const double *x,
           double R1, double R2, int M, int precision, double dt, int nsteps, double *Epot, double *Ekin,
           void *F, double *W, cudaStream_t s, std::string &err) {
  const int nblk = (N + kMdThreads - 1) / kMdThreads;
  const int ngroups = (nblk + kMdGroup - 1) / kMdGroup;
  const size_t sum_bytes = (md_sum_bytes(1, nblk) + 15) / 16 * 16;
  if (c.md_ke.ensure(sum_bytes + (size_t)N * sizeof(double))) {
    err = "device allocation failed";
    return TERSOFF_E_CUDA;
  }
  double *part = c.md_ke.as<double>();
  char *counters = static_cast<char *>(c.md_ke.p) + md_counter_offset(1, nblk);
  double *acc = reinterpret_cast<double *>(static_cast<char *>(c.md_ke.p) + sum_bytes);
  md_accel_kernel<<<nblk, kMdThreads, 0, s>>>(N, mass, acc);
  auto kick = [&](double h, int step) {
    cudaMemsetAsync(counters, 0, (ngroups + 1) * sizeof(unsigned), s);
    if (precision == 64)
      md_kick_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, vel, static_cast<const double *>(F), mass, acc, h, part,
                                                         Ekin + step);
    else
      md_kick_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, vel, static_cast<const float *>(F), mass, acc, h, part,
                                                        Ekin + step);
  };
  int rc = md_force(c, N, pos, boxh, x, R1, R2, M, precision, Epot, F, W, s, err);
  if (rc != TERSOFF_OK) return rc;
  kick(0.0, 0);                                     // kinetic energy of the initial velocities
  for (int k = 1; k <= nsteps; ++k) {
    if (precision == 64)
      md_kick_drift_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, pos, vel, static_cast<const double *>(F), acc, dt);
    else
      md_kick_drift_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, pos, vel, static_cast<const float *>(F), acc, dt);
    rc = md_force(c, N, pos, boxh, x, R1, R2, M, precision, Epot + k, F, W, s, err);
    if (rc != TERSOFF_OK) return rc;
    kick(dt, k);
  }
  const cudaError_t e = launched(2 + 2 * nsteps);   // accelerations, kicks and kick-drifts (the force calls count themselves)
  if (e != cudaSuccess) {
    err = std::string("CUDA error: ") + cudaGetErrorString(e);
    return TERSOFF_E_CUDA;
  }
  return TERSOFF_OK;
}

}  // namespace tsf
