// md.cu -- MD-scale force call: one large periodic cell, one parameter set, neighbour rebuild by a
// cell list plus energy, forces and virial (Eq. 1-14 of arXiv:1909.11474), every call.
//
// Coordinates. Every atom's cell coordinate w = x H^-1 nc is split into its floor C and an in-cell
// coordinate u = w - C in [0, 1), and C into an integer wrap m and a cell index c (C = m nc + c). The
// atom is kept as its in-cell Cartesian position X = u E (FP32; E = the cell edge vectors H_k / nc_k
// as rows). A bond to an atom of a neighbouring cell (offset o in {-1,0,1}^3) is d = o E + (X_j - X_i),
// in FP32 and accurate to ~1e-6 A whatever the box size; its image shift is n = kw + m_i - m_j (kw =
// the periodic wrap of the neighbouring cell). The FP32 d of (j, i) is exactly the negation of that of
// (i, j), so the two atoms of a pair decide membership alike. Membership uses the FP32 distance where
// it is farther than a rounding margin from R2, and the exact FP64 test of the batched build
// otherwise, so the lists equal the batched build's bit for bit; they are sorted to the same (j, n)
// order.
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
// Bricks of the pair search: 4 x 4 x 6 interior cells (the third axis, along which cells are
// consecutive, the longest), and the cells around them
constexpr int kBX = 4, kBY = 4, kBZ = 6;
constexpr int kHX = kBX + 2, kHY = kBY + 2, kHZ = kBZ + 2;
constexpr int kHaloCells = kHX * kHY * kHZ;       // 288
constexpr int kBrickCells = kBX * kBY * kBZ;      // 96
constexpr int kStageCap = 1024;                   // halo atoms staged in shared memory
constexpr int kSearchThreads = 192;               // about the atoms of a brick of a solid
constexpr int kCandCap = 12;                      // candidates (r^2 below the band's upper edge) kept per atom

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

// Cartesian vector of a separation v in cell units: v0 E_0 + v1 E_1 + v2 E_2.
__device__ __forceinline__ float3 md_cart(const MdGeom &G, float v0, float v1, float v2) {
  return make_float3(v0 * G.E[0] + v1 * G.E[3] + v2 * G.E[6], v0 * G.E[1] + v1 * G.E[4] + v2 * G.E[7],
                     v0 * G.E[2] + v1 * G.E[5] + v2 * G.E[8]);
}

// Cell of every atom; the cell's slots hold (X, atom index) so the search reads one record per
// candidate. An atom that gets no slot (non-finite position, full cell) gets cell index -1 and an
// empty list here; no other atom sees it, and the call is flagged. The search writes every other count.
//
// The cell coordinates w = x Hn are formed in FP32 head + tail arithmetic (products split exactly by
// FMA, sums by two-sum), accurate to ~2^-44 |w|; below |w| = 2^16 cells that is under the FP32 rounding
// of u itself. Other positions take FP64 arithmetic. The floor C is then that of head + tail, and
// u = w - C is rounded once to FP32: any consistent (C, u) serves the search and the bond vectors.
__global__ void md_cells_kernel(int N, const double *__restrict__ pos, const MdGeom G,
                                int *__restrict__ cellcnt, float4 *__restrict__ cellx,
                                float4 *__restrict__ x4, int4 *__restrict__ m4, int *__restrict__ cnt,
                                unsigned *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
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
      x4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      m4[i] = make_int4(0, 0, 0, -1);
      cnt[i] = 0;
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
  const float3 X = md_cart(G, uu[0], uu[1], uu[2]);
  x4[i] = make_float4(X.x, X.y, X.z, 0.f);
  const int slot = atomicAdd(&cellcnt[cell], 1);
  if (slot < kMdCap) {
    // the record's index carries in its sign bit whether the atom has a nonzero wrap m (lies outside
    // the primary box), so that the search loads m only for those atoms
    const int tag = i | ((mm[0] | mm[1] | mm[2]) ? (int)0x80000000u : 0);
    cellx[cell * kMdCap + slot] = make_float4(X.x, X.y, X.z, __int_as_float(tag));
  } else {
    set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
    cnt[i] = 0;
  }
  m4[i] = make_int4(mm[0], mm[1], mm[2], slot < kMdCap ? cell : -1);
}

// Offset code of a neighbouring cell o in {-1,0,1}^3: (o0+1) << 4 | (o1+1) << 2 | (o2+1). The code of
// -o is 42 - code.
constexpr unsigned kOffNeg = 42u;

// FP32 separation d = o E + (X_j - X_i) of an atom j of the neighbouring cell with offset code `code`
// (the products o_k E_k are exact, the sums rounded in a fixed order), so the d of (j, i) is exactly
// the negation of that of (i, j).
__device__ __forceinline__ float3 md_sep(const MdGeom &G, unsigned code, float4 xi, float4 xj) {
  const float o0 = (float)((int)(code >> 4) - 1), o1 = (float)((int)((code >> 2) & 3u) - 1),
              o2 = (float)((int)(code & 3u) - 1);
  const float3 b = md_cart(G, o0, o1, o2);
  return make_float3(__fadd_rn(b.x, __fsub_rn(xj.x, xi.x)), __fadd_rn(b.y, __fsub_rn(xj.y, xi.y)),
                     __fadd_rn(b.z, __fsub_rn(xj.z, xi.z)));
}

// Periodic wrap of the coordinate a = c + o (o in {-1, 0, 1}) on an axis of n cells: -1, 0 or 1, and
// the wrapped coordinate g.
__device__ __forceinline__ int md_wrap(int a, int n, int &g) {
  if (a < 0) {
    g = a + n;
    return -1;
  }
  if (a >= n) {
    g = a - n;
    return 1;
  }
  g = a;
  return 0;
}

// Membership of a candidate at FP32 separation d: the FP32 distance decides outside the rounding band
// around R2^2, the exact FP64 test of the batched build inside it (image shift n = wrap + m_i - m_j),
// so that every decision is the exact one.
__device__ __forceinline__ bool md_pair_in(const MdGeom &G, const double *__restrict__ pos,
                                           const int4 *__restrict__ m4, int i, int j, int4 mi, int w0, int w1,
                                           int w2, float3 d) {
  const float r2 = __fmaf_rn(d.z, d.z, __fmaf_rn(d.y, d.y, __fmul_rn(d.x, d.x)));
  if (r2 > G.cut2_hi) return false;
  if (r2 < G.cut2_lo) return true;
  const int4 mj = m4[j];
  const ExactPair e = exact_pair(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], pos[3 * i], pos[3 * i + 1],
                                 pos[3 * i + 2], G.H, w0 + mi.x - mj.x, w1 + mi.y - mj.y, w2 + mi.z - mj.z);
  return e.r2 < G.R2sq;
}

// The full shell of atom i (cell index mi.w, in-cell position xi): every record of the 27 cells around
// its own but i's own is a candidate; visit(key) is called for each member, key = j << 6 | offset code.
// The shell runs as 9 rows (o0, o1) of three cells along the third axis, each row one loop over its
// cells' records in turn (so that the lanes of a warp diverge by row lengths, not cell by cell). The
// FP32 separation here is (o E - X_i) + X_j; any rounding within the band serves, since the band
// sends every near-cutoff candidate to the exact test.
template <typename Visit>
__device__ __forceinline__ void md_shell(const MdGeom &G, const double *__restrict__ pos,
                                         const int4 *__restrict__ m4, const int *__restrict__ cellcnt,
                                         const float4 *__restrict__ cellx, int i, int4 mi, float4 xi,
                                         Visit &&visit) {
  const int nc0 = G.nc[0], nc1 = G.nc[1], nc2 = G.nc[2];
  const int c2 = mi.w % nc2, c1 = (mi.w / nc2) % nc1, c0 = mi.w / (nc2 * nc1);
  int g2[3], w2[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) w2[o] = md_wrap(c2 + o - 1, nc2, g2[o]);
#pragma unroll 1
  for (int ab = 0; ab < 9; ++ab) {
    const int a = ab / 3, b = ab - 3 * a;
    int g0, g1;
    const int w0 = md_wrap(c0 + a - 1, nc0, g0), w1 = md_wrap(c1 + b - 1, nc1, g1);
    const int row = (g0 * nc1 + g1) * nc2;
    const int n0 = min(cellcnt[row + g2[0]], kMdCap), n1 = min(cellcnt[row + g2[1]], kMdCap),
              n2 = min(cellcnt[row + g2[2]], kMdCap);
    // the row's offset o E for o2 = -1, less X_i; o2 = 0 and 1 add the third edge once and twice
    const float fa = (float)(a - 1), fb = (float)(b - 1);
    const float bx = fa * G.E[0] + fb * G.E[3] - G.E[6] - xi.x;
    const float by = fa * G.E[1] + fb * G.E[4] - G.E[7] - xi.y;
    const float bz = fa * G.E[2] + fb * G.E[5] - G.E[8] - xi.z;
    const int n01 = n0 + n1, T = n01 + n2;
    for (int q = 0; q < T; ++q) {
      const int c = q < n0 ? 0 : (q < n01 ? 1 : 2);
      const int slot = q - (c == 0 ? 0 : (c == 1 ? n0 : n01));
      const float4 r = cellx[(size_t)(row + g2[c]) * kMdCap + slot];
      const int j = __float_as_int(r.w) & 0x7fffffff;
      const float fc = (float)c;
      const float dx = __fadd_rn(__fmaf_rn(fc, G.E[6], bx), r.x);
      const float dy = __fadd_rn(__fmaf_rn(fc, G.E[7], by), r.y);
      const float dz = __fadd_rn(__fmaf_rn(fc, G.E[8], bz), r.z);
      if (j != i && md_pair_in(G, pos, m4, i, j, mi, w0, w1, w2[c], make_float3(dx, dy, dz)))
        visit(((unsigned)j << 6) | (unsigned)((a << 4) | (b << 2) | c));
    }
  }
}

// List entry (j, n) of key (j << 6 | offset code) of atom i (wraps m_i, cell (c0, c1, c2)):
// n = wrap + m_i - m_j. Bit 31 of the key marks a partner j with a nonzero m (it is loaded only then).
__device__ __forceinline__ void md_write_entry(const MdGeom &G, const int4 *__restrict__ m4, int4 mi, int c0, int c1,
                                               int c2, unsigned key, size_t at, int *__restrict__ nbr,
                                               char4 *__restrict__ shift) {
  const int j = (int)((key & 0x7fffffffu) >> 6);
  const int4 mj = (key & 0x80000000u) ? m4[j] : make_int4(0, 0, 0, 0);
  int g;
  const int w0 = md_wrap(c0 + (int)((key >> 4) & 3u) - 1, G.nc[0], g);
  const int w1 = md_wrap(c1 + (int)((key >> 2) & 3u) - 1, G.nc[1], g);
  const int w2 = md_wrap(c2 + (int)(key & 3u) - 1, G.nc[2], g);
  nbr[at] = j;
  shift[at] = make_char4((signed char)(w0 + mi.x - mj.x), (signed char)(w1 + mi.y - mj.y),
                         (signed char)(w2 + mi.z - mj.z), 0);
}

// Compare-exchange of two keys by their low 31 bits (bit 31 is a mark that travels with the key).
__device__ __forceinline__ void cas(unsigned &a, unsigned &b) {
  const bool swap = (b << 1) < (a << 1);
  const unsigned lo = swap ? b : a, hi = swap ? a : b;
  a = lo;
  b = hi;
}

// The list of atom i from its members' keys k (count of them; at most kMdMaxM kept, the rest ~0u):
// the count, then the keys sorted (Batcher's odd-even merge sort of 8, 19 compare-exchanges; with at
// most one image of any j, plane spacings of at least 3 R2, the key order is the (j, n) order) into
// the rows of `keys` and the entries (j, n) into the lists.
__device__ __forceinline__ void md_emit(int N, int M, int i, int4 mi, int c0, int c1, int c2, const MdGeom &G,
                                        const int4 *__restrict__ m4, unsigned (&k)[kMdMaxM], int count,
                                        int *__restrict__ cnt, unsigned *__restrict__ keys, int *__restrict__ nbr,
                                        char4 *__restrict__ shift, unsigned *status) {
  cnt[i] = count;
  if (count > M) set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
  const int cm = min(count, M);
  cas(k[0], k[1]); cas(k[2], k[3]); cas(k[4], k[5]); cas(k[6], k[7]);
  cas(k[0], k[2]); cas(k[1], k[3]); cas(k[4], k[6]); cas(k[5], k[7]);
  cas(k[1], k[2]); cas(k[5], k[6]);
  cas(k[0], k[4]); cas(k[1], k[5]); cas(k[2], k[6]); cas(k[3], k[7]);
  cas(k[2], k[4]); cas(k[3], k[5]);
  cas(k[1], k[2]); cas(k[3], k[4]); cas(k[5], k[6]);
#pragma unroll
  for (int e = 0; e < kMdMaxM; ++e)
    if (e < cm) {
      keys[(size_t)e * N + i] = k[e] & 0x7fffffffu;
      md_write_entry(G, m4, mi, c0, c1, c2, k[e], (size_t)e * N + i, nbr, shift);
    }
}

// The whole search of atom i from the cell arrays in global memory (md_shell): the path of bricks
// whose surroundings exceed the stage and of atoms with more than kMdMaxM members. Such an atom
// enumerates its shell a second time, keeps the first M members found in its row of `keys` and
// writes each at its rank among them (the row itself stays in the order found: the force kernel
// flags the atom and gives it no forces).
__device__ __noinline__ void md_search_atom(int N, int M, int i, const double *__restrict__ pos, const MdGeom &G,
                                               const float4 *__restrict__ x4, const int4 *__restrict__ m4,
                                               const int *__restrict__ cellcnt, const float4 *__restrict__ cellx,
                                               int *__restrict__ cnt, unsigned *__restrict__ keys,
                                               int *__restrict__ nbr, char4 *__restrict__ shift, unsigned *status) {
  const int4 mi = m4[i];
  const float4 xi = x4[i];
  const int nc2 = G.nc[2], nc1 = G.nc[1];
  const int c2 = mi.w % nc2, c1 = (mi.w / nc2) % nc1, c0 = mi.w / (nc2 * nc1);
  unsigned k[kMdMaxM];
#pragma unroll
  for (int u = 0; u < kMdMaxM; ++u) k[u] = 0xffffffffu;
  int count = 0;
  md_shell(G, pos, m4, cellcnt, cellx, i, mi, xi, [&](unsigned key) {
#pragma unroll
    for (int u = 0; u < kMdMaxM; ++u)
      if (u == count) k[u] = key | 0x80000000u;   // the partner's m is loaded
    ++count;
  });
  if (count <= kMdMaxM) {
    md_emit(N, M, i, mi, c0, c1, c2, G, m4, k, count, cnt, keys, nbr, shift, status);
    return;
  }
  cnt[i] = count;
  if (count > M) set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
  const int cm = min(count, M);
  int p = 0;
  md_shell(G, pos, m4, cellcnt, cellx, i, mi, xi, [&](unsigned key) {
    if (p < M) keys[(size_t)p * N + i] = key;
    ++p;
  });
  for (int e = 0; e < cm; ++e) {
    const unsigned key = keys[(size_t)e * N + i];
    int rank = 0;
    for (int f = 0; f < cm; ++f) rank += keys[(size_t)f * N + i] < key ? 1 : 0;
    md_write_entry(G, m4, mi, c0, c1, c2, key | 0x80000000u, (size_t)rank * N + i, nbr, shift);
  }
}

// Neighbour lists by bricks of 4x4x6 cells, full shell, no atomics: a CTA stages the records of its
// brick and of the cells around it (6x6x8) in shared memory as brick coordinates (the in-cell
// position plus the halo cell's offset, (h - 1) E), with each record's halo cell beside it. One
// thread per atom of the brick tests the 9 rows (o0, o1) of its shell; the three cells of a row lie
// consecutively in the stage, so a row is one run of records. Members (at most kMdMaxM kept in
// registers) are sorted and written by md_emit. A brick whose surroundings hold more than kStageCap
// atoms, and an atom with more than kMdMaxM members, take the global-memory path (md_search_atom).
__global__ void __launch_bounds__(kSearchThreads, 5) md_search_kernel(
    int N, int M, const double *__restrict__ pos, const __grid_constant__ MdGeom G, const float4 *__restrict__ x4,
    const int4 *__restrict__ m4, const int *__restrict__ cellcnt, const float4 *__restrict__ cellx,
    int *__restrict__ cnt, unsigned *__restrict__ keys, int *__restrict__ nbr, char4 *__restrict__ shift,
    unsigned *status) {
  __shared__ __align__(16) float s_sx[kStageCap], s_sy[kStageCap], s_sz[kStageCap];   // brick coordinates
  __shared__ int s_sj[kStageCap];   // atom index; sign bit: a nonzero wrap m
  __shared__ unsigned short s_h[kStageCap];        // halo cell of each staged record
  // candidates of each thread, [u][tid]; slot kCandCap takes the writes once the list is full
  __shared__ unsigned short s_cand[(kCandCap + 1) * kSearchThreads];
  __shared__ int s_cnt[kHaloCells], s_start[kHaloCells], s_gcell[kHaloCells];
  __shared__ int s_ipre[kBrickCells + 1];
  __shared__ int s_total;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nb2 = (G.nc[2] + kBZ - 1) / kBZ, nb1 = (G.nc[1] + kBY - 1) / kBY;
  const int o0 = (blockIdx.x / (nb2 * nb1)) * kBX, o1 = ((blockIdx.x / nb2) % nb1) * kBY,
            o2 = (blockIdx.x % nb2) * kBZ;   // first interior cell of the brick
  // 1. counts of the halo cells; a halo cell beyond nc is next to no interior cell and stays empty
  for (int h = tid; h < kHaloCells; h += kSearchThreads) {
    const int h0 = h / (kHY * kHZ), h1 = (h / kHZ) % kHY, h2 = h % kHZ;
    const int c0 = o0 + h0 - 1, c1 = o1 + h1 - 1, c2 = o2 + h2 - 1;
    int n = 0, g = 0;
    if (c0 <= G.nc[0] && c1 <= G.nc[1] && c2 <= G.nc[2]) {
      int g0, g1, g2;
      md_wrap(c0, G.nc[0], g0);
      md_wrap(c1, G.nc[1], g1);
      md_wrap(c2, G.nc[2], g2);
      g = (g0 * G.nc[1] + g1) * G.nc[2] + g2;
      n = min(cellcnt[g], kMdCap);
    }
    s_cnt[h] = n;
    s_gcell[h] = g;
  }
  __syncthreads();
  // 2. warp 0: exclusive sums over the halo cells (9 per lane) and over the interior cells (3 per lane)
  static_assert(kHaloCells == 9 * 32 && kBrickCells == 3 * 32, "the scans map 9 and 3 cells onto each lane");
  if (tid < 32) {
    int a[9], tot = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int h = 9 * lane + k;
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
    for (int k = 0; k < 9; ++k) {
      const int h = 9 * lane + k;
      if (h < kHaloCells) s_start[h] = run;
      run += a[k];
    }
    if (lane == 31) s_total = inc;
    int b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int q = 3 * lane + k, q0 = q / (kBY * kBZ), q1 = (q / kBZ) % kBY, q2 = q % kBZ;
      const bool in = o0 + q0 < G.nc[0] && o1 + q1 < G.nc[1] && o2 + q2 < G.nc[2];
      b[k] = in ? s_cnt[((q0 + 1) * kHY + q1 + 1) * kHZ + q2 + 1] : 0;
    }
    const int t2 = b[0] + b[1] + b[2];
    int inc2 = t2;
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc2, off);
      if (lane >= off) inc2 += v;
    }
    s_ipre[3 * lane] = inc2 - t2;
    s_ipre[3 * lane + 1] = inc2 - t2 + b[0];
    s_ipre[3 * lane + 2] = inc2 - t2 + b[0] + b[1];
    if (lane == 31) s_ipre[kBrickCells] = inc2;
  }
  __syncthreads();
  // 3. stage the records, one thread per halo cell (its first four records loaded together)
  const int total = s_total;
  const bool staged = total <= kStageCap;
  if (staged) {
    for (int h = tid; h < kHaloCells; h += kSearchThreads) {
      const int n = s_cnt[h];
      if (n == 0) continue;
      const int h0 = h / (kHY * kHZ), h1 = (h / kHZ) % kHY, h2 = h % kHZ;
      const float3 B = md_cart(G, (float)(h0 - 1), (float)(h1 - 1), (float)(h2 - 1));
      const float4 *src = cellx + (size_t)s_gcell[h] * kMdCap;
      const int t0 = s_start[h];
      float4 r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < n) r[q] = src[q];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < n) {
          s_sx[t0 + q] = B.x + r[q].x;
          s_sy[t0 + q] = B.y + r[q].y;
          s_sz[t0 + q] = B.z + r[q].z;
          s_sj[t0 + q] = __float_as_int(r[q].w);
          s_h[t0 + q] = (unsigned short)h;
        }
      for (int q = 4; q < n; ++q) {
        const float4 v = src[q];
        s_sx[t0 + q] = B.x + v.x;
        s_sy[t0 + q] = B.y + v.y;
        s_sz[t0 + q] = B.z + v.z;
        s_sj[t0 + q] = __float_as_int(v.w);
        s_h[t0 + q] = (unsigned short)h;
      }
    }
  }
  __syncthreads();
  // 4. one thread per atom of the brick
  const int A = s_ipre[kBrickCells];
  for (int a = tid; a < A; a += kSearchThreads) {
    int k = 0;                                     // interior cell of atom a
    for (int step = 64; step > 0; step >>= 1)
      if (k + step < kBrickCells && s_ipre[k + step] <= a) k += step;
    const int k0 = k / (kBY * kBZ), k1 = (k / kBZ) % kBY, k2 = k % kBZ;
    const int hi = ((k0 + 1) * kHY + k1 + 1) * kHZ + k2 + 1;
    const int own = a - s_ipre[k];
    if (!staged) {
      const int i = __float_as_int(cellx[(size_t)s_gcell[hi] * kMdCap + own].w) & 0x7fffffff;
      md_search_atom(N, M, i, pos, G, x4, m4, cellcnt, cellx, cnt, keys, nbr, shift, status);
      continue;
    }
    const int slot = s_start[hi] + own;
    const float4 ei = make_float4(s_sx[slot], s_sy[slot], s_sz[slot], 0.f);
    const int itag = s_sj[slot], i = itag & 0x7fffffff;
    // the scan keeps only the stage positions of the candidates within the band's upper edge (atom i's
    // own record among them), so that the lanes of a warp that find one do little work. It takes the
    // records two at a time (aligned pairs of the stage, in packed FP32), masking the pair members
    // outside the row's run; r^2 is the same as one at a time
    const float2 nx = make_float2(-ei.x, -ei.x), ny = make_float2(-ei.y, -ei.y), nz = make_float2(-ei.z, -ei.z);
    const float2 *sx2 = reinterpret_cast<const float2 *>(s_sx), *sy2 = reinterpret_cast<const float2 *>(s_sy),
                 *sz2 = reinterpret_cast<const float2 *>(s_sz);
    int nc = 0;
#pragma unroll 1
    for (int ab = 0; ab < 9; ++ab) {
      const int ra = ab / 3, rb = ab - 3 * ra;
      const int hc = hi + ((ra - 1) * kHY + (rb - 1)) * kHZ;   // the row's middle cell
      const int p0 = s_start[hc - 1], pend = s_start[hc + 1] + s_cnt[hc + 1];
      for (int k2 = p0 >> 1; 2 * k2 < pend; ++k2) {
        const float2 dx = __fadd2_rn(sx2[k2], nx), dy = __fadd2_rn(sy2[k2], ny), dz = __fadd2_rn(sz2[k2], nz);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const int p = 2 * k2;
        // appended without branches: each record's position is written at the next free slot (a spare
        // slot once the list is full) and the count advances only for a candidate, so the lanes of a
        // warp never diverge here
        const int c0 = (p >= p0 && r2.x <= G.cut2_hi) ? 1 : 0;
        s_cand[min(nc, kCandCap) * kSearchThreads + tid] = (unsigned short)p;
        nc += c0;
        const int c1 = (p + 1 < pend && r2.y <= G.cut2_hi) ? 1 : 0;
        s_cand[min(nc, kCandCap) * kSearchThreads + tid] = (unsigned short)(p + 1);
        nc += c1;
      }
    }
    if (nc > kCandCap) {
      md_search_atom(N, M, i, pos, G, x4, m4, cellcnt, cellx, cnt, keys, nbr, shift, status);
      continue;
    }
    // members among the candidates: the FP32 distance decides below the band, the exact test in it
    const int4 mi = itag < 0 ? m4[i] : make_int4(0, 0, 0, 0);
    const int c0 = o0 + k0, c1 = o1 + k1, c2 = o2 + k2;
    unsigned kk[kMdMaxM];
#pragma unroll
    for (int u = 0; u < kMdMaxM; ++u) kk[u] = 0xffffffffu;
    int count = 0;
    for (int u = 0; u < nc; ++u) {
      const int p = s_cand[u * kSearchThreads + tid];
      if (p == slot) continue;
      const float dx = __fsub_rn(s_sx[p], ei.x), dy = __fsub_rn(s_sy[p], ei.y), dz = __fsub_rn(s_sz[p], ei.z);
      const int jtag = s_sj[p], j = jtag & 0x7fffffff, hj = s_h[p];
      const int d0 = hj / (kHY * kHZ) - (k0 + 1), d1 = (hj / kHZ) % kHY - (k1 + 1), d2 = hj % kHZ - (k2 + 1);
      const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
      bool in = r2 < G.cut2_lo;
      if (!in) {   // in the rounding band: the exact test, with the neighbouring cell's periodic wrap
        int g;
        const int w0 = md_wrap(c0 + d0, G.nc[0], g), w1 = md_wrap(c1 + d1, G.nc[1], g),
                  w2 = md_wrap(c2 + d2, G.nc[2], g);
        in = md_pair_in(G, pos, m4, i, j, mi, w0, w1, w2, make_float3(dx, dy, dz));
      }
      if (in) {
        const unsigned key = ((unsigned)j << 6) | (unsigned)(((d0 + 1) << 4) | ((d1 + 1) << 2) | (d2 + 1)) |
                             ((unsigned)jtag & 0x80000000u);
#pragma unroll
        for (int v = 0; v < kMdMaxM; ++v)
          if (v == count) kk[v] = key;
        ++count;
      }
    }
    if (count > kMdMaxM) {
      md_search_atom(N, M, i, pos, G, x4, m4, cellcnt, cellx, cnt, keys, nbr, shift, status);
      continue;
    }
    md_emit(N, M, i, mi, c0, c1, c2, G, m4, kk, count, cnt, keys, nbr, shift, status);
  }
}

// Passes 1-2 of one atom per thread, M = the warp's largest neighbour count; bonds e >= m of this
// thread are phantoms (f_C = f_C' = 0, unit vector 0), which contribute exactly zero.
template <int M, typename R>
__device__ __forceinline__ void md_atom(const R (&ux)[M], const R (&uy)[M], const R (&uz)[M], const R (&r)[M],
                                        const R (&ir)[M], const R (&fc)[M], const R (&fcp)[M],
                                        const PConsts<R> &K, R &U, R (&Wv)[6], R (&Px)[M], R (&Py)[M],
                                        R (&Pz)[M]) {
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
// quantity k >= 1 to out_rest[k - 1]. The group sums follow the partials; the counters [ngroups + 1]
// are zeroed before the launch. The threads that wrote the block's partials have fenced before the call.
constexpr int kMdGroup = 64;
template <int K>
__device__ __forceinline__ void md_grouped_sum(double *partial, unsigned *counter, int nblk, int b, double *out0,
                                               double *out_rest, double (*red)[7]) {
  __shared__ int s_last;
  const int tid = threadIdx.x, ngroups = (nblk + kMdGroup - 1) / kMdGroup;
  double *gpart = partial + (size_t)K * nblk;
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

// Slot of the reverse entry of key (j << 6 | offset code) of atom i: rank * N + j, the rank of
// (i, -o) among j's keys being its place in j's sorted list; -1 when j's list is not handled (more
// than kMdMaxM entries: flagged by the force kernel) or does not hold it (a truncated list: flagged).
__device__ __forceinline__ int md_reverse_slot(int N, int M, int i, unsigned key, const int *__restrict__ cnt,
                                               const unsigned *__restrict__ keys, unsigned *status) {
  const int j = (int)(key >> 6);
  // the partner's first four keys are loaded beside its count, not after it (entries past the count
  // are ignored below)
  unsigned q[kMdMaxM];
#pragma unroll
  for (int f = 0; f < 4; ++f) q[f] = f < M ? keys[(size_t)f * N + j] : 0xffffffffu;
  const int cj = cnt[j];
  if (cj > kMdMaxM) return -1;
  const int cjm = min(cj, M);
#pragma unroll
  for (int f = 4; f < kMdMaxM; ++f) q[f] = f < cjm ? keys[(size_t)f * N + j] : 0xffffffffu;
  const unsigned want = ((unsigned)i << 6) | (kOffNeg - (key & 63u));
  int rank = 0;
  bool found = false;
#pragma unroll
  for (int f = 0; f < kMdMaxM; ++f)
    if (f < cjm) {
      rank += q[f] < want ? 1 : 0;
      found = found || q[f] == want;
    }
  if (!found) {
    set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
    return -1;
  }
  return rank * N + j;
}

// Passes 1-2 of atom i (m entries) with arrays for M >= m bonds (Mw = the warp's largest count): the
// bond geometry (FP32: the search's separation; FP64: the exact FP64 bond vector), md_atom, and the
// P_ij of every entry: summed over the entries in order into Fo (atom i's own part of F_i), and stored
// at the reverse entry's slot (rank, j) of Prev, so that the gather reads atom i's rows in order.
template <int Mw, typename R>
__device__ __forceinline__ void md_force_atom(int N, int M, int i, int m, const MdGeom &G, const PConsts<R> &K,
                                              const double *__restrict__ pos, const float4 *__restrict__ x4,
                                              const unsigned *__restrict__ keys, const int *__restrict__ cnt,
                                              const int *__restrict__ nbr, const char4 *__restrict__ shift,
                                              float4 xi, typename Vec4<R>::T *__restrict__ Prev,
                                              unsigned *status, R &U, R (&Wv)[6], R (&Fo)[3]) {
  using R4 = typename Vec4<R>::T;
  constexpr int M_ = Mw;
  R ux[M_], uy[M_], uz[M_], r[M_], ir[M_], fc[M_], fcp[M_];
  int rs[M_];
#pragma unroll
  for (int e = 0; e < M_; ++e) {
    ux[e] = R(0); uy[e] = R(0); uz[e] = R(0); r[e] = R(1); ir[e] = R(0); fc[e] = R(0); fcp[e] = R(0);
    rs[e] = -1;
    if (e < m) {
      R dx, dy, dz;
      const unsigned key = keys[(size_t)e * N + i];
      rs[e] = md_reverse_slot(N, M, i, key, cnt, keys, status);
      if constexpr (sizeof(R) == 4) {
        // the search's FP32 separation: neighbouring-cell offset and in-cell positions
        const float3 d = md_sep(G, key & 63u, xi, x4[key >> 6]);
        dx = d.x;
        dy = d.y;
        dz = d.z;
      } else {
        const int j = nbr[(size_t)e * N + i];
        const char4 n = shift[(size_t)e * N + i];
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
  R Px[M_], Py[M_], Pz[M_];
  md_atom<M_, R>(ux, uy, uz, r, ir, fc, fcp, K, U, Wv, Px, Py, Pz);
#pragma unroll
  for (int e = 0; e < M_; ++e)
    if (e < m) {
      Fo[0] += Px[e];
      Fo[1] += Py[e];
      Fo[2] += Pz[e];
      if (rs[e] >= 0) {
        R4 v;
        v.x = Px[e];
        v.y = Py[e];
        v.z = Pz[e];
        v.w = R(0);
        Prev[rs[e]] = v;
      }
    }
}

// The same for the long lists (5-8 entries) as a called function: its many live values do not raise
// the register count of the kernel, which the short lists of solids need.
template <typename R>
struct MdSums {
  R U, W[6], F[3];
};
template <int Mw, typename R>
__device__ __noinline__ MdSums<R> md_force_atom_long(int N, int M, int i, int m, const MdGeom &G,
                                                     const PConsts<R> &K, const double *__restrict__ pos,
                                                     const float4 *__restrict__ x4, const unsigned *__restrict__ keys,
                                                     const int *__restrict__ cnt, const int *__restrict__ nbr,
                                                     const char4 *__restrict__ shift, float4 xi,
                                                     typename Vec4<R>::T *__restrict__ Prev, unsigned *status) {
  MdSums<R> o;
  o.U = R(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) o.W[k] = R(0);
  o.F[0] = o.F[1] = o.F[2] = R(0);
  md_force_atom<Mw, R>(N, M, i, m, G, K, pos, x4, keys, cnt, nbr, shift, xi, Prev, status, o.U, o.W, o.F);
  return o;
}

template <typename R>
__global__ void __launch_bounds__(kMdThreads, sizeof(R) == 4 ? 8 : 1) md_force_kernel(
    int N, int M, const MdGeom G, const PConsts<R> K, const double *__restrict__ pos,
    const float4 *__restrict__ x4, const unsigned *__restrict__ keys, const int *__restrict__ cnt,
    const int *__restrict__ nbr, const char4 *__restrict__ shift, typename Vec4<R>::T *__restrict__ Fown,
    typename Vec4<R>::T *__restrict__ Prev, double *__restrict__ partial, unsigned *counters, double *__restrict__ E,
    double *__restrict__ W, unsigned *status) {
  __shared__ double red[kMdThreads / 32][7];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < N;
  int m = valid ? min(cnt[i], M) : 0;   // a truncated list (count > M) is flagged; its row holds M entries
  if (m > kMdMaxM) {
    set_status(status, TERSOFF_STATUS_MANY_NBRS);
    m = 0;
  }
  float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
  if (sizeof(R) == 4 && valid) xi = x4[i];
  R U = R(0), Wv[6] = {R(0), R(0), R(0), R(0), R(0), R(0)}, Fo[3] = {R(0), R(0), R(0)};
  // arrays sized by the warp's largest neighbour count, so that the common short lists keep few
  // values live
  const int Mw = __reduce_max_sync(0xffffffffu, (unsigned)m);
  switch (Mw) {
#define TSF_MDCASE(MM) \
    case MM: md_force_atom<MM, R>(N, M, i, m, G, K, pos, x4, keys, cnt, nbr, shift, xi, Prev, status, U, Wv, Fo); break;
#define TSF_MDLONG(MM)                                                                      \
    case MM: {                                                                              \
      const MdSums<R> o = md_force_atom_long<MM, R>(N, M, i, m, G, K, pos, x4, keys, cnt, nbr, shift, xi, Prev, status); \
      U = o.U;                                                                              \
      for (int k = 0; k < 6; ++k) Wv[k] = o.W[k];                                           \
      for (int k = 0; k < 3; ++k) Fo[k] = o.F[k];                                           \
      break;                                                                                \
    }
    TSF_MDCASE(1) TSF_MDCASE(2) TSF_MDCASE(3) TSF_MDCASE(4) TSF_MDLONG(5) TSF_MDLONG(6) TSF_MDLONG(7)
    TSF_MDLONG(8)
#undef TSF_MDCASE
#undef TSF_MDLONG
    default: break;
  }
  if (valid) {
    typename Vec4<R>::T f;
    f.x = Fo[0];
    f.y = Fo[1];
    f.z = Fo[2];
    f.w = R(0);
    Fown[i] = f;
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
  md_grouped_sum<7>(partial, counters, nblk, b, E, W, red);
}

// F_i = sum_e P_ij - sum_e P_ji over atom i's entries e = (j, n): the first sum from Fown (the force
// kernel's), P_ji from Prev row e (written there by atom j). An atom with more than kMdMaxM entries
// has no P (the force kernel flags it) and gets F = 0.
template <typename R>
__global__ void md_gather_kernel(int N, int M, const int *__restrict__ cnt, const typename Vec4<R>::T *__restrict__ Fown,
                                 const typename Vec4<R>::T *__restrict__ Prev, R *__restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int ci = cnt[i];
  const int m = ci <= kMdMaxM ? min(ci, M) : 0;
  const auto f = Fown[i];
  R Fx = f.x, Fy = f.y, Fz = f.z;
#pragma unroll
  for (int e = 0; e < kMdMaxM; ++e)
    if (e < m) {
      const auto b = Prev[(size_t)e * N + i];
      Fx -= b.x;
      Fy -= b.y;
      Fz -= b.z;
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
  // FP32 distance error: the in-cell positions X (at most the sum of the cell edges in size) and the
  // offset o E, each rounded, then subtracted and added, stay within ~12 ulp of the cell edge
  // lengths; the band is 128 ulp wide
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
  if (c.md_cellcnt.ensure((ncells + ngroups + 1) * sizeof(int)) || c.md_cells.ensure(ncells * kMdCap * sizeof(float4)) ||
      c.md_pos.ensure((size_t)N * (sizeof(float4) + sizeof(int4))) || c.md_cnt.ensure((size_t)N * sizeof(int)) ||
      c.md_nbr.ensure((size_t)N * M * sizeof(int)) || c.md_shift.ensure((size_t)N * M * sizeof(char4)) ||
      c.md_keys.ensure((size_t)N * M * sizeof(unsigned)) || c.md_Pij.ensure((size_t)N * (kMdMaxM + 1) * 4 * rs) ||
      c.md_red.ensure(md_sum_bytes(7, nblk))) {
    err = "device allocation failed";
    return TERSOFF_E_CUDA;
  }
  c.md_N = N;
  c.md_M = M;
  float4 *x4 = reinterpret_cast<float4 *>(c.md_pos.p);
  int4 *m4 = reinterpret_cast<int4 *>(x4 + N);
  unsigned *st = c.status.as<unsigned>();
  int *cnt = c.md_cnt.as<int>();
  unsigned *keys = c.md_keys.as<unsigned>();
  // cell counts and the force kernel's sum counters, both zero at the start of the call: one memset
  unsigned *sum_counters = c.md_cellcnt.as<unsigned>() + ncells;
  cudaMemsetAsync(c.md_cellcnt.p, 0, (ncells + ngroups + 1) * sizeof(int), s);
  md_cells_kernel<<<nblk, kMdThreads, 0, s>>>(N, pos, G, c.md_cellcnt.as<int>(), c.md_cells.as<float4>(), x4, m4,
                                              cnt, st);
  const long nbricks = (long)((G.nc[0] + kBX - 1) / kBX) * ((G.nc[1] + kBY - 1) / kBY) * ((G.nc[2] + kBZ - 1) / kBZ);
  md_search_kernel<<<(unsigned)nbricks, kSearchThreads, 0, s>>>(N, M, pos, G, x4, m4, c.md_cellcnt.as<int>(), c.md_cells.as<float4>(),
                                               cnt, keys, c.md_nbr.as<int>(), c.md_shift.as<char4>(), st);
  const double D0 = x[0], al = x[1], r0 = x[2], be = x[3], n = x[4], h = x[5];
  const double log2e = 1.4426950408889634;
  if (precision == 64) {
    PConsts<double> K{D0, -al * log2e, r0, -0.5 * al, be, h, n, -0.5 / n};
    dvec4 *Fown = c.md_Pij.as<dvec4>(), *Prev = Fown + N;
    md_force_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, M, G, K, pos, x4, keys, cnt, c.md_nbr.as<int>(),
                                                        c.md_shift.as<char4>(), Fown, Prev, c.md_red.as<double>(), sum_counters,
                                                        E, W, st);
    md_gather_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, M, cnt, Fown, Prev, reinterpret_cast<double *>(F));
  } else {
    PConsts<float> K{(float)D0, (float)(-al * log2e), (float)r0, (float)(-0.5 * al), (float)be, (float)h,
                     (float)n, (float)(-0.5 / n)};
    float4 *Fown = c.md_Pij.as<float4>(), *Prev = Fown + N;
    md_force_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, M, G, K, pos, x4, keys, cnt, c.md_nbr.as<int>(),
                                                       c.md_shift.as<char4>(), Fown, Prev, c.md_red.as<double>(), sum_counters,
                                                       E, W, st);
    md_gather_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, M, cnt, Fown, Prev, reinterpret_cast<float *>(F));
  }
  cudaError_t e = launched(4);   // cells, search, force (with the sums), gather
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
                                                             double *__restrict__ partial, unsigned *counters,
                                                             double *__restrict__ Ekin) {
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
  md_grouped_sum<1>(partial, counters, gridDim.x, blockIdx.x, Ekin, nullptr, red);
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
  unsigned *counters = reinterpret_cast<unsigned *>(static_cast<char *>(c.md_ke.p) + md_counter_offset(1, nblk));
  double *acc = reinterpret_cast<double *>(static_cast<char *>(c.md_ke.p) + sum_bytes);
  md_accel_kernel<<<nblk, kMdThreads, 0, s>>>(N, mass, acc);
  auto kick = [&](double h, int step) {
    cudaMemsetAsync(counters, 0, (ngroups + 1) * sizeof(unsigned), s);
    if (precision == 64)
      md_kick_kernel<double><<<nblk, kMdThreads, 0, s>>>(N, vel, static_cast<const double *>(F), mass, acc, h, part,
                                                         counters, Ekin + step);
    else
      md_kick_kernel<float><<<nblk, kMdThreads, 0, s>>>(N, vel, static_cast<const float *>(F), mass, acc, h, part,
                                                        counters, Ekin + step);
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
