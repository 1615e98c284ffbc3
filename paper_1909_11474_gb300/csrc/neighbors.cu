// neighbors.cu -- neighbour build and parameter-independent geometry cache for batches of small
// periodic cells (the index sets of the sums over j in Eq. 2 and over k in Eq. 7 of
// arXiv:1909.11474, and the cutoff function f_C of Eq. 9).
#include <math.h>

#include "common.cuh"
#include "ctx.hpp"

namespace tsf {

// Per configuration: the inverse box (fractional coordinates s = x H^-1, rows of H = lattice
// vectors) and the three lattice-plane spacings, boxinv[c][0..11] = {Hinv (row-major), gap}, and the
// FP32 constants of the neighbour search, pre32[c][0..23] = {Hinv, R2/gap + margin, H, band}:
// a candidate whose FP32 squared distance is farther than `band` from R2^2 is decided in FP32, the
// rest by the exact FP64 test. `band` bounds the FP32 error of the squared distance: with X the
// largest coordinate magnitude of the configuration, |H| its largest box entry and nmax the largest
// image index a candidate can have, each FP32 component of d = (x_j - x_i) + n.H is within
// delta = 2^-23 (4X + 6 nmax |H|) of the exact value, so |r^2 - r32^2| < 3.5 R2 delta + 12 2^-24 R2^2;
// the band is four times that.
__global__ void box_prep_kernel(int C, const double *__restrict__ box, const float *__restrict__ xmax,
                                double *__restrict__ boxinv, float *__restrict__ pre32, double R2,
                                unsigned *status) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const double *H = box + 9 * c;
  double a0 = H[0], a1 = H[1], a2 = H[2], b0 = H[3], b1 = H[4], b2 = H[5], c0 = H[6], c1 = H[7],
         c2 = H[8];
  // cofactors
  double bxc0 = b1 * c2 - b2 * c1, bxc1 = b2 * c0 - b0 * c2, bxc2 = b0 * c1 - b1 * c0;
  double cxa0 = c1 * a2 - c2 * a1, cxa1 = c2 * a0 - c0 * a2, cxa2 = c0 * a1 - c1 * a0;
  double axb0 = a1 * b2 - a2 * b1, axb1 = a2 * b0 - a0 * b2, axb2 = a0 * b1 - a1 * b0;
  double det = a0 * bxc0 + a1 * bxc1 + a2 * bxc2;
  double *o = boxinv + 12 * c;
  float *f = pre32 + 24 * c;
  bool ok = isfinite(det) && det != 0.0;
  for (int k = 0; k < 9; ++k) ok = ok && isfinite(H[k]);
  if (!ok) {
    set_status(status, TERSOFF_STATUS_NONFINITE);
    for (int k = 0; k < 12; ++k) o[k] = 0.0;
    for (int k = 0; k < 24; ++k) f[k] = 0.f;
    return;
  }
  double id = 1.0 / det;
  // H^-1 columns are (b x c, c x a, a x b) / det, i.e. Hinv[mu][k] = cross_k[mu] / det
  o[0] = bxc0 * id; o[1] = cxa0 * id; o[2] = axb0 * id;
  o[3] = bxc1 * id; o[4] = cxa1 * id; o[5] = axb1 * id;
  o[6] = bxc2 * id; o[7] = cxa2 * id; o[8] = axb2 * id;
  double vol = fabs(det);
  o[9] = vol / sqrt(bxc0 * bxc0 + bxc1 * bxc1 + bxc2 * bxc2);
  o[10] = vol / sqrt(cxa0 * cxa0 + cxa1 * cxa1 + cxa2 * cxa2);
  o[11] = vol / sqrt(axb0 * axb0 + axb1 * axb1 + axb2 * axb2);
  // largest coordinate magnitude (from the FP32 copies: widened by 2^-22 for their rounding)
  const double X = (double)xmax[c] * (1.0 + ldexp(1.0, -22));
  double Hm = 0.0;
  for (int k = 0; k < 9; ++k) Hm = fmax(Hm, fabs(H[k]));
  double nmax = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double col = fabs(o[k]) + fabs(o[3 + k]) + fabs(o[6 + k]);
    nmax = fmax(nmax, ceil(2.0 * X * col + R2 / o[9 + k] + 1.0));
  }
  const double delta = ldexp(4.0 * X + 6.0 * nmax * Hm, -23);
  const double band = 4.0 * (3.5 * R2 * delta + 12.0 * ldexp(R2 * R2, -24));
  for (int k = 0; k < 9; ++k) f[k] = (float)o[k];
  for (int k = 0; k < 3; ++k) f[9 + k] = (float)(R2 / o[9 + k]) + 1e-4f;
  for (int k = 0; k < 9; ++k) f[12 + k] = (float)H[k];
  f[21] = (float)band;
  f[22] = (float)(R2 * R2);
  f[23] = 0.f;
}

// FP32 copies of the positions and, per configuration, the largest coordinate magnitude (xmax must
// be zero on entry; non-negative floats order like their bit patterns, so an integer max suffices).
__global__ void pos32_kernel(int64_t N, const double *__restrict__ pos, const int *__restrict__ atom_cfg,
                             float4 *__restrict__ pos32, float *__restrict__ xmax, unsigned *status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) set_status(status, TERSOFF_STATUS_NONFINITE);
  const float4 v = make_float4((float)x, (float)y, (float)z, 0.f);
  pos32[i] = v;
  const float m = fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z)));
  atomicMax(reinterpret_cast<int *>(xmax) + atom_cfg[i], __float_as_int(m));
}

// Candidate image range of one (i, j) pair on one axis: integers n with |s_j - s_i + n| < rng.
__device__ __forceinline__ void image_range(float ds, float rng, int &lo, int &hi) {
  lo = (int)ceilf(-ds - rng);
  hi = (int)floorf(-ds + rng);
}

// One warp per atom i; lane l tests atoms j = a0 + l, a0 + 32 + l, ... of the same configuration.
// Candidate images are the integers n_k with |s_j - s_i + n_k| < R2 / gap_k (+ margin), found in FP32
// fractional coordinates. Each candidate's squared distance is computed in FP32; outside the rounding
// band around R2^2 that decides it, inside the band the exact FP64 test does, so the result equals the
// exact FP64 test everywhere. The warp runs each block of 32 j twice: first every lane counts its
// accepted entries, then an exclusive warp scan gives each lane its output position, so entries land
// in ascending (j, n0, n1, n2) order.
struct Pre32 {
  float Hi[9], rng[3], H[9], band, R2sq;
};
__device__ __forceinline__ bool member(const Pre32 &q, float dx, float dy, float dz, int n0, int n1, int n2,
                                       const double *xj, const double *xi, const double *H, double R2sq) {
  const float tx = (n0 * q.H[0] + n1 * q.H[3]) + n2 * q.H[6];
  const float ty = (n0 * q.H[1] + n1 * q.H[4]) + n2 * q.H[7];
  const float tz = (n0 * q.H[2] + n1 * q.H[5]) + n2 * q.H[8];
  const float ex = dx + tx, ey = dy + ty, ez = dz + tz;
  const float r2 = ex * ex + ey * ey + ez * ez;
  if (r2 < q.R2sq - q.band) return true;
  if (r2 > q.R2sq + q.band) return false;
  return exact_pair(xj[0], xj[1], xj[2], xi[0], xi[1], xi[2], H, n0, n1, n2).r2 < R2sq;
}

__global__ void __launch_bounds__(128) neighbors_batch_kernel(
    int64_t Ntot, const int *__restrict__ atom_off, const int *__restrict__ atom_cfg,
    const double *__restrict__ pos, const float4 *__restrict__ pos32,
    const double *__restrict__ box, const float *__restrict__ pre32, double R2, int M,
    int *__restrict__ cnt_out, int *__restrict__ nbr, char4 *__restrict__ shift, unsigned *status) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= Ntot) return;   // whole warps only
  const int c = atom_cfg[i];
  const int a0 = atom_off[c], a1 = atom_off[c + 1];
  Pre32 q;
  {
    const float *f = pre32 + 24 * c;
#pragma unroll
    for (int k = 0; k < 9; ++k) q.Hi[k] = f[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) q.rng[k] = f[9 + k];
#pragma unroll
    for (int k = 0; k < 9; ++k) q.H[k] = f[12 + k];
    q.band = f[21];
    q.R2sq = f[22];
  }
  const double *H = box + 9 * c;
  const double R2sq = R2 * R2;
  const double *xi = pos + 3 * i;
  const float4 xi32 = pos32[i];
  int count = 0;
  for (int jb = a0; jb < a1; jb += 32) {
    const int j = jb + lane;
    int lo0 = 1, hi0 = 0, lo1 = 1, hi1 = 0, lo2 = 1, hi2 = 0;
    float dx = 0.f, dy = 0.f, dz = 0.f;
    if (j < a1) {
      const float4 xj = pos32[j];
      dx = xj.x - xi32.x;
      dy = xj.y - xi32.y;
      dz = xj.z - xi32.z;
      image_range(dx * q.Hi[0] + dy * q.Hi[3] + dz * q.Hi[6], q.rng[0], lo0, hi0);
      image_range(dx * q.Hi[1] + dy * q.Hi[4] + dz * q.Hi[7], q.rng[1], lo1, hi1);
      image_range(dx * q.Hi[2] + dy * q.Hi[5] + dz * q.Hi[8], q.rng[2], lo2, hi2);
    }
    const double *xj = pos + 3 * (j < a1 ? j : a0);
    int mine = 0;
    for (int n0 = lo0; n0 <= hi0; ++n0)
      for (int n1 = lo1; n1 <= hi1; ++n1)
        for (int n2 = lo2; n2 <= hi2; ++n2) {
          if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
          if (member(q, dx, dy, dz, n0, n1, n2, xj, xi, H, R2sq)) ++mine;
        }
    int incl = mine;   // inclusive warp scan of the per-lane counts
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (mine) {
      int w = count + incl - mine;
      for (int n0 = lo0; n0 <= hi0; ++n0)
        for (int n1 = lo1; n1 <= hi1; ++n1)
          for (int n2 = lo2; n2 <= hi2; ++n2) {
            if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
            if (member(q, dx, dy, dz, n0, n1, n2, xj, xi, H, R2sq)) {
              if (w < M) {
                nbr[i * M + w] = j;
                shift[i * M + w] = make_char4((signed char)n0, (signed char)n1, (signed char)n2, 0);
              }
              ++w;
            }
          }
    }
    count += total;
  }
  if (lane == 0) {
    cnt_out[i] = count;
    if (count > M) set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
  }
  for (int e = count + lane; e < M; e += 32) {
    nbr[i * M + e] = -1;
    shift[i * M + e] = make_char4(0, 0, 0, 0);
  }
}

// Reverse entry of every bond: entry (i; j, n) <-> (j; i, -n). The exact test is antisymmetric
// (x_i - x_j = -(x_j - x_i) and t(-n) = -t(n) exactly), so the reverse entry always exists.
// One thread per (atom, list slot).
__global__ void reverse_kernel(int64_t Ntot, int M, const int *__restrict__ cnt,
                               const int *__restrict__ nbr, const char4 *__restrict__ shift,
                               const int *__restrict__ boff, int *__restrict__ brev,
                               unsigned *status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / M;
  const int e = (int)(t % M);
  if (i >= Ntot) return;
  const int m = min(cnt[i], M);
  if (e >= m) return;
  const int j = nbr[i * M + e];
  const char4 n = shift[i * M + e];
  const int mj = min(cnt[j], M);
  int found = -1;
  for (int f = 0; f < mj; ++f) {
    const char4 q = shift[(int64_t)j * M + f];
    if (nbr[(int64_t)j * M + f] == (int)i && q.x == -n.x && q.y == -n.y && q.z == -n.z) {
      found = f;
      break;
    }
  }
  if (found < 0) {
    set_status(status, TERSOFF_STATUS_NBR_OVERFLOW);
    found = 0;
  }
  brev[boff[i] + e] = boff[j] + found;
}

// f_C of Eq. 9 and its derivative.
__device__ __forceinline__ void cutoff_fc(double r, double R1, double R2, double &fc, double &fcp) {
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

// Owner atom of bond b: the last atom i with boff[i] <= b (atoms without bonds are skipped).
__device__ __forceinline__ int64_t bond_owner(const int *__restrict__ boff, int64_t Ntot, int b) {
  int64_t lo = 0, hi = Ntot;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (boff[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Per bond: unit vector, r, 2/r, f_C, f_C' and, packed into one int (rev | j << 16), the
// configuration-local indices of the reverse bond and of the neighbour atom (4th slot: as a double,
// or as the bit pattern of the int in the FP32 record). The bond vector d is formed in FP64 by the
// expression of the membership test (where the cancellation happens); FP32 records round it and then
// normalise in FP32, FP64 records (built on the first FP64 evaluation) stay in FP64. One thread per bond.
template <typename R>
__global__ void geometry_bond_kernel(int64_t Ntot, int Btot, int M, const int *__restrict__ atom_cfg,
                                     const int *__restrict__ atom_off, const int *__restrict__ brev,
                                     const double *__restrict__ pos, const double *__restrict__ box,
                                     const int *__restrict__ nbr, const char4 *__restrict__ shift,
                                     const int *__restrict__ boff, double R1, double R2,
                                     typename Vec4<R>::T *__restrict__ gA, typename Vec4<R>::T *__restrict__ gB,
                                     int *__restrict__ outer) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Btot) return;
  const int64_t i = bond_owner(boff, Ntot, b);
  const int e = b - boff[i];
  const int c = atom_cfg[i];
  const double *H = box + 9 * c;
  const int cb0 = boff[atom_off[c]];   // first bond of the configuration
  const int j = nbr[i * M + e];
  // packed: configuration-local index of the reverse bond (bits 0-15) and of atom j (bits 16-31)
  const int rl = (brev[b] - cb0) | ((j - atom_off[c]) << 16);
  const char4 n = shift[i * M + e];
  const ExactPair p = exact_pair(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], pos[3 * i], pos[3 * i + 1],
                                 pos[3 * i + 2], H, n.x, n.y, n.z);
  typename Vec4<R>::T A, Bv;
  if constexpr (sizeof(R) == 4) {
    const float dx = (float)p.dx, dy = (float)p.dy, dz = (float)p.dz;
    const float ir = rsqrtf(dx * dx + dy * dy + dz * dz);
    const float r = (dx * dx + dy * dy + dz * dz) * ir;
    float fc = 1.f, fcp = 0.f;
    if (r > (float)R1) atomicOr(outer + i, 1);   // the atom has a bond beyond R1 (f_C != 1)
    if (r >= (float)R2) {
      fc = 0.f;
    } else if (r > (float)R1) {
      const float w = (r - (float)R1) / (float)(R2 - R1);
      fc = 0.5f * (1.f + cospif(w));
      fcp = (float)(-0.5 * M_PI / (R2 - R1)) * sinpif(w);
    }
    A = make_float4(dx * ir, dy * ir, dz * ir, r);
    Bv = make_float4(ir + ir, fc, fcp, __int_as_float(rl));
  } else {
    const double ir = rsqrt(p.r2);
    const double r = p.r2 * ir;
    double fc, fcp;
    cutoff_fc(r, R1, R2, fc, fcp);
    A = make_dvec4(p.dx * ir, p.dy * ir, p.dz * ir, r);
    Bv = make_dvec4(ir + ir, fc, fcp, (double)rl);
  }
  gA[b] = A;
  gB[b] = Bv;
}

// Per unordered pair (e < f) of an atom's bonds: cos theta from the unit vectors of the records; each
// atom's row is padded to 4 slots with zeros. One thread per (atom, pair slot).
template <typename R>
__global__ void geometry_pair_kernel(int64_t Ntot, int slots, const int *__restrict__ cnt, int M,
                                     const int *__restrict__ boff, const int *__restrict__ poff,
                                     const typename Vec4<R>::T *__restrict__ gA, R *__restrict__ gcos) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / slots;
  const int q = (int)(t % slots);
  if (i >= Ntot) return;
  const int q0 = poff[i], nslot = poff[i + 1] - q0;
  if (q >= nslot) return;
  const int m = min(cnt[i], M);
  // slot q -> (e, f), e < f, row-major over e
  int e = 0, rem = q;
  while (e < m && rem >= m - 1 - e) {
    rem -= m - 1 - e;
    ++e;
  }
  R cs = R(0);
  if (e < m - 1) {
    const int f = e + 1 + rem;
    const auto ue = gA[boff[i] + e], uf = gA[boff[i] + f];
    cs = ue.x * uf.x + ue.y * uf.y + ue.z * uf.z;
  }
  gcos[q0 + q] = cs;
}

// ---------------------------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_box_prep(int C, const double *box, const float *xmax, double *boxinv, float *pre32,
                            double R2, unsigned *status, cudaStream_t s) {
  box_prep_kernel<<<nblk(C, 128), 128, 0, s>>>(C, box, xmax, boxinv, pre32, R2, status);
  return launched(1);
}
cudaError_t launch_pos32(int64_t N, const double *pos, float4 *pos32, const int *atom_cfg, float *xmax,
                         unsigned *status, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  pos32_kernel<<<nblk(N, 256), 256, 0, s>>>(N, pos, atom_cfg, pos32, xmax, status);
  return launched(1);
}
cudaError_t launch_neighbors_batch(int64_t Ntot, const int *atom_off, const int *atom_cfg,
                                   const double *pos, const float4 *pos32, const double *box,
                                   const float *pre32, double R2, int M, int *cnt, int *nbr,
                                   char4 *shift, unsigned *status, cudaStream_t s) {
  if (Ntot == 0) return cudaSuccess;
  neighbors_batch_kernel<<<nblk(Ntot * 32, 128), 128, 0, s>>>(Ntot, atom_off, atom_cfg, pos, pos32, box,
                                                              pre32, R2, M, cnt, nbr, shift, status);
  return launched(1);
}
cudaError_t launch_reverse(int64_t Ntot, int M, const int *cnt, const int *nbr, const char4 *shift,
                           const int *boff, int *brev, unsigned *status, cudaStream_t s) {
  if (Ntot == 0) return cudaSuccess;
  reverse_kernel<<<nblk(Ntot * M, 256), 256, 0, s>>>(Ntot, M, cnt, nbr, shift, boff, brev, status);
  return launched(1);
}
cudaError_t launch_geometry(int precision, int64_t Ntot, int64_t Btot, int M, const int *atom_cfg,
                            const int *atom_off, const int *brev, const double *pos, const double *box,
                            const int *cnt, const int *nbr, const char4 *shift, const int *boff,
                            const int *poff, double R1, double R2, void *gA, void *gB, void *gcos,
                            int max_slots, int *outer, cudaStream_t s) {
  if (Ntot == 0) return cudaSuccess;
  if (outer) {
    cudaError_t e = cudaMemsetAsync(outer, 0, Ntot * sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  if (Btot > 0) {
    if (precision == 64)
      geometry_bond_kernel<double><<<nblk(Btot, 256), 256, 0, s>>>(
          Ntot, (int)Btot, M, atom_cfg, atom_off, brev, pos, box, nbr, shift, boff, R1, R2,
          static_cast<dvec4 *>(gA), static_cast<dvec4 *>(gB), nullptr);
    else
      geometry_bond_kernel<float><<<nblk(Btot, 256), 256, 0, s>>>(
          Ntot, (int)Btot, M, atom_cfg, atom_off, brev, pos, box, nbr, shift, boff, R1, R2,
          static_cast<float4 *>(gA), static_cast<float4 *>(gB), outer);
  }
  if (max_slots > 0) {
    if (precision == 64)
      geometry_pair_kernel<double><<<nblk(Ntot * max_slots, 256), 256, 0, s>>>(
          Ntot, max_slots, cnt, M, boff, poff, static_cast<const dvec4 *>(gA), static_cast<double *>(gcos));
    else
      geometry_pair_kernel<float><<<nblk(Ntot * max_slots, 256), 256, 0, s>>>(
          Ntot, max_slots, cnt, M, boff, poff, static_cast<const float4 *>(gA), static_cast<float *>(gcos));
  }
  return launched((Btot > 0) + (max_slots > 0));
}

}  // namespace tsf
