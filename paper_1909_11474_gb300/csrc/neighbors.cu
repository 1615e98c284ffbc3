// neighbors.cu -- neighbour build and parameter-independent geometry cache for batches of small
// periodic cells (the index sets of the sums over j in Eq. 2 and over k in Eq. 7 of
// arXiv:1909.11474, and the cutoff function f_C of Eq. 9).
#include <math.h>

#include "common.cuh"
#include "ctx.hpp"

namespace tsf {

// Per configuration: the inverse box (fractional coordinates s = x H^-1, rows of H = lattice
// vectors) and the three lattice-plane spacings, boxinv[c][0..11] = {Hinv (row-major), gap}, and the
// FP32 constants of the neighbour prefilter, pre32[c][0..11] = {Hinv, R2/gap + margin}.
__global__ void box_prep_kernel(int C, const double *__restrict__ box, double *__restrict__ boxinv,
                                float *__restrict__ pre32, double R2, unsigned *status) {
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
  bool ok = isfinite(det) && det != 0.0;
  for (int k = 0; k < 9; ++k) ok = ok && isfinite(H[k]);
  if (!ok) {
    set_status(status, TERSOFF_STATUS_NONFINITE);
    for (int k = 0; k < 12; ++k) o[k] = 0.0;
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
  float *f = pre32 + 12 * c;
  for (int k = 0; k < 9; ++k) f[k] = (float)o[k];
  for (int k = 0; k < 3; ++k) f[9 + k] = (float)(R2 / o[9 + k]) + 1e-4f;
}

__global__ void pos32_kernel(int64_t N, const double *__restrict__ pos, float4 *__restrict__ pos32,
                             unsigned *status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) set_status(status, TERSOFF_STATUS_NONFINITE);
  pos32[i] = make_float4((float)x, (float)y, (float)z, 0.f);
}

// Candidate image range of one (i, j) pair on one axis: integers n with |s_j - s_i + n| < rng.
__device__ __forceinline__ void image_range(float ds, float rng, int &lo, int &hi) {
  lo = (int)ceilf(-ds - rng);
  hi = (int)floorf(-ds + rng);
}

// One warp per atom i; lane l tests atoms j = a0 + l, a0 + 32 + l, ... of the same configuration.
// Candidate images are the integers n_k with |s_j - s_i + n_k| < R2 / gap_k (+ margin), found in FP32
// fractional coordinates; each candidate is then decided by the exact FP64 test. The warp runs each
// block of 32 j twice: first every lane counts its accepted entries, then an exclusive warp scan
// gives each lane its output position, so entries land in ascending (j, n0, n1, n2) order.
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
  double H[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) H[k] = box[9 * c + k];
  const float *bi = pre32 + 12 * c;   // no FP64 arithmetic per warp: FP32 prefilter constants
  float Hi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Hi[k] = bi[k];
  const float rng0 = bi[9], rng1 = bi[10], rng2 = bi[11];
  const double R2sq = R2 * R2;
  const double xix = pos[3 * i], xiy = pos[3 * i + 1], xiz = pos[3 * i + 2];
  const float4 xi = pos32[i];
  int count = 0;
  for (int jb = a0; jb < a1; jb += 32) {
    const int j = jb + lane;
    int lo0 = 1, hi0 = 0, lo1 = 1, hi1 = 0, lo2 = 1, hi2 = 0;
    double xjx = 0, xjy = 0, xjz = 0;
    if (j < a1) {
      const float4 xj = pos32[j];
      const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
      image_range(dx * Hi[0] + dy * Hi[3] + dz * Hi[6], rng0, lo0, hi0);
      image_range(dx * Hi[1] + dy * Hi[4] + dz * Hi[7], rng1, lo1, hi1);
      image_range(dx * Hi[2] + dy * Hi[5] + dz * Hi[8], rng2, lo2, hi2);
      xjx = pos[3 * j];
      xjy = pos[3 * j + 1];
      xjz = pos[3 * j + 2];
    }
    int mine = 0;
    for (int n0 = lo0; n0 <= hi0; ++n0)
      for (int n1 = lo1; n1 <= hi1; ++n1)
        for (int n2 = lo2; n2 <= hi2; ++n2) {
          if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
          if (exact_pair(xjx, xjy, xjz, xix, xiy, xiz, H, n0, n1, n2).r2 < R2sq) ++mine;
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
            if (exact_pair(xjx, xjy, xjz, xix, xiy, xiz, H, n0, n1, n2).r2 < R2sq) {
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

// Per bond: unit vector, r, 1/r, f_C, f_C' and, packed into one int (rev | j << 16), the
// configuration-local indices of the reverse bond and of the neighbour atom (stored in the 4th slot:
// as a double, or as the bit pattern of the int in the FP32 record). Computed in FP64 from the same
// d as the membership test, stored in FP64 and rounded to FP32. One thread per (atom, list slot).
__global__ void geometry_bond_kernel(int64_t Ntot, int M, const int *__restrict__ atom_cfg,
                                     const int *__restrict__ atom_off, const int *__restrict__ brev,
                                     const double *__restrict__ pos, const double *__restrict__ box,
                                     const int *__restrict__ cnt, const int *__restrict__ nbr,
                                     const char4 *__restrict__ shift, const int *__restrict__ boff,
                                     double R1, double R2, float4 *__restrict__ gA32,
                                     float4 *__restrict__ gB32, dvec4 *__restrict__ gA64,
                                     dvec4 *__restrict__ gB64) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / M;
  const int e = (int)(t % M);
  if (i >= Ntot) return;
  if (e >= min(cnt[i], M)) return;
  const int c = atom_cfg[i];
  double H[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) H[k] = box[9 * c + k];
  const int b = boff[i] + e;
  const int cb0 = boff[atom_off[c]];   // first bond of the configuration
  const int j = nbr[i * M + e];
  // packed: configuration-local index of the reverse bond (bits 0-15) and of atom j (bits 16-31)
  const int rl = (brev[b] - cb0) | ((j - atom_off[c]) << 16);
  const char4 n = shift[i * M + e];
  ExactPair p = exact_pair(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], pos[3 * i], pos[3 * i + 1],
                           pos[3 * i + 2], H, n.x, n.y, n.z);
  const double ir = rsqrt(p.r2);
  const double r = p.r2 * ir;
  double fc, fcp;
  cutoff_fc(r, R1, R2, fc, fcp);
  const double ux = p.dx * ir, uy = p.dy * ir, uz = p.dz * ir;
  gA64[b] = make_dvec4(ux, uy, uz, r);
  gB64[b] = make_dvec4(ir, fc, fcp, (double)rl);
  gA32[b] = make_float4((float)ux, (float)uy, (float)uz, (float)r);
  gB32[b] = make_float4((float)ir, (float)fc, (float)fcp, __int_as_float(rl));
}

// Per unordered pair (e < f) of an atom's bonds: cos theta from the FP64 unit vectors; each atom's
// row is padded to 4 slots with zeros. One thread per (atom, pair slot).
__global__ void geometry_pair_kernel(int64_t Ntot, int slots, const int *__restrict__ cnt, int M,
                                     const int *__restrict__ boff, const int *__restrict__ poff,
                                     const dvec4 *__restrict__ gA64, float *__restrict__ gcos32,
                                     double *__restrict__ gcos64) {
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
  double cs = 0.0;
  if (e < m - 1) {
    const int f = e + 1 + rem;
    const dvec4 ue = gA64[boff[i] + e], uf = gA64[boff[i] + f];
    cs = ue.x * uf.x + ue.y * uf.y + ue.z * uf.z;
  }
  gcos64[q0 + q] = cs;
  gcos32[q0 + q] = (float)cs;
}

// ---------------------------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_box_prep(int C, const double *box, double *boxinv, float *pre32, double R2, unsigned *status,
                            cudaStream_t s) {
  box_prep_kernel<<<nblk(C, 128), 128, 0, s>>>(C, box, boxinv, pre32, R2, status);
  return cudaGetLastError();
}
cudaError_t launch_pos32(int64_t N, const double *pos, float4 *pos32, const int *, unsigned *status,
                         cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  pos32_kernel<<<nblk(N, 256), 256, 0, s>>>(N, pos, pos32, status);
  return cudaGetLastError();
}
cudaError_t launch_neighbors_batch(int64_t Ntot, const int *atom_off, const int *atom_cfg,
                                   const double *pos, const float4 *pos32, const double *box,
                                   const float *pre32, double R2, int M, int *cnt, int *nbr,
                                   char4 *shift, unsigned *status, cudaStream_t s) {
  if (Ntot == 0) return cudaSuccess;
  neighbors_batch_kernel<<<nblk(Ntot * 32, 128), 128, 0, s>>>(Ntot, atom_off, atom_cfg, pos, pos32, box,
                                                              pre32, R2, M, cnt, nbr, shift, status);
  return cudaGetLastError();
}
cudaError_t launch_reverse(int64_t Ntot, int M, const int *cnt, const int *nbr, const char4 *shift,
                           const int *boff, int *brev, unsigned *status, cudaStream_t s) {
  if (Ntot == 0) return cudaSuccess;
  reverse_kernel<<<nblk(Ntot * M, 256), 256, 0, s>>>(Ntot, M, cnt, nbr, shift, boff, brev, status);
  return cudaGetLastError();
}
cudaError_t launch_geometry(int64_t Ntot, int M, const int *atom_cfg, const int *atom_off,
                            const int *brev, const double *pos,
                            const double *box, const int *cnt, const int *nbr, const char4 *shift,
                            const int *boff, const int *poff, double R1, double R2, float4 *gA32,
                            float4 *gB32, float *gcos32, dvec4 *gA64, dvec4 *gB64,
                            double *gcos64, int max_slots, cudaStream_t s) {
  if (Ntot == 0) return cudaSuccess;
  geometry_bond_kernel<<<nblk(Ntot * M, 256), 256, 0, s>>>(Ntot, M, atom_cfg, atom_off, brev, pos, box, cnt,
                                                           nbr, shift, boff, R1, R2, gA32, gB32, gA64, gB64);
  if (max_slots > 0)
    geometry_pair_kernel<<<nblk(Ntot * max_slots, 256), 256, 0, s>>>(Ntot, max_slots, cnt, M, boff, poff, gA64,
                                                                      gcos32, gcos64);
  return cudaGetLastError();
}

}  // namespace tsf
