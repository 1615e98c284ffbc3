// neighbors.cu -- neighbour build and parameter-independent geometry cache for batches of small
// periodic cells (the index sets of the sums over j in Eq. 2 and over k in Eq. 7 of
// arXiv:1909.11474, and the cutoff function f_C of Eq. 9).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "ctx.hpp"

namespace tsf {

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
// The image indices come as floats (f0, f1, f2: exact small integers) for the FP32 products and as
// ints for the exact test.
__device__ __forceinline__ bool member(const Pre32 &q, float dx, float dy, float dz, float f0, float f1, float f2,
                                       int n0, int n1, int n2, const double *xj, const double *xi, const double *H,
                                       double R2sq) {
  const float tx = (f0 * q.H[0] + f1 * q.H[3]) + f2 * q.H[6];
  const float ty = (f0 * q.H[1] + f1 * q.H[4]) + f2 * q.H[7];
  const float tz = (f0 * q.H[2] + f1 * q.H[5]) + f2 * q.H[8];
  const float ex = dx + tx, ey = dy + ty, ez = dz + tz;
  const float r2 = ex * ex + ey * ey + ez * ez;
  if (r2 < q.R2sq - q.band) return true;
  if (r2 > q.R2sq + q.band) return false;
  return exact_pair(xj[0], xj[1], xj[2], xi[0], xi[1], xi[2], H, n0, n1, n2).r2 < R2sq;
}
__device__ __forceinline__ bool member(const Pre32 &q, float dx, float dy, float dz, int n0, int n1, int n2,
                                       const double *xj, const double *xi, const double *H, double R2sq) {
  return member(q, dx, dy, dz, (float)n0, (float)n1, (float)n2, n0, n1, n2, xj, xi, H, R2sq);
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

// Per bond: unit vector, r, 2/r, f_C, f_C' and, packed into one int (rev | j << 16), the
// configuration-local indices of the reverse bond and of the neighbour atom (4th slot: as a double,
// or as the bit pattern of the int in the FP32 record). FP64 records take the bond vector d of the
// exact membership test and stay in FP64 (built on the first FP64 evaluation by geometry_bond_kernel,
// one thread per bond). FP32 records (built by the fused build kernel) take d rounded to FP32 and
// normalise in FP32; that kernel forms d from FP32 head + tail pairs of the positions and the box
// (bond_component: the FP64 vector rounded to FP32, but for values within ~2^-45 |x| of a rounding
// boundary), so that it needs the device's slow FP64 unit only for configurations whose coordinates
// cannot be split (beyond 2^60).
// FP32 bond record from the FP32 bond vector; R1f, R2f, Wf = R2 - R1 and Kf = -pi / (2 (R2 - R1)) are
// the FP64 cut-off constants rounded to FP32. Returns whether the bond reaches beyond R1.
__device__ __forceinline__ bool bond_record_f32(float dx, float dy, float dz, float R1f, float R2f, float Wf,
                                                float Kf, int rl, float4 &A, float4 &Bv) {
  const float ir = rsqrtf(dx * dx + dy * dy + dz * dz);
  const float r = (dx * dx + dy * dy + dz * dz) * ir;
  float fc = 1.f, fcp = 0.f;
  if (r >= R2f) {
    fc = 0.f;
  } else if (r > R1f) {
    const float w = (r - R1f) / Wf;
    fc = 0.5f * (1.f + cospif(w));
    fcp = Kf * sinpif(w);
  }
  A = make_float4(dx * ir, dy * ir, dz * ir, r);
  Bv = make_float4(ir + ir, fc, fcp, __int_as_float(rl));
  return r > R1f;
}

// The record of one bond from its exact FP64 bond vector: A = (unit vector, r), B = (2/r, f_C, f_C',
// packed indices rl). Returns whether r > R1 (f_C may differ from 1).
template <typename R>
__device__ __forceinline__ bool bond_record(const ExactPair &p, double R1, double R2, int rl,
                                            typename Vec4<R>::T &A, typename Vec4<R>::T &Bv) {
  if constexpr (sizeof(R) == 4) {
    return bond_record_f32((float)p.dx, (float)p.dy, (float)p.dz, (float)R1, (float)R2, (float)(R2 - R1),
                           (float)(-0.5 * M_PI / (R2 - R1)), rl, A, Bv);
  } else {
    const double ir = rsqrt(p.r2);
    const double r = p.r2 * ir;
    double fc, fcp;
    cutoff_fc(r, R1, R2, fc, fcp);
    A = make_dvec4(p.dx * ir, p.dy * ir, p.dz * ir, r);
    Bv = make_dvec4(ir + ir, fc, fcp, (double)rl);
    return r > R1;
  }
}

// FP64 records of the current build (its first FP64 evaluation): one thread per list slot (atom i,
// entry e < min(cnt_i, M)); bond b = boff[i] + e. cb0 = the first bond of i's configuration,
// atom_off[c] * M.
template <typename R>
__global__ void geometry_bond_kernel(int64_t Ntot, int M, const int *__restrict__ atom_cfg,
                                     const int *__restrict__ atom_off, const int *__restrict__ brev,
                                     const double *__restrict__ pos, const double *__restrict__ box,
                                     const int *__restrict__ cnt, const int *__restrict__ nbr,
                                     const char4 *__restrict__ shift, const int *__restrict__ boff, double R1,
                                     double R2, typename Vec4<R>::T *__restrict__ gA,
                                     typename Vec4<R>::T *__restrict__ gB) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / M;
  const int e = (int)(t % M);
  if (i >= Ntot || e >= min(cnt[i], M)) return;
  const int b = boff[i] + e;
  const int c = atom_cfg[i];
  const double *H = box + 9 * c;
  const int cb0 = atom_off[c] * M;   // first bond of the configuration
  const int j = nbr[i * M + e];
  // packed: configuration-local index of the reverse bond (bits 0-15) and of atom j (bits 16-31)
  const int rl = (brev[b] - cb0) | ((j - atom_off[c]) << 16);
  const char4 n = shift[i * M + e];
  const ExactPair p = exact_pair(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], pos[3 * i], pos[3 * i + 1],
                                 pos[3 * i + 2], H, n.x, n.y, n.z);
  typename Vec4<R>::T A, Bv;
  bond_record<R>(p, R1, R2, rl, A, Bv);
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
  const int m = min(cnt[i], M);
  const int q0 = poff[i], nslot = pair_slots(m);
  if (q >= nslot) return;
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
// Neighbour build of a batch of configurations: one launch, one CTA per configuration, two phases
// separated by CTA barriers only. Every configuration's bonds and pair slots start at a fixed base,
// atom_off[c] * M and atom_off[c] * pair_slots(M) (the capacity of full lists), so no configuration
// waits for another's counts.
//  phase 1: FP64 and FP32 copies of the positions, the box constants of the FP32 membership test, the
//    neighbour lists (warp per atom, as described at `member`);
//  phase 2: the bond offsets of the configuration's atoms (block scans), the reverse bond of every
//    bond, the FP32 bond records and the pair cosines.
// Shared memory (dynamic, sized for the largest configuration of the launch): FP32 positions (rounded,
// and as head + tail pairs), per-atom counts, offsets and flags, and, where they fit, the
// configuration's lists and bond unit vectors (the reverse-bond search and the pair cosines then read
// shared memory instead of global memory). Twelve warps per CTA and two CTAs per SM: a 300-cell batch
// runs in one wave.
constexpr int kBuildThreads = 384;
constexpr int kBuildWarps = kBuildThreads / 32;
constexpr size_t kBuildSmemCap = 96 * 1024;   // dynamic shared memory per CTA at most (two CTAs per SM)

struct BuildParams {
  int C, M;
  int64_t Ntot;
  double R1, R2;
  const int *atom_off;
  const double *pos_in, *box_in;   // caller's positions [Ntot][3] and boxes [C][3][3]
  double *pos, *box;               // the context's copies
  int *cnt, *nbr;
  char4 *shift;
  int *boff, *poff, *brev;
  float4 *gA, *gB;
  float *gcos;
  int *ameta;                      // [Ntot]: bonds kept (min(cnt, M)) | (some bond beyond R1) << 16
  int4 *arev;                      // [Ntot]: configuration-local reverse bonds of the first 8 bonds, 16 bits each
  unsigned *status, *build_status; // the context's status word and the build's own (read by the host)
  int nat_max;                     // largest configuration of the launch (shared-memory layout)
  int lists_in_smem;               // the lists and unit vectors fit in shared memory
  int pairmask;                    // the pair-membership bit matrix fits in shared memory (at pm_off)
  int pm_off;
  float R1f, R2f, Wf, Kf;          // R1, R2, R2 - R1 and -pi / (2 (R2 - R1)) rounded to FP32
};

__device__ __forceinline__ void build_flag(const BuildParams &a, unsigned bit) {
  set_status(a.status, bit);
  set_status(a.build_status, bit);
}

// Dynamic shared memory of the build kernel for configurations of up to nat atoms.
__host__ __device__ inline size_t build_smem_base(int nat) {
  return (size_t)4 * nat * sizeof(float4) + (size_t)(4 * nat + 2) * sizeof(int);
}
__host__ __device__ inline size_t build_smem_lists(int nat, int M) {
  return (size_t)nat * M * (sizeof(int2) + sizeof(float4));
}

// Max and exclusive scans over the threads of a block (kBuildThreads), in a fixed order.
__device__ __forceinline__ float block_max_f(float v, float *red) {
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < kBuildWarps; ++w) t = fmaxf(t, red[w]);
  return t;
}
// Exclusive scans of two values at once (v, u), with their totals: one pass, two barriers.
__device__ __forceinline__ int2 block_excl_scan2(int v, int u, int *red, int2 &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int iv = v, iu = u;
  for (int off = 1; off < 32; off <<= 1) {
    const int a = __shfl_up_sync(0xffffffffu, iv, off), b = __shfl_up_sync(0xffffffffu, iu, off);
    if (lane >= off) {
      iv += a;
      iu += b;
    }
  }
  __syncthreads();
  if (lane == 31) {
    red[warp] = iv;
    red[kBuildWarps + warp] = iu;
  }
  __syncthreads();
  int bv = 0, bu = 0;
  total = make_int2(0, 0);
  for (int w = 0; w < kBuildWarps; ++w) {
    if (w < warp) {
      bv += red[w];
      bu += red[kBuildWarps + w];
    }
    total.x += red[w];
    total.y += red[kBuildWarps + w];
  }
  return make_int2(bv + iv - v, bu + iu - u);
}

// Box constants of one configuration for the FP32 membership test: Hinv, the image search range
// R2/gap (+ margin), H and the decision band. `band` bounds the FP32 error of the squared distance:
// with X the largest coordinate magnitude of the configuration, |H| its largest box entry and nmax the
// largest image index a candidate can have, each FP32 component of d = (x_j - x_i) + n.H is within
// delta = 2^-23 (4X + 6 nmax |H|) of the exact value, so |r^2 - r32^2| < 3.5 R2 delta + 12 2^-24 R2^2;
// the band is four times that. Computed by one thread in FP32 (the band is a bound with a factor-4
// margin, the image range has a 1e-4 margin, so FP32 rounding of these constants is immaterial), in
// two parts: box_part1 from the box alone (while the other threads load the positions), box_part2
// once X is known.
struct BoxPart1 {
  float Hinv[9], rgap[3], col[3], Hm;    // rgap = R2 / gap per axis; col = column sums of |Hinv|
  int ok;                                // box finite and non-singular
};
__device__ void box_part1(const double *Hd, double R2, BoxPart1 &o) {
  bool ok = true;
  for (int k = 0; k < 9; ++k) ok = ok && isfinite(Hd[k]);
  float H[9];
  for (int k = 0; k < 9; ++k) H[k] = (float)Hd[k];
  const float a0 = H[0], a1 = H[1], a2 = H[2], b0 = H[3], b1 = H[4], b2 = H[5], c0 = H[6], c1 = H[7],
              c2 = H[8];
  const float bxc0 = b1 * c2 - b2 * c1, bxc1 = b2 * c0 - b0 * c2, bxc2 = b0 * c1 - b1 * c0;
  const float cxa0 = c1 * a2 - c2 * a1, cxa1 = c2 * a0 - c0 * a2, cxa2 = c0 * a1 - c1 * a0;
  const float axb0 = a1 * b2 - a2 * b1, axb1 = a2 * b0 - a0 * b2, axb2 = a0 * b1 - a1 * b0;
  const float det = a0 * bxc0 + a1 * bxc1 + a2 * bxc2;
  ok = ok && isfinite(det) && det != 0.f;
  o.ok = ok ? 1 : 0;
  if (!ok) return;
  const float id = 1.f / det;
  // H^-1 columns are (b x c, c x a, a x b) / det, i.e. Hinv[mu][k] = cross_k[mu] / det
  const float h[9] = {bxc0 * id, cxa0 * id, axb0 * id, bxc1 * id, cxa1 * id, axb1 * id,
                      bxc2 * id, cxa2 * id, axb2 * id};
  for (int k = 0; k < 9; ++k) o.Hinv[k] = h[k];
  const float vol = fabsf(det);
  const float gap[3] = {vol / sqrtf(bxc0 * bxc0 + bxc1 * bxc1 + bxc2 * bxc2),
                        vol / sqrtf(cxa0 * cxa0 + cxa1 * cxa1 + cxa2 * cxa2),
                        vol / sqrtf(axb0 * axb0 + axb1 * axb1 + axb2 * axb2)};
  for (int k = 0; k < 3; ++k) {
    o.rgap[k] = (float)R2 / gap[k];
    o.col[k] = fabsf(h[k]) + fabsf(h[3 + k]) + fabsf(h[6 + k]);
  }
  float Hm = 0.f;
  for (int k = 0; k < 9; ++k) Hm = fmaxf(Hm, fabsf(H[k]));
  o.Hm = Hm;
}
// Returns false for a bad box or an image range beyond the shift encoding.
__device__ bool box_part2(const BoxPart1 &o, const double *H, float xm, double R2, Pre32 &q, int &nmax_out) {
  if (!o.ok) return false;
  // largest coordinate magnitude (from the FP32 copies: widened by 2^-22 for their rounding)
  const float X = xm * (1.f + 0x1p-22f);
  float nmax = 0.f;
  for (int k = 0; k < 3; ++k) nmax = fmaxf(nmax, ceilf(2.f * X * o.col[k] + o.rgap[k] + 1.f));
  const float R2f = (float)R2;
  const float delta = (4.f * X + 6.f * nmax * o.Hm) * 0x1p-23f;
  const float band = 4.f * (3.5f * R2f * delta + 12.f * 0x1p-24f * R2f * R2f);
  for (int k = 0; k < 9; ++k) q.Hi[k] = o.Hinv[k];
  for (int k = 0; k < 3; ++k) q.rng[k] = o.rgap[k] + 1e-4f;
  for (int k = 0; k < 9; ++k) q.H[k] = (float)H[k];
  q.band = band;
  q.R2sq = (float)(R2 * R2);
  nmax_out = (int)fminf(nmax, 127.f);
  return isfinite(band) && nmax <= 127.f;
}

__global__ void __launch_bounds__(kBuildThreads, 2) build_batch_kernel(const BuildParams a) {
  extern __shared__ __align__(16) unsigned char bsm[];
  const int nmax = a.nat_max, M = a.M;
  float4 *s_p32 = reinterpret_cast<float4 *>(bsm);   // positions rounded to FP32 (membership test)
  float4 *s_ph = s_p32 + nmax;                         // FP32 heads and tails of the positions (bond vectors)
  float4 *s_pl = s_ph + nmax;
  float4 *s_fr = s_pl + nmax;                          // fractional coordinates x H^-1 of the FP32 positions
  int *s_m = reinterpret_cast<int *>(s_fr + nmax);
  int *s_boff = s_m + nmax;            // [nmax + 1]
  int *s_poff = s_boff + nmax + 1;     // [nmax + 1]
  int *s_outer = s_poff + nmax + 1;
  int2 *s_list = reinterpret_cast<int2 *>(bsm + (build_smem_base(nmax) + 15) / 16 * 16);   // [nmax * M]
  float4 *s_u = reinterpret_cast<float4 *>(s_list + (size_t)nmax * M);                     // [nmax * M]
  unsigned *s_pm = reinterpret_cast<unsigned *>(bsm + a.pm_off);   // [nmax][ceil(nmax / 32)] pair bits
  __shared__ Pre32 s_q;
  __shared__ BoxPart1 s_b1;
  __shared__ double s_H[9];
  __shared__ float s_Hh[9], s_Hl[9];   // box as FP32 head + tail
  __shared__ int s_ok, s_nmax;
  __shared__ float s_fred[kBuildWarps];
  __shared__ int s_ired[2 * kBuildWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool lists = a.lists_in_smem != 0;
  const int c = blockIdx.x;
  const int a0 = a.atom_off[c], nat = a.atom_off[c + 1] - a0;

  // ---- phase 1: positions, box constants, neighbour lists
  // the last warp's first thread works out the box-only constants while the other warps load the
  // positions
  constexpr int kLoadThreads = kBuildThreads - 32;
  int split = 1;   // every coordinate has an FP32 head + tail (bond vectors without the FP64 unit)
  if (tid == kLoadThreads) {
    double H[9];
    for (int k = 0; k < 9; ++k) {
      H[k] = a.box_in[9 * c + k];
      s_H[k] = H[k];
      a.box[9 * c + k] = H[k];
      float hh, hl;
      split &= split_f64(H[k], hh, hl) ? 1 : 0;
      s_Hh[k] = hh;
      s_Hl[k] = hl;
    }
    box_part1(H, a.R2, s_b1);
  }
  float xm = 0.f;
  int finite = 1;
  for (int t = tid; tid < kLoadThreads && t < nat; t += kLoadThreads) {
    const double *x = a.pos_in + 3 * (int64_t)(a0 + t);
    const double x0 = x[0], x1 = x[1], x2 = x[2];
    double *y = a.pos + 3 * (int64_t)(a0 + t);
    y[0] = x0;
    y[1] = x1;
    y[2] = x2;
    finite &= (isfinite(x0) && isfinite(x1) && isfinite(x2)) ? 1 : 0;
    const float4 v = make_float4((float)x0, (float)x1, (float)x2, 0.f);
    s_p32[t] = v;
    float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
    split &= (split_f64(x0, h.x, l.x) && split_f64(x1, h.y, l.y) && split_f64(x2, h.z, l.z)) ? 1 : 0;
    s_ph[t] = h;
    s_pl[t] = l;
    xm = fmaxf(xm, fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))));
  }
  xm = block_max_f(xm, s_fred);
  finite = __syncthreads_and(finite);
  split = __syncthreads_and(split);
  if (tid == 0) {
    Pre32 q;
    int nimg = 0;
    const bool ok = finite && box_part2(s_b1, s_H, xm, a.R2, q, nimg);
    if (!ok) build_flag(a, TERSOFF_STATUS_NONFINITE);
    s_q = q;
    s_ok = ok ? 1 : 0;
    s_nmax = nimg;
  }
  __syncthreads();
  for (int t = tid; t < nat; t += kBuildThreads) {
    const float4 v = s_p32[t];
    const float *h = s_q.Hi;
    s_fr[t] = make_float4(v.x * h[0] + v.y * h[3] + v.z * h[6], v.x * h[1] + v.y * h[4] + v.z * h[7],
                          v.x * h[2] + v.y * h[5] + v.z * h[8], 0.f);
  }
  __syncthreads();
  {
    const Pre32 q = s_q;
    const bool ok = s_ok != 0;
    const int nimg = s_nmax;
    const double R2sq = a.R2 * a.R2;
    // one warp per atom i, lanes over j; each lane keeps up to kNbrBuf accepted images of its j in
    // registers, so one enumeration suffices (a lane with more enumerates again for the rest); a warp
    // scan of the per-lane counts gives the output positions, so entries land in ascending
    // (j, n0, n1, n2) order
    constexpr int kNbrBuf = 4;
    // with every candidate range narrower than one lattice period (rng < 1/2 on each axis: plane
    // spacings above 2 R2), each j has at most one candidate image; the warp then tests it straight
    // away and places the accepted entries with a ballot (the same candidates and order as the loops)
    const bool single = q.rng[0] < 0.5f && q.rng[1] < 0.5f && q.rng[2] < 0.5f;
    if (single && ok && a.pairmask) {
      // each unordered pair once (the test is symmetric: the FP32 separation of (j, i, -n) is exactly
      // the negated one of (i, j, n), and so is the exact test's), its result a bit in both atoms'
      // rows; then each atom's list from its row, j ascending. The pairs are (i, (i + d) mod nat) for
      // d = 1 .. nat/2 (for an even nat, those of d = nat/2 only with i < nat/2), in blocks of 32
      // consecutive i over the warps
      const int nw = (nat + 31) >> 5, half = nat >> 1, nib = nw;
      for (int t = tid; t < nat * nw; t += kBuildThreads) s_pm[t] = 0u;
      __syncthreads();
      const float lim = (float)nimg;
      for (int b = warp; b < half * nib; b += kBuildWarps) {
        const int d = 1 + b / nib, il = ((b % nib) << 5) + lane;
        const bool act = il < nat && !(2 * d == nat && il >= half);
        int jl = il + d;
        if (jl >= nat) jl -= nat;
        bool acc = false;
        if (act) {
          const float4 xi32 = s_p32[il], si = s_fr[il], xj = s_p32[jl], sj = s_fr[jl];
          const float dx = xj.x - xi32.x, dy = xj.y - xi32.y, dz = xj.z - xi32.z;
          const float f0 = rintf(-(sj.x - si.x)), f1 = rintf(-(sj.y - si.y)), f2 = rintf(-(sj.z - si.z));
          if (fabsf(f0) <= lim && fabsf(f1) <= lim && fabsf(f2) <= lim)
            acc = member(q, dx, dy, dz, f0, f1, f2, (int)f0, (int)f1, (int)f2, a.pos_in + 3 * (int64_t)(a0 + jl),
                         a.pos_in + 3 * (int64_t)(a0 + il), s_H, R2sq);
        }
        if (acc) {
          atomicOr(&s_pm[il * nw + (jl >> 5)], 1u << (jl & 31));
          atomicOr(&s_pm[jl * nw + (il >> 5)], 1u << (il & 31));
        }
      }
      __syncthreads();
      // each atom's list from its row, one thread per atom: the set bits in ascending j, each with the
      // image of the test, n = round(-(s_j - s_i)); entries past M are counted, not written
      for (int li = tid; li < nat; li += kBuildThreads) {
        const int64_t i = a0 + li;
        const float4 si = s_fr[li];
        int count = 0;
        for (int wd = 0; wd < nw; ++wd) {
          unsigned word = s_pm[li * nw + wd];
          while (word) {
            const int jl = (wd << 5) + __ffs(word) - 1;
            word &= word - 1u;
            if (count < M) {
              const float4 sj = s_fr[jl];
              const char4 sh = make_char4((signed char)rintf(-(sj.x - si.x)), (signed char)rintf(-(sj.y - si.y)),
                                          (signed char)rintf(-(sj.z - si.z)), 0);
              a.nbr[i * M + count] = a0 + jl;
              a.shift[i * M + count] = sh;
              if (lists) s_list[li * M + count] = make_int2(jl, *reinterpret_cast<const int *>(&sh));
            }
            ++count;
          }
        }
        a.cnt[i] = count;
        if (count > M) build_flag(a, TERSOFF_STATUS_NBR_OVERFLOW);
        s_m[li] = min(count, M);
        for (int e = count; e < M; ++e) {
          a.nbr[i * M + e] = -1;
          a.shift[i * M + e] = make_char4(0, 0, 0, 0);
        }
      }
    } else
    for (int li = warp; li < nat; li += kBuildWarps) {
      const int64_t i = a0 + li;
      const double *xi = a.pos_in + 3 * i;
      const float4 xi32 = s_p32[li];
      int count = 0;
      const float4 si = s_fr[li];
      for (int jb = 0; single && ok && jb < nat; jb += 32) {
        // at most one candidate image per j: n = round(-(s_j - s_i)), |n| <= nimg. Whether it lies
        // within the image range (|s_j - s_i + n| <= rng) need not be tested: an image outside it is
        // farther than R2 by more than the band, and the membership test rejects it
        const int jl = jb + lane;
        float dx = 0.f, dy = 0.f, dz = 0.f, f0 = 0.f, f1 = 0.f, f2 = 0.f;
        bool cand = false;
        if (jl < nat) {
          const float4 xj = s_p32[jl], sj = s_fr[jl];
          dx = xj.x - xi32.x;
          dy = xj.y - xi32.y;
          dz = xj.z - xi32.z;
          const float d0 = sj.x - si.x, d1 = sj.y - si.y, d2 = sj.z - si.z;
          f0 = rintf(-d0);
          f1 = rintf(-d1);
          f2 = rintf(-d2);
          const float lim = (float)nimg;
          cand = fabsf(f0) <= lim && fabsf(f1) <= lim && fabsf(f2) <= lim &&
                 !(jl == li && f0 == 0.f && f1 == 0.f && f2 == 0.f);
        }
        const int j = a0 + (jl < nat ? jl : 0);
        const double *xj = a.pos_in + 3 * (int64_t)j;
        const int n0 = (int)f0, n1 = (int)f1, n2 = (int)f2;
        const bool acc = cand && member(q, dx, dy, dz, f0, f1, f2, n0, n1, n2, xj, xi, s_H, R2sq);
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        const int w = count + __popc(bal & ((1u << lane) - 1u));
        if (acc && w < M) {
          const char4 sh = make_char4((signed char)n0, (signed char)n1, (signed char)n2, 0);
          a.nbr[i * M + w] = j;
          a.shift[i * M + w] = sh;
          if (lists) s_list[li * M + w] = make_int2(jl, *reinterpret_cast<const int *>(&sh));
        }
        count += __popc(bal);
      }
      for (int jb = 0; !single && ok && jb < nat; jb += 32) {
        const int jl = jb + lane;
        int lo0 = 1, hi0 = 0, lo1 = 1, hi1 = 0, lo2 = 1, hi2 = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f;
        if (jl < nat) {
          const float4 xj = s_p32[jl];
          dx = xj.x - xi32.x;
          dy = xj.y - xi32.y;
          dz = xj.z - xi32.z;
          image_range(dx * q.Hi[0] + dy * q.Hi[3] + dz * q.Hi[6], q.rng[0], lo0, hi0);
          image_range(dx * q.Hi[1] + dy * q.Hi[4] + dz * q.Hi[7], q.rng[1], lo1, hi1);
          image_range(dx * q.Hi[2] + dy * q.Hi[5] + dz * q.Hi[8], q.rng[2], lo2, hi2);
          // every valid image index lies within +-nimg; the clamp only bounds the loops
          lo0 = max(lo0, -nimg); hi0 = min(hi0, nimg);
          lo1 = max(lo1, -nimg); hi1 = min(hi1, nimg);
          lo2 = max(lo2, -nimg); hi2 = min(hi2, nimg);
        }
        const int j = a0 + (jl < nat ? jl : 0);
        const double *xj = a.pos_in + 3 * (int64_t)j;
        int mine = 0;
        int buf[kNbrBuf];
        for (int n0 = lo0; n0 <= hi0; ++n0)
          for (int n1 = lo1; n1 <= hi1; ++n1)
            for (int n2 = lo2; n2 <= hi2; ++n2) {
              if (jl == li && n0 == 0 && n1 == 0 && n2 == 0) continue;
              if (member(q, dx, dy, dz, n0, n1, n2, xj, xi, s_H, R2sq)) {
                const char4 sh = make_char4((signed char)n0, (signed char)n1, (signed char)n2, 0);
#pragma unroll
                for (int u = 0; u < kNbrBuf; ++u)
                  if (u == mine) buf[u] = *reinterpret_cast<const int *>(&sh);
                ++mine;
              }
            }
        int incl = mine;   // inclusive warp scan of the per-lane counts
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int w0 = count + incl - mine;
#pragma unroll
        for (int u = 0; u < kNbrBuf; ++u)
          if (u < mine && w0 + u < M) {
            a.nbr[i * M + w0 + u] = j;
            a.shift[i * M + w0 + u] = *reinterpret_cast<const char4 *>(&buf[u]);
            if (lists) s_list[li * M + w0 + u] = make_int2(jl, buf[u]);
          }
        if (mine > kNbrBuf) {   // rare (small cells): enumerate again for the entries past the buffer
          int u = 0;
          for (int n0 = lo0; n0 <= hi0; ++n0)
            for (int n1 = lo1; n1 <= hi1; ++n1)
              for (int n2 = lo2; n2 <= hi2; ++n2) {
                if (jl == li && n0 == 0 && n1 == 0 && n2 == 0) continue;
                if (member(q, dx, dy, dz, n0, n1, n2, xj, xi, s_H, R2sq)) {
                  if (u >= kNbrBuf && w0 + u < M) {
                    const char4 sh = make_char4((signed char)n0, (signed char)n1, (signed char)n2, 0);
                    a.nbr[i * M + w0 + u] = j;
                    a.shift[i * M + w0 + u] = sh;
                    if (lists) s_list[li * M + w0 + u] = make_int2(jl, *reinterpret_cast<const int *>(&sh));
                  }
                  ++u;
                }
              }
        }
        count += total;
      }
      if (lane == 0) {
        a.cnt[i] = count;
        if (count > M) build_flag(a, TERSOFF_STATUS_NBR_OVERFLOW);
        s_m[li] = min(count, M);
      }
      for (int e = count + lane; e < M; e += 32) {
        a.nbr[i * M + e] = -1;
        a.shift[i * M + e] = make_char4(0, 0, 0, 0);
      }
    }
  }
  __syncthreads();

  // ---- phase 2: bond offsets, reverse bonds, FP32 bond records, pair cosines
  const int64_t base_b = (int64_t)a0 * M, base_q = (int64_t)a0 * pair_slots(M);
  int nb = 0, nq = 0;
  for (int cb = 0; cb < nat; cb += kBuildThreads) {
    const int t = cb + tid;
    const int m = t < nat ? s_m[t] : 0;
    int2 tot;
    const int2 xs = block_excl_scan2(m, t < nat ? pair_slots(m) : 0, s_ired, tot);
    const int xb = xs.x, xq = xs.y, tb = tot.x, tq = tot.y;
    if (t < nat) {
      s_boff[t] = nb + xb;
      s_poff[t] = nq + xq;
      s_outer[t] = 0;
    }
    nb += tb;
    nq += tq;
  }
  if (tid == 0) {
    s_boff[nat] = nb;
    s_poff[nat] = nq;
  }
  __syncthreads();
  for (int t = tid; t < nat; t += kBuildThreads) {
    a.boff[a0 + t] = (int)(base_b + s_boff[t]);
    a.poff[a0 + t] = (int)(base_q + s_poff[t]);
  }
  // one thread per bond: owner atom, reverse entry (j; i, -n), record
  for (int bl = tid; bl < nb; bl += kBuildThreads) {
    int lo = 0, hi = nat;   // last atom t with s_boff[t] <= bl
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_boff[mid] <= bl) lo = mid;
      else hi = mid;
    }
    const int il = lo, e = bl - s_boff[il];
    const int64_t i = a0 + il;
    int jl;
    char4 n;
    if (lists) {
      const int2 le = s_list[il * M + e];
      jl = le.x;
      n = *reinterpret_cast<const char4 *>(&le.y);
    } else {
      jl = a.nbr[i * M + e] - a0;
      n = a.shift[i * M + e];
    }
    const int64_t j = a0 + jl;
    const int mj = s_m[jl];
    int found = -1;
    for (int f = 0; f < mj; ++f) {
      int jf;
      char4 r;
      if (lists) {
        const int2 lf = s_list[jl * M + f];
        jf = lf.x;
        r = *reinterpret_cast<const char4 *>(&lf.y);
      } else {
        jf = a.nbr[j * M + f] - a0;
        r = a.shift[j * M + f];
      }
      if (jf == il && r.x == -n.x && r.y == -n.y && r.z == -n.z) {
        found = f;
        break;
      }
    }
    if (found < 0) {   // the exact test is antisymmetric, so this means an overflowing list
      build_flag(a, TERSOFF_STATUS_NBR_OVERFLOW);
      found = 0;
    }
    const int rev = s_boff[jl] + found;
    a.brev[base_b + bl] = (int)(base_b + rev);
    if (e < 8) reinterpret_cast<unsigned short *>(a.arev + i)[e] = (unsigned short)rev;
    float dx, dy, dz;
    if (split) {
      const float4 hj = s_ph[jl], lj = s_pl[jl], hi = s_ph[il], li = s_pl[il];
      const float n0 = (float)n.x, n1 = (float)n.y, n2 = (float)n.z;
      dx = bond_component(hj.x, lj.x, hi.x, li.x, n0, n1, n2, s_Hh[0], s_Hl[0], s_Hh[3], s_Hl[3], s_Hh[6], s_Hl[6]);
      dy = bond_component(hj.y, lj.y, hi.y, li.y, n0, n1, n2, s_Hh[1], s_Hl[1], s_Hh[4], s_Hl[4], s_Hh[7], s_Hl[7]);
      dz = bond_component(hj.z, lj.z, hi.z, li.z, n0, n1, n2, s_Hh[2], s_Hl[2], s_Hh[5], s_Hl[5], s_Hh[8], s_Hl[8]);
    } else {
      const ExactPair p = exact_pair(a.pos_in[3 * j], a.pos_in[3 * j + 1], a.pos_in[3 * j + 2], a.pos_in[3 * i],
                                     a.pos_in[3 * i + 1], a.pos_in[3 * i + 2], s_H, n.x, n.y, n.z);
      dx = (float)p.dx;
      dy = (float)p.dy;
      dz = (float)p.dz;
    }
    float4 A, Bv;
    if (bond_record_f32(dx, dy, dz, a.R1f, a.R2f, a.Wf, a.Kf, rev | (jl << 16), A, Bv)) atomicOr(&s_outer[il], 1);
    a.gA[base_b + bl] = A;
    a.gB[base_b + bl] = Bv;
    if (lists) s_u[bl] = A;
  }
  __syncthreads();
  for (int t = tid; t < nat; t += kBuildThreads) a.ameta[a0 + t] = s_m[t] | (s_outer[t] ? 0x10000 : 0);
  // one thread per pair slot: cos theta of bonds (e, f), e < f, row-major over e; padding 0
  for (int ql = tid; ql < nq; ql += kBuildThreads) {
    int lo = 0, hi = nat;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_poff[mid] <= ql) lo = mid;
      else hi = mid;
    }
    const int il = lo, m = s_m[il];
    int e = 0, rem = ql - s_poff[il];
    while (e < m && rem >= m - 1 - e) {
      rem -= m - 1 - e;
      ++e;
    }
    float cs = 0.f;
    if (e < m - 1) {
      const int f = e + 1 + rem;
      const float4 ue = lists ? s_u[s_boff[il] + e] : a.gA[base_b + s_boff[il] + e];
      const float4 uf = lists ? s_u[s_boff[il] + f] : a.gA[base_b + s_boff[il] + f];
      cs = ue.x * uf.x + ue.y * uf.y + ue.z * uf.z;
    }
    a.gcos[base_q + ql] = cs;
  }
}

// ---------------------------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_build_batch(const BuildLaunch &L, cudaStream_t s) {
  if (L.C < 1) return cudaSuccess;
  BuildParams a = {};
  a.C = L.C;
  a.M = L.M;
  a.Ntot = L.Ntot;
  a.R1 = L.R1;
  a.R2 = L.R2;
  a.R1f = (float)L.R1;
  a.R2f = (float)L.R2;
  a.Wf = (float)(L.R2 - L.R1);
  a.Kf = (float)(-0.5 * M_PI / (L.R2 - L.R1));
  a.atom_off = L.atom_off;
  a.pos_in = L.pos_in;
  a.box_in = L.box_in;
  a.pos = L.pos;
  a.box = L.box;
  a.cnt = L.cnt;
  a.nbr = L.nbr;
  a.shift = L.shift;
  a.boff = L.boff;
  a.poff = L.poff;
  a.brev = L.brev;
  a.gA = L.gA;
  a.gB = L.gB;
  a.gcos = L.gcos;
  a.ameta = L.ameta;
  a.arev = L.arev;
  a.status = L.status;
  a.build_status = L.build_status;
  a.nat_max = std::max(1, L.nat_max);
  const size_t base = (build_smem_base(a.nat_max) + 15) / 16 * 16;
  const size_t with_lists = base + build_smem_lists(a.nat_max, L.M);
  a.lists_in_smem = with_lists <= kBuildSmemCap ? 1 : 0;
  size_t smem = a.lists_in_smem ? with_lists : base;
  // the pair bit matrix after them, where it fits
  const size_t pm_off = (smem + 15) / 16 * 16;
  const size_t pm_bytes = (size_t)a.nat_max * ((a.nat_max + 31) / 32) * sizeof(unsigned);
  a.pairmask = pm_off + pm_bytes <= kBuildSmemCap ? 1 : 0;
  a.pm_off = (int)pm_off;
  if (a.pairmask) smem = pm_off + pm_bytes;
  // the default 48 KB limit covers the kernel's static shared memory too (a few hundred bytes): opt
  // in with a margin for it
  if (smem + 4096 > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(build_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  build_batch_kernel<<<(unsigned)L.C, kBuildThreads, smem, s>>>(a);
  return launched(1);
}

cudaError_t launch_geometry64(int64_t Ntot, int M, const int *atom_cfg, const int *atom_off, const int *brev,
                              const double *pos, const double *box, const int *cnt, const int *nbr,
                              const char4 *shift, const int *boff, const int *poff, double R1, double R2, void *gA,
                              void *gB, void *gcos, int max_slots, cudaStream_t s) {
  if (Ntot == 0) return cudaSuccess;
  geometry_bond_kernel<double><<<nblk(Ntot * M, 256), 256, 0, s>>>(
      Ntot, M, atom_cfg, atom_off, brev, pos, box, cnt, nbr, shift, boff, R1, R2, static_cast<dvec4 *>(gA),
      static_cast<dvec4 *>(gB));
  if (max_slots > 0)
    geometry_pair_kernel<double><<<nblk(Ntot * max_slots, 256), 256, 0, s>>>(
        Ntot, max_slots, cnt, M, boff, poff, static_cast<const dvec4 *>(gA), static_cast<double *>(gcos));
  return launched(1 + (max_slots > 0));
}

cudaError_t preload_geometry64_kernels() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, geometry_bond_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, geometry_pair_kernel<double>);
  return e;
}

}  // namespace tsf
