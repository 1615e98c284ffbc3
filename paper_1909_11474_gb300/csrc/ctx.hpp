// ctx.hpp -- host-side context of the minimal-Tersoff library and the launchers each .cu exports.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tersoff.h"

namespace tsf {

// Four doubles, 32-byte aligned (one FP64 bond record).
struct __align__(32) dvec4 {
  double x, y, z, w;
};
__host__ __device__ inline dvec4 make_dvec4(double x, double y, double z, double w) {
  dvec4 v;
  v.x = x;
  v.y = y;
  v.z = z;
  v.w = w;
  return v;
}

// Process-wide count of device-buffer (re)allocations: a captured launch sequence is valid only while
// none of the buffers it was captured with has moved.
uint64_t buffer_generation();
void bump_buffer_generation();

// Grow-only device buffer owned by the context.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n) {
    if (n <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    bump_buffer_generation();
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T *as() const {
    return static_cast<T *>(p);
  }
};

// Grow-only pinned host buffer (staging of host <-> device copies).
struct PinnedBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n) {
    if (n <= bytes) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaHostAlloc(&p, n, cudaHostAllocDefault);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T *as() const {
    return static_cast<T *>(p);
  }
};

// Geometry cache of a neighbour build: the bonds of atom i are boff[i] .. boff[i] + m_i - 1 (m_i =
// min(cnt_i, M)), its pair slots poff[i] .. poff[i] + pair_slots(m_i) - 1; the bonds of configuration c
// start at atom_off[c] * M and its pair slots at atom_off[c] * pair_slots(M) (the capacity of full
// lists), so the arrays have gaps between configurations.
struct Geometry {
  const int *boff;      // [Ntot] first bond of atom i
  const int *poff;      // [Ntot] first unordered bond pair of atom i
  const int *brev;      // [Ntot*M] bond index of the reverse entry (j; i, -n)
  const void *gA;       // [Ntot*M] R4: unit vector d/r (x, y, z), r
  const void *gB;       // [Ntot*M] R4: 2/r, f_C(r), f_C'(r), rev | j << 16
  const void *gcos;     // [Ntot*pair_slots(M)] R: cos theta of pair (e, f), e < f, row-major over e
};

// What one cluster rank of the batched evaluation works on, for every parameter tile: atoms
// s0 .. s0+ns-1 of configuration c (its slice when the configuration spans a cluster), bonds
// B0 .. B0+nb-1, padded pair slots Q0 .. Q0+nq-1; cb0 = first bond and nat = atom count of the
// configuration.
struct __align__(16) CtaRec {
  int c, s0, ns, B0;
  int nb, Q0, nq, cb0;
  int nat, pad;
  double inv_nat;   // 1/nat in FP64 (the per-atom energy and virial of Eq. 17-18)
};

// Residual terms the batched fitness writes per (parameter set, configuration), in FP64: the energy,
// virial and force terms of Eq. 17-19 before the sums over configurations.
constexpr int kResidualTerms = 3;
// Largest thread-block cluster a configuration of the batched kernels is split over.
constexpr int kMaxClusterCtas = 16;

// Pair slots per atom: m(m-1)/2 cosines padded to a multiple of 4 (16-byte vector loads).
__host__ __device__ inline int pair_slots(int m) { return ((m * (m - 1) / 2) + 3) & ~3; }

// A launch bucket: items with the same kernel variant.
struct Bucket {
  int mmax;        // 5 or 8: largest neighbour count the variant handles
  int cluster;     // CTAs per configuration (1 = no cluster)
  int precision;   // 32 or 64
  size_t smem;     // dynamic shared memory per CTA
  size_t adj_smem; // dynamic shared memory per CTA of the adjoint kernel (FP32, single-CTA buckets)
  bool adj_split = false;   // gradient through the split path (clusters, or beyond the adjoint's memory)
  size_t adj_split_smem = 0;  // dynamic shared memory per CTA of the split path's tangent kernel
  bool uniform;    // every configuration of the bucket has the same atom and bond counts
  int nitems;      // configurations in the bucket
  int item_off;    // first record of the bucket (records are per configuration and cluster rank)
  size_t smem16 = 0;        // shared memory per CTA of the 16-parameter-set tile variant (0: none)
  size_t smem12 = 0;        // shared memory per CTA of the 12-warp variant (0: none)
  mutable int per_sm = 0;   // resident CTAs per SM of the bucket's kernel variant (0: not queried yet)
  mutable int per_sm16 = 0; // the same for the 16-parameter-set tile variant
  mutable int per_sm12 = 0; // the same for the 12-warp variant
  // schedule chosen by the autotuner for one (P, mode): work items per configuration and whether the
  // last, partly filled parameter tile runs 2 or 4 atoms per warp; otherwise the built-in heuristic
  int tune_P = 0, tune_mode = -1, tune_per_conf = 0, tune_narrow = 1, tune_pt = 32, tune_nw = 8;
};

// Start/stop event pairs recorded around the launches of one kernel family while enabled; read and
// cleared by tersoff_profile_read. Capacity is fixed at enable time; launches past it go untimed.
struct KernelTimer {
  static constexpr int kCap = 4096;
  bool on = false;
  std::vector<cudaEvent_t> ev;   // [2 * kCap]: start, stop, start, stop, ...
  int n = 0;                     // pairs recorded since the last read
  bool begin(cudaStream_t s) {
    if (!on || n >= kCap) return false;
    return cudaEventRecord(ev[2 * n], s) == cudaSuccess;
  }
  void end(cudaStream_t s) {
    if (cudaEventRecord(ev[2 * n + 1], s) == cudaSuccess) ++n;
  }
};

// Process-wide count of kernels launched by the library (every launch site adds to it).
void count_launches(int n);
// cudaGetLastError after n kernel launches; the launches are counted when they were accepted.
inline cudaError_t launched(int n) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) count_launches(n);
  return e;
}

struct BatchPlan {
  int precision = 0;
  uint64_t gen = 0;  // distinct for every plan built (part of the key of captured launch sequences)
  std::vector<Bucket> buckets;
  DevBuf items;    // CtaRec [total CTAs]
};

// A launch sequence captured into a CUDA graph and the key it was captured under (every pointer and
// scalar its launches depend on); replayed while the key matches.
struct GraphCache {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;   // kernel launches in the sequence
};

struct Ctx {
  int device = 0;
  std::string err;
  DevBuf status;   // unsigned [2]: the context's status bits, then those of the last neighbour build alone

  // --- batch build state ---
  bool built = false;
  bool pending = false;               // a build is queued whose counts the host has not checked yet
  bool pending_same_layout = false;   // that build has the previous build's layout
  bool geom64 = false;   // FP64 geometry records built for the current neighbour build
  bool preloaded = false; // fitness kernels loaded on the device (module loading done up front)
  // polls of the batched kernel's bounded staging wait; negative: its built-in bound
  // (tersoff_set_wait_limit)
  int64_t wait_spins = -1;
  int C = 0;
  int64_t Ntot = 0, Btot = 0, Qtot = 0;   // atoms; capacities of the bond and pair-slot arrays
  int64_t nbonds = 0;                      // bonds (neighbour entries kept) of the build
  int M = 0, max_m = 0;
  double R1 = 0, R2 = 0;
  std::vector<int> h_atom_off, h_cnt, h_m, h_boff, h_poff, h_cfg_maxm;   // host mirror of the build's layout
  PinnedBuf hp_stage;   // pinned staging: atom table uploads, neighbour-count readback, offsets
  cudaEvent_t stage_event = nullptr;   // recorded after the staging buffer's last upload
  DevBuf atom_off, atom_cfg, pos, box, cnt, nbr, shift, boff, poff, brev;
  cudaStream_t copy_stream = nullptr;   // the build's count readback runs here, beside later calls
  cudaEvent_t build_done = nullptr;     // recorded after the build kernel on the caller's stream
  DevBuf counters;   // per-launch work counters of the persistent batched kernels
  DevBuf gA32, gB32, gcos32, gA64, gB64, gcos64;
  DevBuf ameta;   // [Ntot] int: bonds kept (min(cnt, M)) | (some bond beyond R1, f_C != 1) << 16
  DevBuf arev;    // [Ntot] int4: configuration-local reverse bonds of the first 8 bonds, 16 bits each
  BatchPlan plan32, plan64;
  DevBuf part, dpart, work, tf4, gpart;
  DevBuf adj_v, adj_ew, adj_aw, adj_gsplit;   // split-path gradient workspaces

  // --- MD state ---
  int md_N = 0, md_M = 0;
  DevBuf md_pos, md_cnt, md_nbr, md_shift, md_cells, md_cellcnt, md_Pij, md_red, md_keys, md_ke;
  DevBuf md_boxd;

  // --- measurement: CUDA events around each batched-kernel launch sequence, on its stream ---
  mutable KernelTimer timer;

  // --- side streams on which the launch buckets of one call run side by side (fork/join by events) ---
  mutable std::vector<cudaStream_t> side;
  mutable std::vector<cudaEvent_t> side_ev;   // [0]: fork, [1 + k]: bucket k done

  // --- launch mode of the per-call launch sequences (CUDA graphs, programmatic dependent launch) ---
  bool graphs = true;
  bool pdl = true;
  int form = 0;            // TERSOFF_FORM_*: parameter vectors of 6 (minimal) or 9 (Tersoff form)
  cudaStream_t cap_stream = nullptr;   // private stream the sequences are captured on
  GraphCache g_fitness;
};

// ---- launchers (defined in the .cu files) ----
// neighbors.cu
// Arguments of the neighbour build (one launch, one CTA per configuration).
struct BuildLaunch {
  int C, M;
  int64_t Ntot;
  double R1, R2;
  const int *atom_off;
  const double *pos_in, *box_in;
  double *pos, *box;
  int *cnt, *nbr;
  char4 *shift;
  int *boff, *poff, *brev;
  float4 *gA, *gB;
  float *gcos;
  int *ameta;
  int4 *arev;
  unsigned *status, *build_status;   // the context's status word and the build's own
  int nat_max;    // largest configuration (atoms)
};
cudaError_t launch_build_batch(const BuildLaunch &L, cudaStream_t s);
// FP64 bond records and pair cosines of the current build (on the first FP64 evaluation)
cudaError_t launch_geometry64(int64_t Ntot, int M, const int *atom_cfg, const int *atom_off, const int *brev,
                              const double *pos, const double *box, const int *cnt, const int *nbr,
                              const char4 *shift, const int *boff, const int *poff, double R1, double R2, void *gA,
                              void *gB, void *gcos, int max_slots, cudaStream_t s);

// batch.cu
struct BatchOut {
  double *E;          // [P][C]
  void *F;            // [P][Ntot][3]
  double *W;          // [P][C][6]
  const double *tE, *tW, *tF;
  const uint8_t *tmask;
  double *part;       // workspace: [P][C][3] FP64 residual terms per (p, c)
  double *dpart;      // workspace: [C][3] per-configuration terms of the target norms D_q (FP64), written
                      // by the batched kernel (fitness)
  void *consts;       // workspace: [P][8] per-parameter-set constants (working precision)
  int *counters;      // workspace: one work counter per launch bucket
  bool pdl = false;   // launch the batched kernels with programmatic stream serialization
  int64_t wait_spins = -1;   // polls of the staging wait before it gives up (negative: built-in bound)
  int form = 0;       // 0: minimal (6 parameters), 1: Tersoff form (9 parameters, Eq. 8, free S)
  int64_t f_ld = 0;   // > 0: F is [Ntot][3][f_ld] (parameter sets fastest) instead of [P][Ntot][3]
  bool split_only = false;   // launch only the buckets whose gradient takes the split path
};
enum BatchMode { kModeEval = 0, kModeFitness = 1 };
cudaError_t launch_batch(const Ctx &ctx, const BatchPlan &plan, const double *params, int P,
                         int mode, const BatchOut &out, cudaStream_t s);
cudaError_t autotune_batch(const Ctx &ctx, BatchPlan &plan, const double *params, int P, int mode,
                           const BatchOut &out, int reps, cudaStream_t s, float *best_ms, int *tried);
// Side streams of the launch buckets, and the module loading of every kernel a fitness call can launch
// (so that later calls neither create resources nor load code on the device).
cudaError_t ensure_side_streams(const Ctx &ctx);
cudaError_t preload_fitness_kernels();
cudaError_t preload_geometry64_kernels();   // neighbors.cu
cudaError_t launch_fitness_finalize(int P, int C, const double *part, const double *dpart,
                                    double we, double wv, double wf, double *Z, double *Zq, double *S, bool pdl,
                                    cudaStream_t s);
// capi.cu: host side of a queued neighbour build; FP64 geometry records on demand
int finish_build(tersoff_ctx *ctx);
int ensure_geom64(tersoff_ctx *ctx, cudaStream_t s);
// noalloc.cu: device address of the allocation-free fitness call's scratch array on `device` (looked up
// once per device, with that device current); nonzero CUDA error code on failure
int static_scratch_address(int device, void **out);

// md.cu
int md_force(Ctx &c, int N, const double *pos, const double *boxh, const double *x, double R1, double R2,
             int M, int precision, double *E, void *F, double *W, cudaStream_t s, std::string &err);
int md_nve(Ctx &c, int N, double *pos, double *vel, const double *mass, const double *boxh, const double *x,
           double R1, double R2, int M, int precision, double dt, int nsteps, double *Epot, double *Ekin,
           void *F, double *W, cudaStream_t s, std::string &err);

// adjoint.cu
size_t adjoint_smem_bytes(int nb, int nq, int nat);
size_t adjoint_split_smem_bytes(int nb, int nq, int ns);   // split-path tangent kernel
cudaError_t launch_param_grad(const Ctx &ctx, const double *params, int P, const double *tE, const double *tW,
                              const double *tF, const uint8_t *tmask, const double *w, int loss, double *L,
                              double *dL, void *consts, void *tf4, double *part, double *dpart, double *gpart,
                              cudaStream_t s);

// plain.cu
cudaError_t launch_plain(const Ctx &ctx, const double *params, int P, double *E, double *F, double *W,
                         cudaStream_t s);

size_t batch_smem_bytes_pt(int precision, int nb, int nq, int nat, int ncta);   // ncta = cluster size
size_t batch_smem_bytes_pt16(int nb, int nq, int nat);   // FP32 single-CTA, 16 parameter sets per tile
size_t batch_smem_bytes_nw12(int nb, int nq, int nat);   // FP32 single-CTA, 12 warps per CTA
int batch_param_tile();
int batch_max_smem_optin();

}  // namespace tsf

// The opaque handle of the C ABI.
struct tersoff_ctx {
  tsf::Ctx c;
};
