/*
 * tersoff.h -- C ABI of the GB300 (sm_103a) minimal-Tersoff library.
 *
 * The library evaluates the minimal Tersoff potential of Fan et al., "A minimal Tersoff potential
 * for diamond silicon with improved descriptions of elastic and phonon transport properties"
 * (arXiv:1909.11474): energy, per-atom forces and virial of many periodic configurations under many
 * parameter sets, the fitness that drives the paper's genetic-algorithm fit (Sec. III.B, Eq. 15-19),
 * and the gradient of that loss with respect to the six parameters.
 *
 * Conventions shared by every call:
 *  - Parameter vector x = [D0 (eV), alpha (1/A), r0 (A), beta, n, h], in the order of Eq. 16.
 *    S is fixed to 2 (Sec. II.B), so Eq. 11-14 give f_R = D0 e^{-2 alpha (r - r0)} and
 *    f_A = 2 D0 e^{-alpha (r - r0)}. R1 and R2 (Eq. 9) are fixed per neighbour build.
 *  - Units: eV and Angstrom. E is the total energy of a configuration (Eq. 1). W is the virial
 *    W_{mu nu} = -dU/d eps_{mu nu} summed over the cell (positive under compression), stored as the
 *    six components xx, yy, zz, xy, yz, zx.
 *  - "device" pointers are CUDA device memory owned by the caller; "host" pointers are ordinary host
 *    memory owned by the caller. The context owns only its own workspace (neighbour lists, geometry
 *    cache, schedules, scratch) and frees it in tersoff_destroy.
 *  - Every call is asynchronous and stream-ordered on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) unless its comment says it synchronises. A call returns a nonzero status for errors it
 *    can see on the host (bad arguments, CUDA launch errors) and then records a message retrievable
 *    with tersoff_last_error. Conditions detected inside kernels (neighbour overflow, a wait that
 *    timed out) set bits of a device status word that tersoff_get_status reads.
 *  - No call falls back to the CPU. A context is not thread-safe; use one context per host thread.
 */
#ifndef TERSOFF_GB300_H
#define TERSOFF_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tersoff_ctx tersoff_ctx;
typedef void *tersoff_stream; /* cudaStream_t */

enum {
  TERSOFF_OK = 0,
  TERSOFF_E_ARG = 1,          /* invalid argument (null pointer, size out of range, bad order)   */
  TERSOFF_E_NBR_OVERFLOW = 2, /* an atom has more neighbours than max_nbr (device status bit 1)   */
  TERSOFF_E_CUDA = 3,         /* a CUDA runtime call failed                                       */
  TERSOFF_E_NONFINITE = 4,    /* non-finite input positions or box (device status bit 4)          */
  TERSOFF_E_TIMEOUT = 5,      /* a bounded device-side wait gave up (device status bit 8)         */
  TERSOFF_E_STATE = 6,        /* call made before tersoff_build_neighbors succeeded               */
  TERSOFF_E_UNSUPPORTED = 7   /* an atom has more neighbours than the evaluation kernels handle   */
};

/* Device status bits, as returned by tersoff_get_status. */
#define TERSOFF_STATUS_NBR_OVERFLOW 1u
#define TERSOFF_STATUS_MANY_NBRS 2u
#define TERSOFF_STATUS_NONFINITE 4u
#define TERSOFF_STATUS_TIMEOUT 8u

/* Loss selector of tersoff_param_grad. */
#define TERSOFF_LOSS_SQ 0 /* L = sum_q w_q S_q / D_q  (smooth)                  */
#define TERSOFF_LOSS_Z 1  /* L = Z = sum_q w_q sqrt(S_q / D_q)  (Eq. 15, 17-19) */

/* Create a context on CUDA device `device`. *out receives the handle. Returns TERSOFF_OK or
 * TERSOFF_E_ARG / TERSOFF_E_CUDA. */
int tersoff_create(tersoff_ctx **out, int device);

/* Free the context and all of its device workspace. Waits for the context's work to finish. */
void tersoff_destroy(tersoff_ctx *ctx);

/* Message of the last host-visible error of this context ("" if none). Owned by the context. */
const char *tersoff_last_error(const tersoff_ctx *ctx);

/* Synchronise `stream`, return the device status word (TERSOFF_STATUS_* bits) and clear it.
 * Returns a negative value if the synchronisation itself failed. */
int tersoff_get_status(tersoff_ctx *ctx, tersoff_stream stream);

/* A batch of periodic configurations. */
typedef struct {
  int32_t C;                /* number of configurations, >= 1                                   */
  const int32_t *atom_off;  /* host [C+1]: atoms of config c are atom_off[c] .. atom_off[c+1]-1;
                               atom_off[0] = 0, non-decreasing, each config 1..1024 atoms          */
  const double *pos;        /* device [Ntot][3], Cartesian positions (A), Ntot = atom_off[C]     */
  const double *box;        /* device [C][3][3], row k = lattice vector k of config c (A)        */
} tersoff_configs;

/* Neighbour build for a batch (the index sets of the sums over j in Eq. 2 and over k in Eq. 7).
 *
 * For every atom i: all entries (j, n) with |x_j - x_i + n0 a + n1 b + n2 c| < R2 and
 * (j, n) != (i, 0), where a periodic image of j is a distinct entry. Membership is decided in FP64
 * with a fixed evaluation order and no fused multiply-add:
 *     t = (n0*a + n1*b) + n2*c,  d = (x_j - x_i) + t,  r^2 = (dx*dx + dy*dy) + dz*dz < R2*R2.
 * Entries are kept in ascending (j, n0, n1, n2) order. The call also builds the parameter-independent
 * geometry cache (bond lengths, unit vectors, f_C and f_C' of Eq. 9, bond-angle cosines; FP32 now,
 * FP64 on the first FP64 evaluation) and the evaluation schedule.
 * The build runs as one kernel queued on `stream` (one CTA per configuration), which copies pos/box
 * into the context: the caller's pos/box must stay unchanged until that kernel has run (stream order
 * suffices). The call returns once the work is queued. The neighbour counts come back to the host on
 * a side stream that waits for the kernel, so that work the caller queues next on `stream` does not
 * wait for the copy; the next call that uses the build (evaluation, fitness, gradient, export,
 * build_info) waits for the counts, checks them and builds the schedule; a rebuild of configurations
 * of the same sizes whose neighbour counts are all unchanged reuses the previous schedule. All
 * device memory of the build (the FP64 geometry records included) is allocated by this call.
 * R1 < R2 (Eq. 9; Sec. II.B uses R1 = 2.8, R2 = 3.2). 1 <= max_nbr <= 32 bounds the entries kept
 * per atom. Argument errors are returned by this call. Errors found by the build kernel are
 * returned by that next call (and set bits of the status word): an atom with more than max_nbr
 * entries TERSOFF_E_NBR_OVERFLOW (TERSOFF_STATUS_NBR_OVERFLOW), positions or boxes that are not
 * finite TERSOFF_E_NONFINITE. */
int tersoff_build_neighbors(tersoff_ctx *ctx, const tersoff_configs *cfg, double R1, double R2,
                            int32_t max_nbr, tersoff_stream stream);

/* Copy the neighbour list of the last build to host memory: cnt [Ntot], nbr [Ntot][max_nbr]
 * (global atom index j, -1 padding), shift [Ntot][max_nbr][3] (n0, n1, n2; 0 padding). Synchronous.
 * Any output pointer may be NULL. */
int tersoff_export_neighbors(tersoff_ctx *ctx, int32_t *cnt, int32_t *nbr, int8_t *shift);

/* Number of atoms, bonds (neighbour entries) and the largest neighbour count of the last build
 * (waits for the build as described at tersoff_build_neighbors). */
int tersoff_build_info(tersoff_ctx *ctx, int64_t *ntot, int64_t *nbonds, int32_t *max_m);

/* Energy, forces and virial for every (parameter set p, configuration c) of the last build
 * (Eq. 1-14; forces F_i = -dU/dx_i and the virial above).
 *  params    device [P][6] double (order of Eq. 16), P >= 1; [P][9] in the Tersoff form
 *            (tersoff_set_form)
 *  precision 32: per-pair arithmetic in FP32; each warp sums its atoms' energy and virial terms in
 *            FP32; the sum of a CTA's per-warp partial sums is their exact sum rounded once to FP64
 *            (fixed-point integer accumulation), and the sums over cluster ranks are FP64 additions,
 *            all in a fixed order; F in float;
 *            64: everything in FP64, F in double
 *  E         device [P][C] double, total energy (eV)             -- may be NULL
 *  F         device [P][Ntot][3] float or double (see precision) -- may be NULL
 *  W         device [P][C][6] double, total virial (eV)          -- may be NULL
 * Atoms with more than 8 neighbours are not supported by the evaluation kernels: the build reports
 * them and this call returns TERSOFF_E_UNSUPPORTED. */
int tersoff_eval(tersoff_ctx *ctx, const double *params, int32_t P, int32_t precision, double *E,
                 void *F, double *W, tersoff_stream stream);

/* Training targets (Eq. 17-19); energies and virials per atom, forces per atom as they are. */
typedef struct {
  const double *E;       /* device [C], target energy per atom (eV/atom)                      */
  const double *W;       /* device [C][6], target virial per atom (eV/atom), xx yy zz xy yz zx  */
  const double *F;       /* device [Ntot][3], target forces (eV/A)                             */
  const uint8_t *mask;   /* device [C]: bit 0 = E, bit 1 = W, bit 2 = F present for config c    */
} tersoff_targets;

/* Fitness of every parameter set (Eq. 15, 17-19):
 *   S_e = sum_c (E_c/N_c - E*_c)^2, S_v = sum_c sum_6 (W_c/N_c - W*_c)^2, S_f = sum_i |F_i - F*_i|^2
 *   over configs whose mask has the bit; D_q = the same sums over the targets alone;
 *   Zq[p][q] = sqrt(S_q / D_q) (0 if D_q = 0); Z[p] = sum_q w_q Zq[p][q]; +inf if any predicted
 *   value of parameter set p is not finite.
 *  params device [P][6] ([P][9] in the Tersoff form); w host [3] = (w_e, w_v, w_f); precision 32
 *  or 64 as in tersoff_eval;
 *  Z device [P] double; Zq device [P][3] double (may be NULL); S device [P][3] double (may be NULL).
 * Residual sums are accumulated in FP64 in a fixed order (deterministic). */
int tersoff_fitness(tersoff_ctx *ctx, const double *params, int32_t P, const tersoff_targets *tg,
                    const double *w, int32_t precision, double *Z, double *Zq, double *S,
                    tersoff_stream stream);

/* tersoff_fitness without device allocation. The paper has no counterpart; this entry point exists
 * for callers that cannot let a library call cudaMalloc: cudaMalloc stalls the whole device until it
 * returns, which a caller that keeps other streams busy or runs one generation after another cannot
 * afford, and a caller whose device memory was reserved up front by another allocator (a framework's
 * caching allocator, say) may have none left to give. tersoff_build_neighbors allocates every device
 * buffer this call uses (the FP64 geometry records and the work-schedule records included), creates
 * the side streams and loads the code of the kernels; tersoff_create looks up the device address of
 * one fixed 8 MiB scratch array that every device loading the library keeps until the process exits.
 * The call itself allocates nothing, also as the first call after a build: it may then wait for the
 * build's neighbour counts, fill the schedule records with synchronous host-to-device copies and, in
 * FP64, launch the kernels that compute the FP64 geometry into the buffers the build allocated.
 *  Arguments, results and arithmetic are those of tersoff_fitness, and so are the results.
 *  Limit: P*8*8 + P*C*24 + C*24 + 256 bytes (each part rounded up to 256) must fit in 8 MiB, e.g.
 *  P = 200 parameter sets over C = 300 cells of 64 atoms needs 1.5 MB; a larger request returns
 *  TERSOFF_E_ARG with the byte count in tersoff_last_error and launches nothing.
 *  If the address look-up in tersoff_create failed, the first call on that device repeats it; make
 *  that call before any stream capture. Every call shares the one array and leaves its contents
 *  behind; the call's first kernel zeroes its work counters (the only part that must start at zero)
 *  on `stream`. Two calls whose work overlaps on the GPU (different streams, or
 *  different contexts on the same device) race on the array: serialise them. */
int tersoff_fitness_static(tersoff_ctx *ctx, const double *params, int32_t P,
                           const tersoff_targets *tg, const double *w, int32_t precision, double *Z,
                           double *Zq, double *S, tersoff_stream stream);

/* Autotuner of the batched schedule; the paper has no counterpart. For the current build and these
 * tersoff_fitness arguments (P, targets, precision; params is read as the workload), times every
 * candidate schedule of each launch bucket -- work items per configuration (chunks of the parameter
 * tiles claimed by the persistent CTAs) and, for the FP32 single-CTA variant of up to 4 neighbours,
 * the tile width and warps per CTA (32 parameter sets with 8 or 12 warps, or 16 with two atoms per
 * warp and three CTAs per SM) and
 * whether a partly filled last tile runs more atoms per warp -- over whole launches (the best of
 * `reps` timed launches after one warm-up, CUDA events on `stream`), and keeps the fastest in the
 * context. Later tersoff_fitness / tersoff_fitness_static / tersoff_eval calls with the same P use
 * it until a rebuild changes the neighbour counts. Results of a tuned schedule equal the untuned
 * ones up to the FP32 summation order of the warps' atom groups. Synchronises `stream`.
 *  reps 1..100; best_ms (host, may be NULL) receives the tuned launch time in ms; tried (host, may
 *  be NULL) the number of candidates timed. Writes only the context's workspace. */
int tersoff_autotune(tersoff_ctx *ctx, const double *params, int32_t P, const tersoff_targets *tg,
                     int32_t precision, int32_t reps, double *best_ms, int32_t *tried, tersoff_stream stream);

/* Set the batched fitness schedule by hand (what tersoff_autotune would choose); the paper has no
 * counterpart. For every launch bucket of `precision` and calls with this P: tile = 32 parameter
 * sets per tile (one atom per warp), or 16 (two atoms per warp, three CTAs per SM; only for the FP32
 * single-CTA variant of up to 4 neighbours, others keep 32); warps = 8 or 12 per CTA (12: 32-wide
 * tiles of that same variant only, at most 80 registers, two CTAs per SM); items_per_config >= 1 work items per
 * configuration (the parameter tiles split into that many chunks, capped at the tile count);
 * narrow = 1 lets a partly filled last tile run with more atoms per warp. Kept until a rebuild
 * changes the neighbour counts or tersoff_autotune runs. */
int tersoff_set_schedule(tersoff_ctx *ctx, int32_t precision, int32_t P, int32_t tile, int32_t warps,
                         int32_t items_per_config, int32_t narrow);

/* The batched work schedule of the current build; the paper has no counterpart. bucket < 0: info[0]
 * receives the number of launch buckets. Otherwise info (host, 8 int32) receives for that bucket:
 * largest neighbour count of its kernel variant, CTAs per configuration (cluster size), number of
 * configurations, the P its fitness schedule was set for (0: none, built-in heuristic), tile width,
 * work items per configuration (0: heuristic), narrow last tile (0/1), warps per CTA. */
int tersoff_schedule_info(tersoff_ctx *ctx, int32_t precision, int32_t bucket, int32_t *info);

/* One generation of the genetic algorithm of Sec. III.B on the device (needs no context): rank the
 * N_pop = P individuals by fitness (ascending Z; a non-finite Z ranks last; ties keep index order),
 * keep the N_par best as parents in rank order (the elite first, never altered), refill with
 * P - N_par children by uniform crossover (a child draws two parents uniformly from the N_par and
 * takes each gene from the first with probability 1/2), then replace each gene of every individual
 * but the elite with probability `rate` by a fresh uniform value.
 *  n_genes = G: genes per individual, 1..16 (6 for the minimal potential, 9 for the Tersoff form).
 *  Z device [P] double; genes_in, genes_out device [P][G] double in [0, 1] (distinct buffers);
 *  uniforms device double in [0, 1): (G+2)(P - N_par) + 2G(P - 1) values laid out as: child c uses
 *  u[(G+2)c], u[(G+2)c+1] to pick its parents (index floor(u N_par)) and u[(G+2)c+2+g] < 1/2 to
 *  take gene g from the first; from base = (G+2)(P - N_par), individual i >= 1 uses
 *  u[base + 2G(i-1) + 2g] < rate to mutate gene g and u[base + 2G(i-1) + 2g + 1] as its new value;
 *  lo, hi device [G]: parameter limits, params_out device [P][G] = lo + genes_out (hi - lo)
 *  (Sec. III.B, step 1); order device [P] int32 (may be NULL): individuals from best to worst.
 * 1 <= N_par <= P <= 4096, 1 <= G <= 16, 0 <= rate <= 1, else TERSOFF_E_ARG. Stream-ordered, one
 * kernel. */
int tersoff_ga_step(int32_t P, int32_t n_genes, int32_t n_par, double rate, const double *Z,
                    const double *genes_in, const double *uniforms, const double *lo, const double *hi,
                    double *genes_out, double *params_out, int32_t *order, tersoff_stream stream);

/* Loss and its gradient with respect to x = [D0, alpha, r0, beta, n, h] for every parameter set
 *  (x = [D0, alpha, r0, S, n, h, gamma, c, d] in the Tersoff form, tersoff_set_form), Eq. 15-19, for
 *  configurations of every size the batched evaluation takes (large ones through a split path:
 *  evaluation, residual weights, tangent passes per atom slice).
 *  loss TERSOFF_LOSS_SQ or TERSOFF_LOSS_Z (the latter has a zero gradient term where S_q = 0);
 *  L device [P] double; dL device [P][6] ([P][9] in the Tersoff form) double. FP32 per-pair arithmetic with FP64 accumulation of
 *  the residual sums and of the gradient. Forces enter through the directional derivative
 *  sum_i v_i . dF_i/dx = -d/dx [ sum_i sum_j (v_j - v_i) . dU_i/dd_ij ] with v_i = dL/dF_i. */
int tersoff_param_grad(tersoff_ctx *ctx, const double *params, int32_t P, const tersoff_targets *tg,
                       const double *w, int32_t loss, double *L, double *dL, tersoff_stream stream);

/* Plain FP64 path: the same E, F, W as tersoff_eval(precision = 64), computed with one kernel launch
 * per (p, c), one thread per atom, bond geometry recomputed from positions (no batching, no
 * geometry cache). It is the comparison baseline for the batched path.
 *  params device [P][6]; E device [P][C]; F device [P][Ntot][3] double; W device [P][C][6]. */
int tersoff_eval_plain(tersoff_ctx *ctx, const double *params, int32_t P, double *E, double *F,
                       double *W, tersoff_stream stream);

/* MD-scale force call for one large periodic cell: neighbour rebuild (cell list) plus E, F, W.
 *  N atoms (>= 1, <= 2^24), pos device [N][3] double, box host [3][3] (rows = lattice vectors; every
 *  plane spacing must exceed 3*R2 so that each atom has at most one image of any other within R2),
 *  params host [6]; precision 32 or 64; E device [1] double; F device [N][3] float or double;
 *  W device [6] double. The neighbour list is the same set, in the same canonical order, as
 *  tersoff_build_neighbors would produce. max_nbr as above, except that when an atom has more than
 *  max_nbr neighbours (flagged) which of them are kept is unspecified. */
int tersoff_md_force(tersoff_ctx *ctx, int32_t N, const double *pos, const double *box,
                     const double *params, double R1, double R2, int32_t max_nbr, int32_t precision,
                     double *E, void *F, double *W, tersoff_stream stream);

/* Velocity-Verlet NVE steps driven by the MD-scale force call. The integrator is not part of the
 *  paper's method (its MD runs, Sec. IV, use an external code); it is the step toward them.
 *  Units: eV, A, amu, fs.
 *  - pos, vel: device [N][3] double, updated in place. Positions are never wrapped into the box.
 *  - mass: device [N] double (amu).
 *  - box, params, R1, R2, max_nbr, precision: as in tersoff_md_force.
 *  - dt: the time step (fs, > 0); nsteps >= 0 steps.
 *  The call evaluates the forces at the initial positions, then takes nsteps steps, each of
 *  v += F dt / 2m, x += v dt, F = F(x), v += F dt / 2m.
 *  Outputs (device):
 *  - Epot, Ekin: [nsteps + 1] double, the potential and kinetic energy before the first step and
 *    after every step. Ekin is summed in a fixed order, so it is deterministic.
 *  - F: [N][3] float (precision 32) or double (64), the forces at the final positions.
 *  - W: [6] double, the virial at the final positions.
 *  Errors: TERSOFF_E_ARG for bad arguments (pos == vel, dt <= 0, nsteps < 0, ...); device problems
 *  are flagged in the status word as for tersoff_md_force. */
int tersoff_md_nve(tersoff_ctx *ctx, int32_t N, double *pos, double *vel, const double *mass, const double *box,
                   const double *params, double R1, double R2, int32_t max_nbr, int32_t precision, double dt,
                   int32_t nsteps, double *Epot, double *Ekin, void *F, double *W, tersoff_stream stream);

/* Neighbour list of the last tersoff_md_force call, like tersoff_export_neighbors. Synchronous. */
int tersoff_md_export_neighbors(tersoff_ctx *ctx, int32_t *cnt, int32_t *nbr, int8_t *shift);

/* Launch mode of the per-call kernel sequences (bits, default both); the paper has no counterpart.
 *  TERSOFF_LAUNCH_GRAPHS: tersoff_fitness captures its launch sequence (preparation, batched kernel,
 *    finalize) into a CUDA graph on a private stream the first time and replays it with one graph
 *    launch while the arguments (pointers, P, weights, precision), the neighbour build's work
 *    schedule and the context's buffers are unchanged; any change re-captures. Calls made while
 *    kernel timing (tersoff_profile) is on, or on a stream that is being captured, launch directly.
 *  TERSOFF_LAUNCH_PDL: the batched and finalize kernels are launched with programmatic stream
 *    serialization, so each may start while its predecessor finishes (it waits before reading the
 *    predecessor's results).
 * Results are identical in every mode. Returns TERSOFF_E_ARG for a null context or unknown bits. */
#define TERSOFF_LAUNCH_GRAPHS 1
#define TERSOFF_LAUNCH_PDL 2
int tersoff_set_launch_mode(tersoff_ctx *ctx, int32_t mode);

/* Bound of the device-side wait of this context's later calls; the paper has no counterpart. One kernel
 * waits on other work: the batched kernel waits for the bulk copies that stage a configuration's
 * geometry in shared memory (tersoff_eval, tersoff_fitness, tersoff_fitness_static, tersoff_autotune).
 * The wait polls at most `spins` times (0: it gives up at once unless the copies have already landed);
 * a negative value restores the built-in bound (2^22 polls, far beyond any wait that can end). A wait
 * that gives up sets TERSOFF_STATUS_TIMEOUT in the status word, and its CTA stops without its results
 * after a second wait, with the built-in bound, for the copies already in flight: the call's outputs
 * are then undefined. It exists so that the timeout path can be exercised; nothing is left behind,
 * and the next call with the default bound runs normally. Returns TERSOFF_E_ARG for a null context or
 * spins >= 2^32. */
int tersoff_set_wait_limit(tersoff_ctx *ctx, int64_t spins);

/* Functional form of the potential for the context's later tersoff_eval and tersoff_fitness calls
 * (Sec. II.A-B):
 *  TERSOFF_FORM_MINIMAL (default): the minimal Tersoff potential, params [P][6] =
 *    (D0, alpha, r0, beta, n, h) (Eq. 16), g = beta (cos - h)^2 (Eq. 10), S = 2.
 *  TERSOFF_FORM_TERSOFF: the general form, params [P][9] = (D0, alpha, r0, S, n, h, gamma, c, d):
 *    the original angular function g^T = gamma (1 + c^2/d^2 - c^2/(d^2 + (cos - h)^2)) (Eq. 8) and
 *    a free S in Eq. 11-14 (S != 1).
 * In the Tersoff form tersoff_param_grad returns dL [P][9], and tersoff_autotune,
 * tersoff_eval_plain, tersoff_fitness_static, tersoff_md_force and tersoff_md_nve return
 * TERSOFF_E_UNSUPPORTED.
 * Errors: TERSOFF_E_ARG for an unknown form. */
#define TERSOFF_FORM_MINIMAL 0
#define TERSOFF_FORM_TERSOFF 1
int tersoff_set_form(tersoff_ctx *ctx, int32_t form);

/* Measurement helpers; the paper has no counterpart.
 * tersoff_kernel_launches: number of kernels the library has launched in this process, all contexts
 * and devices together (a count kept on the host when each launch is accepted). */
int64_t tersoff_kernel_launches(void);

/* Arithmetic throughput of CUDA device `device`, measured by microbenchmarks (independent dependency
 * chains in every thread of a grid that fills every SM, timed with CUDA events, best of three
 * launches); the paper has no counterpart. out (host, 6 doubles) receives, in operations per second:
 *  [0] FP32 FMA, as FLOP/s (2 per FMA);   [1] packed FP32x2 FMA (__ffma2_rn), as FLOP/s (4 per instruction);
 *  [2] FP64 FMA, as FLOP/s (2 per FMA);   [3] FP64 add, op/s;
 *  [4] special-function unit 2^x (ex2.approx.f32), op/s;   [5] FP32 -> FP64 -> FP32 conversions, op/s.
 * Synchronous (allocates and frees a small device buffer; runs for a few milliseconds). Returns
 * TERSOFF_E_ARG for a bad device or a null pointer, TERSOFF_E_CUDA on a CUDA error. */
int tersoff_measure_peaks(int32_t device, double *out);

/* Start (enable = 1) or stop (enable = 0) timing the batched E/F/W kernel of this context: while on,
 * every tersoff_eval / tersoff_fitness / tersoff_fitness_static records a CUDA event pair on its own
 * stream around its batched-kernel launches (prep and finalize kernels excluded). Enabling clears
 * earlier records. At most 4096 launch sequences are timed between two reads; later ones are not.
 * Returns TERSOFF_E_ARG for a null context, TERSOFF_E_CUDA if an event cannot be created. */
int tersoff_profile(tersoff_ctx *ctx, int32_t enable);

/* Synchronise on the recorded events and return, in host memory, the number of timed launch
 * sequences (*count) and their summed duration in milliseconds (*ms); clears the records. */
int tersoff_profile_read(tersoff_ctx *ctx, int64_t *count, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* TERSOFF_GB300_H */
