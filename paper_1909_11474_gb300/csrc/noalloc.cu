// noalloc.cu -- tersoff_fitness_static: the fitness call of tersoff_fitness with no device
// allocation at call time. Its per-call scratch (per-parameter-set constants, the per-(parameter set,
// configuration) residual terms and the per-configuration target-norm terms) lives in one file-scope __device__ array of fixed size instead of context buffers
// that grow on demand. Everything else it uses is allocated by tersoff_build_neighbors.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "ctx.hpp"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB, held by every device that loads the library
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_fitness_scratch[kScratchBytes];

// Device address of g_fitness_scratch, looked up once per device. Host code must not use the
// symbol's name as an address: on the host it names a stand-in, not device memory.
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int set_error(tersoff_ctx *ctx, int code, const char *msg) {
  if (ctx) ctx->c.err = msg;
  return code;
}

}  // namespace

namespace tsf {
// Looked up by tersoff_create on its device, and again by the entry point if that failed.
int static_scratch_address(int device, void **out) {
  *out = nullptr;
  if (device < 0 || device >= kMaxDevices) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != device) e = cudaSetDevice(device);
    void *ptr = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&ptr, g_fitness_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess || !ptr) return (int)(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    g_scratch_addr[device] = ptr;
  }
  *out = g_scratch_addr[device];
  return 0;
}
}  // namespace tsf

extern "C" int tersoff_fitness_static(tersoff_ctx *ctx, const double *params, int32_t P,
                                      const tersoff_targets *tg, const double *w, int32_t precision,
                                      double *Z, double *Zq, double *S, tersoff_stream stream) {
  if (!ctx) return TERSOFF_E_ARG;
  tsf::Ctx &c = ctx->c;
  if (c.form != 0) return set_error(ctx, TERSOFF_E_UNSUPPORTED, "the allocation-free fitness takes the minimal form only");
  if (int rc = tsf::finish_build(ctx)) return rc;
  if (!params || P < 1 || !tg || !w || !Z) return set_error(ctx, TERSOFF_E_ARG, "null argument or P < 1");
  if (!tg->E || !tg->W || !tg->F || !tg->mask) return set_error(ctx, TERSOFF_E_ARG, "null target pointer");
  if (precision != 32 && precision != 64) return set_error(ctx, TERSOFF_E_ARG, "precision must be 32 or 64");
  if (c.max_m > 8) return set_error(ctx, TERSOFF_E_UNSUPPORTED, "an atom has more than 8 neighbours");
  const tsf::BatchPlan &plan = precision == 64 ? c.plan64 : c.plan32;
  if (plan.buckets.empty()) return set_error(ctx, TERSOFF_E_STATE, "no work schedule for this build");
  if (c.device < 0 || c.device >= kMaxDevices) return set_error(ctx, TERSOFF_E_ARG, "device index out of range");

  // scratch layout, each part 256-byte aligned
  const size_t b_consts = align256((size_t)P * 8 * sizeof(double));
  const size_t b_part = align256((size_t)P * c.C * tsf::kResidualTerms * sizeof(double));
  const size_t b_dpart = align256((size_t)c.C * 3 * sizeof(double));
  const size_t b_count = align256(64 * sizeof(int));
  const size_t need = b_consts + b_part + b_dpart + b_count;
  if (need > kScratchBytes) {
    char buf[200];
    std::snprintf(buf, sizeof(buf), "tersoff_fitness_static needs %zu bytes of scratch for P=%d, C=%d; "
                  "the static limit is %zu", need, (int)P, c.C, kScratchBytes);
    return set_error(ctx, TERSOFF_E_ARG, buf);
  }

  if (cudaSetDevice(c.device) != cudaSuccess) return set_error(ctx, TERSOFF_E_CUDA, "cudaSetDevice failed");
  unsigned char *base = nullptr;
  {
    void *ptr = nullptr;
    const int e = tsf::static_scratch_address(c.device, &ptr);
    if (e != 0) {
      char buf[160];
      std::snprintf(buf, sizeof(buf), "cudaGetSymbolAddress of the static scratch failed: %s",
                    cudaGetErrorString((cudaError_t)e));
      return set_error(ctx, TERSOFF_E_CUDA, buf);
    }
    base = static_cast<unsigned char *>(ptr);
  }

  // every scratch element read by the kernels is written earlier in the same call (the constants by
  // the prep kernel, every (p, c) residual term and every configuration's target-norm terms by the
  // batch kernel); the work counters, which must start at zero, are zeroed by the prep kernel
  tsf::BatchOut o = {};
  o.tE = tg->E;
  o.tW = tg->W;
  o.tF = tg->F;
  o.tmask = tg->mask;
  o.consts = base;
  o.part = reinterpret_cast<double *>(base + b_consts);
  o.dpart = reinterpret_cast<double *>(base + b_consts + b_part);
  o.counters = reinterpret_cast<int *>(base + b_consts + b_part + b_dpart);
  o.pdl = c.pdl;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == 64) {
    const int rc = tsf::ensure_geom64(ctx, s);   // kernels into buffers allocated by the neighbour build
    if (rc) return rc;
  }
  cudaError_t e = tsf::launch_batch(c, plan, params, P, tsf::kModeFitness, o, s);
  if (e == cudaSuccess)
    e = tsf::launch_fitness_finalize(P, c.C, o.part, o.dpart, w[0], w[1], w[2], Z, Zq, S, o.pdl, s);
  if (e != cudaSuccess) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "CUDA error: %s", cudaGetErrorString(e));
    return set_error(ctx, TERSOFF_E_CUDA, buf);
  }
  return TERSOFF_OK;
}
