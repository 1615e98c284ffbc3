// ga.cu -- one generation of the genetic algorithm that fits the minimal Tersoff parameters
// (arXiv:1909.11474, Sec. III.B): rank the population by fitness, keep the elite, keep the N_par best
// as parents, refill the population with children made by uniform crossover, mutate genes. One CTA
// does the whole population (N_pop <= 4096) of G genes each (6 for the minimal potential, 9 for the
// Tersoff form); the random numbers are drawn by the caller and passed in.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "ctx.hpp"

namespace tsf {

constexpr int kGaThreads = 1024;
constexpr int kGaMaxPop = 4096;
constexpr int kGaMaxGenes = 16;

// Ranking: the position of individual i is the number of individuals that precede it (smaller key,
// or equal key and smaller index), key = Z where finite, +inf otherwise. O(N_pop^2) comparisons in
// one CTA, which is far below the cost of the fitness evaluation that precedes it.
__global__ void __launch_bounds__(kGaThreads) ga_step_kernel(
    int P, int G, int n_par, double rate, const double *__restrict__ Z, const double *__restrict__ genes_in,
    const double *__restrict__ u, const double *__restrict__ lo, const double *__restrict__ hi,
    double *__restrict__ genes_out, double *__restrict__ params_out, int *__restrict__ order_out) {
  __shared__ double s_key[kGaMaxPop];
  __shared__ int s_order[kGaMaxPop];
  const int tid = threadIdx.x;
  for (int i = tid; i < P; i += kGaThreads) {
    const double z = Z[i];
    s_key[i] = isfinite(z) ? z : INFINITY;
  }
  __syncthreads();
  for (int i = tid; i < P; i += kGaThreads) {
    const double ki = s_key[i];
    int pos = 0;
    for (int j = 0; j < P; ++j) {
      const double kj = s_key[j];
      pos += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
    }
    s_order[pos] = i;
  }
  __syncthreads();
  const int base = (G + 2) * (P - n_par);
  for (int t = tid; t < P * G; t += kGaThreads) {
    const int i = t / G, g = t % G;
    double v;
    if (i < n_par) {
      v = genes_in[s_order[i] * G + g];                  // elite first, then the other parents
    } else {                                             // uniform crossover of two drawn parents
      const int c = i - n_par;
      const int pa = min((int)(u[(G + 2) * c] * (double)n_par), n_par - 1);
      const int pb = min((int)(u[(G + 2) * c + 1] * (double)n_par), n_par - 1);
      const int src = u[(G + 2) * c + 2 + g] < 0.5 ? pa : pb;
      v = genes_in[s_order[src] * G + g];
    }
    if (i >= 1) {                                        // mutation, the elite excepted
      const int k = base + 2 * G * (i - 1) + 2 * g;
      if (u[k] < rate) v = u[k + 1];
    }
    genes_out[t] = v;
    params_out[t] = __dadd_rn(lo[g], __dmul_rn(v, __dsub_rn(hi[g], lo[g])));   // lo + gene (hi - lo), unfused
  }
  if (order_out)
    for (int i = tid; i < P; i += kGaThreads) order_out[i] = s_order[i];
}

}  // namespace tsf

extern "C" int tersoff_ga_step(int32_t P, int32_t n_genes, int32_t n_par, double rate, const double *Z,
                               const double *genes_in, const double *uniforms, const double *lo, const double *hi,
                               double *genes_out, double *params_out, int32_t *order, tersoff_stream stream) {
  if (P < 1 || P > tsf::kGaMaxPop || n_par < 1 || n_par > P) return TERSOFF_E_ARG;
  if (n_genes < 1 || n_genes > tsf::kGaMaxGenes) return TERSOFF_E_ARG;
  if (!Z || !genes_in || !uniforms || !lo || !hi || !genes_out || !params_out) return TERSOFF_E_ARG;
  if (genes_in == genes_out || !(rate >= 0.0 && rate <= 1.0)) return TERSOFF_E_ARG;
  tsf::ga_step_kernel<<<1, tsf::kGaThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      P, n_genes, n_par, rate, Z, genes_in, uniforms, lo, hi, genes_out, params_out, order);
  return tsf::launched(1) == cudaSuccess ? TERSOFF_OK : TERSOFF_E_CUDA;
}
