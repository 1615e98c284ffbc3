// batch_launch.cuh -- launch of one bucket of the batched evaluation kernel (shared by the minimal-form
// launchers in batch.cu and the Tersoff-form launchers in batch_gen.cu).
#pragma once
#include <algorithm>

#include "batch_kernel.cuh"

namespace tsf {

constexpr int kPT = 32;   // parameter sets per warp: one atom per warp

template <int PTV, int MMAX, bool CLUSTER, int MINB, typename R, int NW = kNW, bool GEN = false>
inline cudaError_t launch_variant(BatchParams bp, const Bucket &b, bool pdl, cudaStream_t s) {
  auto kern = batch_kernel<PTV, MMAX, CLUSTER, MINB, R, NW, GEN>;
  const size_t smem = PTV != kPT ? b.smem16 : NW != kNW ? b.smem12 : b.smem;
  int gen_per_sm = 0;                              // Tersoff-form variants: occupancy queried per launch
  int &per_sm = GEN ? gen_per_sm : PTV != kPT ? b.per_sm16 : NW != kNW ? b.per_sm12 : b.per_sm;
  constexpr int kThr = NW * kWarp;
  bp.ntiles = (bp.P + PTV - 1) / PTV;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int cluster = CLUSTER ? b.cluster : 1, ncta = cluster;
  // resident CTAs of this variant, rounded down to whole clusters
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThr, smem);
    if (e != cudaSuccess) return e;
  }
  const int slots = std::max(1, per_sm * nsm / ncta);
  const int nconf = b.nitems;
  // work items: whole configurations when they are all alike and fit in one wave of CTAs (the
  // geometry is then staged once per configuration); otherwise each configuration's tiles are split
  // into chunks so that about four items per CTA slot balance the dynamically claimed work; the
  // autotuner's choice for this (P, mode) overrides both
  int per_conf = 1;
  if (!(b.uniform && nconf <= slots)) per_conf = std::min(bp.ntiles, std::max(1, (4 * slots + nconf - 1) / nconf));
  bp.narrow = 1;
  if (b.tune_P == bp.P && b.tune_mode == bp.mode && b.tune_per_conf > 0) {
    per_conf = std::min(bp.ntiles, b.tune_per_conf);
    bp.narrow = b.tune_narrow;
  }
  bp.nconf = nconf;
  bp.chunk_tiles = (bp.ntiles + per_conf - 1) / per_conf;
  bp.nchunks = (bp.ntiles + bp.chunk_tiles - 1) / bp.chunk_tiles;
  const int nitems = nconf * bp.nchunks;
  const int grid_clusters = std::min(nitems, slots);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(grid_clusters * ncta));
  cfg.blockDim = dim3(kThr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  // programmatic dependent launch: the kernel may start while its predecessor (the preparation kernel
  // or the previous bucket) runs; it waits for it before reading the per-call constants
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if constexpr (CLUSTER) {
    if (cluster > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = cluster;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.numAttrs = 2;
  }
  const cudaError_t el = cudaLaunchKernelEx(&cfg, kern, bp);
  if (el == cudaSuccess) count_launches(1);
  return el;
}


// One bucket in the Tersoff form (batch_gen.cu): the default schedule of the minimal form's kernels,
// instantiated with the Tersoff-form per-atom core.
cudaError_t launch_bucket_tersoff_form(BatchParams bp, const Bucket &b, bool f64, bool pdl, cudaStream_t s);

}  // namespace tsf
