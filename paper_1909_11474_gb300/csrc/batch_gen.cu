// batch_gen.cu -- the batched evaluation kernel in the Tersoff form (Eq. 8 angular function, free S
// in Eq. 11-14), in a translation unit of its own so that it compiles beside the minimal form's.
#include "batch_launch.cuh"

namespace tsf {

cudaError_t launch_bucket_tersoff_form(BatchParams bp, const Bucket &b, bool f64, bool pdl, cudaStream_t s) {
  const bool cl = b.cluster > 1;
  if (!f64) {
    if (!cl && b.mmax <= 4) return launch_variant<kPT, 4, false, 2, float, kNW, true>(bp, b, pdl, s);
    if (!cl) return launch_variant<kPT, 8, false, 2, float, kNW, true>(bp, b, pdl, s);
    return launch_variant<kPT, 8, true, 2, float, kNW, true>(bp, b, pdl, s);
  }
  if (!cl) return launch_variant<kPT, 8, false, 1, double, kNW, true>(bp, b, pdl, s);
  return launch_variant<kPT, 8, true, 1, double, kNW, true>(bp, b, pdl, s);
}

}  // namespace tsf
