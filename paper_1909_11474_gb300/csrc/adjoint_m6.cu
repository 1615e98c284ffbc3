// adjoint_m6.cu -- the parameter-gradient kernel for atoms of up to 6 neighbours, minimal form.
#include "adjoint_kernel.cuh"

namespace tsf {
template cudaError_t launch_adjoint_variant<6, false>(const AdjParams &, size_t, unsigned, cudaStream_t);
template cudaError_t launch_tangent_split<6, false>(const AdjParams &, const AdjSplit &, size_t, unsigned,
                                                     cudaStream_t);
}  // namespace tsf
