// adjoint_gen_m8.cu -- the parameter-gradient kernel for atoms of up to 8 neighbours, Tersoff form (Eq. 8, free S).
#include "adjoint_kernel.cuh"

namespace tsf {
template cudaError_t launch_adjoint_variant<8, true>(const AdjParams &, size_t, unsigned, cudaStream_t);
template cudaError_t launch_tangent_split<8, true>(const AdjParams &, const AdjSplit &, size_t, unsigned,
                                                     cudaStream_t);
}  // namespace tsf
