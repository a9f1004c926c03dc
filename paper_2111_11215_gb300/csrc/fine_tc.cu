// fine_tc.cu -- colour queries of the fine stage with the BF16 tensor-core MLP (tcgen05).
#include "dvgo_internal.cuh"

namespace dvgo {

int launch_fine_colour_fwd_tc(const RenderArgs &, cudaStream_t) { return DVGO_ERR_UNSUPPORTED; }
int launch_fine_colour_bwd_tc(const RenderArgs &, cudaStream_t) { return DVGO_ERR_UNSUPPORTED; }

}  // namespace dvgo
