// MIX-32 scheme (Sec. 4.1.3): placeholder until the FP32 kernels land.
#include "dp_internal.cuh"

namespace dp {

dp_status compute_mix32(dp_model *, dp_nlist *, double *, double *, double *, double *, double *, cudaStream_t)
{
    set_error("MIX-32 is not built into this library yet");
    return DP_ERR_UNSUPPORTED;
}

}  // namespace dp
