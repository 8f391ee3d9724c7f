// step_fused.cu -- row-streaming fused FP32 D2Q9 step for the walled cavity.
#include "internal.h"

namespace lbm {

int fused_d2q9_blocks(int, int) { return 0; }

cudaError_t launch_fused_d2q9(const StepParams &, const float *, float *, int *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace lbm
