// FP32 instantiations of the stage (a) kernel.
#include "moments.cuh"

namespace mp3 {

cudaError_t launch_moments_f32(const MomentArgs<float>& a, int n_sm, cudaStream_t st)
{
    return launch_moments_dispatch<float>(a, n_sm, st);
}

}  // namespace mp3
