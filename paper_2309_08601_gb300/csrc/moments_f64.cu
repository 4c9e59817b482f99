// FP64 instantiations of the stage (a) kernel (the plain double-precision path).
#include "moments.cuh"

namespace mp3 {

cudaError_t launch_moments_f64(const MomentArgs<double>& a, int n_sm, cudaStream_t st)
{
    return launch_moments_dispatch<double>(a, n_sm, st);
}

}  // namespace mp3
