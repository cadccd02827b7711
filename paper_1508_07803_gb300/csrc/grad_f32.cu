// float instantiations of the gradient kernel (grad.cuh).
#include "grad.cuh"

namespace robast {

cudaError_t launch_grad_f32(const GradArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
    return a.stage ? launch_grad_one<float, 128, true>(a, grid, smem, s) : launch_grad_one<float, 128, false>(a, grid, 0, s);
}

}  // namespace robast
