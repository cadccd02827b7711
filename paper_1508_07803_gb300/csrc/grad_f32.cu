// float instantiations of the gradient kernel (grad.cuh): FP32 search, FP32 derivative passes.
#include "grad.cuh"

namespace robast {

int grad_blocks_per_sm_f32(size_t smem) { return grad_occupancy<float, float>(smem); }

cudaError_t launch_grad_f32(const GradArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
    return a.stage ? launch_grad_one<float, float, 128, true>(a, grid, smem, s)
                   : launch_grad_one<float, float, 128, false>(a, grid, 0, s);
}

}  // namespace robast
