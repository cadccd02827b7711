// float instantiations of the gradient kernel (grad.cuh) with FP64 derivative passes: geometries
// with Bezier cone walls, whose grazing roots lose their derivatives in FP32.
#include "grad.cuh"

namespace robast {

int grad_blocks_per_sm_f32_r64(size_t smem) { return grad_occupancy<float, double>(smem); }

cudaError_t launch_grad_f32_r64(const GradArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
    return a.stage ? launch_grad_one<float, double, 128, true>(a, grid, smem, s)
                   : launch_grad_one<float, double, 128, false>(a, grid, 0, s);
}

}  // namespace robast
