// double instantiations of the gradient kernel (grad.cuh) and the kernel that turns the
// fixed-point sums into parameter gradients.
#include "grad.cuh"

namespace robast {

// d_params[p] += d_obj * gradient, from the fixed-point sums of the pass (the sums of the
// variant the parameter's surface belongs to)
__global__ void grad_finish(const unsigned long long* acc, const unsigned long long* vals_all, const int* surf_var,
                            int n_params, int objective, double d_obj, double* out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_params) return;
    const unsigned long long* V = vals_all + (size_t)surf_var[p / 16] * 16;
    const unsigned long long* c = acc + (size_t)p * 6;
    const double W = fx_value(V + 0);
    double g = 0.0;
    if (objective == 1) {
        const double N = fx_value(V + 14);
        g = N > 0 ? fx_value(c) / N : 0.0;
    } else if (W > 0) {
        const double qx = fx_value(V + 2) / W, qy = fx_value(V + 4) / W;
        if (objective == 0) g = 2.0 / W * (fx_value(c) - qx * fx_value(c + 2) - qy * fx_value(c + 4));
        if (objective == 2) g = fx_value(c + 2) / W;
        if (objective == 3) g = fx_value(c + 4) / W;
    }
    out[p] += d_obj * g;
}

double grad_fx_value(const unsigned long long* a) { return fx_value(a); }

int grad_blocks_per_sm_f64(size_t smem) { return grad_occupancy<double, double>(smem); }

cudaError_t launch_grad_f64(const GradArgs<double>& a, int grid, size_t smem, cudaStream_t s) {
    return a.stage ? launch_grad_one<double, double, 128, true>(a, grid, smem, s)
                   : launch_grad_one<double, double, 128, false>(a, grid, 0, s);
}
cudaError_t launch_grad_finish(const unsigned long long* acc, const unsigned long long* vals, const int* surf_var,
                               int n_params, int objective, double d_obj, double* out, cudaStream_t s) {
    grad_finish<<<(n_params + 255) / 256, 256, 0, s>>>(acc, vals, surf_var, n_params, objective, d_obj, out);
    return cudaGetLastError();
}

}  // namespace robast
