// Internal interface between the host translation unit and the two kernel
// translation units (FP32 and FP64 instantiations of the trace kernel).
#pragma once
#include <cuda_runtime.h>

#include "trace.cuh"

namespace robast {

// Occupancy: resident blocks of trace_kernel<T, block> per SM for `smem`
// bytes of dynamic shared memory (0 if the configuration cannot launch); prof: the feature
// profile (FT_ALL, FT_TELESCOPE for plain traces, FT_CONCENTRATOR for source mode).  The
// source-mode halves live in their own translation units (trace_f32_src.cu, trace_f64_src.cu).
int trace_blocks_per_sm_f32(int block, size_t smem, bool src, unsigned prof);
int trace_blocks_per_sm_f64(int block, size_t smem, bool src, unsigned prof);
int trace_blocks_per_sm_f32_src(int block, size_t smem, unsigned prof);
int trace_blocks_per_sm_f64_src(int block, size_t smem, unsigned prof);

// Gradient pass (grad.cuh): frozen-path objective sums and per-parameter sums, 128-bit fixed
// point (two u64 words each: fraction, integer part).
constexpr int GRAD_SLOTS = 16 * 3 * 2;  // u64 words per surface: 16 parameters x 3 sums x 2
template <typename T>
struct GradArgs {
    Tables tab;              // precision T: the nearest-hit search
    const double* surf64;    // FP64 surface records: the dual-number re-intersection
    const double* grec;      // per surface: d rows / d tilt_x (9), d rows / d tilt_y (9)
    const T* o;
    const T* d;
    const T* lam;
    const int* vop;
    long long n;
    unsigned long long seed;
    long long first_id;
    int max_bounces;
    int stage;
    T eps;
    T newton_tol;
    double newton_tol64;  // Newton tolerance of the FP64 re-intersections (forward values, FP64 passes)
    int objective;
    double tau;
    unsigned long long* acc;   // [n_surf * GRAD_SLOTS]
    unsigned long long* vals;  // [n_variants * 8 * 2]
    unsigned long long* units; // optional [3]: FP64 interactions of the forward passes, interactions
                               // replayed by the reverse sweeps, dual-number interactions
    const int* order;          // optional processing order (work index -> photon index)
};
// resident blocks of 128 threads per SM; _r64: FP32 search with FP64 derivative passes (cones)
int grad_blocks_per_sm_f32(size_t smem);
int grad_blocks_per_sm_f32_r64(size_t smem);
int grad_blocks_per_sm_f64(size_t smem);
cudaError_t launch_grad_f32(const GradArgs<float>& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_grad_f32_r64(const GradArgs<float>& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_grad_f64(const GradArgs<double>& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_grad_finish(const unsigned long long* acc, const unsigned long long* vals, const int* surf_var,
                               int n_params, int objective, double d_obj, double* out, cudaStream_t s);
// value of a 128-bit fixed-point sum
double grad_fx_value(const unsigned long long* a);

// Coherent processing order (order.cu): scratch bytes for n photons, and the
// permutation (work index -> photon index) built in `scratch` on stream s.
long long order_scratch_bytes(long long n);
cudaError_t build_order_f32(const float* o, long long n, void* scratch, int** order, int sms, cudaStream_t s);
cudaError_t build_order_f64(const double* o, long long n, void* scratch, int** order, int sms, cudaStream_t s);

// Source mode: the FP32-rounded origins (x then y, [2 nw]) of photons base .. base + nw - 1 of
// the groups, generated as the trace kernel generates them (the coherent-order sort's input).
cudaError_t launch_src_origins(const SrcGroup* groups, int n_groups, long long base, long long nw,
                               long long first_id, unsigned long long seed, float* xy, int sms, cudaStream_t s);

// Launch the persistent trace kernel; returns the cudaError_t of the launch.
cudaError_t launch_trace_f32(const TraceArgs<float>& a, int block, int grid, size_t smem, cudaStream_t s,
                             unsigned prof);
cudaError_t launch_trace_f32_src(const TraceArgs<float>& a, int block, int grid, size_t smem, cudaStream_t s,
                                 unsigned prof);
cudaError_t launch_trace_f64(const TraceArgs<double>& a, int block, int grid, size_t smem, cudaStream_t s,
                             unsigned prof);
cudaError_t launch_trace_f64_src(const TraceArgs<double>& a, int block, int grid, size_t smem, cudaStream_t s,
                                 unsigned prof);

// FP64 re-trace of the FP32 photons queued by the accuracy guard (block 128; prof: the FP32
// launch's feature profile).
int retrace_blocks_per_sm(size_t smem, bool src, unsigned prof);
cudaError_t launch_retrace(const TraceArgs<double, float>& a, int grid, size_t smem, cudaStream_t s, unsigned prof);

}  // namespace robast
