// Internal interface between the host translation unit and the two kernel
// translation units (FP32 and FP64 instantiations of the trace kernel).
#pragma once
#include <cuda_runtime.h>

#include "trace.cuh"

namespace robast {

// Occupancy: resident blocks of trace_kernel<T, block> per SM for `smem`
// bytes of dynamic shared memory (0 if the configuration cannot launch).
int trace_blocks_per_sm_f32(int block, size_t smem, bool src);
int trace_blocks_per_sm_f64(int block, size_t smem, bool src);

// Launch the persistent trace kernel; returns the cudaError_t of the launch.
cudaError_t launch_trace_f32(const TraceArgs<float>& a, int block, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_trace_f64(const TraceArgs<double>& a, int block, int grid, size_t smem, cudaStream_t s);

}  // namespace robast
