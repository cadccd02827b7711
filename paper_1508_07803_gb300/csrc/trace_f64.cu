// double instantiations of the persistent trace kernel (see trace.cuh).
#include "launch.h"

namespace robast {

template <int BLOCK, bool C, bool STAGED, bool SRC = false>
static cudaError_t launch_one(const TraceArgs<double>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = trace_kernel<double, BLOCK, C, STAGED, SRC>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int BLOCK>
static int occupancy_one(size_t smem, bool src) {
    auto k = src ? (smem ? trace_kernel<double, BLOCK, false, true, true> : trace_kernel<double, BLOCK, false, false, true>)
                 : (smem ? trace_kernel<double, BLOCK, false, true> : trace_kernel<double, BLOCK, false, false>);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, BLOCK, smem) != cudaSuccess) return 0;
    return nb;
}

int trace_blocks_per_sm_f64(int block, size_t smem, bool src) {
    switch (block) {
        case 64: return occupancy_one<64>(smem, src);
        case 128: return occupancy_one<128>(smem, src);
        case 256: return occupancy_one<256>(smem, src);
    }
    return 0;
}

cudaError_t launch_trace_f64(const TraceArgs<double>& a, int block, int grid, size_t smem, cudaStream_t s) {
    const bool st = a.stage != 0;
    if (a.groups) {
        if (a.units) return cudaErrorInvalidConfiguration;
        switch (block) {
            case 64: return st ? launch_one<64, false, true, true>(a, grid, smem, s) : launch_one<64, false, false, true>(a, grid, smem, s);
            case 128: return st ? launch_one<128, false, true, true>(a, grid, smem, s) : launch_one<128, false, false, true>(a, grid, smem, s);
            case 256: return st ? launch_one<256, false, true, true>(a, grid, smem, s) : launch_one<256, false, false, true>(a, grid, smem, s);
        }
        return cudaErrorInvalidConfiguration;
    }
    if (a.units) {
        if (block != 128) return cudaErrorInvalidConfiguration;
        return st ? launch_one<128, true, true>(a, grid, smem, s) : launch_one<128, true, false>(a, grid, smem, s);
    }
    switch (block) {
        case 64: return st ? launch_one<64, false, true>(a, grid, smem, s) : launch_one<64, false, false>(a, grid, smem, s);
        case 128: return st ? launch_one<128, false, true>(a, grid, smem, s) : launch_one<128, false, false>(a, grid, smem, s);
        case 256: return st ? launch_one<256, false, true>(a, grid, smem, s) : launch_one<256, false, false>(a, grid, smem, s);
    }
    return cudaErrorInvalidConfiguration;
}

// The FP64 re-trace of FP32 photons (accuracy guard): FP64 arithmetic on the FP32 arrays,
// block 128, photons from a device queue.
template <bool STAGED, bool SRC>
static cudaError_t launch_re(const TraceArgs<double, float>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = trace_kernel<double, 128, false, STAGED, SRC, float>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

int retrace_blocks_per_sm(size_t smem, bool src) {
    auto k = src ? (smem ? trace_kernel<double, 128, false, true, true, float> : trace_kernel<double, 128, false, false, true, float>)
                 : (smem ? trace_kernel<double, 128, false, true, false, float> : trace_kernel<double, 128, false, false, false, float>);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 128, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_retrace(const TraceArgs<double, float>& a, int grid, size_t smem, cudaStream_t s) {
    const bool st = a.stage != 0;
    if (a.groups) return st ? launch_re<true, true>(a, grid, smem, s) : launch_re<false, true>(a, grid, smem, s);
    return st ? launch_re<true, false>(a, grid, smem, s) : launch_re<false, false>(a, grid, smem, s);
}

}  // namespace robast
