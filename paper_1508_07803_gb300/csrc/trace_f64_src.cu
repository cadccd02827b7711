// double instantiations of the source-mode trace kernel (photons generated on the device from
// source groups; full and concentrator profiles) and of the accuracy guard's FP64 re-trace of
// FP32 photons (see trace.cuh).
#include "launch.h"

namespace robast {

template <int BLOCK, bool STAGED, unsigned FEAT>
static cudaError_t launch_one(const TraceArgs<double>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = trace_kernel<double, BLOCK, false, STAGED, true, double, FEAT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int BLOCK, unsigned FEAT>
static int occupancy_one(size_t smem) {
    auto k = smem ? trace_kernel<double, BLOCK, false, true, true, double, FEAT>
                  : trace_kernel<double, BLOCK, false, false, true, double, FEAT>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, BLOCK, smem) != cudaSuccess) return 0;
    return nb;
}

int trace_blocks_per_sm_f64_src(int block, size_t smem, unsigned prof) {
    const bool cc = prof == FT_CONCENTRATOR;
    switch (block) {
        case 64: return cc ? occupancy_one<64, FT_CONCENTRATOR>(smem) : occupancy_one<64, FT_ALL>(smem);
        case 128: return cc ? occupancy_one<128, FT_CONCENTRATOR>(smem) : occupancy_one<128, FT_ALL>(smem);
        case 256: return cc ? occupancy_one<256, FT_CONCENTRATOR>(smem) : occupancy_one<256, FT_ALL>(smem);
    }
    return 0;
}

template <int BLOCK>
static cudaError_t launch_prof(const TraceArgs<double>& a, int grid, size_t smem, cudaStream_t s, unsigned prof) {
    const bool st = a.stage != 0;
    if (prof == FT_CONCENTRATOR)
        return st ? launch_one<BLOCK, true, FT_CONCENTRATOR>(a, grid, smem, s)
                  : launch_one<BLOCK, false, FT_CONCENTRATOR>(a, grid, smem, s);
    return st ? launch_one<BLOCK, true, FT_ALL>(a, grid, smem, s) : launch_one<BLOCK, false, FT_ALL>(a, grid, smem, s);
}

cudaError_t launch_trace_f64_src(const TraceArgs<double>& a, int block, int grid, size_t smem, cudaStream_t s,
                                 unsigned prof) {
    if (a.units) return cudaErrorInvalidConfiguration;
    switch (block) {
        case 64: return launch_prof<64>(a, grid, smem, s, prof);
        case 128: return launch_prof<128>(a, grid, smem, s, prof);
        case 256: return launch_prof<256>(a, grid, smem, s, prof);
    }
    return cudaErrorInvalidConfiguration;
}

// The FP64 re-trace of FP32 photons (accuracy guard): FP64 arithmetic on the FP32 arrays,
// block 128, photons from a device queue; the FP32 launch's feature profile.
template <bool STAGED, bool SRC, unsigned FEAT>
static auto retrace_kernel_of() {
    return trace_kernel<double, 128, false, STAGED, SRC, float, FEAT>;
}

template <bool SRC, unsigned FEAT>
static int retrace_occupancy(size_t smem) {
    auto k = smem ? retrace_kernel_of<true, SRC, FEAT>() : retrace_kernel_of<false, SRC, FEAT>();
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 128, smem) != cudaSuccess) return 0;
    return nb;
}

int retrace_blocks_per_sm(size_t smem, bool src, unsigned prof) {
    if (src)
        return prof == FT_CONCENTRATOR ? retrace_occupancy<true, FT_CONCENTRATOR>(smem)
                                       : retrace_occupancy<true, FT_ALL>(smem);
    if (prof == FT_TELESCOPE) return retrace_occupancy<false, FT_TELESCOPE>(smem);
    if (prof == FT_CONCENTRATOR) return retrace_occupancy<false, FT_CONCENTRATOR>(smem);
    return retrace_occupancy<false, FT_ALL>(smem);
}

template <bool SRC, unsigned FEAT>
static cudaError_t launch_re(const TraceArgs<double, float>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = a.stage ? retrace_kernel_of<true, SRC, FEAT>() : retrace_kernel_of<false, SRC, FEAT>();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_retrace(const TraceArgs<double, float>& a, int grid, size_t smem, cudaStream_t s, unsigned prof) {
    if (a.groups)
        return prof == FT_CONCENTRATOR ? launch_re<true, FT_CONCENTRATOR>(a, grid, smem, s)
                                       : launch_re<true, FT_ALL>(a, grid, smem, s);
    if (prof == FT_TELESCOPE) return launch_re<false, FT_TELESCOPE>(a, grid, smem, s);
    if (prof == FT_CONCENTRATOR) return launch_re<false, FT_CONCENTRATOR>(a, grid, smem, s);
    return launch_re<false, FT_ALL>(a, grid, smem, s);
}

}  // namespace robast
