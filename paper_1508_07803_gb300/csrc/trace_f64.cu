// double instantiations of the plain persistent trace kernel (see trace.cuh): the full,
// telescope and concentrator profiles for every launch shape, and the counting build; the
// source-mode and re-trace instantiations are in trace_f64_src.cu.
#include "launch.h"

namespace robast {

template <int BLOCK, bool C, bool STAGED, unsigned FEAT>
static cudaError_t launch_one(const TraceArgs<double>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = trace_kernel<double, BLOCK, C, STAGED, false, double, FEAT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int BLOCK, unsigned FEAT>
static int occupancy_one(size_t smem) {
    auto k = smem ? trace_kernel<double, BLOCK, false, true, false, double, FEAT>
                  : trace_kernel<double, BLOCK, false, false, false, double, FEAT>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, BLOCK, smem) != cudaSuccess) return 0;
    return nb;
}

template <int BLOCK>
static int occupancy_prof(size_t smem, unsigned prof) {
    if (prof == FT_TELESCOPE) return occupancy_one<BLOCK, FT_TELESCOPE>(smem);
    if (prof == FT_CONCENTRATOR) return occupancy_one<BLOCK, FT_CONCENTRATOR>(smem);
    return occupancy_one<BLOCK, FT_ALL>(smem);
}

int trace_blocks_per_sm_f64(int block, size_t smem, bool src, unsigned prof) {
    if (src) return trace_blocks_per_sm_f64_src(block, smem, prof);
    switch (block) {
        case 64: return occupancy_prof<64>(smem, prof);
        case 128: return occupancy_prof<128>(smem, prof);
        case 256: return occupancy_prof<256>(smem, prof);
    }
    return 0;
}

template <int BLOCK>
static cudaError_t launch_prof(const TraceArgs<double>& a, int grid, size_t smem, cudaStream_t s, unsigned prof) {
    const bool st = a.stage != 0;
    if (prof == FT_TELESCOPE)
        return st ? launch_one<BLOCK, false, true, FT_TELESCOPE>(a, grid, smem, s)
                  : launch_one<BLOCK, false, false, FT_TELESCOPE>(a, grid, smem, s);
    if (prof == FT_CONCENTRATOR)
        return st ? launch_one<BLOCK, false, true, FT_CONCENTRATOR>(a, grid, smem, s)
                  : launch_one<BLOCK, false, false, FT_CONCENTRATOR>(a, grid, smem, s);
    return st ? launch_one<BLOCK, false, true, FT_ALL>(a, grid, smem, s)
              : launch_one<BLOCK, false, false, FT_ALL>(a, grid, smem, s);
}

cudaError_t launch_trace_f64(const TraceArgs<double>& a, int block, int grid, size_t smem, cudaStream_t s,
                             unsigned prof) {
    const bool st = a.stage != 0;
    if (a.groups) return launch_trace_f64_src(a, block, grid, smem, s, prof);
    if (a.units) {  // counting build (full profile, block 128)
        if (block != 128) return cudaErrorInvalidConfiguration;
        return st ? launch_one<128, true, true, FT_ALL>(a, grid, smem, s)
                  : launch_one<128, true, false, FT_ALL>(a, grid, smem, s);
    }
    switch (block) {
        case 64: return launch_prof<64>(a, grid, smem, s, prof);
        case 128: return launch_prof<128>(a, grid, smem, s, prof);
        case 256: return launch_prof<256>(a, grid, smem, s, prof);
    }
    return cudaErrorInvalidConfiguration;
}

}  // namespace robast
