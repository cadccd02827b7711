// float instantiations of the plain persistent trace kernel (see trace.cuh): the full profile,
// the telescope profile (mirrors, masts and camera boxes) and the concentrator profile (cones
// and refracting faces) for every launch shape; the source-mode instantiations are in
// trace_f32_src.cu (a separate unit, compiled in parallel).
#include "launch.h"

namespace robast {

template <int BLOCK, bool C, bool STAGED, bool SRC, unsigned FEAT>
static cudaError_t launch_one(const TraceArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = trace_kernel<float, BLOCK, C, STAGED, SRC, float, FEAT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int BLOCK, bool SRC, unsigned FEAT>
static int occupancy_one(size_t smem) {
    auto k = smem ? trace_kernel<float, BLOCK, false, true, SRC, float, FEAT>
                  : trace_kernel<float, BLOCK, false, false, SRC, float, FEAT>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, BLOCK, smem) != cudaSuccess) return 0;
    return nb;
}

template <int BLOCK, bool SRC>
static int occupancy_prof(size_t smem, unsigned prof) {
    if (prof == FT_TELESCOPE) return occupancy_one<BLOCK, SRC, FT_TELESCOPE>(smem);
    if (prof == FT_CONCENTRATOR) return occupancy_one<BLOCK, SRC, FT_CONCENTRATOR>(smem);
    return occupancy_one<BLOCK, SRC, FT_ALL>(smem);
}

int trace_blocks_per_sm_f32(int block, size_t smem, bool src, unsigned prof) {
    if (src) return trace_blocks_per_sm_f32_src(block, smem, prof);
    switch (block) {
        case 64: return occupancy_prof<64, false>(smem, prof);
        case 128: return occupancy_prof<128, false>(smem, prof);
        case 256: return occupancy_prof<256, false>(smem, prof);
        case 512: return occupancy_prof<512, false>(smem, prof);
    }
    return 0;
}

template <int BLOCK, bool SRC>
static cudaError_t launch_prof(const TraceArgs<float>& a, int grid, size_t smem, cudaStream_t s, unsigned prof) {
    const bool st = a.stage != 0;
    if (prof == FT_TELESCOPE)
        return st ? launch_one<BLOCK, false, true, SRC, FT_TELESCOPE>(a, grid, smem, s)
                  : launch_one<BLOCK, false, false, SRC, FT_TELESCOPE>(a, grid, smem, s);
    if (prof == FT_CONCENTRATOR)
        return st ? launch_one<BLOCK, false, true, SRC, FT_CONCENTRATOR>(a, grid, smem, s)
                  : launch_one<BLOCK, false, false, SRC, FT_CONCENTRATOR>(a, grid, smem, s);
    return st ? launch_one<BLOCK, false, true, SRC, FT_ALL>(a, grid, smem, s)
              : launch_one<BLOCK, false, false, SRC, FT_ALL>(a, grid, smem, s);
}

cudaError_t launch_trace_f32(const TraceArgs<float>& a, int block, int grid, size_t smem, cudaStream_t s,
                             unsigned prof) {
    const bool st = a.stage != 0;
    if (a.groups) return launch_trace_f32_src(a, block, grid, smem, s, prof);
    if (a.units) {  // counting build (full profile, block 128)
        if (block != 128) return cudaErrorInvalidConfiguration;
        return st ? launch_one<128, true, true, false, FT_ALL>(a, grid, smem, s)
                  : launch_one<128, true, false, false, FT_ALL>(a, grid, smem, s);
    }
    switch (block) {
        case 64: return launch_prof<64, false>(a, grid, smem, s, prof);
        case 128: return launch_prof<128, false>(a, grid, smem, s, prof);
        case 256: return launch_prof<256, false>(a, grid, smem, s, prof);
        case 512: return launch_prof<512, false>(a, grid, smem, s, prof);
    }
    return cudaErrorInvalidConfiguration;
}

}  // namespace robast
