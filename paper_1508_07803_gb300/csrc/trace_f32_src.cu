// float instantiations of the source-mode trace kernel (see trace.cuh): photons generated on the
// device from source groups; the full profile and the concentrator profile (cones and refracting
// faces), and the counting build.
#include "launch.h"

namespace robast {

template <int BLOCK, bool C, bool STAGED, unsigned FEAT>
static cudaError_t launch_one(const TraceArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = trace_kernel<float, BLOCK, C, STAGED, true, float, FEAT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int BLOCK, unsigned FEAT>
static int occupancy_one(size_t smem) {
    auto k = smem ? trace_kernel<float, BLOCK, false, true, true, float, FEAT>
                  : trace_kernel<float, BLOCK, false, false, true, float, FEAT>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, BLOCK, smem) != cudaSuccess) return 0;
    return nb;
}

int trace_blocks_per_sm_f32_src(int block, size_t smem, unsigned prof) {
    const bool cc = prof == FT_CONCENTRATOR;
    switch (block) {
        case 64: return cc ? occupancy_one<64, FT_CONCENTRATOR>(smem) : occupancy_one<64, FT_ALL>(smem);
        case 128: return cc ? occupancy_one<128, FT_CONCENTRATOR>(smem) : occupancy_one<128, FT_ALL>(smem);
        case 256: return cc ? occupancy_one<256, FT_CONCENTRATOR>(smem) : occupancy_one<256, FT_ALL>(smem);
    }
    return 0;
}

template <int BLOCK>
static cudaError_t launch_prof(const TraceArgs<float>& a, int grid, size_t smem, cudaStream_t s, unsigned prof) {
    const bool st = a.stage != 0;
    if (prof == FT_CONCENTRATOR)
        return st ? launch_one<BLOCK, false, true, FT_CONCENTRATOR>(a, grid, smem, s)
                  : launch_one<BLOCK, false, false, FT_CONCENTRATOR>(a, grid, smem, s);
    return st ? launch_one<BLOCK, false, true, FT_ALL>(a, grid, smem, s)
              : launch_one<BLOCK, false, false, FT_ALL>(a, grid, smem, s);
}

cudaError_t launch_trace_f32_src(const TraceArgs<float>& a, int block, int grid, size_t smem, cudaStream_t s,
                                 unsigned prof) {
    const bool st = a.stage != 0;
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
