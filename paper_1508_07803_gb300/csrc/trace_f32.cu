// float instantiations of the persistent trace kernel (see trace.cuh).
#include "launch.h"

namespace robast {

template <int BLOCK, bool C, bool STAGED, bool SRC = false>
static cudaError_t launch_one(const TraceArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = trace_kernel<float, BLOCK, C, STAGED, SRC>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int BLOCK>
static int occupancy_one(size_t smem, bool src) {
    auto k = src ? (smem ? trace_kernel<float, BLOCK, false, true, true> : trace_kernel<float, BLOCK, false, false, true>)
                 : (smem ? trace_kernel<float, BLOCK, false, true> : trace_kernel<float, BLOCK, false, false>);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, BLOCK, smem) != cudaSuccess) return 0;
    return nb;
}

// 512 threads: the plain FP32 trace only (one copy of the staged tables per SM)
static int occupancy_512(size_t smem) {
    auto k = smem ? trace_kernel<float, 512, false, true> : trace_kernel<float, 512, false, false>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 512, smem) != cudaSuccess) return 0;
    return nb;
}

int trace_blocks_per_sm_f32(int block, size_t smem, bool src) {
    switch (block) {
        case 64: return occupancy_one<64>(smem, src);
        case 128: return occupancy_one<128>(smem, src);
        case 256: return occupancy_one<256>(smem, src);
        case 512: return src ? 0 : occupancy_512(smem);
    }
    return 0;
}

cudaError_t launch_trace_f32(const TraceArgs<float>& a, int block, int grid, size_t smem, cudaStream_t s) {
    const bool st = a.stage != 0;
    if (a.groups) {
        if (a.units) {  // counting build of the source-mode kernel (block 128)
            if (block != 128) return cudaErrorInvalidConfiguration;
            return st ? launch_one<128, true, true, true>(a, grid, smem, s) : launch_one<128, true, false, true>(a, grid, smem, s);
        }
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
        case 512: return st ? launch_one<512, false, true>(a, grid, smem, s) : launch_one<512, false, false>(a, grid, smem, s);
    }
    return cudaErrorInvalidConfiguration;
}

}  // namespace robast
