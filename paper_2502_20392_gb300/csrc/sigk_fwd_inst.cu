// sigk_fwd_inst.cu -- instantiates the forward solver for one edge degree P
// (compiled once per P with -DSIGK_P=<P>) and the supported D in {4, 8, 16}.
#include "sigk_fwd.cuh"
#include "sigk_launch.h"

#ifndef SIGK_P
#error "compile with -DSIGK_P=<edge degree>"
#endif

namespace sigk {

template <int P, int D>
static int info_impl(KernelInfo* info) {
    constexpr int R = rows_per_lane(P, D);
    const int threads = 128;
    const int smem = (threads / 32) * FwdSmem<P, D>::per_warp * (int)sizeof(float);
    auto kern = fwd_kernel<P, D, R>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess)
        return -1;
    info->rows_per_lane = R;
    info->smem_bytes = smem;
    info->threads = threads;
    info->blocks_per_sm = nb;
    return 0;
}

template <int P, int D>
static cudaError_t launch_impl(const SolverArgs& a, int grid, cudaStream_t s) {
    constexpr int R = rows_per_lane(P, D);
    const int smem = 4 * FwdSmem<P, D>::per_warp * (int)sizeof(float);
    auto kern = fwd_kernel<P, D, R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

template <>
int fwd_info<SIGK_P>(int D, KernelInfo* info) {
    switch (D) {
        case 4: return info_impl<SIGK_P, 4>(info);
        case 8: return info_impl<SIGK_P, 8>(info);
        case 16: return info_impl<SIGK_P, 16>(info);
        default: return -1;
    }
}

template <>
cudaError_t fwd_launch<SIGK_P>(int D, const SolverArgs& a, int grid, cudaStream_t s) {
    switch (D) {
        case 4: return launch_impl<SIGK_P, 4>(a, grid, s);
        case 8: return launch_impl<SIGK_P, 8>(a, grid, s);
        case 16: return launch_impl<SIGK_P, 16>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sigk
