// sigk_fwd_inst.cu -- instantiates, for one edge degree P (compiled once per P
// with -DSIGK_P=<P>) and D in {4, 8, 16}: the inference forward solver, the
// one-row-per-lane training forward, and the backward (adjoint) kernel.
#include "sigk_bwd.cuh"
#include "sigk_fwd.cuh"
#include "sigk_fwd_cm.cuh"
#include "sigk_launch.h"

#ifndef SIGK_P
#error "compile with -DSIGK_P=<edge degree>"
#endif

namespace sigk {

template <typename K>
static int occupancy(K kern, int threads, int smem, int R, KernelInfo* info) {
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

template <int P, int D, int R>
static int fwd_info_impl(KernelInfo* info) {
    const int smem = 4 * FwdSmem<P, D>::per_warp * (int)sizeof(float);
    return occupancy(fwd_kernel<P, D, R>, 128, smem, R, info);
}

template <int P, int D, int R>
static cudaError_t fwd_launch_impl(const SolverArgs& a, int grid, cudaStream_t s) {
    const int smem = 4 * FwdSmem<P, D>::per_warp * (int)sizeof(float);
    auto kern = fwd_kernel<P, D, R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

template <int P, int D>
static int bwd_info_impl(KernelInfo* info) {
    const int smem = 4 * BwdSmem<P, D>::per_warp * (int)sizeof(float);
    return occupancy(bwd_kernel<P, D>, 128, smem, 1, info);
}

template <int P, int D>
static cudaError_t bwd_launch_impl(const BwdArgs& a, int grid, cudaStream_t s) {
    const int smem = 4 * BwdSmem<P, D>::per_warp * (int)sizeof(float);
    auto kern = bwd_kernel<P, D>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

#define SIGK_DISPATCH_D(FN, ...)            \
    switch (D) {                            \
        case 4: return FN<SIGK_P, 4>(__VA_ARGS__);   \
        case 8: return FN<SIGK_P, 8>(__VA_ARGS__);   \
        case 16: return FN<SIGK_P, 16>(__VA_ARGS__); \
        default: break;                     \
    }

template <>
int fwd_info<SIGK_P>(int D, int R, KernelInfo* info) {
    if (R == 1) {
        switch (D) {
            case 4: return fwd_info_impl<SIGK_P, 4, 1>(info);
            case 8: return fwd_info_impl<SIGK_P, 8, 1>(info);
            case 16: return fwd_info_impl<SIGK_P, 16, 1>(info);
            default: return -1;
        }
    }
    switch (D) {
        case 4: return fwd_info_impl<SIGK_P, 4, rows_per_lane(SIGK_P, 4)>(info);
        case 8: return fwd_info_impl<SIGK_P, 8, rows_per_lane(SIGK_P, 8)>(info);
        case 16: return fwd_info_impl<SIGK_P, 16, rows_per_lane(SIGK_P, 16)>(info);
        default: return -1;
    }
}

template <>
cudaError_t fwd_launch<SIGK_P>(int D, int R, const SolverArgs& a, int grid, cudaStream_t s) {
    if (R == 1) {
        switch (D) {
            case 4: return fwd_launch_impl<SIGK_P, 4, 1>(a, grid, s);
            case 8: return fwd_launch_impl<SIGK_P, 8, 1>(a, grid, s);
            case 16: return fwd_launch_impl<SIGK_P, 16, 1>(a, grid, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (D) {
        case 4: return fwd_launch_impl<SIGK_P, 4, rows_per_lane(SIGK_P, 4)>(a, grid, s);
        case 8: return fwd_launch_impl<SIGK_P, 8, rows_per_lane(SIGK_P, 8)>(a, grid, s);
        case 16: return fwd_launch_impl<SIGK_P, 16, rows_per_lane(SIGK_P, 16)>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static int fwd_cm_info_impl(KernelInfo* info) {
    return occupancy(fwd_cm_kernel<SIGK_P, T>, 128, CmSmem<SIGK_P, T>::bytes, 1, info);
}

template <typename T>
static cudaError_t fwd_cm_launch_impl(const SolverArgs& a, void* cscratch, int64_t cstride,
                                      int grid, cudaStream_t s) {
    const int smem = CmSmem<SIGK_P, T>::bytes;
    auto kern = fwd_cm_kernel<SIGK_P, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, s>>>(a, static_cast<T*>(cscratch), cstride);
    return cudaGetLastError();
}

template <>
int fwd_cm_info<SIGK_P>(bool f64, KernelInfo* info) {
    return f64 ? fwd_cm_info_impl<double>(info) : fwd_cm_info_impl<float>(info);
}

template <>
cudaError_t fwd_cm_launch<SIGK_P>(bool f64, const SolverArgs& a, void* cscratch, int64_t cstride,
                                  int grid, cudaStream_t s) {
    return f64 ? fwd_cm_launch_impl<double>(a, cscratch, cstride, grid, s)
               : fwd_cm_launch_impl<float>(a, cscratch, cstride, grid, s);
}

template <>
int bwd_info<SIGK_P>(int D, KernelInfo* info) {
    SIGK_DISPATCH_D(bwd_info_impl, info)
    return -1;
}

template <>
cudaError_t bwd_launch<SIGK_P>(int D, const BwdArgs& a, int grid, cudaStream_t s) {
    SIGK_DISPATCH_D(bwd_launch_impl, a, grid, s)
    return cudaErrorInvalidValue;
}

}  // namespace sigk
