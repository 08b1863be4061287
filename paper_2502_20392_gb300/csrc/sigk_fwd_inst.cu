// sigk_fwd_inst.cu -- instantiates, for one edge degree P and ring count NR
// (compiled once per pair with -DSIGK_P=<P> -DSIGK_NR=<NR>) and D in
// {4, 8, 16}: the forward solver (inference, and training with every 32-row
// seam stored, with or without every tile's record) and the backward
// (adjoint) kernel; the two-phase solver in FP32 and FP64; and the
// tensor-core solver for large d.
#include "sigk_bwd.cuh"
#include "sigk_bwd2.cuh"
#include "sigk_fwd.cuh"
#include "sigk_fwd_cm.cuh"
#include "sigk_fwd_tc.cuh"
#include "sigk_launch.h"

#ifndef SIGK_P
#error "compile with -DSIGK_P=<edge degree>"
#endif
#ifndef SIGK_NR
#error "compile with -DSIGK_NR=<ring count>"
#endif
static_assert(SIGK_NR >= 1 && SIGK_NR <= SIGK_P && SIGK_NR <= sigk::kMaxRings, "bad ring count");

namespace sigk {

template <typename K>
static int occupancy(K kern, int threads, int smem, int R, KernelInfo* info) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -1;
    // the whole unified L1 / shared memory as shared memory: several CTAs of
    // tens of KB each per SM (a default carveout left one CTA per SM)
    if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
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

template <int D, int R, bool REC>
static int fwd_info_impl(KernelInfo* info) {
    const int smem = 4 * FwdSmem<SIGK_P, D, R, REC>::per_warp * (int)sizeof(float);
    return occupancy(fwd_kernel<SIGK_P, D, R, SIGK_NR, REC>, 128, smem, R, info);
}

template <int D, int R, bool REC>
static cudaError_t fwd_launch_impl(const SolverArgs& a, int grid, cudaStream_t s) {
    const int smem = 4 * FwdSmem<SIGK_P, D, R, REC>::per_warp * (int)sizeof(float);
    auto kern = fwd_kernel<SIGK_P, D, R, SIGK_NR, REC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

// compensated chunk sums in the FP32 two-phase kernel from this dimension on
constexpr int kCompDim = 1024;

template <typename T, bool COMP>
static int fwd_cm_info_impl(KernelInfo* info) {
    return occupancy(fwd_cm_kernel<SIGK_P, T, SIGK_NR, COMP>, 128, CmSmem<SIGK_P, T>::bytes, 1, info);
}

template <typename T, bool COMP>
static cudaError_t fwd_cm_launch_impl(const SolverArgs& a, void* cscratch, int64_t cstride,
                                      int grid, cudaStream_t s) {
    const int smem = CmSmem<SIGK_P, T>::bytes;
    auto kern = fwd_cm_kernel<SIGK_P, T, SIGK_NR, COMP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, s>>>(a, static_cast<T*>(cscratch), cstride);
    return cudaGetLastError();
}

constexpr int kR4 = rows_per_lane(SIGK_P, 4);
constexpr int kR8 = rows_per_lane(SIGK_P, 8);
constexpr int kR16 = rows_per_lane(SIGK_P, 16);
constexpr int kQ4 = rec_rows_per_lane(SIGK_P, 4);
constexpr int kQ8 = rec_rows_per_lane(SIGK_P, 8);
constexpr int kQ16 = rec_rows_per_lane(SIGK_P, 16);

// variant 0: inference, or training with the strip seams stored
// (rows_per_lane(P, D) rows per lane); variant 1: training that also stores
// every tile's record for the adjoint (rec_rows_per_lane(P, D) rows).
template <>
int fwd_info<SIGK_P, SIGK_NR>(int D, int variant, KernelInfo* info) {
    if (variant != 0 && variant != 1) return -1;
    switch (D) {
        case 4: return variant ? fwd_info_impl<4, kQ4, true>(info) : fwd_info_impl<4, kR4, false>(info);
        case 8: return variant ? fwd_info_impl<8, kQ8, true>(info) : fwd_info_impl<8, kR8, false>(info);
        case 16:
            return variant ? fwd_info_impl<16, kQ16, true>(info) : fwd_info_impl<16, kR16, false>(info);
        default: return -1;
    }
}

template <>
cudaError_t fwd_launch<SIGK_P, SIGK_NR>(int D, int variant, const SolverArgs& a, int grid,
                                        cudaStream_t s) {
    if (variant != 0 && variant != 1) return cudaErrorInvalidValue;
    switch (D) {
        case 4:
            return variant ? fwd_launch_impl<4, kQ4, true>(a, grid, s)
                           : fwd_launch_impl<4, kR4, false>(a, grid, s);
        case 8:
            return variant ? fwd_launch_impl<8, kQ8, true>(a, grid, s)
                           : fwd_launch_impl<8, kR8, false>(a, grid, s);
        case 16:
            return variant ? fwd_launch_impl<16, kQ16, true>(a, grid, s)
                           : fwd_launch_impl<16, kR16, false>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

// (both FP32 variants share the launch shape: the occupancy is the lower one)
template <>
int fwd_cm_info<SIGK_P, SIGK_NR>(bool f64, KernelInfo* info) {
    if (f64) return fwd_cm_info_impl<double, false>(info);
    KernelInfo a, b;
    if (fwd_cm_info_impl<float, false>(&a) != 0 || fwd_cm_info_impl<float, true>(&b) != 0) return -1;
    *info = a.blocks_per_sm <= b.blocks_per_sm ? a : b;
    return 0;
}

template <>
cudaError_t fwd_cm_launch<SIGK_P, SIGK_NR>(bool f64, const SolverArgs& a, void* cscratch,
                                           int64_t cstride, int grid, cudaStream_t s) {
    if (f64) return fwd_cm_launch_impl<double, false>(a, cscratch, cstride, grid, s);
    return a.d > kCompDim ? fwd_cm_launch_impl<float, true>(a, cscratch, cstride, grid, s)
                          : fwd_cm_launch_impl<float, false>(a, cscratch, cstride, grid, s);
}

template <>
int bwd2_info<SIGK_P, SIGK_NR>(KernelInfo* info) {
    const int smem = 4 * Bwd2Smem<SIGK_P>::per_warp * (int)sizeof(float);
    return occupancy(bwd2_kernel<SIGK_P, SIGK_NR>, 128, smem, 1, info);
}

template <>
cudaError_t bwd2_launch<SIGK_P, SIGK_NR>(const BwdArgs& a, float* cs, int64_t cstride, int grid,
                                         cudaStream_t s) {
    const int smem = 4 * Bwd2Smem<SIGK_P>::per_warp * (int)sizeof(float);
    auto kern = bwd2_kernel<SIGK_P, SIGK_NR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, s>>>(a, cs, cstride);
    return cudaGetLastError();
}

template <>
int fwd_tc_info<SIGK_P, SIGK_NR>(KernelInfo* info) {
    const int r = occupancy(fwd_tc_kernel<SIGK_P, SIGK_NR>, kTcThreads, TcSmem<SIGK_P>::bytes, 1, info);
    // one CTA per SM: it holds all of TMEM
    if (r == 0 && info->blocks_per_sm > 1) info->blocks_per_sm = 1;
    return r;
}

template <>
cudaError_t fwd_tc_launch<SIGK_P, SIGK_NR>(const TcArgs& a, int grid, cudaStream_t s) {
    const int smem = TcSmem<SIGK_P>::bytes;
    auto kern = fwd_tc_kernel<SIGK_P, SIGK_NR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kTcThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sigk
