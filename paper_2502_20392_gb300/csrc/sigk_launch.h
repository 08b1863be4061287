// sigk_launch.h -- host-side entry points of the per-order kernel translation
// units (one TU per edge degree P keeps the build parallel).
#pragma once
#include <cuda_runtime.h>
#include "sigk_device.cuh"

namespace sigk {

struct KernelInfo {
    int rows_per_lane;   // R
    int smem_bytes;      // dynamic shared memory per CTA
    int threads;         // threads per CTA
    int blocks_per_sm;   // occupancy
};

// Rows per lane as a function of (P, D): fewer rows when the register
// footprint (R*(P + D) state floats) would push occupancy too low.  Four rows
// amortise the per-step shuffles, seam staging and control over four tiles:
// at P = 6, D = 16 (168 registers, three CTAs per SM) the 64-path Gram's
// forward took 12.2 ms against 13.8 ms with two rows at four CTAs per SM;
// at P = 12, D = 16 one row per lane at four CTAs per SM was slower than two
// (30.8 against 26.0 ms).
constexpr int rows_per_lane(int P, int D) { return ((P + D) <= 16 || (D == 16 && P <= 6)) ? 4 : 2; }
// The same for the training forward that stores the tile records (its
// per-row record state adds registers): two rows while that fits without
// spills, else one.  The records are laid out per work item and step, so a
// step's 32 * R records are one contiguous block whatever R is.
constexpr int rec_rows_per_lane(int P, int D) { return (P <= 10 && P + D <= 24) ? 2 : 1; }

// Entry points of the kernel translation units, one unit per (edge degree P,
// ring count NR); NR is a compile-time constant of every solver kernel, so
// the truncated ring sums carry no run-time predicates.
//
// variant 0: inference, or training (SolverArgs::store set: the seam after
// every 32-row strip is stored), rows_per_lane(P, D) rows per lane; variant
// 1: training that also stores every tile's record for the adjoint,
// rec_rows_per_lane(P, D) rows per lane.
template <int P, int NR> int fwd_info(int D, int variant, KernelInfo* info);
template <int P, int NR>
cudaError_t fwd_launch(int D, int variant, const SolverArgs& a, int grid, cudaStream_t s);

// Two-phase kernel (strip coefficients first, then the sweep): d > 16 in
// FP32, or any d in FP64 (f64 = true).  cscratch holds float or double strips.
template <int P, int NR> int fwd_cm_info(bool f64, KernelInfo* info);
template <int P, int NR>
cudaError_t fwd_cm_launch(bool f64, const SolverArgs& a, void* cscratch, int64_t cstride, int grid,
                          cudaStream_t s);

// Tensor-core solver for large d (increment Gram on tcgen05, float-float
// coefficients, FP32 sweep); one CTA per 128-row block.
struct TcArgs;
template <int P, int NR> int fwd_tc_info(KernelInfo* info);
template <int P, int NR> cudaError_t fwd_tc_launch(const TcArgs& a, int grid, cudaStream_t s);

// The adjoint kernel (any d): phase 0 coefficients, replay, reverse sweep,
// contraction to the increments; cs: per-warp strip areas of cstride floats.
struct BwdArgs;
template <int P, int NR> int bwd2_info(KernelInfo* info);
template <int P, int NR>
cudaError_t bwd2_launch(const BwdArgs& a, float* cs, int64_t cstride, int grid, cudaStream_t s);

}  // namespace sigk
