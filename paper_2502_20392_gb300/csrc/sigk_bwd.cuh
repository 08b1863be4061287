// sigk_bwd.cuh -- arguments of the reverse-mode (adjoint) sweep.
//
// The adjoint runs after a training forward that stored the right-edge seam
// after every 32-row strip (the checkpointed wavefront boundaries) and, when
// they fit the device memory budget, every tile's record (the row's incoming
// left edge and the exponent decisions, P + 2 floats).  One work item =
// (pair, strip of 32 rows, one row per lane), strips of a pair in DECREASING
// order (the schedule's k-th item of a pair is strip n_strips - 1 - k).  The
// kernel is bwd2_kernel (sigk_bwd2.cuh).
#pragma once
#include "sigk_device.cuh"

namespace sigk {

struct BwdArgs {
    const PairDesc* pairs;
    Schedule sched;              // item k of a pair is its strip n_strips - 1 - k
    int32_t n_pairs;
    int32_t inc_mode;
    int32_t d;
    int32_t nr;
    const float* store;          // forward seams, per pair (training forward)
    const int64_t* store_off;    // [n_pairs] float offsets into store
    const int32_t* pair_exp;     // [n_pairs] exponent of the final value
    const double* pair_w;        // [n_pairs] upstream weight of each pair
    float* rec;                  // per-warp records (replay)
    int64_t rec_stride;          // floats per warp
    // records stored by the training forward (SolverArgs::rec layout, items
    // of rec_rows strips); with rec_off != nullptr pass A is skipped
    const float* rec_store;
    const int64_t* rec_off;
    int32_t rec_rows;
    int32_t nslot;               // adjoint seam ring
    int32_t wcols;
    float* aseam;
    unsigned long long* prod;
    unsigned long long* cons;
    long long* done;
    int* item_counter;
    int* status;
    unsigned long long* counters;
    // extents, for the bounds checks of SIGK_DEBUG builds
    int64_t store_cap;           // floats of store
    int64_t rec_cap;             // floats of rec_store
    int64_t rec_total;           // floats of the per-warp replay records
};

}  // namespace sigk
