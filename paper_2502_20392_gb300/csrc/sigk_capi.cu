// sigk_capi.cu -- C-ABI of libsigk.so (declared in include/sigk.h).
//
// Host responsibilities: argument validation, workspace layout, choosing the
// kernel instantiation and grid, launching the device-side planner (which
// builds the pair table and strip counts from DEVICE length vectors, so no
// host synchronisation and no host lengths are needed), the persistent
// solver, and the FP64 reductions (Gram mirror, MMD^2).  The library never
// allocates device memory.
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>
#include <cmath>

#include <cuda_runtime.h>

#include "../../include/sigk.h"
#include "sigk_bwd.cuh"
#include "sigk_stats.cuh"
#include "sigk_device.cuh"
#include "sigk_fwd_tc.cuh"
#include "sigk_launch.h"

namespace sigk {

static thread_local std::string g_last_error;
static thread_local cudaEvent_t g_ev_start = nullptr;
static thread_local cudaEvent_t g_ev_stop = nullptr;

static sigk_status fail(sigk_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

static sigk_status cuda_fail(cudaError_t e, const char* where) {
    return fail(SIGK_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// options

struct Opts {
    int order;     // P (even, 4..16)
    int rings;     // nr
    int flags;
    int grid_ctas;
    int64_t max_len;
    float refine_c;  // 0: no refinement
    int wait_ms;     // bounded-wait budget
    float ring_tol;  // per-tile ring count (0: fixed)
};

static bool resolve_opts(const sigk_opts* o, Opts* r) {
    r->order = 8;
    r->rings = 4;
    r->flags = 0;
    r->grid_ctas = 0;
    r->max_len = 8193;
    r->refine_c = 0.0f;
    r->wait_ms = 4000;
    r->ring_tol = 0.0f;
    if (o) {
        if (o->order) r->order = o->order;
        if (o->rings) r->rings = o->rings;
        r->flags = o->flags;
        r->grid_ctas = o->grid_ctas;
        if (o->max_len > 0) r->max_len = o->max_len;
        r->refine_c = o->refine_c;
        if (o->wait_ms) r->wait_ms = o->wait_ms;
        r->ring_tol = o->ring_tol;
    }
    if (!(r->ring_tol >= 0.0f) || r->ring_tol > 1.0f) return false;
    if (r->wait_ms < 1 || r->wait_ms > 600000) return false;
    if (!(r->refine_c >= 0.0f) || r->refine_c > 1e30f) return false;
    if (r->order < 4 || r->order > kMaxP) return false;
    r->order += (r->order & 1);
    int nrmax = r->order < kMaxRings ? r->order : kMaxRings;
    if (r->rings < 1 || r->rings > nrmax) return false;
    // odd ring counts are compiled for the FP32 solvers; the FP64 solver,
    // which keeps the square truncation at any order, and a single ring
    // round up to even (nrmax is even)
    if ((r->flags & SIGK_FLAG_FP64) || r->rings < 2) r->rings += (r->rings & 1);
    // The FP32 solvers keep the tile-matrix entries of weighted degree
    // 2m + k <= 2 rings + 1 (keep_entry): no entry reaches an edge degree
    // above 2 rings, so a larger order would only carry zeros.  The FP64
    // solver keeps the whole square truncation of order P.
    if (!(r->flags & SIGK_FLAG_FP64) && r->order > 2 * r->rings) r->order = 2 * r->rings;
    if (r->grid_ctas < 0 || r->max_len > (int64_t)INT32_MAX) return false;
    return true;
}

// register-resident increments for d <= 16; larger d uses the two-phase
// kernel (bucket 0), up to kMaxDim
constexpr int kMaxDim = 8192;
static int dim_bucket(int d) {
    return d <= 4 ? 4 : (d <= 8 ? 8 : (d <= 16 ? 16 : (d <= kMaxDim ? 0 : -1)));
}

// (edge degree P, ring count NR) pairs compiled: P even in 4..16, NR even in
// 2..min(P, 8), and NR in {3, 5, 7} with NR <= P <= 2 NR (the FP32 solvers,
// which clamp P to 2 NR; the FP64 solver rounds odd ring counts up).
#define SIGK_DISPATCH_PNR(FN, ...)                  \
    switch (P * 16 + NR) {                          \
        case 66: return FN<4, 2>(__VA_ARGS__); \
        case 68: return FN<4, 4>(__VA_ARGS__); \
        case 98: return FN<6, 2>(__VA_ARGS__); \
        case 100: return FN<6, 4>(__VA_ARGS__); \
        case 102: return FN<6, 6>(__VA_ARGS__); \
        case 130: return FN<8, 2>(__VA_ARGS__); \
        case 132: return FN<8, 4>(__VA_ARGS__); \
        case 134: return FN<8, 6>(__VA_ARGS__); \
        case 136: return FN<8, 8>(__VA_ARGS__); \
        case 162: return FN<10, 2>(__VA_ARGS__); \
        case 164: return FN<10, 4>(__VA_ARGS__); \
        case 166: return FN<10, 6>(__VA_ARGS__); \
        case 168: return FN<10, 8>(__VA_ARGS__); \
        case 194: return FN<12, 2>(__VA_ARGS__); \
        case 196: return FN<12, 4>(__VA_ARGS__); \
        case 198: return FN<12, 6>(__VA_ARGS__); \
        case 200: return FN<12, 8>(__VA_ARGS__); \
        case 226: return FN<14, 2>(__VA_ARGS__); \
        case 228: return FN<14, 4>(__VA_ARGS__); \
        case 230: return FN<14, 6>(__VA_ARGS__); \
        case 232: return FN<14, 8>(__VA_ARGS__); \
        case 258: return FN<16, 2>(__VA_ARGS__); \
        case 260: return FN<16, 4>(__VA_ARGS__); \
        case 262: return FN<16, 6>(__VA_ARGS__); \
        case 264: return FN<16, 8>(__VA_ARGS__); \
        case 67: return FN<4, 3>(__VA_ARGS__); \
        case 99: return FN<6, 3>(__VA_ARGS__); \
        case 101: return FN<6, 5>(__VA_ARGS__); \
        case 133: return FN<8, 5>(__VA_ARGS__); \
        case 135: return FN<8, 7>(__VA_ARGS__); \
        case 165: return FN<10, 5>(__VA_ARGS__); \
        case 167: return FN<10, 7>(__VA_ARGS__); \
        case 199: return FN<12, 7>(__VA_ARGS__); \
        case 231: return FN<14, 7>(__VA_ARGS__); \
        default: break;                             \
    }

static int fwd_info_dispatch(int P, int NR, int D, int R, KernelInfo* info) {
    SIGK_DISPATCH_PNR(fwd_info, D, R, info)
    return -1;
}

static cudaError_t fwd_launch_dispatch(int P, int NR, int D, int R, const SolverArgs& a, int grid,
                                       cudaStream_t s) {
    SIGK_DISPATCH_PNR(fwd_launch, D, R, a, grid, s)
    return cudaErrorInvalidValue;
}

static int fwd_cm_info_dispatch(int P, int NR, bool f64, KernelInfo* info) {
    SIGK_DISPATCH_PNR(fwd_cm_info, f64, info)
    return -1;
}

static cudaError_t fwd_cm_launch_dispatch(int P, int NR, bool f64, const SolverArgs& a, void* cs,
                                          int64_t cstride, int grid, cudaStream_t s) {
    SIGK_DISPATCH_PNR(fwd_cm_launch, f64, a, cs, cstride, grid, s)
    return cudaErrorInvalidValue;
}

static int fwd_tc_info_dispatch(int P, int NR, KernelInfo* info) {
    SIGK_DISPATCH_PNR(fwd_tc_info, info)
    return -1;
}

static cudaError_t fwd_tc_launch_dispatch(int P, int NR, const TcArgs& a, int grid, cudaStream_t s) {
    SIGK_DISPATCH_PNR(fwd_tc_launch, a, grid, s)
    return cudaErrorInvalidValue;
}

static int bwd2_info_dispatch(int P, int NR, KernelInfo* info) {
    SIGK_DISPATCH_PNR(bwd2_info, info)
    return -1;
}

static cudaError_t bwd2_launch_dispatch(int P, int NR, const BwdArgs& a, float* cs, int64_t cstride,
                                        int grid, cudaStream_t s) {
    SIGK_DISPATCH_PNR(bwd2_launch, a, cs, cstride, grid, s)
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// workspace layout

struct Layout {
    size_t hdr, ox, oy, sx, sy, pairs, item_start, order, lvl, prod, cons, done, seam, gram, total;
    bool strip_major;    // the ring in use can hold whole strips: strip-major allowed
    // backward sections (train == true)
    size_t store, store_off, pair_exp, pair_w, rec, bprod, bcons, bdone, aseam, bcs;
    int64_t bcstride;
    int64_t store_floats, rec_stride;
    bool stored_rec;     // the training forward stores every tile's record
    int rec_rows;        // its rows per lane (records are grouped per item of that many strips)
    size_t rstore, rec_off;
    int64_t rstore_floats;
    int bnslot, bwcols, bgrid, bnwarps;
    KernelInfo binfo;
    bool train;
    bool cm;             // two-phase kernel (d > 16, or FP64)
    bool f64;            // FP64 solve (SIGK_FLAG_FP64)
    bool tc;             // tensor-core increment Gram (d > 16, FP32, d <= kTcMaxDim)
    int d_pad;           // its digit rows: d rounded up to 16
    int64_t n_slots;     // paths of the call (digit cache slots)
    size_t ycache, yexp, ablk, cst;  // its sections
    int64_t cst_stride;
    int strip_quantum;   // the pair table's strips per work unit (tc: 4)
    size_t elem;         // bytes per seam / strip element (4 or 8)
    size_t cscratch;     // its per-warp coefficient strips
    int64_t cstride;
    int64_t n_pairs, n_paths_x, n_paths_y;
    int nslot, wcols, grid, nwarps, rows_per_strip, stride;
    int fwd_shift;       // training: forward items are 2^fwd_shift table strips
    size_t item_start2, lvl2;
    int64_t nwords;
    KernelInfo info;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Strip-major schedule limits: strips per pair the level arrays hold, and the
// largest seam ring (bytes) it may take.
constexpr int kLevelCap = 4096;
constexpr double kStripMajorBudget = 8.0 * 1024 * 1024 * 1024;
constexpr int64_t kStripMajorMinPairs = 64;
// Largest store of tile records (bytes) the training forward may write for
// the adjoint; above it (or with SIGK_FLAG_REPLAY) the adjoint replays each
// strip from its seam instead.
constexpr double kRecordBudget = 128.0 * 1024 * 1024 * 1024;

// Number of pair entries solved by an op.
static int64_t pair_count(int op, int64_t n_x, int64_t n_y, int flags) {
    if (op == SIGK_OP_PAIRS) return n_x;
    if (op == SIGK_OP_GRAM) {
        if (n_y > 0) return n_x * n_y;
        return (flags & SIGK_FLAG_GRAM_FULL) ? n_x * n_x : n_x * (n_x + 1) / 2;
    }
    // MMD: Gram of the concatenated sample, upper triangle
    int64_t n = n_x + n_y;
    return n * (n + 1) / 2;
}

static sigk_status make_layout(int op, int64_t n_x, int64_t n_y, int d, const Opts& o, Layout* L,
                               bool train = false, bool allow_sm = true) {
    const int D = dim_bucket(d);
    if (D < 0) return fail(SIGK_ERR_UNSUPPORTED, "d must be in 1..8192");
    L->train = train;
    L->f64 = (o.flags & SIGK_FLAG_FP64) != 0;
    L->cm = (D == 0) || L->f64;
    L->elem = L->f64 ? sizeof(double) : sizeof(float);
    if (L->f64 && train)
        return fail(SIGK_ERR_UNSUPPORTED, "the backward runs in FP32 only (no SIGK_FLAG_FP64)");
    if (L->cm && train && d > kTcMaxDim)
        return fail(SIGK_ERR_UNSUPPORTED, "the backward supports d <= 1024");
    // stored tile records: (pair, 32-row strip) x (max_len + 32) blocks of
    // 32 records; the training forward then runs with one row per lane
    L->stored_rec = false;
    L->rec_rows = 1;
    L->rstore_floats = 0;
    if (train && !(o.flags & SIGK_FLAG_REPLAY) && !L->cm) {
        // (pair, item of R strips) x (max_len + 32) blocks of 32 R records
        // (d > 16: the two-phase training forward keeps the seams only)
        const int R = rec_rows_per_lane(o.order, D);
        const int64_t items = ((o.max_len + 31) / 32 + R - 1) / R;
        const double fl = (double)pair_count(op, n_x, n_y, o.flags) * (double)items *
                          (double)(o.max_len + 32) * 32.0 * R * (double)rec_floats(o.order);
        if (fl * sizeof(float) <= kRecordBudget) {
            L->stored_rec = true;
            L->rec_rows = R;
            L->rstore_floats = (int64_t)fl;
        }
    }
    L->tc = L->cm && !L->f64 && !train && d <= kTcMaxDim && !(o.flags & SIGK_FLAG_NO_TENSOR);
    L->d_pad = (d + kTcK - 1) / kTcK * kTcK;
    L->strip_quantum = L->tc ? 4 : 1;
    const int qinfo = L->tc ? fwd_tc_info_dispatch(o.order, o.rings, &L->info)
                      : L->cm ? fwd_cm_info_dispatch(o.order, o.rings, L->f64, &L->info)
                            : fwd_info_dispatch(o.order, o.rings, D, L->stored_rec ? 1 : 0, &L->info);
    if (qinfo != 0 || L->info.blocks_per_sm <= 0)
        return fail(SIGK_ERR_CUDA, "kernel occupancy query failed");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return fail(SIGK_ERR_CUDA, "cannot query SM count");
    const int full_grid = sms * L->info.blocks_per_sm;
    L->grid = o.grid_ctas > 0 ? (o.grid_ctas < full_grid ? o.grid_ctas : full_grid) : full_grid;
    L->nwarps = L->grid * (L->info.threads / 32);
    if (L->tc) allow_sm = false;  // blocks of four consecutive strips: pair-major schedules only
    // the pair table counts strips of 32 * R rows; in training it counts
    // 32-row strips (the adjoint's unit) and the forward takes R of them
    L->rows_per_strip = train ? 32 : 32 * L->info.rows_per_lane;
    L->fwd_shift = 0;
    if (train)
        for (int r = L->info.rows_per_lane; r > 1; r >>= 1) ++L->fwd_shift;
    L->stride = o.order + 4;
    L->n_pairs = pair_count(op, n_x, n_y, o.flags);
    // Seam ring, pair-major: nslot > concurrent warps; wcols large enough that
    // the warps in flight can always hold a whole sweep between them (nwarps *
    // wcols >= 2 * max_len), so a producer never waits on a consumer that
    // cannot start.  Strip-major (when the ring fits the budget): a slot holds
    // a whole strip (wcols >= max_len, no flow control) and nslot covers the
    // producer-consumer distance (<= n_pairs items) plus the warps in flight,
    // so a slot is reused only after an item at least nwarps earlier is done.
    const int64_t wfull = (o.max_len + 31) & ~(int64_t)31;
    const int64_t nslot_sm = L->n_pairs + L->nwarps + 64;
    // strip-major needs many pairs (a producer is one level, i.e. the pairs
    // with more strips, ahead of its consumer); with few pairs it only costs
    // ring memory
    if ((o.flags & SIGK_FLAG_PAIR_MAJOR) || pair_count(op, n_x, n_y, o.flags) < kStripMajorMinPairs)
        allow_sm = false;
    L->strip_major = allow_sm && !train && nslot_sm <= (int64_t)INT32_MAX / 2 &&
                     (double)nslot_sm * (double)wfull * (double)L->stride * (double)L->elem <=
                         kStripMajorBudget;
    L->nslot = L->strip_major ? (int)nslot_sm : L->nwarps + 64;
    // training: one progress word per work item (seams are not reused)
    L->nwords = L->nslot;
    if (train) {
        const int64_t items = (int64_t)pair_count(op, n_x, n_y, o.flags) *
                              ((o.max_len + L->rows_per_strip - 1) / L->rows_per_strip);
        if (items > L->nwords) L->nwords = items;
    }
    int64_t w = 2 * o.max_len / L->nwarps + 64;
    if (w < 256) w = 256;
    if (w > o.max_len) w = o.max_len;
    w = (w + 31) & ~(int64_t)31;
    if (w < 32) w = 32;
    // the tensor-core solver's producer runs ahead of its sweeps, so its
    // seam slots hold whole strips (no flow control between strips)
    if (L->strip_major || L->tc) w = wfull < 32 ? 32 : wfull;
    L->wcols = (int)w;
    L->n_paths_x = n_x;
    L->n_paths_y = (op == SIGK_OP_GRAM && n_y == 0) ? 0 : n_y;
    size_t off = 0;
    L->hdr = off; off = align256(off + 256);
    L->ox = off; off = align256(off + sizeof(int64_t) * (size_t)(n_x + 1));
    L->oy = off; off = align256(off + sizeof(int64_t) * (size_t)(n_y + 1));
    L->sx = off; off = align256(off + sizeof(int32_t) * (size_t)(n_x + 1));
    L->sy = off; off = align256(off + sizeof(int32_t) * (size_t)(n_y + 1));
    L->pairs = off; off = align256(off + sizeof(PairDesc) * (size_t)L->n_pairs);
    L->item_start = off; off = align256(off + sizeof(int32_t) * (size_t)(L->n_pairs + 1));
    L->order = off; off = align256(off + sizeof(int32_t) * (size_t)(L->n_pairs + 1));
    L->item_start2 = off; off = align256(off + sizeof(int32_t) * (size_t)(L->n_pairs + 1));
    L->lvl2 = off; off = align256(off + sizeof(int32_t) * (size_t)(kLevelCap + 2));
    L->lvl = off; off = align256(off + sizeof(int32_t) * 2 * (size_t)(kLevelCap + 2));
    L->prod = off; off = align256(off + sizeof(unsigned long long) * (size_t)L->nwords);
    L->cons = off; off = align256(off + sizeof(unsigned long long) * (size_t)L->nwords);
    L->done = off; off = align256(off + sizeof(long long) * (size_t)L->nwords);
    L->seam = off; off = align256(off + L->elem * (size_t)L->nslot * L->wcols * L->stride);
    L->gram = off;
    if (op == SIGK_OP_MMD) off = align256(off + sizeof(double) * (size_t)(n_x + n_y) * (n_x + n_y));
    L->cstride = 0;
    L->cscratch = off;
    L->n_slots = n_x + L->n_paths_y;
    L->cst_stride = 0;
    L->ycache = L->yexp = L->ablk = L->cst = off;
    if (L->tc) {
        // digits of every path's first max_len segments (a tiled matrix of
        // whole 64-row chunks per path), exponents; per CTA the digits of a
        // block's rows and the skewed (c, clo) of its strips
        L->ycache = off;
        off = align256(off + sizeof(uint16_t) * (size_t)L->n_slots * (size_t)tc_cache_rows(o.max_len) *
                                 kTcDigits * L->d_pad);
        L->yexp = off; off = align256(off + sizeof(int32_t) * (size_t)L->n_slots * o.max_len);
        const size_t ctas = (size_t)L->grid;
        L->ablk = off; off = align256(off + sizeof(uint16_t) * ctas * kTcDigits * kTcRows * L->d_pad);
        L->cst_stride = (o.max_len + 32 + kTcPF) * 32;
        L->cst = off; off = align256(off + sizeof(float2) * ctas * kTcSlots * 4 * L->cst_stride);
    } else if (L->cm) {  // one [max_len][32] coefficient strip per warp
        L->cstride = 32 * ((o.max_len + 31) & ~(int64_t)31);
        off = align256(off + L->elem * (size_t)L->nwarps * L->cstride);
    }
    if (train) {
        if (bwd2_info_dispatch(o.order, o.rings, &L->binfo) != 0 || L->binfo.blocks_per_sm <= 0)
            return fail(SIGK_ERR_CUDA, "backward occupancy query failed");
        L->bgrid = sms * L->binfo.blocks_per_sm;
        if (o.grid_ctas > 0 && o.grid_ctas < L->bgrid) L->bgrid = o.grid_ctas;
        L->bnwarps = L->bgrid * (L->binfo.threads / 32);
        const int64_t bnslot_sm = L->n_pairs + L->bnwarps + 64;
        L->strip_major = allow_sm && bnslot_sm <= (int64_t)INT32_MAX / 2 &&
                         (double)bnslot_sm * (double)wfull * (double)adj_seam_floats(o.order) * 4.0 <=
                             kStripMajorBudget;
        L->bnslot = L->strip_major ? (int)bnslot_sm : L->bnwarps + 64;
        int64_t bw = 2 * o.max_len / L->bnwarps + 64;
        if (bw < 256) bw = 256;
        if (bw > o.max_len) bw = o.max_len;
        bw = (bw + 31) & ~(int64_t)31;
        if (bw < 32) bw = 32;
        if (L->strip_major) bw = wfull < 32 ? 32 : wfull;
        L->bwcols = (int)bw;
        // forward seams of every strip boundary: (strips - 1) x swept columns
        const int64_t strips = (o.max_len + 31) / 32;
        L->store_floats = L->n_pairs * (strips > 1 ? strips - 1 : 0) * o.max_len * L->stride;
        L->rec_stride = (o.max_len + 31) * (int64_t)rec_floats(o.order) * 32;
        L->store = off; off = align256(off + sizeof(float) * (size_t)L->store_floats);
        L->store_off = off; off = align256(off + sizeof(int64_t) * (size_t)L->n_pairs);
        L->pair_exp = off; off = align256(off + sizeof(int32_t) * (size_t)L->n_pairs);
        L->pair_w = off; off = align256(off + sizeof(double) * (size_t)L->n_pairs);
        L->rec = off;
        if (!L->stored_rec) off = align256(off + sizeof(float) * (size_t)L->bnwarps * L->rec_stride);
        L->rec_off = off; off = align256(off + sizeof(int64_t) * (size_t)L->n_pairs);
        L->rstore = off; off = align256(off + sizeof(float) * (size_t)L->rstore_floats);
        L->bprod = off; off = align256(off + sizeof(unsigned long long) * (size_t)L->bnslot);
        L->bcons = off; off = align256(off + sizeof(unsigned long long) * (size_t)L->bnslot);
        L->bdone = off; off = align256(off + sizeof(long long) * (size_t)L->bnslot);
        L->aseam = off;
        off = align256(off + sizeof(float) * (size_t)L->bnslot * L->bwcols * adj_seam_floats(o.order));
        // per adjoint warp: its strip's coefficients, then g, skewed
        L->bcstride = (o.max_len + 32 + kB2PF) * 32;
        L->bcs = off;
        off = align256(off + sizeof(float) * (size_t)L->bnwarps * L->bcstride);
    }
    L->total = off;
    return SIGK_OK;
}

// Header of the workspace (first 256 bytes).
struct Header {
    int status;
    int item_counter;
    int bwd_item_counter;
    int nonfinite;      // a non-finite output was met (record_nonfinite writes status + 3)
    unsigned long long counters[4];
    int sched[4];  // schedule: mode, n_levels, n_items (Schedule::hdr)
    int sched2[4];  // training forward's schedule (items of 2^fwd_shift strips)
    long long train_sig;  // signature of the training forward whose state the workspace holds (0: none)
    unsigned ring_hist[4];  // tiles solved with <= 2, 3-4, 5-6, 7-8 rings (adaptive forwards)
    int pad2[6];
    long long diag[3];  // first timed-out wait: address, target, value seen (byte 128)
    long long wait_ns;  // budget of the bounded waits of the current launch (byte 152)
};
static_assert(offsetof(Header, diag) == 128, "record_timeout writes the diagnosis at byte 128");
static_assert(offsetof(Header, wait_ns) == kHdrWaitNs, "wait_budget reads the budget at kHdrWaitNs");
static_assert(offsetof(Header, nonfinite) == 3 * sizeof(int), "record_nonfinite writes status + 3");
static_assert(sizeof(Header) <= 256, "the header occupies the first 256 bytes of the workspace");

// ---------------------------------------------------------------------------
// device-side planner: one CTA builds prefix offsets, the pair table and the
// strip counts, and resets the seam synchronisation words.

struct PlanArgs {
    int op;
    int flags;
    int inc_mode;
    int d;
    const float* X;
    const int64_t* len_x;
    int64_t n_x;
    const float* Y;
    const int64_t* len_y;
    int64_t n_y;        // 0: Gram of X with itself
    int64_t max_len;
    int rows_per_strip;
    int strip_quantum;  // strip counts are rounded up to a multiple of this (>= 1)
    int64_t n_pairs;
    int64_t* ox;
    int64_t* oy;
    const int32_t* sX;  // per-path refinement factors (null: 1)
    const int32_t* sY;
    PairDesc* pairs;
    int32_t* item_start;
    int32_t* order;     // strip-major schedule: pairs by decreasing strip count
    int32_t* lvl;       // level starts [lvl_cap + 2], then a scratch of the same size
    int lvl_cap;        // largest strip count the level arrays hold
    int allow_sm;       // strip-major allowed (the seam ring holds whole strips)
    int fwd_shift;      // training: the forward solves 2^fwd_shift strips per item
    int32_t* item_start2;  // training forward's item starts [pairs + 1]
    int32_t* lvl2;         // training forward's level starts
    unsigned long long* prod;
    unsigned long long* cons;
    long long* done;
    int nslot;
    Header* hdr;
    double* out;        // output (k values / Gram)
    int64_t out_ld;     // leading dimension of the Gram output
    // training (backward) extras; train == 0 leaves them unused
    int phase;          // 1: prefix sums; 2: pair table, items, resets; 3: both
    long long wait_ns;  // budget of the bounded waits (written to the header)
    int train;
    int stride;         // seam entry floats (P + 4)
    int64_t store_cap;  // floats available for the forward seam store
    int64_t* store_off;
    int64_t* rec_off;   // stored tile records: per-pair offsets (null: replay)
    int64_t rec_cap;    // floats available for them
    int rec_rows;       // rows per lane of the forward that writes them
    int rec_block;      // floats per block (32 * rec_rows records)
    long long train_sig;  // training: signature recorded once the plan succeeded
    double* pair_w;
    const double* grad_out;
    float* gX;
    float* gY;
    unsigned long long* bprod;
    unsigned long long* bcons;
    long long* bdone;
    int bnslot;
};

constexpr int kPlanThreads = 1024;

// Exclusive prefix sum of v[0..n) (int64) into out[0..n], one CTA.
__device__ void block_exclusive_scan(const int64_t* v, int64_t n, int64_t* out, int64_t* sh,
                                     bool segments, int inc_mode, int* bad) {
    const int t = threadIdx.x;
    const int64_t chunk = (n + kPlanThreads - 1) / kPlanThreads;
    const int64_t b0 = t * chunk, b1 = (b0 + chunk < n) ? b0 + chunk : n;
    int64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) {
        int64_t x = v[i];
        if (segments) {
            int64_t mn = inc_mode ? 0 : 1;
            if (x < mn || x > (int64_t)INT32_MAX) atomicExch(bad, 1);
        }
        s += x;
    }
    sh[t] = s;
    __syncthreads();
    for (int o = 1; o < kPlanThreads; o <<= 1) {
        int64_t add = (t >= o) ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    int64_t run = sh[t] - s;
    for (int64_t i = b0; i < b1; ++i) {
        out[i] = run;
        run += v[i];
    }
    if (t == kPlanThreads - 1) out[n] = sh[t];
    __syncthreads();
}

// Exclusive prefix over n pairs (pair i = order[i], or i when order is
// null) of their items, ceil(n_strips / 2^shift), into out[0..n]; one CTA.
__device__ void block_prefix_items(const PairDesc* pairs, const int32_t* order, int64_t n,
                                   int shift, int32_t* out, int64_t* sh) {
    const int t = threadIdx.x;
    const int64_t chunk = (n + kPlanThreads - 1) / kPlanThreads;
    const int64_t b0 = t * chunk, b1 = (b0 + chunk < n) ? b0 + chunk : n;
    auto units = [&](int64_t i) -> int64_t {
        const int ns = pairs[order ? order[i] : i].n_strips;
        return (ns + (1 << shift) - 1) >> shift;
    };
    int64_t sum = 0;
    for (int64_t i = b0; i < b1; ++i) sum += units(i);
    sh[t] = sum;
    __syncthreads();
    for (int o = 1; o < kPlanThreads; o <<= 1) {
        int64_t add = (t >= o) ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    int64_t run = sh[t] - sum;
    for (int64_t i = b0; i < b1; ++i) {
        out[i] = (int32_t)run;
        run += units(i);
    }
    if (t == kPlanThreads - 1) out[n] = (int32_t)sh[t];
    __syncthreads();
}

// Per-pair offsets out[i] = sum_{i' < i} sz(pairs[i']) by a block scan; sets
// SIGK_ERR_WORKSPACE when the total exceeds cap.  One CTA of kPlanThreads.
template <typename F>
__device__ void pair_offsets(const PlanArgs& A, int64_t* sh, int64_t* out, int64_t cap, F sz) {
    const int t = threadIdx.x;
    const int64_t n = A.n_pairs;
    const int64_t chunk = (n + kPlanThreads - 1) / kPlanThreads;
    const int64_t b0 = t * chunk, b1 = (b0 + chunk < n) ? b0 + chunk : n;
    int64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += sz(A.pairs[i]);
    sh[t] = s;
    __syncthreads();
    for (int o = 1; o < kPlanThreads; o <<= 1) {
        int64_t add = (t >= o) ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    int64_t run = sh[t] - s;
    for (int64_t i = b0; i < b1; ++i) {
        out[i] = run;
        run += sz(A.pairs[i]);
    }
    if (t == kPlanThreads - 1 && sh[t] > cap) atomicCAS(&A.hdr->status, 0, kErrWorkspace);
    __syncthreads();
}

// Pair p of the op -> the paths (a, b) it couples and its output entries
// o0, o1 (o1 >= 0: the mirrored entry of a symmetric Gram).  nz: paths of
// the square matrix (MMD: both samples; Gram: n_x).
__device__ void pair_index(const PlanArgs& A, bool self, int64_t p, int64_t& a, int64_t& b,
                           int64_t& o0, int64_t& o1) {
    const int64_t nx = A.n_x;
    const int64_t nz = (A.op == SIGK_OP_MMD) ? A.n_x + A.n_y : (self ? nx : A.n_y);
    const bool tri = (A.op == SIGK_OP_MMD) || (self && !(A.flags & SIGK_FLAG_GRAM_FULL));
    o0 = -1;
    o1 = -1;
    if (A.op == SIGK_OP_PAIRS) {
        a = p; b = p; o0 = p;
    } else if (tri) {
        // p -> (a, b), a <= b, row-major upper triangle of an nz x nz matrix
        const int64_t n = nz;
        double disc = (double)(2 * n + 1) * (double)(2 * n + 1) - 8.0 * (double)p;
        int64_t aa = (int64_t)(((double)(2 * n + 1) - sqrt(disc)) * 0.5);
        if (aa < 0) aa = 0;
        while (aa > 0 && aa * n - aa * (aa - 1) / 2 > p) --aa;
        while ((aa + 1) * n - (aa + 1) * aa / 2 <= p) ++aa;
        a = aa;
        b = p - (aa * n - aa * (aa - 1) / 2) + aa;
        o0 = a * A.out_ld + b;
        o1 = (a != b) ? b * A.out_ld + a : -1;
    } else {
        const int64_t ny = self ? nx : A.n_y;
        a = p / ny; b = p % ny;
        o0 = a * A.out_ld + b;
    }
}

// Path z of the pair table's side: (from Y?, index within X or Y).  MMD
// numbers X then Y; a Gram of X with itself takes both sides from X.
__device__ __forceinline__ void pair_side(const PlanArgs& A, bool self, int64_t z, bool second,
                                          bool* from_y, int64_t* idx) {
    if (A.op == SIGK_OP_MMD) {
        *from_y = z >= A.n_x;
        *idx = z < A.n_x ? z : z - A.n_x;
    } else {
        *from_y = second && !(A.op == SIGK_OP_GRAM && self);
        *idx = z;
    }
}

__global__ void __launch_bounds__(kPlanThreads) plan_kernel(PlanArgs A) {
    __shared__ int64_t sh[kPlanThreads];
    __shared__ int bad;
    __shared__ int max_strips;
    const int t = threadIdx.x;
    const bool self = (A.op == SIGK_OP_GRAM && A.n_y == 0);
    if (A.phase & 1) {
        if (t == 0) {
            bad = 0;
            A.hdr->status = 0;  // errors are reported per call
            A.hdr->nonfinite = 0;
            A.hdr->train_sig = 0;  // no training state until this plan succeeds
            A.hdr->wait_ns = A.wait_ns;
        }
        __syncthreads();
        block_exclusive_scan(A.len_x, A.n_x, A.ox, sh, true, A.inc_mode, &bad);
        if (!self) block_exclusive_scan(A.len_y, A.n_y, A.oy, sh, true, A.inc_mode, &bad);
        __syncthreads();
        if (bad) {
            if (t == 0) atomicCAS(&A.hdr->status, 0, kErrLength);
            return;
        }
    }
    if (!(A.phase & 2)) return;
    if (ld_volatile_s32(&A.hdr->status) != 0) return;
    const int RS = A.rows_per_strip;
    // pair table (the adjoint's upstream weights and gradient pointers are
    // set later, by adjoint_prep_kernel)
    for (int64_t p = t; p < A.n_pairs; p += kPlanThreads) {
        int64_t a, b, o0, o1;
        pair_index(A, self, p, a, b, o0, o1);
        // resolve path pointers and segment counts
        const float* pa;
        const float* pb;
        int64_t la, lb;
        int32_t ra = 1, rb = 1;
        int32_t slot_a = 0, slot_b = 0;
        auto path = [&](int64_t z, bool second, const float** ptr, int64_t* segs, int32_t* rf) {
            bool from_y;
            int64_t i;
            pair_side(A, self, z, second, &from_y, &i);
            (second ? slot_b : slot_a) = (int32_t)(from_y ? A.n_x + i : i);
            const float* base = from_y ? A.Y : A.X;
            const int64_t* off = from_y ? A.oy : A.ox;
            const int64_t* len = from_y ? A.len_y : A.len_x;
            const int32_t* sf = from_y ? A.sY : A.sX;
            *ptr = base + off[i] * A.d;
            *rf = sf ? sf[i] : 1;
            *segs = (A.inc_mode ? len[i] : len[i] - 1) * (int64_t)(*rf);
        };
        path(a, false, &pa, &la, &ra);
        path(b, true, &pb, &lb, &rb);
        PairDesc pd;
        pd.out0 = o0;
        pd.out1 = o1;
        // orientation: rows = the path that minimises padded work
        // ceil(rows/RS)*RS*(cols + 31), subject to cols <= max_len
        const int64_t RQ = (int64_t)RS * (A.strip_quantum > 1 ? A.strip_quantum : 1);
        const int64_t cost_ab = ((la + RQ - 1) / RQ) * RQ * (lb + 31);
        const int64_t cost_ba = ((lb + RQ - 1) / RQ) * RQ * (la + 31);
        bool swap = cost_ba < cost_ab;
        if (swap && la > A.max_len) swap = false;
        if (!swap && lb > A.max_len) swap = true;
        if ((swap ? la : lb) > A.max_len) atomicCAS(&A.hdr->status, 0, kErrLength);
        pd.xr = swap ? pb : pa;
        pd.yr = swap ? pa : pb;
        pd.gxr = nullptr;
        pd.gyr = nullptr;
        pd.sx = swap ? rb : ra;
        pd.sy = swap ? ra : rb;
        pd.xslot = swap ? slot_b : slot_a;
        pd.yslot = swap ? slot_a : slot_b;
        if (la > (int64_t)INT32_MAX || lb > (int64_t)INT32_MAX) atomicCAS(&A.hdr->status, 0, kErrLength);
        pd.L1 = (int32_t)(swap ? lb : la);
        pd.L2 = (int32_t)(swap ? la : lb);
        pd.swapped = swap ? 1 : 0;
        if (pd.L1 == 0 || pd.L2 == 0) {
            pd.n_strips = 0;
            if (o0 >= 0) A.out[o0] = 1.0;  // a one-point path: k = 1
            if (o1 >= 0) A.out[o1] = 1.0;
        } else {
            const int q = A.strip_quantum > 1 ? A.strip_quantum : 1;
            pd.n_strips = ((pd.L1 + RS - 1) / RS + q - 1) / q * q;
        }
        A.pairs[p] = pd;
    }
    __syncthreads();
    // item_start = exclusive prefix of n_strips (int32 result, int64 scan)
    {
        const int64_t n = A.n_pairs;
        const int64_t chunk = (n + kPlanThreads - 1) / kPlanThreads;
        const int64_t b0 = t * chunk, b1 = (b0 + chunk < n) ? b0 + chunk : n;
        int64_t s = 0;
        for (int64_t i = b0; i < b1; ++i) s += A.pairs[i].n_strips;
        sh[t] = s;
        __syncthreads();
        for (int o = 1; o < kPlanThreads; o <<= 1) {
            int64_t add = (t >= o) ? sh[t - o] : 0;
            __syncthreads();
            sh[t] += add;
            __syncthreads();
        }
        int64_t run = sh[t] - s;
        for (int64_t i = b0; i < b1; ++i) {
            A.item_start[i] = (int32_t)run;
            run += A.pairs[i].n_strips;
        }
        if (t == kPlanThreads - 1) {
            if (sh[t] > (int64_t)INT32_MAX) atomicCAS(&A.hdr->status, 0, kErrLength);
            // training: one progress word per item
            if (A.train && sh[t] > (int64_t)A.nslot) atomicCAS(&A.hdr->status, 0, kErrWorkspace);
            A.item_start[n] = (int32_t)sh[t];
        }
    }
    // schedule.  With at most lvl_cap strips per pair the pairs are sorted by
    // decreasing strip count (counting sort).  Strip-major (mode 1) when it is
    // allowed and the strip counts are even (the longest pair has at most
    // twice the mean): level l holds strip l of every pair that has one.
    // Otherwise pair-major over the sorted pairs (mode 2): the pairs with the
    // longest chains of strips start first.  Beyond lvl_cap: pair-major in
    // index order (mode 0).
    if (t == 0) max_strips = 0;
    __syncthreads();
    {
        int mx = 0;
        for (int64_t p = t; p < A.n_pairs; p += kPlanThreads) mx = max(mx, A.pairs[p].n_strips);
        atomicMax(&max_strips, mx);
    }
    __syncthreads();
    const int ms = max_strips;
    if (ms > 0 && ms <= A.lvl_cap) {
        int32_t* lvl = A.lvl;
        int32_t* cur = A.lvl + A.lvl_cap + 2;
        for (int i = t; i <= ms + 1; i += kPlanThreads) cur[i] = 0;
        __syncthreads();
        for (int64_t p = t; p < A.n_pairs; p += kPlanThreads) {
            const int n = A.pairs[p].n_strips;
            if (n > 0) atomicAdd(&cur[n], 1);
        }
        __syncthreads();
        if (t == 0) {
            int above = 0;  // cur[n] := pairs with more than n strips
            for (int n = ms; n >= 0; --n) {
                const int h = cur[n];
                cur[n] = above;
                above += h;
            }
            int run = 0;
            for (int l = 0; l < ms; ++l) {
                lvl[l] = run;
                run += cur[l];
            }
            lvl[ms] = run;
            const int active = cur[0];  // pairs with at least one strip
            const bool even = (int64_t)ms * active <= 2 * (int64_t)run;
            A.hdr->sched[0] = (A.allow_sm && even) ? 1 : 2;
            A.hdr->sched[1] = (A.allow_sm && even) ? ms : active;
            A.hdr->sched[2] = run;
        }
        __syncthreads();
        for (int64_t p = t; p < A.n_pairs; p += kPlanThreads) {
            const int n = A.pairs[p].n_strips;
            if (n > 0) A.order[atomicAdd(&cur[n], 1)] = (int32_t)p;
        }
        __syncthreads();
        if (A.hdr->sched[0] == 2)  // item_start over the sorted pairs
            block_prefix_items(A.pairs, A.order, A.hdr->sched[1], 0, A.item_start, sh);
    } else if (t == 0) {
        A.hdr->sched[0] = 0;
        A.hdr->sched[1] = 0;
        A.hdr->sched[2] = A.item_start[A.n_pairs];
    }
    __syncthreads();
    // training: the forward's own schedule in items of 2^fwd_shift strips,
    // same mode and pair order (the adjoint keeps the 32-row schedule)
    if (A.train) {
        const int sh2 = A.fwd_shift;
        const int mode = A.hdr->sched[0];
        if (mode == 1) {
            if (t == 0) {
                const int n2 = (ms + (1 << sh2) - 1) >> sh2;
                int run = 0;
                for (int l = 0; l < n2; ++l) {
                    A.lvl2[l] = run;
                    const int n = l << sh2;  // pairs with more than n strips
                    run += A.lvl[n + 1] - A.lvl[n];
                }
                A.lvl2[n2] = run;
                A.hdr->sched2[0] = 1;
                A.hdr->sched2[1] = n2;
                A.hdr->sched2[2] = run;
            }
        } else {
            const int64_t n = mode == 2 ? A.hdr->sched[1] : A.n_pairs;
            block_prefix_items(A.pairs, mode == 2 ? A.order : nullptr, n, sh2, A.item_start2, sh);
            if (t == 0) {
                A.hdr->sched2[0] = mode;
                A.hdr->sched2[1] = mode == 2 ? A.hdr->sched[1] : 0;
                A.hdr->sched2[2] = A.item_start2[n];
            }
        }
    }
    __syncthreads();
    // reset the seam synchronisation words and the work counter
    for (int i = t; i < A.nslot; i += kPlanThreads) {
        A.prod[i] = 0ull;
        A.cons[i] = 0ull;
        A.done[i] = -1ll;
    }
    if (t == 0) {
        A.hdr->item_counter = 0;
        A.hdr->bwd_item_counter = 0;
        A.hdr->counters[0] = 0;
        A.hdr->counters[1] = 0;
        A.hdr->counters[2] = 0;
        A.hdr->counters[3] = 0;
        for (int q = 0; q < 4; ++q) A.hdr->ring_hist[q] = 0u;
    }
    if (!A.train) return;
    // per-pair offsets of the forward seam store: (strips - 1) x L2 x stride
    __syncthreads();
    pair_offsets(A, sh, A.store_off, A.store_cap, [&](const PairDesc& q) -> int64_t {
        return q.n_strips > 1 ? (int64_t)(q.n_strips - 1) * q.L2 * A.stride : 0;
    });
    // and of the stored tile records: items of rec_rows strips x (L2 + 32)
    // blocks
    if (A.rec_off) {
        __syncthreads();
        pair_offsets(A, sh, A.rec_off, A.rec_cap, [&](const PairDesc& q) -> int64_t {
            return (int64_t)((q.n_strips + A.rec_rows - 1) / A.rec_rows) * (q.L2 + 32) * A.rec_block;
        });
    }
    __syncthreads();
    if (t == 0 && ld_volatile_s32(&A.hdr->status) == 0) A.hdr->train_sig = A.train_sig;
}

// Adjoint set-up, run before every adjoint launch on a workspace that holds
// a training forward: the upstream weight of every pair's k value (from
// grad_out), the gradient pointers of the pair table, zeroed gradient outputs
// (accumulated with atomics) and reset adjoint synchronisation words.  A
// grid-stride kernel; block 0 resets the counters.
__global__ void adjoint_prep_kernel(PlanArgs A) {
    const bool self = (A.op == SIGK_OP_GRAM && A.n_y == 0);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    // the workspace must hold a successful training forward of this call's
    // op, sizes and options; otherwise touch nothing (the adjoint kernel then
    // sees the error status and exits before reading the workspace)
    if (A.train_sig == 0 || *(volatile long long*)&A.hdr->train_sig != A.train_sig) {
        if (tid == 0) atomicCAS(&A.hdr->status, 0, kErrArg);
        return;
    }
    if (tid == 0) {
        A.hdr->bwd_item_counter = 0;
        A.hdr->counters[2] = 0;
        A.hdr->counters[3] = 0;
        A.hdr->wait_ns = A.wait_ns;
    }
    for (int64_t p = tid; p < A.n_pairs; p += nth) {
        int64_t a, b, o0, o1;
        pair_index(A, self, p, a, b, o0, o1);
        double w = 0.0;
        if (A.op == SIGK_OP_PAIRS) {
            w = A.grad_out[p];
        } else if (A.op == SIGK_OP_GRAM) {
            w = A.grad_out[o0];
            if (o1 >= 0) w += A.grad_out[o1];
        } else {  // MMD^2 = mean k(x,x') + mean k(y,y') - 2 mean k(x,y)
            const int64_t m = A.n_x, n = A.n_y;
            const bool unb = !(A.flags & SIGK_FLAG_MMD_BIASED);
            double cf;
            if (a < m && b < m) {
                cf = (a == b) ? (unb ? 0.0 : 1.0 / ((double)m * m))
                              : (unb ? 2.0 / ((double)m * (m - 1)) : 2.0 / ((double)m * m));
            } else if (a >= m && b >= m) {
                cf = (a == b) ? (unb ? 0.0 : 1.0 / ((double)n * n))
                              : (unb ? 2.0 / ((double)n * (n - 1)) : 2.0 / ((double)n * n));
            } else {
                cf = -2.0 / ((double)m * n);
            }
            w = A.grad_out[0] * cf;
        }
        A.pair_w[p] = w;
        auto grad = [&](int64_t z, bool second) -> float* {
            bool from_y;
            int64_t i;
            pair_side(A, self, z, second, &from_y, &i);
            float* g = from_y ? A.gY : A.gX;
            return g ? g + (from_y ? A.oy : A.ox)[i] * A.d : nullptr;
        };
        float* ga = grad(a, false);
        float* gb = grad(b, true);
        PairDesc& pd = A.pairs[p];
        pd.gxr = pd.swapped ? gb : ga;
        pd.gyr = pd.swapped ? ga : gb;
    }
    if (A.gX) {
        const int64_t nxf = (int64_t)A.ox[A.n_x] * A.d;
        for (int64_t i = tid; i < nxf; i += nth) A.gX[i] = 0.0f;
    }
    if (A.gY && !self) {
        const int64_t nyf = (int64_t)A.oy[A.n_y] * A.d;
        for (int64_t i = tid; i < nyf; i += nth) A.gY[i] = 0.0f;
    }
    for (int64_t i = tid; i < A.bnslot; i += nth) {
        A.bprod[i] = 0ull;
        A.bcons[i] = 0ull;
        A.bdone[i] = -1ll;
    }
}

// Per-path refinement factors: s = the power of two >= max_i |dz_i| /
// sqrt(refine_c), clamped to [1, 64]; one warp per path.  The planner multiplies the path's
// segment count by s and the kernels read segment v / s scaled by 1/s.
__global__ void refine_kernel(const float* Z, const int64_t* len, const int64_t* offs, int64_t n,
                              int d, int inc_mode, float refine_c, int32_t* s_out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n; p += warps) {
        const int64_t off = offs[p];
        const int64_t segs = inc_mode ? len[p] : len[p] - 1;
        const float* z = Z + off * d;
        float mx = 0.0f;
        for (int64_t i = lane; i < segs; i += 32) {
            float n2 = 0.0f;
            for (int e = 0; e < d; ++e) {
                const float v = inc_mode ? z[i * d + e] : z[(i + 1) * d + e] - z[i * d + e];
                n2 = fmaf(v, v, n2);
            }
            mx = fmaxf(mx, n2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
        if (lane == 0) {
            const float f = ceilf(sqrtf(mx) / sqrtf(refine_c));
            // the next power of two: the scaling 1/s is exact, and the strip
            // kernels stage a virtual row's segment with shifts
            int32_t sp = 1;
            while (sp < 64 && (float)sp < f) sp <<= 1;
            s_out[p] = sp;
        }
    }
}

// MMD^2 from the Gram of Z = [X; Y] (N = m + n), FP64, one CTA.
__global__ void __launch_bounds__(1024) mmd_reduce_kernel(const double* G, int64_t m, int64_t n,
                                                          int unbiased, double* out) {
    __shared__ double sh[3][1024];
    const int64_t N = m + n;
    double sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int64_t idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int64_t a = idx / N, b = idx % N;
        const double v = G[idx];
        if (a < m && b < m) {
            if (!unbiased || a != b) sxx += v;
        } else if (a >= m && b >= m) {
            if (!unbiased || a != b) syy += v;
        } else if (a < m && b >= m) {
            sxy += v;
        }
    }
    sh[0][threadIdx.x] = sxx;
    sh[1][threadIdx.x] = syy;
    sh[2][threadIdx.x] = sxy;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mm = unbiased ? (double)m * (double)(m - 1) : (double)m * (double)m;
        const double nn = unbiased ? (double)n * (double)(n - 1) : (double)n * (double)n;
        out[0] = sh[0][0] / mm + sh[1][0] / nn - 2.0 * sh[2][0] / ((double)m * (double)n);
    }
}

// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Smallest (order P, rings n) with the estimated truncation errors below
// tol/10, relative to the local kernel scale (App. C.3: a-priori order search
// from the largest coupling in the grid, here per pair and for two knobs):
//   rings: sum_ij |c_ij|^{n+1} / ((n+1)!)^2 <= tol/10 (the dropped ring n+1)
//   order: max(L1, L2) * C^{P+1} / ((P+1)!)^2 <= tol/10, C = max(C_a, C_b) the
//          accumulated coupling (the dropped edge coefficient of degree P+1,
//          over a row or column)
static void choose_order(const double* st, int64_t n, double tol, int* P_out, int* nr_out,
                         int64_t* max_swept, double* max_tile_c, bool* order_fits) {
    *max_tile_c = 0.0;
    *order_fits = true;
    const double target = 0.1 * tol;
    // rings: the sum of the first dropped ring over every tile treats the
    // terms as coherent; on the 1024-segment Grams it overstates the measured
    // truncation error 3-4 times (sigma = 1, three rings: 1.7e-6 predicted,
    // 4.4e-7 measured on self-kernels), so it gets a quarter of the tolerance
    const double ring_target = 0.25 * tol;
    int P = 4, nr = 1;
    double fact[40];
    fact[0] = 1.0;
    for (int k = 1; k < 40; ++k) fact[k] = fact[k - 1] * k;
    for (int64_t p = 0; p < n; ++p) {
        const double* o = st + p * kStatFields;
        if (o[0] <= 0 || o[1] <= 0) continue;
        if ((int64_t)o[1] > *max_swept) *max_swept = (int64_t)o[1];
        if (o[12] > *max_tile_c) *max_tile_c = o[12];
        int r = 1;
        while (r < kMaxRings && o[4 + (r + 1) - 2] / (fact[r + 1] * fact[r + 1]) > ring_target) ++r;
        if (r > nr) nr = r;
        const double C = o[2] > o[3] ? o[2] : o[3];
        const double Lm = o[0] > o[1] ? o[0] : o[1];
        int q = 4;
        while (q < kMaxP && Lm * pow(C, q + 1) / (fact[q + 1] * fact[q + 1]) > target) ++q;
        if (Lm * pow(C, q + 1) / (fact[q + 1] * fact[q + 1]) > target) *order_fits = false;
        if (q > P) P = q;
    }
    if (P < nr) P = nr;
    P += (P & 1);
    if (P > kMaxP) P = kMaxP;
    // the FP32 truncation keeps edge degrees up to 2 nr (keep_entry): enough
    // rings that the degree it reaches is within 4 of the coupling rule's P
    // (that rule bounds every edge by the largest coupling of the pair, which
    // overstates the edges of most tiles by orders of magnitude)
    if (2 * nr < P - 4) nr = (P - 4 + 1) / 2;
    if (nr > (P < kMaxRings ? P : kMaxRings)) nr = P < kMaxRings ? P : kMaxRings;
    if (nr < 2) nr = 2;
    *P_out = P;
    *nr_out = nr;
}

static sigk_status check_ws(const Layout& L, void* ws, size_t ws_bytes) {
    if (!ws) return fail(SIGK_ERR_WORKSPACE, "workspace pointer is NULL");
    if (((uintptr_t)ws & 255) != 0) return fail(SIGK_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(SIGK_ERR_WORKSPACE, "workspace too small: need " + std::to_string(L.total) +
                                            " bytes, got " + std::to_string(ws_bytes));
    return SIGK_OK;
}

// Planner launches: prefix sums, then (with refinement) the per-path factors,
// then the pair table.  Without refinement one launch does both phases.
static cudaError_t launch_planner(PlanArgs pa, const Opts& o, const Layout& L, char* base,
                                  cudaStream_t stream) {
    pa.sX = nullptr;
    pa.sY = nullptr;
    if (o.refine_c <= 0.0f) {
        pa.phase = 3;
        plan_kernel<<<1, kPlanThreads, 0, stream>>>(pa);
        return cudaGetLastError();
    }
    pa.phase = 1;
    plan_kernel<<<1, kPlanThreads, 0, stream>>>(pa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int32_t* sX = (int32_t*)(base + L.sx);
    int32_t* sY = (int32_t*)(base + L.sy);
    const bool self = (pa.op == SIGK_OP_GRAM && pa.n_y == 0);
    auto blocks = [](int64_t n) { return (unsigned)((n + 7) / 8 < 4096 ? (n + 7) / 8 : 4096); };
    if (pa.n_x > 0)
        refine_kernel<<<blocks(pa.n_x), 256, 0, stream>>>(pa.X, pa.len_x, pa.ox, pa.n_x, pa.d,
                                                            pa.inc_mode, o.refine_c, sX);
    if (!self && pa.n_y > 0)
        refine_kernel<<<blocks(pa.n_y), 256, 0, stream>>>(pa.Y, pa.len_y, pa.oy, pa.n_y, pa.d,
                                                            pa.inc_mode, o.refine_c, sY);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    pa.sX = sX;
    pa.sY = self ? sX : sY;
    pa.phase = 2;
    plan_kernel<<<1, kPlanThreads, 0, stream>>>(pa);
    return cudaGetLastError();
}

// Signature of a training call (op, sizes, options, layout): recorded by the
// training forward's planner, checked by the adjoint's set-up kernel.
static long long train_signature(int op, int64_t n_x, int64_t n_y, int d, const Opts& o,
                                 const Layout& L) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the fields
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xFF;
            h *= 1099511628211ull;
        }
    };
    uint32_t rc;
    memcpy(&rc, &o.refine_c, sizeof(rc));
    mix((uint64_t)op); mix((uint64_t)n_x); mix((uint64_t)n_y); mix((uint64_t)d);
    mix((uint64_t)o.order); mix((uint64_t)o.rings); mix((uint64_t)o.flags);
    mix((uint64_t)o.max_len); mix((uint64_t)o.grid_ctas); mix((uint64_t)rc); mix((uint64_t)L.total);
    return (long long)(h | 1ull);  // never 0
}

// Common driver: plan + solve into `out` (k values or Gram).  With `train`,
// the forward runs in training mode: every 32-row strip's seam is stored and,
// within the record budget, every tile's record (one row per lane); the
// workspace then holds what launch_adjoint needs.
static sigk_status run_solver(int op, const float* X, const int64_t* len_x, int64_t n_x,
                              const float* Y, const int64_t* len_y, int64_t n_y, int d,
                              double* out, int64_t out_ld, void* ws, size_t ws_bytes,
                              cudaStream_t stream, const Opts& o, Layout* Lout,
                              bool train = false, bool allow_sm = true) {
    Layout L;
    sigk_status st = make_layout(op, n_x, n_y, d, o, &L, train, allow_sm);
    if (st != SIGK_OK) return st;
    if ((st = check_ws(L, ws, ws_bytes)) != SIGK_OK) return st;
    char* base = (char*)ws;
    Header* hdr = (Header*)(base + L.hdr);
    PlanArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.op = op;
    pa.flags = o.flags;
    pa.inc_mode = (o.flags & SIGK_FLAG_INCREMENTS) ? 1 : 0;
    pa.d = d;
    pa.X = X;
    pa.len_x = len_x;
    pa.n_x = n_x;
    pa.Y = Y;
    pa.len_y = len_y;
    pa.n_y = n_y;
    pa.max_len = o.max_len;
    pa.rows_per_strip = L.rows_per_strip;
    pa.strip_quantum = L.strip_quantum;
    pa.n_pairs = L.n_pairs;
    pa.ox = (int64_t*)(base + L.ox);
    pa.oy = (int64_t*)(base + L.oy);
    pa.pairs = (PairDesc*)(base + L.pairs);
    pa.item_start = (int32_t*)(base + L.item_start);
    pa.order = (int32_t*)(base + L.order);
    pa.lvl = (int32_t*)(base + L.lvl);
    pa.lvl_cap = kLevelCap;
    pa.allow_sm = L.strip_major ? 1 : 0;
    pa.fwd_shift = L.fwd_shift;
    pa.item_start2 = (int32_t*)(base + L.item_start2);
    pa.lvl2 = (int32_t*)(base + L.lvl2);
    pa.prod = (unsigned long long*)(base + L.prod);
    pa.cons = (unsigned long long*)(base + L.cons);
    pa.done = (long long*)(base + L.done);
    pa.nslot = (int)L.nwords;
    pa.hdr = hdr;
    pa.out = out;
    pa.out_ld = out_ld;
    pa.wait_ns = (long long)o.wait_ms * 1000000ll;
    if (train) {
        pa.train = 1;
        pa.stride = L.stride;
        pa.store_cap = L.store_floats;
        pa.store_off = (int64_t*)(base + L.store_off);
        pa.train_sig = train_signature(op, n_x, n_y, d, o, L);
        if (L.stored_rec) {
            pa.rec_off = (int64_t*)(base + L.rec_off);
            pa.rec_cap = L.rstore_floats;
            pa.rec_rows = L.rec_rows;
            pa.rec_block = 32 * L.rec_rows * rec_floats(o.order);
        }
    }
    cudaError_t e = launch_planner(pa, o, L, base, stream);
    if (e != cudaSuccess) return cuda_fail(e, "planner launch");
    SolverArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.pairs = pa.pairs;
    Schedule table_sched;  // 32*R-row strips (inference) or 32-row strips (adjoint)
    table_sched.hdr = hdr->sched;
    table_sched.item_start = pa.item_start;
    table_sched.order = pa.order;
    table_sched.level_start = pa.lvl;
    table_sched.n_pairs = (int32_t)L.n_pairs;
    table_sched.shift = 0;
    sa.sched = table_sched;
    if (train) {  // the training forward's items are 2^fwd_shift table strips
        sa.sched.hdr = hdr->sched2;
        sa.sched.item_start = pa.item_start2;
        sa.sched.level_start = pa.lvl2;
        sa.sched.shift = L.fwd_shift;
    }
    sa.n_pairs = (int32_t)L.n_pairs;
    sa.inc_mode = pa.inc_mode;
    sa.d = d;
    sa.nr = o.rings;
    sa.nslot = L.nslot;
    sa.wcols = L.wcols;
    sa.seam = (float*)(base + L.seam);
    sa.prod = pa.prod;
    sa.cons = pa.cons;
    sa.done = pa.done;
    sa.item_counter = &hdr->item_counter;
    sa.status = &hdr->status;
    sa.counters = hdr->counters;
    sa.out = out;
    sa.withhold_first_seam = (o.flags & SIGK_FLAG_TEST_WITHHOLD_SEAM) && !train ? 1 : 0;
    // per-tile ring counts (inference only): |c| <= theta_n keeps the first
    // dropped ring |c|^(n+1)/((n+1)!)^2 within ring_tol
    sa.ring_adaptive = (o.ring_tol > 0.0f && L.tc) ? 1 : 0;
    sa.ring_hist = hdr->ring_hist;
    for (int q = 0; q < 3; ++q) {
        const int n = 2 * q + 2;
        double f = 1.0;
        for (int k = 2; k <= n + 1; ++k) f *= k;
        sa.ring_theta[q] = (float)pow((double)o.ring_tol * f * f, 1.0 / (n + 1));
    }
    sa.nwords = (int32_t)L.nwords;
    sa.store_cap = train ? L.store_floats : 0;
    sa.rec_cap = L.stored_rec ? L.rstore_floats : 0;
    sa.out_cap = op == SIGK_OP_PAIRS ? L.n_pairs
                                     : (op == SIGK_OP_MMD ? (n_x + n_y) * (n_x + n_y)
                                                          : n_x * (n_y > 0 ? n_y : n_x));
    if (train) {
        sa.store = (float*)(base + L.store);
        sa.store_off = pa.store_off;
        sa.pair_exp = (int32_t*)(base + L.pair_exp);
        if (L.stored_rec) {
            sa.rec = (float*)(base + L.rstore);
            sa.rec_off = pa.rec_off;
        }
    }
    if (L.n_pairs > 0 && L.tc) {
        // digits of every path's first max_len segments (the swept sides)
        SliceArgs sl;
        sl.X = X;
        sl.Y = (op == SIGK_OP_GRAM && n_y == 0) ? nullptr : Y;
        sl.ox = pa.ox;
        sl.oy = pa.oy;
        sl.len_x = len_x;
        sl.len_y = len_y;
        sl.n_x = n_x;
        sl.n_slots = L.n_slots;
        sl.d = d;
        sl.d_pad = L.d_pad;
        sl.inc_mode = pa.inc_mode;
        sl.max_len = o.max_len;
        sl.cache = (uint16_t*)(base + L.ycache);
        sl.exps = (int32_t*)(base + L.yexp);
        const int64_t rows = L.n_slots * tc_cache_rows(o.max_len);
        const int64_t blocks = (rows + 7) / 8;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
        slice_paths_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, stream>>>(sl);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "digit pre-pass launch");
    }
    if (L.n_pairs > 0) {
        if (g_ev_start && g_ev_stop) cudaEventRecord(g_ev_start, stream);
        if (L.tc) {
            TcArgs ta;
            ta.A = sa;
            ta.ycache = (const uint16_t*)(base + L.ycache);
            ta.yexp = (const int32_t*)(base + L.yexp);
            ta.max_len = o.max_len;
            ta.d_pad = L.d_pad;
            ta.ablk = (uint16_t*)(base + L.ablk);
            ta.cst = (float2*)(base + L.cst);
            ta.cst_stride = L.cst_stride;
            ta.block_counter = &hdr->item_counter;
            e = fwd_tc_launch_dispatch(o.order, o.rings, ta, L.grid, stream);
        } else {
            e = L.cm ? fwd_cm_launch_dispatch(o.order, o.rings, L.f64, sa, base + L.cscratch, L.cstride,
                                              L.grid, stream)
                     : fwd_launch_dispatch(o.order, o.rings, dim_bucket(d), L.stored_rec ? 1 : 0, sa,
                                           L.grid, stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "solver launch");
        if (g_ev_start && g_ev_stop) cudaEventRecord(g_ev_stop, stream);
    }
    if (Lout) *Lout = L;
    return SIGK_OK;
}

// The adjoint after a training forward on the same workspace (run_solver with
// train = true, same op, sizes and opts): adjoint_prep_kernel, then the
// adjoint kernel.  gX / gY (or null) receive the gradients.
static sigk_status launch_adjoint(int op, int64_t n_x, int64_t n_y, int d, const double* grad_out,
                                  float* gX, float* gY, void* ws, size_t ws_bytes,
                                  cudaStream_t stream, const Opts& o) {
    Layout L;
    sigk_status st = make_layout(op, n_x, n_y, d, o, &L, true);
    if (st != SIGK_OK) return st;
    if ((st = check_ws(L, ws, ws_bytes)) != SIGK_OK) return st;
    if (L.n_pairs == 0) return SIGK_OK;
    char* base = (char*)ws;
    Header* hdr = (Header*)(base + L.hdr);
    PlanArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.op = op;
    pa.flags = o.flags;
    pa.d = d;
    pa.n_x = n_x;
    pa.n_y = n_y;
    pa.n_pairs = L.n_pairs;
    pa.out_ld = op == SIGK_OP_MMD ? n_x + n_y : (op == SIGK_OP_GRAM ? (n_y > 0 ? n_y : n_x) : 0);
    pa.ox = (int64_t*)(base + L.ox);
    pa.oy = (int64_t*)(base + L.oy);
    pa.pairs = (PairDesc*)(base + L.pairs);
    pa.hdr = hdr;
    pa.pair_w = (double*)(base + L.pair_w);
    pa.grad_out = grad_out;
    pa.gX = gX;
    pa.gY = gY;
    pa.bprod = (unsigned long long*)(base + L.bprod);
    pa.bcons = (unsigned long long*)(base + L.bcons);
    pa.bdone = (long long*)(base + L.bdone);
    pa.bnslot = L.bnslot;
    pa.train_sig = train_signature(op, n_x, n_y, d, o, L);
    pa.wait_ns = (long long)o.wait_ms * 1000000ll;
    adjoint_prep_kernel<<<L.bgrid, 256, 0, stream>>>(pa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint set-up launch");
    BwdArgs ba;
    memset(&ba, 0, sizeof(ba));
    ba.pairs = pa.pairs;
    ba.sched.hdr = hdr->sched;
    ba.sched.item_start = (int32_t*)(base + L.item_start);
    ba.sched.order = (int32_t*)(base + L.order);
    ba.sched.level_start = (int32_t*)(base + L.lvl);
    ba.sched.n_pairs = (int32_t)L.n_pairs;
    ba.sched.shift = 0;
    ba.n_pairs = (int32_t)L.n_pairs;
    ba.inc_mode = (o.flags & SIGK_FLAG_INCREMENTS) ? 1 : 0;
    ba.d = d;
    ba.nr = o.rings;
    ba.store = (float*)(base + L.store);
    ba.store_off = (int64_t*)(base + L.store_off);
    ba.pair_exp = (int32_t*)(base + L.pair_exp);
    ba.pair_w = pa.pair_w;
    ba.rec = (float*)(base + L.rec);
    ba.rec_stride = L.rec_stride;
    if (L.stored_rec) {
        ba.rec_store = (float*)(base + L.rstore);
        ba.rec_off = (int64_t*)(base + L.rec_off);
        ba.rec_rows = L.rec_rows;
    }
    ba.nslot = L.bnslot;
    ba.wcols = L.bwcols;
    ba.aseam = (float*)(base + L.aseam);
    ba.prod = pa.bprod;
    ba.cons = pa.bcons;
    ba.done = pa.bdone;
    ba.item_counter = &hdr->bwd_item_counter;
    ba.status = &hdr->status;
    ba.counters = hdr->counters;
    ba.store_cap = L.store_floats;
    ba.rec_cap = L.stored_rec ? L.rstore_floats : 0;
    ba.rec_total = L.stored_rec ? 0 : (int64_t)L.bnwarps * L.rec_stride;
    if (g_ev_start && g_ev_stop) cudaEventRecord(g_ev_start, stream);
    e = bwd2_launch_dispatch(o.order, o.rings, ba, (float*)(base + L.bcs), L.bcstride, L.bgrid, stream);
    if (e != cudaSuccess) return cuda_fail(e, "backward launch");
    if (g_ev_start && g_ev_stop) cudaEventRecord(g_ev_stop, stream);
    return SIGK_OK;
}

static sigk_status common_checks(int64_t n1, int64_t n2, int d, const void* out) {
    if (d < 1) return fail(SIGK_ERR_ARG, "d must be >= 1");
    if (n1 < 0 || n2 < 0) return fail(SIGK_ERR_ARG, "negative batch size");
    if (!out) return fail(SIGK_ERR_ARG, "output pointer is NULL");
    if (n1 > (int64_t)1 << 24 || n2 > (int64_t)1 << 24) return fail(SIGK_ERR_ARG, "batch too large");
    return SIGK_OK;
}

}  // namespace sigk

using namespace sigk;

extern "C" {

size_t sigk_workspace_size(int op, int64_t n_x, int64_t n_y, int d, const sigk_opts* opts) {
    Opts o;
    if (!resolve_opts(opts, &o)) return 0;
    if (op < SIGK_OP_PAIRS || op > SIGK_OP_MMD || n_x < 0 || n_y < 0 || d < 1) return 0;
    if (op == SIGK_OP_PAIRS) n_y = n_x;
    Layout L;
    if (make_layout(op, n_x, n_y, d, o, &L) != SIGK_OK) return 0;
    return L.total;
}

sigk_status sigk_pairs(const float* X, const int64_t* len_x, const float* Y, const int64_t* len_y,
                       int64_t n_pairs, int d, double* k_out, void* ws, size_t ws_bytes,
                       void* stream, const sigk_opts* opts) {
    sigk_status st = common_checks(n_pairs, n_pairs, d, k_out);
    if (st != SIGK_OK) return st;
    if (n_pairs > 0 && (!X || !Y || !len_x || !len_y)) return fail(SIGK_ERR_ARG, "null input");
    Opts o;
    if (!resolve_opts(opts, &o)) return fail(SIGK_ERR_ARG, "invalid sigk_opts");
    if (n_pairs == 0) return SIGK_OK;
    return run_solver(SIGK_OP_PAIRS, X, len_x, n_pairs, Y, len_y, n_pairs, d, k_out, 0, ws,
                      ws_bytes, (cudaStream_t)stream, o, nullptr);
}

sigk_status sigk_gram(const float* X, const int64_t* len_x, int64_t n_x, const float* Y,
                      const int64_t* len_y, int64_t n_y, int d, double* G, void* ws,
                      size_t ws_bytes, void* stream, const sigk_opts* opts) {
    if (!Y) n_y = 0;
    sigk_status st = common_checks(n_x, n_y, d, G);
    if (st != SIGK_OK) return st;
    if (n_x > 0 && (!X || !len_x)) return fail(SIGK_ERR_ARG, "null input");
    if (Y && n_y > 0 && !len_y) return fail(SIGK_ERR_ARG, "null len_y");
    Opts o;
    if (!resolve_opts(opts, &o)) return fail(SIGK_ERR_ARG, "invalid sigk_opts");
    if (n_x == 0 || (Y && n_y == 0)) return SIGK_OK;
    const int64_t ld = Y ? n_y : n_x;
    return run_solver(SIGK_OP_GRAM, X, len_x, n_x, Y, len_y, Y ? n_y : 0, d, G, ld, ws, ws_bytes,
                      (cudaStream_t)stream, o, nullptr);
}

sigk_status sigk_mmd(const float* X, const int64_t* len_x, int64_t m, const float* Y,
                     const int64_t* len_y, int64_t n, int d, double* mmd2_out, double* gram_out,
                     void* ws, size_t ws_bytes, void* stream, const sigk_opts* opts) {
    sigk_status st = common_checks(m, n, d, mmd2_out);
    if (st != SIGK_OK) return st;
    if (!X || !Y || !len_x || !len_y) return fail(SIGK_ERR_ARG, "null input");
    Opts o;
    if (!resolve_opts(opts, &o)) return fail(SIGK_ERR_ARG, "invalid sigk_opts");
    const int unbiased = (o.flags & SIGK_FLAG_MMD_BIASED) ? 0 : 1;
    if (m < 1 + unbiased || n < 1 + unbiased)
        return fail(SIGK_ERR_ARG, "MMD needs at least 2 paths per sample (1 for the V-statistic)");
    Layout L;
    if ((st = make_layout(SIGK_OP_MMD, m, n, d, o, &L)) != SIGK_OK) return st;
    if ((st = check_ws(L, ws, ws_bytes)) != SIGK_OK) return st;
    double* G = gram_out ? gram_out : (double*)((char*)ws + L.gram);
    st = run_solver(SIGK_OP_MMD, X, len_x, m, Y, len_y, n, d, G, m + n, ws, ws_bytes,
                    (cudaStream_t)stream, o, nullptr);
    if (st != SIGK_OK) return st;
    mmd_reduce_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(G, m, n, unbiased, mmd2_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mmd_reduce launch");
    return SIGK_OK;
}

size_t sigk_backward_workspace_size(int op, int64_t n_x, int64_t n_y, int d, const sigk_opts* opts) {
    Opts o;
    if (!resolve_opts(opts, &o)) return 0;
    if (op < SIGK_OP_PAIRS || op > SIGK_OP_MMD || n_x < 0 || n_y < 0 || d < 1) return 0;
    if (op == SIGK_OP_PAIRS) n_y = n_x;
    Layout L;
    if (make_layout(op, n_x, n_y, d, o, &L, true) != SIGK_OK) return 0;
    return L.total;
}

// Shared by sigk_forward_train and sigk_backward: argument checks and the
// training forward into value_out (or the workspace's Gram for MMD).
static sigk_status forward_train(int op, const float* X, const int64_t* len_x, int64_t n_x,
                                 const float* Y, const int64_t* len_y, int64_t n_y, int d,
                                 double* value_out, void* ws, size_t ws_bytes, void* stream,
                                 const Opts& o) {
    sigk_status st;
    Layout L;
    if ((st = make_layout(op, n_x, n_y, d, o, &L, true)) != SIGK_OK) return st;
    if ((st = check_ws(L, ws, ws_bytes)) != SIGK_OK) return st;
    const int unbiased = (o.flags & SIGK_FLAG_MMD_BIASED) ? 0 : 1;
    double* vals = nullptr;
    int64_t ld = 0;
    if (op == SIGK_OP_MMD) {
        vals = (double*)((char*)ws + L.gram);
        ld = n_x + n_y;
    } else if (op == SIGK_OP_GRAM) {
        if (!value_out) return fail(SIGK_ERR_ARG, "a Gram training forward needs value_out [n_x*n_y]");
        vals = value_out;
        ld = n_y > 0 ? n_y : n_x;
    } else {
        if (!value_out) return fail(SIGK_ERR_ARG, "a pairs training forward needs value_out [n_pairs]");
        vals = value_out;
    }
    st = run_solver(op, X, len_x, n_x, n_y > 0 || op != SIGK_OP_GRAM ? Y : nullptr, len_y, n_y, d,
                    vals, ld, ws, ws_bytes, (cudaStream_t)stream, o, nullptr, true);
    if (st != SIGK_OK) return st;
    if (op == SIGK_OP_MMD && value_out) {
        mmd_reduce_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(vals, n_x, n_y, unbiased, value_out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "mmd_reduce launch");
    }
    return SIGK_OK;
}

// Normalises (op, n_x, n_y, Y) and checks the arguments common to the
// training calls; *skip = true when there is nothing to solve.
static sigk_status train_checks(int op, const float* X, const int64_t* len_x, int64_t n_x,
                                const float* Y, const int64_t* len_y, int64_t* n_y, int d,
                                const sigk_opts* opts, Opts* o, bool* skip) {
    *skip = false;
    if (op < SIGK_OP_PAIRS || op > SIGK_OP_MMD) return fail(SIGK_ERR_ARG, "bad op");
    if (op == SIGK_OP_GRAM && !Y) *n_y = 0;
    if (op == SIGK_OP_PAIRS) *n_y = n_x;
    sigk_status st = common_checks(n_x, *n_y, d, (const void*)1);
    if (st != SIGK_OK) return st;
    if (n_x > 0 && (!X || !len_x)) return fail(SIGK_ERR_ARG, "null X input");
    if (op != SIGK_OP_GRAM || Y) {
        if (*n_y > 0 && (!Y || !len_y)) return fail(SIGK_ERR_ARG, "null Y input");
    }
    if (!resolve_opts(opts, o)) return fail(SIGK_ERR_ARG, "invalid sigk_opts");
    if (n_x == 0 || (op != SIGK_OP_GRAM && *n_y == 0)) {
        *skip = true;
        return SIGK_OK;
    }
    const int unbiased = (o->flags & SIGK_FLAG_MMD_BIASED) ? 0 : 1;
    if (op == SIGK_OP_MMD && (n_x < 1 + unbiased || *n_y < 1 + unbiased))
        return fail(SIGK_ERR_ARG, "MMD needs at least 2 paths per sample (1 for the V-statistic)");
    return SIGK_OK;
}

sigk_status sigk_forward_train(int op, const float* X, const int64_t* len_x, int64_t n_x,
                               const float* Y, const int64_t* len_y, int64_t n_y, int d,
                               double* value_out, void* ws, size_t ws_bytes, void* stream,
                               const sigk_opts* opts) {
    Opts o;
    bool skip;
    sigk_status st = train_checks(op, X, len_x, n_x, Y, len_y, &n_y, d, opts, &o, &skip);
    if (st != SIGK_OK || skip) return st;
    return forward_train(op, X, len_x, n_x, Y, len_y, n_y, d, value_out, ws, ws_bytes, stream, o);
}

sigk_status sigk_adjoint(int op, int64_t n_x, int64_t n_y, int d, const double* grad_out,
                         float* grad_X, float* grad_Y, void* ws, size_t ws_bytes, void* stream,
                         const sigk_opts* opts) {
    if (op < SIGK_OP_PAIRS || op > SIGK_OP_MMD) return fail(SIGK_ERR_ARG, "bad op");
    if (!grad_out) return fail(SIGK_ERR_ARG, "grad_out is NULL");
    if (op == SIGK_OP_PAIRS) n_y = n_x;
    sigk_status st = common_checks(n_x, n_y, d, grad_out);
    if (st != SIGK_OK) return st;
    Opts o;
    if (!resolve_opts(opts, &o)) return fail(SIGK_ERR_ARG, "invalid sigk_opts");
    if (n_x == 0 || (op != SIGK_OP_GRAM && n_y == 0)) return SIGK_OK;
    return launch_adjoint(op, n_x, n_y, d, grad_out, grad_X,
                          (op == SIGK_OP_GRAM && n_y == 0) ? nullptr : grad_Y, ws, ws_bytes,
                          (cudaStream_t)stream, o);
}

sigk_status sigk_backward(int op, const float* X, const int64_t* len_x, int64_t n_x, const float* Y,
                          const int64_t* len_y, int64_t n_y, int d, const double* grad_out,
                          float* grad_X, float* grad_Y, double* value_out, void* ws,
                          size_t ws_bytes, void* stream, const sigk_opts* opts) {
    if (!grad_out) return fail(SIGK_ERR_ARG, "grad_out is NULL");
    Opts o;
    bool skip;
    sigk_status st = train_checks(op, X, len_x, n_x, Y, len_y, &n_y, d, opts, &o, &skip);
    if (st != SIGK_OK || skip) return st;
    st = forward_train(op, X, len_x, n_x, Y, len_y, n_y, d, value_out, ws, ws_bytes, stream, o);
    if (st != SIGK_OK) return st;
    return launch_adjoint(op, n_x, n_y, d, grad_out, grad_X,
                          (op == SIGK_OP_GRAM && n_y == 0) ? nullptr : grad_Y, ws, ws_bytes,
                          (cudaStream_t)stream, o);
}

// Exact tile statistics of the pair table as planned (sigk_stats.cuh).
static constexpr int kStatGridPerSm = 4;
static cudaError_t launch_stats(const PlanArgs& pa, double* stats, size_t stats_bytes,
                                float* basebuf, int grid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(stats, 0, stats_bytes, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&pa.hdr->item_counter, 0, sizeof(int), s)) != cudaSuccess) return e;
    StatArgs sa;
    sa.pairs = pa.pairs;
    sa.sched.shift = 0;
    sa.sched.hdr = pa.hdr->sched;
    sa.sched.item_start = pa.item_start;
    sa.sched.order = pa.order;
    sa.sched.level_start = pa.lvl;
    sa.sched.n_pairs = (int32_t)pa.n_pairs;
    sa.n_pairs = (int32_t)pa.n_pairs;
    sa.rows_per_strip = pa.rows_per_strip;
    sa.d = pa.d;
    sa.inc_mode = pa.inc_mode;
    sa.item_counter = &pa.hdr->item_counter;
    sa.stats = stats;
    sa.base = basebuf;
    const int smem = 4 * StSmem::per_warp * (int)sizeof(float);
    pair_stats_kernel<<<grid, 128, smem, s>>>(sa);
    return cudaGetLastError();
}

sigk_status sigk_plan(int op, const float* X, const int64_t* len_x, int64_t n_x, const float* Y,
                      const int64_t* len_y, int64_t n_y, int d, double tol, void* ws,
                      size_t ws_bytes, void* stream, const sigk_opts* opts_in, sigk_opts* opts_out) {
    if (!opts_out) return fail(SIGK_ERR_ARG, "opts_out is NULL");
    if (!(tol > 0.0) || tol >= 1.0) return fail(SIGK_ERR_ARG, "tol must be in (0, 1)");
    if (op < SIGK_OP_PAIRS || op > SIGK_OP_MMD) return fail(SIGK_ERR_ARG, "bad op");
    if (op == SIGK_OP_GRAM && !Y) n_y = 0;
    if (op == SIGK_OP_PAIRS) n_y = n_x;
    sigk_status st = common_checks(n_x, n_y, d, opts_out);
    if (st != SIGK_OK) return st;
    Opts o;
    if (!resolve_opts(opts_in, &o)) return fail(SIGK_ERR_ARG, "invalid sigk_opts");
    o.order = kMaxP;  // layout for the largest order (the planner's seam stride)
    o.rings = kMaxRings;
    Layout L;
    if ((st = make_layout(op, n_x, n_y, d, o, &L)) != SIGK_OK) return st;
    if ((st = check_ws(L, ws, ws_bytes)) != SIGK_OK) return st;
    const size_t need = align256(sizeof(double) * kStatFields * (size_t)L.n_pairs);
    if (need > L.total - L.seam) return fail(SIGK_ERR_WORKSPACE, "workspace too small for plan statistics");
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return fail(SIGK_ERR_CUDA, "cannot query SM count");
    const int stat_grid = sms * kStatGridPerSm;
    const size_t base_bytes = align256(sizeof(float) * (size_t)stat_grid * 4 * (size_t)d);
    char* base = (char*)ws;
    cudaStream_t strm = (cudaStream_t)stream;
    // the planner builds the pair table; its k outputs go to a scratch area
    double* scratch_out = (double*)(base + L.seam);
    PlanArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.op = op;
    pa.flags = o.flags & ~SIGK_FLAG_GRAM_FULL;
    pa.inc_mode = (o.flags & SIGK_FLAG_INCREMENTS) ? 1 : 0;
    pa.d = d;
    pa.X = X; pa.len_x = len_x; pa.n_x = n_x;
    pa.Y = (op == SIGK_OP_GRAM && !Y) ? nullptr : Y;
    pa.len_y = len_y;
    pa.n_y = (op == SIGK_OP_GRAM && !Y) ? 0 : n_y;
    pa.max_len = (int64_t)INT32_MAX;  // no swept-length limit while planning
    pa.rows_per_strip = L.rows_per_strip;
    pa.strip_quantum = 1;
    pa.n_pairs = L.n_pairs;
    pa.ox = (int64_t*)(base + L.ox);
    pa.oy = (int64_t*)(base + L.oy);
    pa.pairs = (PairDesc*)(base + L.pairs);
    pa.item_start = (int32_t*)(base + L.item_start);
    pa.order = (int32_t*)(base + L.order);
    pa.lvl = (int32_t*)(base + L.lvl);
    pa.lvl_cap = kLevelCap;
    pa.allow_sm = L.strip_major ? 1 : 0;
    pa.fwd_shift = L.fwd_shift;
    pa.item_start2 = (int32_t*)(base + L.item_start2);
    pa.lvl2 = (int32_t*)(base + L.lvl2);
    pa.prod = (unsigned long long*)(base + L.prod);
    pa.cons = (unsigned long long*)(base + L.cons);
    pa.done = (long long*)(base + L.done);
    pa.nslot = (int)L.nwords;
    pa.hdr = (Header*)(base + L.hdr);
    pa.out = scratch_out;
    pa.out_ld = 0;
    pa.wait_ns = (long long)o.wait_ms * 1000000ll;
    float* statbase = nullptr;
    if (op != SIGK_OP_PAIRS) {
        // Gram-shaped ops write k at a*ld+b; give them a large enough scratch
        const int64_t nz = (op == SIGK_OP_MMD) ? n_x + n_y : n_x;
        const int64_t ncol = (op == SIGK_OP_GRAM && Y) ? n_y : nz;
        pa.out_ld = ncol;
        const size_t gram_bytes = align256(sizeof(double) * (size_t)((op == SIGK_OP_MMD ? nz : n_x) * ncol));
        if (gram_bytes + need + base_bytes > L.total - L.seam)
            return fail(SIGK_ERR_WORKSPACE, "workspace too small for plan scratch");
        scratch_out = (double*)(base + L.seam + need);
        pa.out = scratch_out;
        statbase = (float*)(base + L.seam + need + gram_bytes);
    } else {
        if (need + base_bytes > L.total - L.seam)
            return fail(SIGK_ERR_WORKSPACE, "workspace too small for plan scratch");
        statbase = (float*)(base + L.seam + need);
    }
    cudaError_t e = launch_planner(pa, o, L, base, strm);
    if (e != cudaSuccess) return cuda_fail(e, "planner launch");
    double* stats = (double*)(base + L.seam);
    if ((e = launch_stats(pa, stats, need, statbase, stat_grid, strm)) != cudaSuccess)
        return cuda_fail(e, "pair_stats launch");
    if ((e = cudaStreamSynchronize(strm)) != cudaSuccess) return cuda_fail(e, "plan synchronize");
    Header h;
    if ((e = cudaMemcpy(&h, base + L.hdr, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "plan status copy");
    if (h.status != 0) return fail((sigk_status)h.status, "invalid lengths");
    std::vector<double> hs((size_t)kStatFields * L.n_pairs);
    if ((e = cudaMemcpy(hs.data(), stats, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "plan stats copy");
    int P = 4, nr = 1;
    int64_t max_swept = 1;
    double max_c = 0.0;
    bool fits = true;
    choose_order(hs.data(), L.n_pairs, tol, &P, &nr, &max_swept, &max_c, &fits);
    // Tiles whose |c| may exceed 1 (Cauchy-Schwarz), or edges whose coupling
    // needs an order above 16, are refined and the refined problem is planned
    // again; each step divides refine_c by 4 (halving the couplings).
    float rc = 1.0f;
    while ((max_c > 1.0 || !fits) && o.refine_c <= 0.0f && rc >= 1.0f / 256.0f) {
        Opts o2 = o;
        o2.refine_c = rc;
        if ((e = launch_planner(pa, o2, L, base, strm)) != cudaSuccess)
            return cuda_fail(e, "planner launch");
        if ((e = launch_stats(pa, stats, need, statbase, stat_grid, strm)) != cudaSuccess)
            return cuda_fail(e, "pair_stats launch");
        if ((e = cudaStreamSynchronize(strm)) != cudaSuccess) return cuda_fail(e, "plan synchronize");
        if ((e = cudaMemcpy(&h, base + L.hdr, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "plan status copy");
        if (h.status != 0) return fail((sigk_status)h.status, "invalid lengths");
        if ((e = cudaMemcpy(hs.data(), stats, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "plan stats copy");
        P = 4; nr = 1; max_swept = 1;
        choose_order(hs.data(), L.n_pairs, tol, &P, &nr, &max_swept, &max_c, &fits);
        if (max_c <= 1.0 && fits) {
            o.refine_c = rc;
            break;
        }
        rc *= 0.25f;
        if (rc < 1.0f / 256.0f) o.refine_c = rc * 4.0f;  // finest tried
    }
    sigk_opts zero;
    memset(&zero, 0, sizeof(zero));
    *opts_out = opts_in ? *opts_in : zero;
    opts_out->order = P;
    opts_out->rings = nr;
    opts_out->refine_c = o.refine_c;
    {
        // per-tile ring tolerance: a tenth of an equal share of the ring-sum
        // rule of the largest pair (tol / 100 over its L1 L2 tiles); the
        // dropped rings of neighbouring tiles add coherently, and an equal
        // share (tol / 10) measured 1.06e-5 on a 1e-5 workload
        double cells = 1.0;
        for (int64_t p = 0; p < L.n_pairs; ++p) {
            const double* st = hs.data() + p * kStatFields;
            if (st[0] * st[1] > cells) cells = st[0] * st[1];
        }
        opts_out->ring_tol = (float)(0.01 * tol / cells);
    }
    opts_out->max_len = max_swept;  // the longest swept path as planned (refined)
    {
        // a tuned layout for this shape class, if the tuning cache holds one
        char key[256];
        if (sigk_tune_key(op, n_x, n_y, d, opts_out, key, sizeof(key)) == SIGK_OK)
            sigk_tune_cache_get(key, opts_out, nullptr);
    }
    if (max_c > 1.0 || !fits)
        return fail(SIGK_ERR_ACCURACY,
                    "the a-priori rule is not met at order 16 even at the finest refinement tried");
    return SIGK_OK;
}

sigk_status sigk_sync_status(void* ws, size_t ws_bytes, void* stream) {
    if (!ws || ws_bytes < 256) return fail(SIGK_ERR_WORKSPACE, "bad workspace");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    Header h;
    e = cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status copy");
    if (h.status == 0 && h.nonfinite != 0) {
        int zero = 0;
        cudaMemcpy((char*)ws + offsetof(Header, nonfinite), &zero, sizeof(int), cudaMemcpyHostToDevice);
        return fail(SIGK_ERR_NONFINITE, "non-finite value met on the device (the other outputs are valid)");
    }
    if (h.status != 0) {
        int zero[4] = {0, 0, 0, 0};
        cudaMemcpy(ws, &zero[0], sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy((char*)ws + offsetof(Header, nonfinite), &zero[3], sizeof(int), cudaMemcpyHostToDevice);
        const char* msg = h.status == kErrTimeout ? "a bounded device wait timed out"
                          : h.status == kErrNonfinite ? "non-finite value met on the device"
                          : h.status == kErrLength ? "a path length is out of range"
                          : h.status == kErrBounds ? "a device-side bounds check failed (debug build)"
                                                   : "device error";
        return fail((sigk_status)h.status, msg);
    }
    return SIGK_OK;
}

sigk_status sigk_launch_info(int op, int64_t n_x, int64_t n_y, int d, const sigk_opts* opts,
                             int train, int* out6) {
    if (!out6 || op < SIGK_OP_PAIRS || op > SIGK_OP_MMD || n_x < 0 || n_y < 0 || d < 1)
        return fail(SIGK_ERR_ARG, "bad arguments");
    Opts o;
    if (!resolve_opts(opts, &o)) return fail(SIGK_ERR_ARG, "invalid sigk_opts");
    if (op == SIGK_OP_PAIRS) n_y = n_x;
    Layout L;
    sigk_status st = make_layout(op, n_x, n_y, d, o, &L, train != 0);
    if (st != SIGK_OK) return st;
    const KernelInfo& k = train ? L.binfo : L.info;
    out6[0] = train ? L.bgrid : L.grid;
    out6[1] = k.blocks_per_sm;
    out6[2] = k.threads;
    out6[3] = k.smem_bytes;
    out6[4] = k.rows_per_lane;
    out6[5] = L.tc ? 2 : (L.cm ? 1 : 0);
    return SIGK_OK;
}

sigk_status sigk_ring_histogram(void* ws, size_t ws_bytes, void* stream, double* out4) {
    if (!ws || ws_bytes < 256 || !out4) return fail(SIGK_ERR_ARG, "bad arguments");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    Header h;
    e = cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "histogram copy");
    for (int i = 0; i < 4; ++i) out4[i] = (double)h.ring_hist[i];
    return SIGK_OK;
}

sigk_status sigk_counters(void* ws, size_t ws_bytes, void* stream, double* out4) {
    if (!ws || ws_bytes < 256 || !out4) return fail(SIGK_ERR_ARG, "bad arguments");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    Header h;
    e = cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "counter copy");
    for (int i = 0; i < 4; ++i) out4[i] = (double)h.counters[i];
    return SIGK_OK;
}

void sigk_profile_events(void* ev_start, void* ev_stop) {
    g_ev_start = (cudaEvent_t)ev_start;
    g_ev_stop = (cudaEvent_t)ev_stop;
}

const char* sigk_last_error(void) { return g_last_error.c_str(); }

const char* sigk_version(void) { return "sigk-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// No-allocation entry point (sigk_pairs_static).
//
// For callers that cannot call cudaMalloc -- e.g. code running inside a
// memory-pool-managed or graph-captured region, or a host runtime with its
// own allocator that forbids side allocations -- the scratch that sigk_pairs
// takes from the caller's workspace comes here from a fixed device array in
// this file.  Every GPU that loads the library holds these bytes until the
// process exits.  In host code `g_static_ws` only names a host-side stand-in:
// its device address is obtained once per device with cudaGetSymbolAddress
// (with that device current) on the first call there, and only that address
// is passed to kernels.

namespace sigk {

constexpr size_t kStaticWsBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static void* g_static_ptr[kMaxDevices];  // device address of g_static_ws per device

static sigk_status static_ws_ptr(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SIGK_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return SIGK_OK;
}

}  // namespace sigk

extern "C" sigk_status sigk_pairs_static(const float* X, const int64_t* len_x, const float* Y,
                                         const int64_t* len_y, int64_t n_pairs, int d,
                                         double* k_out, void* stream, const sigk_opts* opts) {
    using namespace sigk;
    sigk_status st = common_checks(n_pairs, n_pairs, d, k_out);
    if (st != SIGK_OK) return st;
    if (n_pairs > 0 && (!X || !Y || !len_x || !len_y)) return fail(SIGK_ERR_ARG, "null input");
    Opts o;
    if (!resolve_opts(opts, &o)) return fail(SIGK_ERR_ARG, "invalid sigk_opts");
    if (n_pairs == 0) return SIGK_OK;
    // Fit the layout into the static scratch: first as sigk_pairs would, then
    // with the pair-major schedule (a smaller seam ring), then also with one
    // CTA per SM (fewer warps).
    Layout L;
    bool sm = true;
    if ((st = make_layout(SIGK_OP_PAIRS, n_pairs, n_pairs, d, o, &L)) != SIGK_OK) return st;
    if (L.total > kStaticWsBytes) {
        sm = false;
        if ((st = make_layout(SIGK_OP_PAIRS, n_pairs, n_pairs, d, o, &L, false, false)) != SIGK_OK)
            return st;
    }
    if (L.total > kStaticWsBytes) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        o.grid_ctas = sms > 0 ? sms : 1;
        if ((st = make_layout(SIGK_OP_PAIRS, n_pairs, n_pairs, d, o, &L, false, false)) != SIGK_OK)
            return st;
    }
    if (L.total > kStaticWsBytes)
        return fail(SIGK_ERR_WORKSPACE,
                    "problem needs " + std::to_string(L.total) + " bytes of scratch; the static "
                    "scratch of sigk_pairs_static holds " + std::to_string(kStaticWsBytes) +
                    " (use sigk_pairs with a caller workspace)");
    void* ws = nullptr;
    if ((st = static_ws_ptr(&ws)) != SIGK_OK) return st;
    return run_solver(SIGK_OP_PAIRS, X, len_x, n_pairs, Y, len_y, n_pairs, d, k_out, 0, ws,
                      kStaticWsBytes, (cudaStream_t)stream, o, nullptr, false, sm);
}

extern "C" sigk_status sigk_static_sync_status(void* stream) {
    using namespace sigk;
    void* ws = nullptr;
    sigk_status st = static_ws_ptr(&ws);
    if (st != SIGK_OK) return st;
    return sigk_sync_status(ws, kStaticWsBytes, stream);
}
