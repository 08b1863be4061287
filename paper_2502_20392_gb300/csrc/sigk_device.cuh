// sigk_device.cuh -- device building blocks of the sm_103a signature-kernel
// solver: the per-tile map of the tile-centred expansion, float-float corner
// arithmetic, power-of-two renormalisation, and bounded inter-warp waits.
//
// Tile map (Sec. 2.3, Proposition "tile-centred expansion", with the
// orientation of its proof in App. A.6).  On the unit tile with coefficient
// c = <dx_i, dy_j>, bottom edge K(u,0) = sum_r a_r u^r and left edge
// K(0,v) = sum_r b_r v^r (a_0 = b_0 = corner), the solution is
//   K(u,v) = sum_{p,q} c^min(p,q) w_pq B_pq u^p v^q,
//   w_pq = |p-q|! / (p! q!),  B_pq = b_{q-p} (q >= p) or a_{p-q} (p > q).
// The top edge a'_p = sum_q (.)_pq and the right edge b'_q = sum_p (.)_pq are
// the next tiles' boundary data.  Truncation to p,q <= P is the (N+1)x(N+1)
// truncation of App. A.7 with N = P.
//
// Factorial scaling.  The kernel stores ah_p = p! a_p and bh_q = q! b_q.  With
// ch_m = c^m / m! the map becomes
//   ah'_p = sum_{m=0}^{p-1} ch_m ah_{p-m} + c^p sum_{r=0}^{P-p} bh_r/(p+r)!
//   bh'_q = sum_{m=0}^{q-1} ch_m bh_{q-m} + c^q sum_{r=0}^{P-q} ah_r/(q+r)!
//   b'_0  = b_0 + sum_{p>=1} ah_p / p!
// (ah_0 := bh_0 := b_0, the corner value; a_0 is never used, as in the proof
// where the diagonal carries the left-edge constant).  Rings m = min(p,q) are
// the Neumann iterates T^m of Sec. 2.2.2; only m <= nr are kept (the local
// Neumann iteration count, App. C.3: the a-priori order choice), and of those
// only the entries of weighted degree 2m + k <= 2 nr + 1, k = |p - q| the
// degree of the edge coefficient they carry (keep_entry below).  Every
// constant is a compile-time entry of a __constant__ table, so each term is
// one FFMA.
//
// Precision.  The corner value b_0 is carried as an unevaluated float-float
// pair (hi, lo): it is the only O(1) quantity that accumulates an O(1)
// rounding error per tile.  All other coefficients are FP32.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sigk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kG = 32;            // columns per seam block (one warp width)
constexpr int kMaxP = 16;         // maximum edge degree
constexpr int kMaxRings = 8;      // maximum Neumann iterations per tile
// adjoint, passes A and B: coefficient loads in flight per lane (the
// per-warp strip area holds max_len + 32 + kB2PF rows of 32 entries); four
// in flight measured 79.5 against 68.3 ms on the 64-path Gram
constexpr int kB2PF = 2;

// 1/k! for k = 0..33, rounded to FP32 (all normal numbers; the tile map
// indexes at most k = 16).  Each translation unit holds its own copy.
static __constant__ float c_inv_fact[34] = {1.0f, 1.0f, 0.5f, 0.166666667f, 0.0416666667f, 0.00833333333f, 0.00138888889f, 0.000198412698f, 2.48015873e-05f, 2.75573192e-06f, 2.75573192e-07f, 2.50521084e-08f, 2.0876757e-09f, 1.60590438e-10f, 1.14707456e-11f, 7.64716373e-13f, 4.77947733e-14f, 2.81145725e-15f, 1.5619207e-16f, 8.22063525e-18f, 4.11031762e-19f, 1.95729411e-20f, 8.89679139e-22f, 3.86817017e-23f, 1.61173757e-24f, 6.44695028e-26f, 2.47959626e-27f, 9.18368986e-29f, 3.27988924e-30f, 1.13099629e-31f, 3.76998763e-33f, 1.21612504e-34f, 3.80039075e-36f, 1.15163356e-37f};

enum : int {
    kOK = 0, kErrArg = -1, kErrLength = -2, kErrNonfinite = -3, kErrWorkspace = -4,
    kErrCuda = -5, kErrTimeout = -6, kErrBounds = -9
};

struct PairDesc {
    const float* xr;   // row path (split into strips over warp lanes)
    const float* yr;   // swept path
    int32_t L1;        // segments of the row path
    int32_t L2;        // segments of the swept path
    int32_t n_strips;  // ceil(L1 / rows per strip)
    int32_t swapped;   // 1 if the row path is the caller's y
    int32_t sx;        // refinement of the row path: each segment in sx pieces
    int32_t sy;        // refinement of the swept path
    int32_t xslot;     // index of the row path among the call's paths (X, then Y)
    int32_t yslot;     // index of the swept path among the call's paths
    int64_t out0;      // output index, or -1
    int64_t out1;      // mirrored output index, or -1
    float* gxr;        // gradient rows of the row path (backward), or null
    float* gyr;        // gradient rows of the swept path (backward), or null
};

// Work schedule written by the planner (three ints in the workspace header):
// [0] mode, [1] n_levels (mode 1) or sorted pairs (mode 2), [2] n_items.
//   mode 0, pair-major in index order: the strips of a pair are consecutive
//     items (item_start prefix sums over the pairs); a strip consumes the seam
//     of item - 1.
//   mode 1, strip-major: level l holds strip l of every pair that has one,
//     pairs ordered by decreasing strip count (order[]); level_start[l] is
//     the first item of level l.  A strip's producer is a whole level earlier,
//     so a consumer rarely waits.  Used when the strip counts are even.
//   mode 2, pair-major over order[]: item_start holds the prefix sums in that
//     order, so the pairs with the longest chains of strips start first.
//
// A schedule may count work in units of 2^shift strips (the training forward
// solves 32*R rows per item while the table counts 32-row strips): a pair
// with n strips has ceil(n / 2^shift) items.
struct Schedule {
    const int* hdr;                // mode, n_levels / sorted pairs, n_items
    const int32_t* item_start;     // modes 0, 2: [pairs + 1] prefix sums of the items per pair
    const int32_t* order;          // modes 1, 2: pairs by decreasing strip count
    const int32_t* level_start;    // mode 1: [n_levels + 1]
    int32_t n_pairs;
    int32_t shift;                 // items are 2^shift strips
};

struct ItemRef {
    int pair;   // index into the pair table
    int k;      // position of the strip in the pair's sequence (0 first)
    int prev;   // item that produces this strip's incoming seam, or -1
    int next;   // item that consumes this strip's outgoing seam, or -1
};

// Floats in a tile record (written by the training forward or the adjoint's
// replay, read by the reverse sweep): [0] the incoming corner (high part),
// [1] b1 with its low part added, [q] b_q for q = 2..P, [P + 1] the exponent
// word -- P + 2 floats for the even orders, moved as 8-byte pairs.
__host__ __device__ constexpr int rec_floats(int P) { return (P + 3) / 2 * 2; }

// Floats per column of the adjoint seam (corner adjoint, b1..bP adjoints):
// padded to a multiple of 4 (128-bit shared loads and stores) up to P = 12;
// at P >= 14 the padding would cost the adjoint its third CTA per SM.
__host__ __device__ constexpr int adj_seam_floats(int P) { return P <= 12 ? (P + 4) / 4 * 4 : P + 1; }

// Largest i in [0, n) with v[i] <= x (v non-decreasing, v[0] <= x).
__device__ __forceinline__ int upper_index(const int32_t* v, int n, int x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (v[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ ItemRef decode_item(const Schedule& S, const PairDesc* pairs, int item) {
    ItemRef r;
    if (S.hdr[0] == 1) {
        const int nl = S.hdr[1];
        const int l = upper_index(S.level_start, nl, item);
        const int rank = item - S.level_start[l];
        r.pair = S.order[rank];
        r.k = l;
        r.prev = l > 0 ? S.level_start[l - 1] + rank : -1;
        r.next = (l + 1 < nl && rank < S.level_start[l + 2] - S.level_start[l + 1])
                     ? S.level_start[l + 1] + rank : -1;
    } else {
        const bool sorted = S.hdr[0] == 2;
        const int q = upper_index(S.item_start, sorted ? S.hdr[1] : S.n_pairs, item);
        const int p = sorted ? S.order[q] : q;
        r.pair = p;
        r.k = item - S.item_start[q];
        r.prev = r.k > 0 ? item - 1 : -1;
        const int units = (pairs[p].n_strips + (1 << S.shift) - 1) >> S.shift;
        r.next = r.k + 1 < units ? item + 1 : -1;
    }
    return r;
}

struct SolverArgs {
    const PairDesc* pairs;
    Schedule sched;
    int32_t n_pairs;
    int32_t inc_mode;              // rows of xr/yr are increments (else points)
    int32_t d;
    int32_t nr;                    // Neumann rings kept per tile
    int32_t nslot;                 // seam ring slots
    int32_t wcols;                 // columns per slot (multiple of kG)
    float* seam;                   // nslot * wcols * stride floats
    unsigned long long* prod;      // [nslot] (item << 32) | columns published
    unsigned long long* cons;      // [nslot] (consumer item << 32) | columns read
    long long* done;               // [nslot] last finished item with that residue
    int* item_counter;
    int* status;
    unsigned long long* counters;  // [0] tiles, [1] lane-tiles incl. padding
    double* out;
    // training forward (backward pass follows): every strip's right-edge seam
    // goes to a per-pair store instead of the ring, and the final exponent of
    // each pair is recorded.  store == nullptr: inference.
    float* store;
    const int64_t* store_off;      // [n_pairs] float offsets into store
    int32_t* pair_exp;             // [n_pairs] or null
    // training with stored tile records: every tile's record as the adjoint
    // reads it, per work item (pair, R strips of 32 rows) (L2 + 32) blocks of
    // 32 * R records of rec_floats(P) floats -- block t holds the records of
    // the item's rows at step t (row lane*R + k at column t - lane), block
    // L2 + 31 the rows' bottom-edge states after the last column.  rec ==
    // nullptr: the adjoint replays the strips instead.
    float* rec;
    const int64_t* rec_off;        // [n_pairs] float offsets into rec
    // fault-injection hook (tests of the bounded waits): the schedule's first
    // item does not publish its outgoing seam
    int32_t withhold_first_seam;
    // per-tile ring count (inference forwards; 0 = the fixed count NR): a
    // tile whose |c| is at most ring_theta[k] needs at most 2k + 2 rings (its
    // first dropped ring |c|^(n+1)/((n+1)!)^2 stays below the ring tolerance);
    // a warp uses the largest count any of its tiles of the step needs
    int32_t ring_adaptive;
    float ring_theta[3];
    unsigned* ring_hist;           // [4] tiles solved with 2, 4, 6, 8 rings (adaptive launches)
    // extents of the buffers above, for the bounds checks of SIGK_DEBUG builds
    int32_t nwords;                // progress words (prod, cons, done)
    int64_t store_cap;             // floats of store
    int64_t rec_cap;               // floats of rec
    int64_t out_cap;               // entries of out
};

// Tile records (layout above).  rec_put_head stores every pair but the last,
// which holds the exponent word (known only after the tile); rec_put_tail
// stores that pair (b_P as recorded, the exponent word).
template <int P>
__device__ __forceinline__ void rec_put_head(float* dst, float hi, float b1lo, const float (&b)[P + 1]) {
    constexpr int RS = rec_floats(P);
    float rv[RS];
    rv[0] = hi;
    rv[1] = b[1] + b1lo;
#pragma unroll
    for (int q = 2; q <= P; ++q) rv[q] = b[q];
#pragma unroll
    for (int q = P + 1; q < RS; ++q) rv[q] = 0.0f;
    float2* d2 = reinterpret_cast<float2*>(dst);
#pragma unroll
    for (int g = 0; g < RS / 2 - 1; ++g) d2[g] = make_float2(rv[2 * g], rv[2 * g + 1]);
}
template <int P>
__device__ __forceinline__ void rec_put_tail(float* dst, float bP, int expw) {
    constexpr int RS = rec_floats(P);
    static_assert(RS == P + 2, "the last pair is (b_P, exponent word)");
    reinterpret_cast<float2*>(dst)[RS / 2 - 1] = make_float2(bP, __int_as_float(expw));
}
template <int P>
__device__ __forceinline__ void rec_get(const float* src, float& hi, float (&b)[P + 1], int& expw) {
    constexpr int RS = rec_floats(P);
    float rv[RS];
    const float2* s2 = reinterpret_cast<const float2*>(src);
#pragma unroll
    for (int g = 0; g < RS / 2; ++g) {
        const float2 v = s2[g];
        rv[2 * g] = v.x;
        rv[2 * g + 1] = v.y;
    }
    hi = rv[0];
    b[0] = 0.0f;
#pragma unroll
    for (int q = 1; q <= P; ++q) b[q] = rv[q];
    expw = __float_as_int(rv[P + 1]);
}
// A row's final bottom-edge state (a1lo, a_1..a_P) in a record slot.
template <int P>
__device__ __forceinline__ void rec_put_state(float* dst, float a1lo, const float (&a)[P + 1]) {
    constexpr int RS = rec_floats(P);
    float fv[RS];
    fv[0] = a1lo;
#pragma unroll
    for (int p = 1; p <= P; ++p) fv[p] = a[p];
#pragma unroll
    for (int q = P + 1; q < RS; ++q) fv[q] = 0.0f;
    float2* d2 = reinterpret_cast<float2*>(dst);
#pragma unroll
    for (int g = 0; g < RS / 2; ++g) d2[g] = make_float2(fv[2 * g], fv[2 * g + 1]);
}
template <int P>
__device__ __forceinline__ void rec_get_state(const float* src, float& a1lo, float (&a)[P + 1]) {
    constexpr int RS = rec_floats(P);
    float fv[RS];
    const float2* s2 = reinterpret_cast<const float2*>(src);
#pragma unroll
    for (int g = 0; g < RS / 2; ++g) {
        const float2 v = s2[g];
        fv[2 * g] = v.x;
        fv[2 * g + 1] = v.y;
    }
    a1lo = fv[0];
#pragma unroll
    for (int p = 1; p <= P; ++p) a[p] = fv[p];
}

// ---------------------------------------------------------------------------
// memory-order helpers
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_acquire_s64(const long long* p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_s64(long long* p, long long v) {
    asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_s32(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A non-finite result (NaN or Inf in the data, or beyond the range of the
// power-of-two exponent) is recorded in the word after the three work
// counters of the header (status + 3), not in the status word: it is an
// error of that output alone, and the launch carries on with every other
// pair (the status word stops the launch).
__device__ __forceinline__ void record_nonfinite(int* status) { atomicExch(status + 3, 1); }

// First time-out of a launch: the status word, then (for diagnosis) the
// waited-on address, the target and the value last seen, as three 64-bit
// words at byte 128 of the status word's 256-byte header.
__device__ __forceinline__ void record_timeout(int* status, const void* p, long long target,
                                               long long seen) {
    if (atomicCAS(status, 0, kErrTimeout) == 0) {
        long long* diag = reinterpret_cast<long long*>(status + 32);
        diag[0] = (long long)(uintptr_t)p;
        diag[1] = target;
        diag[2] = seen;
    }
}

// Bounds checks of the SIGK_DEBUG build: a region a work item is about to
// touch must lie inside its buffer.  On a violation the first one is recorded
// (status kErrBounds; diagnosis: check site, offending offset, limit) and the
// caller skips the access; in other builds the check is compiled out.
__device__ __forceinline__ bool dbg_in(int* status, int site, long long off, long long lim) {
#ifdef SIGK_DEBUG
    if (off >= 0 && off <= lim) return true;
    if (atomicCAS(status, 0, kErrBounds) == 0) {
        long long* diag = reinterpret_cast<long long*>(status + 32);
        diag[0] = site;
        diag[1] = off;
        diag[2] = lim;
    }
    return false;
#else
    (void)status; (void)site; (void)off; (void)lim;
    return true;
#endif
}

// Bounded wait until *p >= target.  Gives up after the call's wait budget
// (the 64-bit word kHdrWaitNs bytes after the status word, in nanoseconds of
// %globaltimer; 0 means 4 s), or a hard iteration cap, or as soon as another
// warp has recorded an error; on time-out it records kErrTimeout.  Returns
// true when the condition holds.
constexpr unsigned long long kWaitNs = 4000000000ull;
constexpr int kWaitMaxIter = 1 << 24;
constexpr int kHdrWaitNs = 152;  // byte offset of the budget from the status word

__device__ __forceinline__ unsigned long long wait_budget(const int* status) {
    const unsigned long long b =
        *reinterpret_cast<const volatile unsigned long long*>(reinterpret_cast<const char*>(status) + kHdrWaitNs);
    return b ? b : kWaitNs;
}

__device__ __forceinline__ bool wait_ge_u64(const unsigned long long* p,
                                            unsigned long long target, int* status) {
    if (ld_acquire_u64(p) >= target) return true;
    const unsigned long long t0 = global_ns();
    const unsigned long long budget = wait_budget(status);
    for (int it = 0; it < kWaitMaxIter; ++it) {
        __nanosleep(it < 64 ? 32 : 256);
        if (ld_acquire_u64(p) >= target) return true;
        if ((it & 31) == 31) {
            if (ld_volatile_s32(status) != 0) return false;
            if (global_ns() - t0 > budget) break;
        }
    }
    record_timeout(status, p, (long long)target, (long long)ld_acquire_u64(p));
    return false;
}

__device__ __forceinline__ bool wait_ge_s64(const long long* p, long long target, int* status) {
    if (ld_acquire_s64(p) >= target) return true;
    const unsigned long long t0 = global_ns();
    const unsigned long long budget = wait_budget(status);
    for (int it = 0; it < kWaitMaxIter; ++it) {
        __nanosleep(it < 64 ? 32 : 256);
        if (ld_acquire_s64(p) >= target) return true;
        if ((it & 31) == 31) {
            if (ld_volatile_s32(status) != 0) return false;
            if (global_ns() - t0 > budget) break;
        }
    }
    record_timeout(status, p, target, ld_acquire_s64(p));
    return false;
}

// ---------------------------------------------------------------------------
// Asynchronous copies.  Shared-memory addresses for PTX operands:
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// make this thread's generic-proxy writes to shared memory visible to the
// async proxy (before a bulk store reads them)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Before item writes seam slot item % nslot: the slot's previous user u =
// item - nslot must have been read completely by u's consumer.  Lane 0 waits
// (bounded); the result is broadcast to the warp.
__device__ __forceinline__ bool wait_slot_free(const Schedule& S, const PairDesc* pairs, int item,
                                               int nslot, const long long* done, int* status) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0 && item >= nslot) {
        const int c = decode_item(S, pairs, item - nslot).next;
        if (c >= 0) ok = wait_ge_s64(&done[c % nslot], (long long)c, status);
    }
    return __shfl_sync(kFull, ok, 0);
}

// Asynchronous 8-byte global -> shared copies of one thread (cp.async),
// committed as a group; wait_group N waits until at most N of this thread's
// groups are still in flight.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)), "l"(gsrc)
                 : "memory");
}
// 16-byte copy of which only the first src_bytes (0 or 16) are read; the rest
// of the 16 bytes is filled with zeros.  Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16z(void* smem_dst, const void* gsrc, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// A seam entry (corner hi, lo, b1lo, b_1..b_P, exponent: S = P + 4 floats,
// even) between shared memory and registers in the widest aligned words:
// 16-byte accesses when S is a multiple of 4 (the entry then starts on a
// 16-byte boundary), else 8-byte ones.  One lane reads or writes a whole
// entry per step, so the width sets how many shared-memory instructions the
// warp issues for it.
template <int S>
__device__ __forceinline__ void seam_entry_load(const float* src, float (&v)[S]) {
    static_assert(S % 2 == 0, "seam entries hold an even number of floats");
    if constexpr (S % 4 == 0) {
#pragma unroll
        for (int g = 0; g < S / 4; ++g) {
            const float4 w = reinterpret_cast<const float4*>(src)[g];
            v[4 * g] = w.x; v[4 * g + 1] = w.y; v[4 * g + 2] = w.z; v[4 * g + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int g = 0; g < S / 2; ++g) {
            const float2 w = reinterpret_cast<const float2*>(src)[g];
            v[2 * g] = w.x; v[2 * g + 1] = w.y;
        }
    }
}
template <int S>
__device__ __forceinline__ void seam_entry_store(float* dst, const float (&v)[S]) {
    static_assert(S % 2 == 0, "seam entries hold an even number of floats");
    if constexpr (S % 4 == 0) {
#pragma unroll
        for (int g = 0; g < S / 4; ++g)
            reinterpret_cast<float4*>(dst)[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
    } else {
#pragma unroll
        for (int g = 0; g < S / 2; ++g) reinterpret_cast<float2*>(dst)[g] = make_float2(v[2 * g], v[2 * g + 1]);
    }
}
// Pack / unpack the left edge of one lane as a seam entry.
template <int P>
__device__ __forceinline__ void seam_pack(float (&v)[P + 4], float hi, float lo, float b1lo,
                                          const float (&b)[P + 1], int E) {
    v[0] = hi; v[1] = lo; v[2] = b1lo;
#pragma unroll
    for (int q = 1; q <= P; ++q) v[2 + q] = b[q];
    v[P + 3] = __int_as_float(E);
}
template <int P>
__device__ __forceinline__ void seam_unpack(const float (&v)[P + 4], float& hi, float& lo, float& b1lo,
                                            float (&b)[P + 1], int& F) {
    hi = v[0]; lo = v[1]; b1lo = v[2];
#pragma unroll
    for (int q = 1; q <= P; ++q) b[q] = v[2 + q];
    F = __float_as_int(v[P + 3]);
}

// Bulk (TMA) store of `bytes` from shared to global memory, in this
// thread's bulk async-group; both addresses 16-byte aligned, bytes a
// multiple of 16.  The async proxy is outside the ordering of generic
// fences, so a later __threadfence does not wait for it.
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most N of this thread's bulk groups may still be reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// all of this thread's bulk groups complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 2^n as a float for n <= 0 (0 below the normal range).
__device__ __forceinline__ float exp2_nonpos(int n) {
    return n < -126 ? 0.0f : __int_as_float((127 + n) << 23);
}
__device__ __forceinline__ float exp2_nonneg(int n) {
    return __int_as_float((127 + (n > 127 ? 127 : n)) << 23);
}

// Exponent word of a tile record: bbump (bit 31) | F/64 (14 bits) |
// E_before/64 (16 bits) | abump (bit 0).  F is the exponent of the tile's
// incoming left edge, E_before that of the row's bottom-edge state before the
// tile (both non-negative multiples of 64), abump = 1 when the row's
// bottom-edge state was rescaled by 2^-64 after the tile, bbump = 1 when the
// tile's outgoing right edge was.  With one row per lane the two bumps
// coincide; with several rows per lane only the last row's right edge leaves
// the lane, and only it is rescaled.
__device__ __forceinline__ int pack_exp(int F, int Eb, int abump, int bbump) {
    return (int)(((unsigned)bbump << 31) | ((unsigned)((F >> 6) & 0x3FFF) << 17) |
                 ((unsigned)((Eb >> 6) & 0xFFFF) << 1) | (unsigned)abump);
}
// True when the record's tile needed no exponent handling: the incoming edge
// had the row's exponent and nothing was rescaled (the common case).
__device__ __forceinline__ bool exp_plain(int w) {
    const unsigned u = (unsigned)w;
    return (u & 0x80000001u) == 0u && ((u >> 17) & 0x3FFFu) == ((u >> 1) & 0xFFFFu);
}
__device__ __forceinline__ void unpack_exp(int w, int& F, int& Eb, int& abump, int& bbump) {
    abump = w & 1;
    bbump = (int)((unsigned)w >> 31);
    Eb = (int)(((unsigned)w >> 1) & 0xFFFF) * 64;
    F = (int)(((unsigned)w >> 17) & 0x3FFF) * 64;
}

// Rings a tile with coefficient magnitude ac needs (2, 4, 6 or 8) under the
// launch's thresholds (SolverArgs::ring_theta).
__device__ __forceinline__ int rings_needed(float ac, const float (&th)[3]) {
    return ac <= th[0] ? 2 : (ac <= th[1] ? 4 : (ac <= th[2] ? 6 : 8));
}

// Entries of the tile matrix that the truncation keeps.  An entry of ring m
// (the power c^m, 1 <= m <= nr) multiplies an edge coefficient of degree k
// (k = 0: the corner); it is kept when its total degree m + k is at most P
// and its weighted degree 2m + k at most 2 NT + 1, NT being the launch's ring
// count.  Each power of c counts twice: a tile coefficient is the product of
// two increments, a coupling (which sets the size of an edge coefficient of
// degree k, ~ C^k / (k!)^2) is the product of an increment and a whole path
// prefix, so c is of the order of C^2 or smaller on Brownian-type paths.  An
// FP64 emulation of the scheme on the 1024-segment Grams measured the error
// of this truncation against the exact kernel at 2.4e-10 (sigma = 1, P = 8,
// NT = 4: 36 of the square's 48 entries) and 1.9e-8 (sigma = 4, NT = 6: 78
// of 156 entries at P = 16).  No entry reaches degree 2 NT + 1, so an edge
// degree P > 2 NT computes exactly what P = 2 NT computes (the solver
// launches with P clamped to 2 NT).
__host__ __device__ constexpr bool keep_entry(int P, int NT, int nr, int m, int k) {
    return m >= 1 && m <= nr && k >= 0 && m + k <= P && 2 * m + k <= 2 * NT + 1;
}

// ---------------------------------------------------------------------------
// One tile.  a[1..P]: scaled bottom edge (overwritten by the top edge);
// (hi, lo), b[1..P]: scaled left edge (overwritten by the right edge).  NT:
// the launch's ring count (the truncation's weighted degree); nr <= NT: the
// rings of this tile (a compile-time constant at every call site).
//
// CLO: the coefficient is the unevaluated float-float pair c + clo (an
// increment Gram computed beyond FP32 precision).  Rounding c to one float
// perturbs every tile by a relative 2^-24, and over the millions of tiles of
// a long, strongly coupled pair these perturbations reach the 1e-5 level of
// k (CPU emulation of this sweep: 1.1e-5 with the FP32 dot products, 3e-6
// with c correctly rounded, 8e-7 with the pair).  The low part enters where
// the result is first order in c: the m = 1 ring of every edge coefficient
// (clo * a_{p-1}) and the first-order coefficients, whose product c * ha_1 is
// then formed exactly (TwoProduct) before the compensated accumulation.
template <int P, int NT, bool CLO = false>
__device__ __forceinline__ void tile_update(float c, float (&a)[P + 1], float& a1lo, float& hi,
                                            float& lo, float (&b)[P + 1], float& b1lo, int nr,
                                            float clo = 0.0f) {
    constexpr int NRM = P < NT ? P : NT;
    float cp[NRM + 1], ch[NRM + 1];
    cp[1] = c;
    ch[1] = c;
#pragma unroll
    for (int m = 2; m <= NRM; ++m) {
        cp[m] = cp[m - 1] * c;
        ch[m] = cp[m] * c_inv_fact[m];
    }
    // ring-p Hankel sums of the incoming edges over the kept offsets
    // (b_0 = a_0 := hi)
    float ha[NRM + 1], hb[NRM + 1];
#pragma unroll
    for (int p = 1; p <= NRM; ++p) {
        ha[p] = 0.0f;
        hb[p] = 0.0f;
        if (p <= nr) {
            float sa = hi * c_inv_fact[p];
            float sb = sa;
#pragma unroll
            for (int r = 1; r <= P - p; ++r) {
                if (keep_entry(P, NT, nr, p, r)) {
                    sa = fmaf(b[r], c_inv_fact[p + r], sa);
                    sb = fmaf(a[r], c_inv_fact[p + r], sb);
                }
            }
            ha[p] = sa;
            hb[p] = sb;
        }
    }
    // bottom edge evaluated at u = 1 (without its constant term)
    float S = a1lo;
#pragma unroll
    for (int p = P; p >= 1; --p) S = fmaf(a[p], c_inv_fact[p], S);
    // top edge (in place, high degree first: reads only lower, older entries)
#pragma unroll
    for (int p = P; p >= 2; --p) {
        float v = a[p];
#pragma unroll
        for (int m = 1; m < p && m <= NRM; ++m)
            if (keep_entry(P, NT, nr, m, p - m)) v = fmaf(ch[m], a[p - m], v);
        if (p <= NRM && p <= nr) v = fmaf(cp[p], ha[p], v);
        if constexpr (CLO)
            if (keep_entry(P, NT, nr, 1, p - 1)) v = fmaf(clo, a[p - 1], v);
        a[p] = v;
    }
    // right edge
#pragma unroll
    for (int q = P; q >= 2; --q) {
        float v = b[q];
#pragma unroll
        for (int m = 1; m < q && m <= NRM; ++m)
            if (keep_entry(P, NT, nr, m, q - m)) v = fmaf(ch[m], b[q - m], v);
        if (q <= NRM && q <= nr) v = fmaf(cp[q], hb[q], v);
        if constexpr (CLO)
            if (keep_entry(P, NT, nr, 1, q - 1)) v = fmaf(clo, b[q - 1], v);
        b[q] = v;
    }
    // first-order coefficients: compensated (TwoSum) accumulation.  Along a
    // long row or column they gather ~L increments of only a few ulps each,
    // whose plain FP32 rounding is biased rather than random.
    // The pair is renormalised (Fast2Sum) so that the high part stays the
    // nearest float to the full value: the Hankel sums and convolutions read
    // only the high part.
    {
        const float da = cp[1] * ha[1], db = cp[1] * hb[1];
        const float sa = a[1] + da, sb = b[1] + db;
        const float ta = sa - a[1], tb = sb - b[1];
        float la = a1lo + ((a[1] - (sa - ta)) + (da - ta));
        float lb = b1lo + ((b[1] - (sb - tb)) + (db - tb));
        if constexpr (CLO) {  // exact product error of c * ha_1, and the low part of c
            la += fmaf(clo, ha[1], fmaf(c, ha[1], -da));
            lb += fmaf(clo, hb[1], fmaf(c, hb[1], -db));
        }
        a[1] = sa + la;
        b[1] = sb + lb;
        a1lo = la - (a[1] - sa);
        b1lo = lb - (b[1] - sb);
    }
    // corner value b'_0 = b_0 + S in float-float: TwoSum, then Fast2Sum
    // renormalisation so that hi is the nearest float to hi + lo (hi is what
    // the next tiles' Hankel sums read)
    const float s = hi + S;
    const float bb = s - hi;
    const float t = lo + ((hi - (s - bb)) + (S - bb));
    hi = s + t;
    lo = t - (hi - s);
}

// Inverse of the bottom-to-top edge update of tile_update, given the tile's
// left edge (hi, b) and its top edge a2: the update is unit lower triangular
// in the degree (a'_p = a_p + sum_m ch_m a_{p-m} + c^p ha_p(b) over the kept
// entries), so the bottom edge is recovered degree by degree.  Used by the
// reverse sweep to rebuild each tile's inputs from the stored left edges
// instead of storing every tile.  ha (rings p <= nr) is returned for the
// adjoint.
template <int P, int NT>
__device__ __forceinline__ void tile_inverse_a(float c, const float (&a2)[P + 1], float hi,
                                               const float (&b)[P + 1], int nr,
                                               float (&a)[P + 1], float (&ha)[P + 1]) {
    constexpr int NRM = P < NT ? P : NT;
    float cp[NRM + 1], ch[NRM + 1];
    cp[1] = c;
    ch[1] = c;
#pragma unroll
    for (int m = 2; m <= NRM; ++m) {
        cp[m] = cp[m - 1] * c;
        ch[m] = cp[m] * c_inv_fact[m];
    }
#pragma unroll
    for (int p = 1; p <= P; ++p) {
        float v = a2[p];
        ha[p] = 0.0f;
        if (p <= NRM && p <= nr) {
            float sa = hi * c_inv_fact[p];
#pragma unroll
            for (int r = 1; r <= P - p; ++r)
                if (keep_entry(P, NT, nr, p, r)) sa = fmaf(b[r], c_inv_fact[p + r], sa);
            ha[p] = sa;
            v = fmaf(-cp[p], sa, v);
        }
        // highest ring first: a[p - 1], the value computed last, enters last,
        // so the degree-by-degree recovery waits one FMA per degree
#pragma unroll
        for (int m = (p - 1 < NRM ? p - 1 : NRM); m >= 1; --m)
            if (keep_entry(P, NT, nr, m, p - m)) v = fmaf(-ch[m], a[p - m], v);
        a[p] = v;
    }
    a[0] = 0.0f;
}

// Reverse-mode adjoint of tile_update (the exact derivative of the truncated
// FP32 scheme, with the float-float corner treated as one real b0 = hi + lo).
// Forward inputs: c, a (bottom edge), hi, b (left edge), ha (ring Hankel sums
// of b, from tile_inverse_a).  Adjoint inputs: A2 (top edge), B02 (corner),
// B2 (right edge).  Outputs overwrite them with the adjoints of the bottom edge
// (A), the corner (B0) and the left edge (B); returns dk/dc.
template <int P, int NT>
__device__ __forceinline__ float tile_adjoint(float c, const float (&a)[P + 1], float hi,
                                              const float (&b)[P + 1], const float (&ha)[P + 1],
                                              float (&A)[P + 1], float& B0, float (&B)[P + 1],
                                              int nr) {
    constexpr int NRM = P < NT ? P : NT;
    float cp[NRM + 1], ch[NRM + 1];
    cp[1] = c;
    ch[1] = c;
#pragma unroll
    for (int m = 2; m <= NRM; ++m) {
        cp[m] = cp[m - 1] * c;
        ch[m] = cp[m] * c_inv_fact[m];
    }
    // hb from the bottom edge (as in the forward)
    float hb[NRM + 1];
#pragma unroll
    for (int p = 1; p <= NRM; ++p) {
        hb[p] = 0.0f;
        if (p <= nr) {
            float sb = hi * c_inv_fact[p];
#pragma unroll
            for (int r = 1; r <= P - p; ++r)
                if (keep_entry(P, NT, nr, p, r)) sb = fmaf(a[r], c_inv_fact[p + r], sb);
            hb[p] = sb;
        }
    }
    // c-bar contributions: d ch_m / dc = ch_{m-1}, d cp_m / dc = m cp_{m-1}
    float cbar = 0.0f;
    // correlation sums chb_m = sum_p A2_p a_{p-m} + B2_p b_{p-m} (kept entries)
#pragma unroll
    for (int m = 1; m <= NRM; ++m) {
        if (m <= nr) {
            // two independent accumulators (bottom- and left-edge terms)
            float chA = 0.0f, chB = 0.0f;
#pragma unroll
            for (int p = m + 1; p <= P; ++p) {
                if (keep_entry(P, NT, nr, m, p - m)) {
                    chA = fmaf(A[p], a[p - m], chA);
                    chB = fmaf(B[p], b[p - m], chB);
                }
            }
            const float dch = (m == 1) ? 1.0f : ch[m - 1];
            cbar = fmaf(chA + chB, dch, cbar);
            // ring-m Hankel term: d/dcp_m (cp_m (A2_m ha_m + B2_m hb_m))
            const float dcp = (m == 1) ? 1.0f : (float)m * cp[m - 1];
            cbar = fmaf(fmaf(A[m], ha[m], B[m] * hb[m]), dcp, cbar);
        }
    }
    // transposed Hankel: hab_p = cp_p A2_p feeds B_r and the corner
    float hab[NRM + 1], hbb[NRM + 1];
#pragma unroll
    for (int p = 1; p <= NRM; ++p) {
        hab[p] = (p <= nr) ? cp[p] * A[p] : 0.0f;
        hbb[p] = (p <= nr) ? cp[p] * B[p] : 0.0f;
    }
    // transposed convolution (low degree first: reads only higher, older entries)
    const float Sbar = B0;
#pragma unroll
    for (int s = 1; s <= P; ++s) {
        float va = A[s], vb = B[s];
#pragma unroll
        for (int m = 1; m <= NRM && s + m <= P; ++m)
            if (keep_entry(P, NT, nr, m, s)) {
                va = fmaf(ch[m], A[s + m], va);
                vb = fmaf(ch[m], B[s + m], vb);
            }
        va = fmaf(Sbar, c_inv_fact[s], va);  // corner b0' = b0 + sum_p a_p / p!
#pragma unroll
        for (int p = 1; p <= NRM && p + s <= P; ++p) {
            if (keep_entry(P, NT, nr, p, s)) {
                va = fmaf(hbb[p], c_inv_fact[p + s], va);  // hb_p reads a_s
                vb = fmaf(hab[p], c_inv_fact[p + s], vb);  // ha_p reads b_s
            }
        }
        A[s] = va;
        B[s] = vb;
    }
    float b0 = B0;
#pragma unroll
    for (int p = 1; p <= NRM; ++p) b0 = fmaf(hab[p] + hbb[p], c_inv_fact[p], b0);
    B0 = b0;
    A[0] = 0.0f;
    B[0] = 0.0f;
    return cbar;
}

// Kept entries of the tile matrix: 1 for a diagonal entry (k = 0), 2 for an
// off-diagonal one (it appears above and below the diagonal).
__host__ __device__ constexpr int kept_entries(int P, int NT, int nr) {
    int n = 0;
    for (int m = 1; m <= P; ++m)
        for (int k = 0; k <= P; ++k)
            if (keep_entry(P, NT, nr, m, k)) n += (k == 0) ? 1 : 2;
    return n;
}

// FP32 operations of tile_update (FMA counted as 2), for the roofline.
__host__ __device__ constexpr long long tile_flops(int P, int NT, int nr) {
    long long f = 0;
    const int nrm = P < NT ? P : NT;
    if (nr > nrm) nr = nrm;
    f += 2 * (nr - 1);                           // powers
    f += 2 * nr;                                 // corner terms of the Hankel sums (1 mul each)
    f += 2 * 2 * kept_entries(P, NT, nr);        // 2 FMAs per kept entry (one per outgoing edge)
    f += 2 * P;                                  // S
    f += 10;                                     // float-float corner
    f += 18;                                     // compensated a1, b1
    return f;
}

// The kept-entry counts and per-tile operation counts that the roofline
// figures use (bench.py mirrors them; tests/test_bench_cpu.py pins the same
// numbers), checked here against keep_entry itself.
static_assert(kept_entries(8, 4, 4) == 36 && kept_entries(6, 3, 3) == 21 && kept_entries(12, 6, 6) == 78,
              "kept entries of the weighted-degree truncation");
static_assert(kept_entries(16, 6, 6) == kept_entries(12, 6, 6), "no kept entry above degree 2n");
static_assert(tile_flops(8, 4, 4) == 234 - 2 * 16 && tile_flops(6, 3, 3) == 166 - 2 * 16 &&
                  tile_flops(12, 6, 6) == 418 - 2 * 16,
              "tile operations without the increment inner product");

}  // namespace sigk
