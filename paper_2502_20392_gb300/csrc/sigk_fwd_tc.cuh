// sigk_fwd_tc.cuh -- forward solver for paths of large dimension d with the
// increment Gram c_ij = <dx_i, dy_j> on the tensor cores (tcgen05), in
// float-float precision, and the FP32 wavefront sweep.
//
// The coefficient of every tile is a dense contraction over d (the rho of the
// coefficient on all tiles, Sec. 2.1; the rho step of the App. C.1 algorithm).
// It is formed here exactly enough to be carried as an unevaluated pair
// c + clo: each increment row is scaled by a power of two 2^e so that its
// largest entry lies in [64, 128), and written as four signed 8-bit digits,
//     x = 2^e (t0 + t1 2^-8 + t2 2^-16 + t3 2^-24) + r,  |r| <= 2^(e-25),
// each digit an integer in [-128, 128] and therefore exact in BF16.  Digit
// products summed over d are integers that the tensor core accumulates in
// FP32 without rounding while they stay below 2^24 (d <= 1024 for the leading
// group); the products of digit orders k + l = g are summed into one TMEM
// accumulator per g = 0..3, and
//     c = 2^(e_i + e_j) (G0 + 2^-8 G1 + 2^-16 G2 + 2^-24 G3)
// is rounded once into (c, clo).  The dropped products (k + l >= 4) and the
// digit remainders leave c correct to about 2^-31 of the rows' largest
// products, far below FP32 rounding.
//
// Work unit: a block of 128 rows = four 32-row strips of one pair (the pair
// table counts 32-row strips, padded to a multiple of four; the schedule is
// pair-major, so the four strips are consecutive work items).  One CTA per SM
// (it holds all of TMEM) splits the work between a producer and sweepers:
//   producer (warps 0-3)  claims a block whenever one of the CTA's kTcSlots
//            block slots is free, cuts the block's rows into digits in a
//            per-CTA global area, and forms the coefficients 64 columns at a
//            time: a four-stage cp.async pipeline stages the digit tiles (16
//            dimensions per step) in the tensor core's shared-memory layout,
//            one thread issues the ten 128x64x16 MMAs of each step into one
//            of two TMEM buffers, and the previous chunk is read back
//            (tcgen05.ld) meanwhile into the strips' coefficient areas,
//            skewed so that the 32 values a warp's lanes read in one sweep
//            step are contiguous; each finished chunk is published;
//   sweepers (kTcSlots x 4 warps)  warp q of a slot sweeps strip q of the
//            slot's block (one row per lane), waiting only for the chunks
//            it is about to read, with seams between strips and blocks through
//            the global seam ring as in every other solver.
// The L1 x L2 coefficient matrix is never stored: only the strips of the
// blocks in a CTA's slots exist at a time.
#pragma once
#include <type_traits>
#include "sigk_device.cuh"
#include "sigk_fwd.cuh"

namespace sigk {

constexpr int kTcRows = 128;       // rows per block: the MMA's M (four strips)
constexpr int kTcN = 64;           // columns per chunk: the MMA's N
constexpr int kTcK = 16;           // contraction per MMA (BF16)
constexpr int kTcDigits = 4;       // 8-bit digits per operand
constexpr int kTcMaxDim = 1024;    // exact accumulation of the leading group
constexpr int kTcPF = 2;           // sweep: coefficient loads in flight per lane
constexpr int kTcStages = 4;       // operand stages of the producer's copy pipeline
constexpr int kTcSlots = 3;        // blocks being swept at once per CTA
constexpr int kTcSweepWarps = 4 * kTcSlots;
constexpr int kTcThreads = 128 + 32 * kTcSweepWarps;  // producer group + sweep warps
// TMEM columns: two chunk buffers of four digit-order accumulators
constexpr int kTcTmemCols = 2 * 4 * kTcN;
static_assert(kTcTmemCols <= 512, "TMEM holds 512 columns");

// Named barrier of the producer group (barrier 0 is __syncthreads).
__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Dynamic shared memory of the tensor-core kernel (bytes): the producer's
// operand stages (A: 4 digits x 128 rows x 16 dimensions, B: 4 digits x 64
// columns x 16 dimensions, BF16, 24 KB per stage) and every sweep warp's
// seam-in and seam-out blocks; 1 KB of slack to align the operand tiles.
template <int P>
struct TcSmem {
    static constexpr int a_tile = kTcRows * kTcK * 2;           // one digit of A: 4 KB
    static constexpr int b_tile = kTcN * kTcK * 2;              // one digit of B: 2 KB
    static constexpr int stage = kTcDigits * (a_tile + b_tile);  // 24 KB
    static constexpr int stages = kTcStages * stage;
    static constexpr int seams = kTcSweepWarps * 2 * kG * (P + 4) * 4;
    static constexpr int bytes = stages + seams + 1024;
    static_assert(bytes <= 200 * 1024, "fits the SM with the static shared memory");
};

struct TcArgs {
    SolverArgs A;                  // pair table, schedule (items = 32-row strips), seams, outputs
    const uint16_t* ycache;        // digits of every path's segments: per slot a tiled matrix of
                                   // tc_cache_rows(max_len) rows (tile_index; BF16 bits)
    const int32_t* yexp;           // their exponents [slot][max_len]
    int64_t max_len;               // segments per slot
    int32_t d_pad;                 // d rounded up to a multiple of 16
    uint16_t* ablk;                // per CTA: digits of the block's 128 rows, tiled (16 row groups)
    float2* cst;                   // per CTA: skewed (c, clo) of kTcSlots x 4 strips
    int64_t cst_stride;            // float2 per strip: (max_len + 32 + kTcPF) * 32
    int* block_counter;
};

// ---------------------------------------------------------------------------
// digits

// Exponent of a row from its largest magnitude m: 2^e * [64, 128) holds m.
__device__ __forceinline__ int digit_exponent(float m) {
    return m > 0.0f ? ilogbf(m) - 6 : 0;
}

// The four BF16 digits of x * 2^-e (|x * 2^-e| < 128), as raw bit patterns.
// Every step is exact in FP32: the scaled value has at most 24 significant
// bits above 2^-17, the remainder after an integer digit is a multiple of the
// value's ulp below 1/2, and scaling by 2^8 is exact.
__device__ __forceinline__ void digits4(float x, int e, uint16_t (&t)[kTcDigits]) {
    float u = ldexpf(x, -e);
#pragma unroll
    for (int k = 0; k < kTcDigits; ++k) {
        const float dk = rintf(u);
        t[k] = (uint16_t)(__float_as_uint(dk) >> 16);  // integers |dk| <= 128: exact in BF16
        u = (u - dk) * 256.0f;
    }
}

// Digits in global memory are kept in the operand layout of the MMAs: for
// digit k and 16-dimension step s, the rows in groups of eight, each group
// one 256-byte block [half h of the step][row & 7][8 dimensions] -- the
// core-matrix layout of the shared-memory tiles (kTcLbo = 128, kTcSbo = 256
// bytes), so that one bulk copy moves a whole tile of consecutive rows.
// Element offset of (row r, dimension e, digit k) in a matrix of nrg row
// groups and ks steps of 16 dimensions:
__host__ __device__ constexpr int64_t tile_index(int64_t r, int e, int k, int ks, int64_t nrg) {
    return ((((int64_t)k * ks + (e >> 4)) * nrg + (r >> 3)) << 7) + (((e >> 3) & 1) << 6) + ((r & 7) << 3) +
           (e & 7);
}
// Rows of a path's digit matrix in the cache: max_len rounded up to whole
// 64-row chunks, so that a chunk's tile never runs past the matrix.
__host__ __device__ constexpr int64_t tc_cache_rows(int64_t max_len) { return (max_len + 63) / 64 * 64; }

// One warp cuts row `row` of a path (points or increments; `valid` false: a
// zero row) into digits, stored as row `trow` of the tiled matrix at base
// (nrg row groups, d_pad / 16 steps); returns the exponent (lane-uniform).
// esub is subtracted from the exponent (the refinement scale 1/s of a virtual
// row).
__device__ __forceinline__ int slice_row(const float* z, int64_t row, bool valid, int d, int d_pad,
                                         int inc_mode, int esub, uint16_t* base, int64_t trow, int64_t nrg,
                                         int lane) {
    float m = 0.0f;
    for (int e = lane; e < d; e += 32) {
        const float v = valid ? (inc_mode ? z[row * d + e] : z[(row + 1) * d + e] - z[row * d + e]) : 0.0f;
        m = fmaxf(m, fabsf(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    const int ex = digit_exponent(m);
    for (int e = lane; e < d_pad; e += 32) {
        const float v = (valid && e < d) ? (inc_mode ? z[row * d + e] : z[(row + 1) * d + e] - z[row * d + e]) : 0.0f;
        uint16_t t[kTcDigits];
        digits4(v, ex, t);
#pragma unroll
        for (int k = 0; k < kTcDigits; ++k) base[tile_index(trow, e, k, d_pad >> 4, nrg)] = t[k];
    }
    return m > 0.0f ? ex - esub : 0;
}

// Pre-pass: the digits of every path's first min(segments, max_len) segments
// (unrefined), one warp per segment, into the path's tiled matrix of
// tc_cache_rows(max_len) rows (rows past the path are zero digits); a path
// can be the swept path of a pair only within that range.
struct SliceArgs {
    const float* X;
    const float* Y;
    const int64_t* ox;             // point (or increment) offsets of X paths [n_x + 1]
    const int64_t* oy;
    const int64_t* len_x;
    const int64_t* len_y;
    int64_t n_x;
    int64_t n_slots;               // n_x (+ n_y)
    int32_t d, d_pad, inc_mode;
    int64_t max_len;
    uint16_t* cache;
    int32_t* exps;
};

static __global__ void __launch_bounds__(256) slice_paths_kernel(SliceArgs S) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t rows = tc_cache_rows(S.max_len);
    const int64_t total = S.n_slots * rows;
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < total; w += warps) {
        const int64_t slot = w / rows, r = w % rows;
        const bool fy = slot >= S.n_x;
        const int64_t i = fy ? slot - S.n_x : slot;
        const int64_t segs = S.inc_mode ? (fy ? S.len_y : S.len_x)[i] : (fy ? S.len_y : S.len_x)[i] - 1;
        const float* z = (fy ? S.Y : S.X) + (fy ? S.oy : S.ox)[i] * S.d;
        const int ex = slice_row(z, r, r < segs, S.d, S.d_pad, S.inc_mode, 0,
                                 S.cache + slot * rows * kTcDigits * S.d_pad, r, rows >> 3, lane);
        if (lane == 0 && r < S.max_len) S.exps[slot * S.max_len + r] = ex;
    }
}

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier helpers (single CTA; no cluster, no multicast)

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of
// 8 rows x 16 bytes (rows 16 bytes apart), lbo = byte distance of core
// matrices adjacent along K, sbo = along M/N; version field 1.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor: D FP32, A and B BF16, both K-major, N = kTcN, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);
// Byte offsets of the tiles' core matrices: two along K (lbo), rows in
// groups of eight (sbo).
constexpr uint32_t kTcLbo = 128, kTcSbo = 256;

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
                 "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(mbar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Bounded wait for the completion of the mbarrier phase with this parity;
// records kErrTimeout when it runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int* status) {
    if (mbar_try(mbar, parity)) return true;
    const unsigned long long t0 = global_ns();
    const unsigned long long budget = wait_budget(status);
    for (int it = 0; it < kWaitMaxIter; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > budget) break;
    }
    record_timeout(status, mbar, (long long)parity, -1);
    return false;
}
__device__ __forceinline__ void cp_async16(uint32_t sdst, const void* gsrc, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sdst), "l"(gsrc), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Arrive on an mbarrier expecting `bytes` of bulk copies (the phase completes
// when they have landed), or arrive without copies.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on mbar.
__device__ __forceinline__ void bulk_g2s(uint32_t sdst, const void* gsrc, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sdst),
                 "l"(gsrc), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

template <int NC>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                   "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---------------------------------------------------------------------------
// phase 2: the sweep of one 32-row strip with (c, clo) from the skewed area

// CTA-scope acquire load of a shared-memory word.
__device__ __forceinline__ int ld_acquire_cta(const int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(int* p, int v) {
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

// Bounded wait (every lane) until the producer has published `need` chunks
// of this strip's coefficients (*ready >= need); false when the wait runs
// out (kErrTimeout recorded) or the CTA aborts (*err set).
__device__ __forceinline__ bool wait_chunks(const int* ready, int need, const int* err, int* status) {
    if (ld_acquire_cta(ready) >= need) return true;
    const unsigned long long t0 = global_ns();
    const unsigned long long budget = wait_budget(status);
    for (int it = 0; it < kWaitMaxIter; ++it) {
        if (ld_acquire_cta(ready) >= need) return true;
        if (ld_acquire_cta(err)) return false;
        __nanosleep(64);
        if ((it & 63) == 63 && global_ns() - t0 > budget) break;
    }
    record_timeout(status, ready, need, ld_acquire_cta(ready));
    return false;
}

// The sweep reads coefficient entry t * 32 + l (row l, column t - l) at step
// t - kTcPF; entry t is complete once the chunk holding column t is: before
// step t (a multiple of kTcN) the strip needs the chunks of the columns up to
// t + kTcN - 1 + kTcPF.
__device__ __forceinline__ int chunks_needed(int t, int nch) {
    const int n = (t + kTcN - 1 + kTcPF) / kTcN + 1;
    return n < nch ? n : nch;
}

template <int P, int NR>
__device__ __forceinline__ bool sweep_strip_tc(const SolverArgs& A, const PairDesc& pd, int lo_p,
                                               int s, int item, int prev, int next, const float2* cw,
                                               float* sin_, float* sout,
                                               unsigned long long& tiles_done,
                                               unsigned long long& lane_tiles, unsigned (&rhist)[4],
                                               const int* ready, const int* err) {
    constexpr int S = P + 4;
    const int lane = threadIdx.x & 31;
    const int L1 = pd.L1, L2 = pd.L2;
    const bool has_in = prev >= 0;
    const bool has_out = next >= 0;
    const int slot_in = has_in ? prev % A.nslot : 0;
    const int slot_out = item % A.nslot;
    const int i0 = s * 32;
    bool ok = true;
    float a[P + 1], a1lo = 0.0f;
#pragma unroll
    for (int p = 0; p <= P; ++p) a[p] = 0.0f;
    int E = 0;
    float ohi = 1.0f, olo = 0.0f, ob1lo = 0.0f, ob[P + 1];
#pragma unroll
    for (int q = 0; q <= P; ++q) ob[q] = 0.0f;
    int oE = 0;
    const int Tn = L2 + 31;
    const bool has_row = i0 + lane < L1;
    const int nch = (L2 + kTcN - 1) / kTcN;
    // coefficients of step t at cw[t * 32 + lane]: loads kTcPF steps ahead,
    // each chunk of columns once the producer has published it
    ok = wait_chunks(ready, chunks_needed(0, nch), err, A.status);
    float2 cq[kTcPF];
#pragma unroll
    for (int k = 0; k < kTcPF; ++k) cq[k] = __ldcg(cw + k * 32 + lane);
    for (int t = 0; t < Tn && ok; ++t) {
        if (t > 0 && t % kTcN == 0 && t < L2 && !wait_chunks(ready, chunks_needed(t, nch), err, A.status)) {
            ok = false;
            break;
        }
        const float2 cc = cq[0];
#pragma unroll
        for (int k = 0; k + 1 < kTcPF; ++k) cq[k] = cq[k + 1];
        cq[kTcPF - 1] = __ldcg(cw + (t + kTcPF) * 32 + lane);
        if ((t & 31) == 0 && t < L2 && has_in) {
            const int nb = min(32, L2 - t);
            const unsigned long long need = ((unsigned long long)prev << 32) | (unsigned)(t + nb);
            bool okl = true;
            if (lane == 0) okl = wait_ge_u64(&A.prod[slot_in], need, A.status);
            ok = __shfl_sync(kFull, okl, 0);
            if (ok) {
                warp_copy_cg<S>(sin_, A.seam + ((size_t)slot_in * A.wcols + (t % A.wcols)) * S, nb * S, lane);
                __syncwarp();
                if (lane == 0)
                    st_release_u64(&A.cons[slot_in], ((unsigned long long)item << 32) | (unsigned)(t + nb));
            }
            __syncwarp();
            if (!ok) break;
        }
        float hi = __shfl_up_sync(kFull, ohi, 1);
        float lo = __shfl_up_sync(kFull, olo, 1);
        float b1lo = __shfl_up_sync(kFull, ob1lo, 1);
        float b[P + 1];
        b[0] = 0.0f;
#pragma unroll
        for (int q = 1; q <= P; ++q) b[q] = __shfl_up_sync(kFull, ob[q], 1);
        int F = __shfl_up_sync(kFull, oE, 1);
        if (lane == 0) {
            if (has_in && t < L2) {
                float v[S];
                seam_entry_load<S>(sin_ + (t & 31) * S, v);
                seam_unpack<P>(v, hi, lo, b1lo, b, F);
            } else {
                hi = 1.0f; lo = 0.0f; b1lo = 0.0f; F = 0;
#pragma unroll
                for (int q = 1; q <= P; ++q) b[q] = 0.0f;
            }
        }
        const int j = t - lane;
        // the warp's ring count for this step (the largest its tiles need)
        int nw = NR;
        if (A.ring_adaptive) {
            const int nl = (j >= 0 && j < L2) ? rings_needed(fabsf(cc.x), A.ring_theta) : 0;
            nw = min((int)__reduce_max_sync(kFull, (unsigned)nl), NR);
            if (j >= 0 && j < L2 && has_row) {
#pragma unroll
                for (int q = 0; q < 4; ++q) rhist[q] += ((nw + 1) / 2 - 1 == q) ? 1u : 0u;
            }
        }
        if (j >= 0 && j < L2) {
            if (F != E) {
                if (F > E) {
                    const float sc = exp2_nonpos(E - F);
                    a1lo *= sc;
#pragma unroll
                    for (int p = 1; p <= P; ++p) a[p] *= sc;
                    E = F;
                } else {
                    const float sc = exp2_nonpos(F - E);
                    hi *= sc; lo *= sc; b1lo *= sc;
#pragma unroll
                    for (int q = 1; q <= P; ++q) b[q] *= sc;
                }
            }
            // rows past the end of the path have zero digits: c = clo = 0
            auto tile = [&](auto nrc) {
                tile_update<P, NR, true>(cc.x, a, a1lo, hi, lo, b, b1lo, decltype(nrc)::value, cc.y);
            };
            if (nw == NR) tile(std::integral_constant<int, NR>{});
            else if (nw <= 2) tile(std::integral_constant<int, 2>{});
            else if (NR > 4 && nw == 4) tile(std::integral_constant<int, (NR > 4 ? 4 : NR)>{});
            else tile(std::integral_constant<int, (NR > 6 ? 6 : NR)>{});
            if (fabsf(hi) > 1.8446744e19f) {  // 2^64
                const float sc = 5.421011e-20f;  // 2^-64
                a1lo *= sc;
#pragma unroll
                for (int p = 1; p <= P; ++p) a[p] *= sc;
                hi *= sc; lo *= sc; b1lo *= sc;
#pragma unroll
                for (int q = 1; q <= P; ++q) b[q] *= sc;
                E += 64;
            }
            ohi = hi; olo = lo; ob1lo = b1lo; oE = E;
#pragma unroll
            for (int q = 1; q <= P; ++q) ob[q] = b[q];
            tiles_done += has_row ? 1ull : 0ull;
            lane_tiles += 1;
            if (lane == 31) {
                if (has_out) {
                    float v[S];
                    seam_pack<P>(v, hi, lo, b1lo, b, E);
                    seam_entry_store<S>(sout + (j & 31) * S, v);
                } else if (j == L2 - 1) {
                    double k = (double)hi + (double)lo + (double)b1lo;
                    double fq = 1.0;
#pragma unroll
                    for (int q = 1; q <= P; ++q) {
                        fq *= (double)q;
                        k += (double)b[q] / fq;
                    }
                    k = ldexp(k, E);
                    if (!isfinite(k)) record_nonfinite(A.status);
                    if (pd.out0 >= 0) A.out[pd.out0] = k;
                    if (pd.out1 >= 0) A.out[pd.out1] = k;
                }
            }
        }
        const int jj = t - 31;
        if (has_out && jj >= 0 && jj < L2 && (((jj & 31) == 31) || jj == L2 - 1)) {
            __syncwarp();
            const int start = jj & ~31;
            const int nb = jj - start + 1;
            if (start + nb > A.wcols) {
                const unsigned long long need = ((unsigned long long)next << 32) |
                                                (unsigned)(start + nb - A.wcols);
                bool okl = true;
                if (lane == 0) okl = wait_ge_u64(&A.cons[slot_out], need, A.status);
                ok = __shfl_sync(kFull, okl, 0);
            }
            if (ok) {
                float* dst = A.seam + ((size_t)slot_out * A.wcols + (start % A.wcols)) * S;
                for (int idx = lane; idx < nb * S; idx += 32) __stcg(dst + idx, sout[idx]);
                __threadfence();
                __syncwarp();
                if (lane == 0)
                    st_release_u64(&A.prod[slot_out], ((unsigned long long)item << 32) | (unsigned)(start + nb));
            }
            __syncwarp();
        }
    }
    return ok;
}

// ---------------------------------------------------------------------------

// State of one CTA shared between its producer group and its sweep warps.
struct TcShared {
    uint64_t mbar[kTcStages];     // stage s: the MMAs that read it have completed
    uint64_t full[kTcStages];     // stage s: its operand tiles have landed (bulk copies)
    uint32_t tmem_base;
    int blk;                      // the producer's block (broadcast within the group)
    int stop;                     // no more blocks (the normal end)
    int err;                      // abort: a wait ran out
    int slot_seq[kTcSlots];       // blocks published into each slot so far
    int slot_blk[kTcSlots];       // the slot's current block
    int slot_ready[kTcSlots];     // chunks of its coefficients published
    int slot_done[kTcSlots];      // of its four strips swept (4: the slot is free)
    int aexp[kTcRows];            // exponents of the producer's block rows
};

__device__ __forceinline__ bool producer_and(bool v) {
    int r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.s32 p, %1, 0;\nbar.red.and.pred q, 1, 128, p;\nselp.s32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((int)v)
                 : "memory");
    return r != 0;
}

// Bounded wait of the producer's thread 0 for a free slot; returns its index,
// or -1 (abort, or the wait ran out: kErrTimeout recorded).
__device__ __forceinline__ int wait_free_slot(TcShared& sh, int* status) {
    const unsigned long long t0 = global_ns();
    const unsigned long long budget = wait_budget(status);
    for (int it = 0; it < kWaitMaxIter; ++it) {
#pragma unroll
        for (int k = 0; k < kTcSlots; ++k)
            if (ld_acquire_cta(&sh.slot_done[k]) == 4) return k;
        if (ld_acquire_cta(&sh.err)) return -1;
        __nanosleep(128);
        if ((it & 63) == 63 && global_ns() - t0 > budget) break;
    }
    record_timeout(status, &sh.slot_done[0], 4, ld_acquire_cta(&sh.slot_done[0]));
    return -1;
}

// Bounded wait of a sweep warp for the next block of its slot; false at the
// end (no more blocks) or on abort.
__device__ __forceinline__ bool wait_slot_block(TcShared& sh, int slot, int gen, int* status) {
    const unsigned long long t0 = global_ns();
    const unsigned long long budget = wait_budget(status);
    for (int it = 0; it < kWaitMaxIter; ++it) {
        if (ld_acquire_cta(&sh.slot_seq[slot]) > gen) return true;
        if (ld_acquire_cta(&sh.err)) return false;
        if (ld_acquire_cta(&sh.stop)) return ld_acquire_cta(&sh.slot_seq[slot]) > gen;
        __nanosleep(128);
        if ((it & 63) == 63 && global_ns() - t0 > budget) break;
    }
    record_timeout(status, &sh.slot_seq[slot], gen + 1, ld_acquire_cta(&sh.slot_seq[slot]));
    return false;
}

// The producer group (threads 0..127 of the CTA): claims blocks while a slot
// is free, cuts the block's rows into digits, and forms the coefficients of
// the block's four strips 64 columns at a time: a kTcStages-deep pipeline of
// cp.async copies of the digit tiles (16 dimensions per step), thread 0 issues
// each step's ten 128x64x16 MMAs and commits them to the stage's mbarrier,
// and the chunk's (c, clo) are read back from TMEM (warp w: rows 32w..32w+31,
// strip w) while the tensor core already works on the next chunk (two TMEM
// buffers).  Each finished chunk is published to the slot's sweep warps.
template <int P>
__device__ __forceinline__ void tc_producer(const TcArgs& T, TcShared& sh, unsigned char* stg, int tid) {
    const SolverArgs& A = T.A;
    using Sm = TcSmem<P>;
    constexpr int S = kTcStages;
    const int lane = tid & 31, warp = tid >> 5;
    const int d = A.d, d_pad = T.d_pad, KS = d_pad / kTcK;
    uint16_t* ablk = T.ablk + (int64_t)blockIdx.x * kTcDigits * kTcRows * d_pad;
    const int n_blocks = A.sched.hdr[2] >> 2;
    const uint32_t tmem = sh.tmem_base;
    uint32_t gstep = 0;   // operand steps so far: stage g % S, its use number g / S
    uint32_t gchunk = 0;  // chunks so far: TMEM buffer gchunk & 1
    int64_t issued = -1, waited = -1;
    int64_t filled = -1, consumed = -1;  // thread 0: last step whose bulk copies were issued / awaited
    bool ok = true;
    for (;;) {
        // ---- a free slot, and the next block -------------------------------
        if (tid == 0) {
            int blk = -1;
            const int slot = wait_free_slot(sh, A.status);
            if (slot >= 0) {
                blk = atomicAdd(T.block_counter, 1);
                if (blk >= n_blocks || ld_volatile_s32(A.status) != 0) blk = -1;
            }
            sh.blk = blk < 0 ? -1 : blk * kTcSlots + slot;
        }
        producer_sync();
        const int code = sh.blk;
        producer_sync();  // read before thread 0 can overwrite it
        if (code < 0) break;
        const int blk = code / kTcSlots, slot = code % kTcSlots;
        const ItemRef ir = decode_item(A.sched, A.pairs, 4 * blk);
        const PairDesc pd = A.pairs[ir.pair];
        const int L1 = pd.L1, L2 = pd.L2;
        const int r0 = ir.k * 32;  // the block's first row (strips come in fours)
#ifdef SIGK_DEBUG
        ok = dbg_in(A.status, 41, ir.pair, A.n_pairs - 1) &&
             dbg_in(A.status, 42, (int64_t)(L2 + 31 + kTcPF) * 32, T.cst_stride) &&
             dbg_in(A.status, 47, (int64_t)(L2 + pd.sy - 1) / pd.sy, T.max_len) &&
             dbg_in(A.status, 48, (int64_t)(ir.k & 3), 0);
        ok = producer_and(ok);
        if (!ok) break;
#endif
        // ---- digits of the block's 128 rows (32 per warp) -------------------
        {
            const int lsx = 31 - __clz(pd.sx);  // refinement factors are powers of two
            for (int rr = 0; rr < 32; ++rr) {
                const int r = warp * 32 + rr;
                const int v = r0 + r;  // virtual row
                const int ex = slice_row(pd.xr, (int64_t)(v >> lsx), v < L1, d, d_pad, A.inc_mode, lsx,
                                         ablk, r, kTcRows / 8, lane);
                if (lane == 0) sh.aexp[r] = ex;
            }
        }
        __threadfence_block();
        // the bulk copies (async proxy) read what these generic stores wrote
        asm volatile("fence.proxy.async.global;" ::: "memory");
        producer_sync();
        // ---- publish the block to the slot's sweep warps --------------------
        if (tid == 0) {
            sh.slot_blk[slot] = blk;
            sh.slot_ready[slot] = 0;
            sh.slot_done[slot] = 0;
            st_release_cta(&sh.slot_seq[slot], sh.slot_seq[slot] + 1);
        }
        // ---- the coefficients, kTcN columns at a time -----------------------
        const int lsy = 31 - __clz(pd.sy);
        const int64_t yrows = tc_cache_rows(T.max_len);
        const uint16_t* yc = T.ycache + (int64_t)pd.yslot * yrows * kTcDigits * d_pad;
        // an unrefined swept path: a chunk's 64 columns are consecutive rows
        // of the path's tiled digit matrix, so every operand tile of a step
        // is one contiguous block and leaves global memory in one bulk copy
        // (issued by thread 0, completing on the stage's `full` mbarrier);
        // a refined one repeats rows, and all producer threads copy 16-byte
        // pieces (cp.async)
        const bool bulk = pd.sy == 1;
        const int32_t* ye = T.yexp + (int64_t)pd.yslot * T.max_len;
        float2* cw = T.cst + ((int64_t)blockIdx.x * kTcSlots + slot) * 4 * T.cst_stride + (int64_t)warp * T.cst_stride;
        const int nch = (L2 + kTcN - 1) / kTcN;
        const int nst = nch * KS;
        // copies of step n (chunk n / KS, dimensions 16 (n % KS)) into stage (gstep + n) % S
        auto issue = [&](int n) {
            const int c0 = (n / KS) * kTcN, kk = n % KS;
            unsigned char* sa = stg + ((gstep + n) % S) * Sm::stage;
            unsigned char* sb = sa + kTcDigits * Sm::a_tile;
            // A: 4 digits x 128 rows x 2 halves of 8 dims; B: 4 digits x 64 columns x 2 halves
            for (int idx = tid; idx < kTcDigits * kTcRows * 2; idx += 128) {
                const int h = idx & 1, r = (idx >> 1) & (kTcRows - 1), k = idx >> 8;
                cp_async16(smem_u32(sa + k * Sm::a_tile + (r >> 3) * kTcSbo + h * kTcLbo + (r & 7) * 16),
                           ablk + tile_index(r, kk * kTcK + 8 * h, k, KS, kTcRows / 8), 16u);
            }
            for (int idx = tid; idx < kTcDigits * kTcN * 2; idx += 128) {
                const int h = idx & 1, jj = (idx >> 1) & (kTcN - 1), k = idx >> 7;
                const int j = c0 + jj;
                const bool in = j < L2;
                cp_async16(smem_u32(sb + k * Sm::b_tile + (jj >> 3) * kTcSbo + h * kTcLbo + (jj & 7) * 16),
                           yc + tile_index(in ? (j >> lsy) : 0, kk * kTcK + 8 * h, k, KS, yrows >> 3),
                           in ? 16u : 0u);
            }
        };
        // thread 0: the eight tiles of step n (four digits of A and of B) into
        // stage (gstep + n) % S, one bulk copy each
        auto issue_bulk = [&](int n) {
            const int c0 = (n / KS) * kTcN, kk = n % KS;
            const uint32_t st = (gstep + n) % S;
            unsigned char* sa = stg + st * Sm::stage;
            unsigned char* sb = sa + kTcDigits * Sm::a_tile;
            mbar_expect_tx(&sh.full[st], (uint32_t)(kTcDigits * (Sm::a_tile + Sm::b_tile)));
#pragma unroll
            for (int k = 0; k < kTcDigits; ++k) {
                bulk_g2s(smem_u32(sa + k * Sm::a_tile), ablk + tile_index(0, kk * kTcK, k, KS, kTcRows / 8),
                         (uint32_t)Sm::a_tile, &sh.full[st]);
                bulk_g2s(smem_u32(sb + k * Sm::b_tile), yc + tile_index(c0, kk * kTcK, k, KS, yrows >> 3),
                         (uint32_t)Sm::b_tile, &sh.full[st]);
            }
            filled = (int64_t)gstep + n;
        };
        // (c, clo) of chunk c from TMEM into the strips' skewed areas, then
        // published: chunk c's last MMAs are complete once its last step's
        // commit has arrived
        auto epilogue = [&](int c) {
            const uint32_t m = gstep + (uint32_t)((c + 1) * KS - 1);
            if (!mbar_wait(&sh.mbar[m % S], (m / S) & 1, A.status)) ok = false;
            waited = m;
            tc_fence_after();
            const int c0 = c * kTcN;
            const int ea = sh.aexp[warp * 32 + lane];
            // column exponents, lane l: columns c0 + l and c0 + 32 + l
            int ecol[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = c0 + 32 * h + lane;
                ecol[h] = j < L2 ? ye[j >> lsy] - lsy : 0;
            }
            const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16) + ((gchunk + c) & 1) * 4 * kTcN;
#pragma unroll 1
            for (int qt = 0; qt < kTcN / 16; ++qt) {
                uint32_t g0[16], g1[16], g2[16], g3[16];
                tmem_ld16<16>(tl + 0 * kTcN + 16 * qt, g0);
                tmem_ld16<16>(tl + 1 * kTcN + 16 * qt, g1);
                tmem_ld16<16>(tl + 2 * kTcN + 16 * qt, g2);
                tmem_ld16<16>(tl + 3 * kTcN + 16 * qt, g3);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int jj = 16 * qt + q;
                    const int j = c0 + jj;
                    const int eb = __shfl_sync(kFull, ecol[jj >> 5], jj & 31);
                    // c = 2^(ea + eb) (G0 + G1 2^-8 + G2 2^-16 + G3 2^-24), rounded once to (hi, lo)
                    const float s0 = __uint_as_float(g0[q]);
                    const float t1 = __uint_as_float(g1[q]) * 0.00390625f;
                    const float sh_ = s0 + t1;
                    const float bv = sh_ - s0;
                    float e = (s0 - (sh_ - bv)) + (t1 - bv);
                    e += fmaf(__uint_as_float(g2[q]), 1.52587890625e-05f,
                              __uint_as_float(g3[q]) * 5.9604644775390625e-08f);
                    const float hi = sh_ + e;
                    const float lo = e - (hi - sh_);
                    const int ex = ea + eb;
                    if (j < L2) cw[(int64_t)(j + lane) * 32 + lane] = make_float2(ldexpf(hi, ex), ldexpf(lo, ex));
                }
            }
            tc_fence_before();
            __threadfence_block();
            producer_sync();  // every warp's rows of the chunk are written; its TMEM buffer is free
            if (tid == 0) st_release_cta(&sh.slot_ready[slot], c + 1);
        };
#pragma unroll 1
        for (int n = 0; n < S - 1; ++n) {
            if (bulk) {
                if (tid == 0 && n < nst) issue_bulk(n);
            } else {
                if (n < nst) issue(n);
                cp_async_commit();
            }
        }
#pragma unroll 1
        for (int n = 0; n < nst; ++n) {
            const uint32_t g = gstep + n;
            bool ready = true;
            if (bulk) {
                // step n's tiles have landed (thread 0 issues the MMAs)
                if (tid == 0) {
                    ready = mbar_wait(&sh.full[g % S], (g / S) & 1, A.status);
                    consumed = g;
                }
            } else {
                asm volatile("cp.async.wait_group %0;" ::"n"(S - 2) : "memory");  // step n's copies (this thread's)
                fence_proxy_async_smem();
                producer_sync();  // every thread's copies of step n have landed
                // one arrival per step keeps the stage's `full` phases in step
                // with the bulk blocks
                if (tid == 0) mbar_arrive(&sh.full[g % S]);
            }
            if (!ready) ok = false;
            const int c = n / KS, kk = n % KS;
            if (tid == 0 && ready) {
                tc_fence_after();
                unsigned char* sa = stg + (g % S) * Sm::stage;
                unsigned char* sb = sa + kTcDigits * Sm::a_tile;
                const uint32_t dbuf = tmem + ((gchunk + c) & 1) * 4 * kTcN;
                // digit orders k + l = q accumulate at TMEM columns dbuf + 64 q
#pragma unroll
                for (int q = 0; q < 4; ++q) {
#pragma unroll
                    for (int k = 0; k <= q; ++k) {
                        const uint64_t da = tc_desc(smem_u32(sa + k * Sm::a_tile), kTcLbo, kTcSbo);
                        const uint64_t db = tc_desc(smem_u32(sb + (q - k) * Sm::b_tile), kTcLbo, kTcSbo);
                        tc_mma(dbuf + kTcN * q, da, db, (kk > 0 || k > 0) ? 1u : 0u);
                    }
                }
                tc_commit(&sh.mbar[g % S]);
            }
            issued = g;
            // refill: step n + S - 1 goes to stage (g - 1) % S, which the MMAs of step g - 1 read
            if (n + S - 1 < nst) {
                if (bulk) {
                    if (tid == 0 && ok) {
                        if (g >= 1 && !mbar_wait(&sh.mbar[(g - 1) % S], ((g - 1) / S) & 1, A.status)) ok = false;
                        if (ok) issue_bulk(n + S - 1);
                    }
                } else {
                    if (g >= 1 && !mbar_wait(&sh.mbar[(g - 1) % S], ((g - 1) / S) & 1, A.status)) ok = false;
                    issue(n + S - 1);
                }
            }
            if (!bulk) cp_async_commit();
            // the previous chunk's epilogue overlaps this chunk's MMAs
            if (kk == 0 && c >= 1) epilogue(c - 1);
            ok = producer_and(ok);
            if (!ok) break;
        }
        if (ok && nst > 0) epilogue(nch - 1);
        asm volatile("cp.async.wait_all;" ::: "memory");
        gstep += nst;
        gchunk += nch;
        ok = producer_and(ok);
        if (!ok) break;
    }
    // the end of the blocks, or an abort
    if (tid == 0) {
        if (!ok) st_release_cta(&sh.err, 1);
        st_release_cta(&sh.stop, 1);
    }
    // MMAs still in flight (after an abort) complete before TMEM is freed
    if (issued > waited) mbar_wait(&sh.mbar[issued % S], (uint32_t)(issued / S) & 1, A.status);
    // and bulk copies still in flight land before the CTA's shared memory is released
    if (tid == 0)
        for (int64_t q = consumed + 1; q <= filled; ++q)
            if (!mbar_wait(&sh.full[q % S], (uint32_t)(q / S) & 1, A.status)) break;
}

// One CTA per SM (it holds all of TMEM): warps 0-3 are the producer group,
// warps 4 .. 4 + kTcSweepWarps - 1 sweep: warp 4 + 4 k + q sweeps strip q of
// the block in slot k, reading its chunks as the producer publishes them.
// Deadlock freedom: a block is claimed only when a slot (four sweep warps) is
// free, the producer never waits on a sweep while it forms a block, and the
// seam ring holds whole strips (no flow control), so every wait of a sweep
// points to a lower work item or to its own producer.
template <int P, int NR>
__global__ void __launch_bounds__(kTcThreads, 1) fwd_tc_kernel(TcArgs T) {
    const SolverArgs& A = T.A;
    constexpr int S = P + 4;
    using Sm = TcSmem<P>;
    extern __shared__ float4 smem_tc_raw[];
    __shared__ TcShared sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // operand stages 1 KB aligned (the dynamic area is 1 KB larger than needed)
    unsigned char* stg = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_tc_raw) + 1023) & ~(uintptr_t)1023);
    float* seams = reinterpret_cast<float*>(stg + Sm::stages);
    unsigned long long tiles_done = 0, lane_tiles = 0;
    unsigned rhist[4] = {0u, 0u, 0u, 0u};  // tiles by ring count (adaptive launches)

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kTcStages; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.mbar[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.full[k])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.stop = 0;
        sh.err = 0;
#pragma unroll
        for (int k = 0; k < kTcSlots; ++k) {
            sh.slot_seq[k] = 0;
            sh.slot_blk[k] = 0;
            sh.slot_ready[k] = 0;
            sh.slot_done[k] = 4;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp < 4) {
        tc_producer<P>(T, sh, stg, threadIdx.x);
    } else {
        const int sw = warp - 4, slot = sw >> 2, q = sw & 3;
        float* seam_w = seams + sw * 2 * kG * S;
        for (int gen = 0;; ++gen) {
            if (!wait_slot_block(sh, slot, gen, A.status)) break;
            const int blk = sh.slot_blk[slot];
            const int item = 4 * blk + q;
            const ItemRef ir = decode_item(A.sched, A.pairs, item);
            const PairDesc pd = A.pairs[ir.pair];
            const float2* cw = T.cst + ((int64_t)blockIdx.x * kTcSlots + slot) * 4 * T.cst_stride +
                               (int64_t)q * T.cst_stride;
            bool ok = true;
#ifdef SIGK_DEBUG
            ok = dbg_in(A.status, 43, item % A.nslot, A.nslot - 1) &&
                 dbg_in(A.status, 45, pd.out0, A.out_cap - 1) &&
                 dbg_in(A.status, 46, pd.out1 < 0 ? 0 : pd.out1, A.out_cap - 1) &&
                 dbg_in(A.status, 49, (int64_t)(ir.k & 3), q) && dbg_in(A.status, 49, (int64_t)q, ir.k & 3);
            ok = __all_sync(kFull, ok);
#endif
            if (ok && ir.next >= 0) ok = wait_slot_free(A.sched, A.pairs, item, A.nslot, A.done, A.status);
            if (ok)
                ok = sweep_strip_tc<P, NR>(A, pd, ir.pair, ir.k, item, ir.prev, ir.next, cw, seam_w,
                                           seam_w + kG * S, tiles_done, lane_tiles, rhist,
                                           &sh.slot_ready[slot], &sh.err);
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                st_release_s64(&A.done[item % A.nslot], (long long)item);
                if (!ok) st_release_cta(&sh.err, 1);
                atomicAdd(&sh.slot_done[slot], 1);
            }
            __syncwarp();
            if (!ok) break;
        }
    }
    tc_fence_before();
    __syncthreads();  // the producer's MMAs are complete and every TMEM read is done
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem_base), "r"(kTcTmemCols));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tiles_done += __shfl_down_sync(kFull, tiles_done, o);
        lane_tiles += __shfl_down_sync(kFull, lane_tiles, o);
    }
    if (lane == 0) {
        atomicAdd(&A.counters[0], tiles_done);
        atomicAdd(&A.counters[1], lane_tiles);
    }
    if (A.ring_adaptive) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            unsigned v = rhist[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
            if (lane == 0 && v) atomicAdd(&A.ring_hist[k], v);
        }
    }
}

}  // namespace sigk
