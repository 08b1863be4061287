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
// pair-major, so the four strips are consecutive work items).  A group of
// four warps owns a block (four groups per CTA, one CTA per SM):
//   phase 1  the block's rows are cut into digits in a per-CTA global area;
//            for every 32-column chunk of the swept path, the CTA stages the
//            digit tiles (16 dimensions per step, two stages, cp.async) in the
//            tensor core's shared-memory layout, one thread issues the ten
//            128x32x16 MMAs of each step into TMEM, and every warp reads its
//            32 rows back (tcgen05.ld) and stores (c, clo) into its strip's
//            coefficient area, skewed so that the 32 values a warp's lanes
//            read in one sweep step are contiguous;
//   phase 2  warp w sweeps strip w of the block (the wavefront sweep of
//            sigk_fwd_cm.cuh with one row per lane), seams between strips and
//            blocks through the global seam ring as in every other solver.
// The groups of a CTA are in different phases, so the tensor-core phase of
// one overlaps the FMA sweep of the others.  The L1 x L2 coefficient
// matrix is never stored: only one block's strips per CTA exist at a time.
#pragma once
#include <type_traits>
#include "sigk_device.cuh"
#include "sigk_fwd.cuh"

namespace sigk {

constexpr int kTcRows = 128;       // rows per block: the MMA's M (four strips)
constexpr int kTcN = 32;           // columns per chunk: the MMA's N
constexpr int kTcK = 16;           // contraction per MMA (BF16)
constexpr int kTcDigits = 4;       // 8-bit digits per operand
constexpr int kTcMaxDim = 1024;    // exact accumulation of the leading group
constexpr int kTcPF = 2;           // sweep: coefficient loads in flight per lane
// A CTA of this kernel holds TMEM, and the occupancy calculation then allows
// one CTA per SM whatever its shared memory (measured on this GPU: a kernel
// that contains tcgen05.alloc gets 1 CTA per SM at 16 KB of shared memory, the
// same kernel without it 13).  So one CTA per SM runs kTcGroups independent
// 4-warp groups, each a block worker with its own quarter of TMEM.
constexpr int kTcGroups = 4;

// Barriers of one 128-thread group (named barrier 1 + gr; barrier 0 is
// __syncthreads).
__device__ __forceinline__ void group_sync(int gr) {
    asm volatile("bar.sync %0, 128;" ::"r"(gr + 1) : "memory");
}
__device__ __forceinline__ bool group_and(int gr, bool v) {
    int r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.s32 p, %1, 0;\nbar.red.and.pred q, %2, 128, p;\nselp.s32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((int)v), "r"(gr + 1)
                 : "memory");
    return r != 0;
}

// Dynamic shared memory of the tensor-core kernel (bytes).  Phase 1: two
// stages of the digit tiles (A: 4 digits x 128 rows x 16 dims, B: 4 digits x
// 32 columns x 16 dims, BF16); phase 2: per warp the seam-in and seam-out
// blocks.  The two phases share one region.  The total is padded so that at
// most four CTAs fit an SM (their TMEM: 4 x 128 columns).
template <int P>
struct TcSmem {
    static constexpr int a_tile = kTcRows * kTcK * 2;           // one digit of A: 4 KB
    static constexpr int b_tile = kTcN * kTcK * 2;              // one digit of B: 1 KB
    static constexpr int stage = kTcDigits * (a_tile + b_tile);  // 20 KB
    static constexpr int phase1 = 2 * stage;
    static constexpr int phase2 = 4 * 2 * kG * (P + 4) * 4;
    // per group, 1 KB aligned (tcgen05 operand tiles)
    static constexpr int group = ((phase1 > phase2 ? phase1 : phase2) + 1023) / 1024 * 1024;
    static constexpr int bytes = kTcGroups * group + 1024;  // + 1 KB alignment slack
    static_assert(bytes <= 227 * 1024, "one CTA of kTcGroups groups per SM");
};

struct TcArgs {
    SolverArgs A;                  // pair table, schedule (items = 32-row strips), seams, outputs
    const uint16_t* ycache;        // digits of every path's segments [slot][max_len][4][d_pad] (BF16 bits)
    const int32_t* yexp;           // their exponents [slot][max_len]
    int64_t max_len;               // segments per slot
    int32_t d_pad;                 // d rounded up to a multiple of 16
    uint16_t* ablk;                // per CTA: digits of the block's rows [4][128][d_pad]
    int32_t* aexp;                 // per CTA: their exponents [128]
    float2* cst;                   // per CTA: skewed (c, clo) of the four strips
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

// One warp cuts row `row` of a path (points or increments; `valid` false: a
// zero row) into digits: dst[k * kstride + e] for k < 4, e < d_pad; returns
// the exponent (lane-uniform).  esub is subtracted from the exponent (the
// refinement scale 1/s of a virtual row).
__device__ __forceinline__ int slice_row(const float* z, int64_t row, bool valid, int d, int d_pad,
                                         int inc_mode, int esub, uint16_t* dst, int64_t kstride,
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
        for (int k = 0; k < kTcDigits; ++k) dst[k * kstride + e] = t[k];
    }
    return m > 0.0f ? ex - esub : 0;
}

// Pre-pass: the digits of every path's first min(segments, max_len) segments
// (unrefined), one warp per segment; a path can be the swept path of a pair
// only within that range.
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
    const int64_t total = S.n_slots * S.max_len;
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < total; w += warps) {
        const int64_t slot = w / S.max_len, r = w % S.max_len;
        const bool fy = slot >= S.n_x;
        const int64_t i = fy ? slot - S.n_x : slot;
        const int64_t segs = S.inc_mode ? (fy ? S.len_y : S.len_x)[i] : (fy ? S.len_y : S.len_x)[i] - 1;
        if (r >= segs) continue;  // warp-uniform
        const float* z = (fy ? S.Y : S.X) + (fy ? S.oy : S.ox)[i] * S.d;
        const int ex = slice_row(z, r, true, S.d, S.d_pad, S.inc_mode, 0,
                                 S.cache + w * kTcDigits * S.d_pad, S.d_pad, lane);
        if (lane == 0) S.exps[w] = ex;
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
// Instruction descriptor: D FP32, A and B BF16, both K-major, N = 32, M = 128.
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

template <int P, int NR>
__device__ __forceinline__ bool sweep_strip_tc(const SolverArgs& A, const PairDesc& pd, int lo_p,
                                               int s, int item, int prev, int next, const float2* cw,
                                               float* sin_, float* sout,
                                               unsigned long long& tiles_done,
                                               unsigned long long& lane_tiles, unsigned (&rhist)[4]) {
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
    // coefficients of step t at cw[t * 32 + lane]: loads kTcPF steps ahead
    float2 cq[kTcPF];
#pragma unroll
    for (int k = 0; k < kTcPF; ++k) cq[k] = __ldcg(cw + k * 32 + lane);
    for (int t = 0; t < Tn && ok; ++t) {
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
                const float* e_ = sin_ + (t & 31) * S;
                hi = e_[0];
                lo = e_[1];
                b1lo = e_[2];
#pragma unroll
                for (int q = 1; q <= P; ++q) b[q] = e_[2 + q];
                F = __float_as_int(e_[P + 3]);
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
                for (int q = 0; q < 4; ++q) rhist[q] += ((nw >> 1) - 1 == q) ? 1u : 0u;
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
                tile_update<P, true>(cc.x, a, a1lo, hi, lo, b, b1lo, decltype(nrc)::value, cc.y);
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
                    float* e_ = sout + (j & 31) * S;
                    e_[0] = hi; e_[1] = lo; e_[2] = b1lo;
#pragma unroll
                    for (int q = 1; q <= P; ++q) e_[2 + q] = b[q];
                    e_[P + 3] = __int_as_float(E);
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

template <int P, int NR>
__global__ void __launch_bounds__(kTcGroups * 128, 1) fwd_tc_kernel(TcArgs T) {
    const SolverArgs& A = T.A;
    constexpr int S = P + 4;
    using Sm = TcSmem<P>;
    extern __shared__ float4 smem_tc_raw[];
    __shared__ __align__(8) uint64_t mbar_g[kTcGroups][2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int blk_g[kTcGroups], st_g[kTcGroups], stop_g[kTcGroups];
    __shared__ int32_t yexp_g[kTcGroups][2][kTcN];  // column exponents of the chunk (double buffered)
    // group gr = warps 4 gr .. 4 gr + 3: an independent block worker with its
    // own shared memory, TMEM columns [128 gr, 128 gr + 128), mbarriers and
    // named barrier 1 + gr; warp w % 4 of a group reaches TMEM lanes 32 (w % 4)
    const int gr = threadIdx.x >> 7;
    const int tid = threadIdx.x & 127, lane = tid & 31, warp = tid >> 5;
    const int wid = (int)(blockIdx.x * kTcGroups + gr);  // worker index: per-worker scratch
    uint64_t* mbar = mbar_g[gr];
    int& blk_s = blk_g[gr];
    int& st_s = st_g[gr];
    int& stop_s = stop_g[gr];
    int32_t (*yexp_s)[kTcN] = yexp_g[gr];
    const int d = A.d, d_pad = T.d_pad;
    const int KS = d_pad / kTcK;
    uint16_t* ablk = T.ablk + (int64_t)wid * kTcDigits * kTcRows * d_pad;
    int32_t* aexp = T.aexp + (int64_t)wid * kTcRows;
    float2* cblk = T.cst + (int64_t)wid * 4 * T.cst_stride;
    // operand tiles 1 KB aligned (the dynamic area is 1 KB larger than needed)
    unsigned char* st0 = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_tc_raw) + 1023) & ~(uintptr_t)1023) + gr * Sm::group;
    float* seam_w = reinterpret_cast<float*>(st0) + warp * 2 * kG * S;  // phase 2 (aliases phase 1)
    unsigned long long tiles_done = 0, lane_tiles = 0;

    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(128 * kTcGroups));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stop_s = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base_s + 128 * gr;
    unsigned rhist[4] = {0u, 0u, 0u, 0u};  // tiles by ring count (adaptive launches)
    uint32_t step = 0;         // MMA steps of this CTA so far (stage = step & 1)
    int64_t issued = -1;       // last step whose MMAs were committed (CTA-uniform)
    int64_t waited = -1;       // last step whose completion was observed
    const int n_blocks = A.sched.hdr[2] >> 2;

    for (;;) {
        if (tid == 0) {
            blk_s = atomicAdd(T.block_counter, 1);
            st_s = ld_volatile_s32(A.status);
        }
        group_sync(gr);
        const int blk = blk_s, st = st_s;
        group_sync(gr);  // read before thread 0 can overwrite them
        if (blk >= n_blocks || st != 0) break;
        const int item = 4 * blk + warp;
        const ItemRef ir = decode_item(A.sched, A.pairs, item);
        const int lo_p = ir.pair;
        const PairDesc pd = A.pairs[lo_p];
        const int s = ir.k;                   // this warp's strip
        const int L1 = pd.L1, L2 = pd.L2;
        const int r0 = (s & ~3) * 32;         // first row of the block
        bool ok = true;
#ifdef SIGK_DEBUG
        ok = dbg_in(A.status, 41, lo_p, A.n_pairs - 1) && dbg_in(A.status, 42, (int64_t)(L2 + 31 + kTcPF) * 32, T.cst_stride) &&
             dbg_in(A.status, 43, item % A.nslot, A.nslot - 1) &&
             dbg_in(A.status, 45, pd.out0, A.out_cap - 1) && dbg_in(A.status, 46, pd.out1 < 0 ? 0 : pd.out1, A.out_cap - 1) &&
             dbg_in(A.status, 47, (int64_t)(L2 + pd.sy - 1) / pd.sy, T.max_len) &&
             dbg_in(A.status, 48, (int64_t)(s & 3), warp) && dbg_in(A.status, 49, (int64_t)warp, s & 3);
#endif
        ok = group_and(gr, ok);

        // ---- phase 1a: digits of the block's 128 rows (32 per warp) -----------
        if (ok) {
            const int lsx = 31 - __clz(pd.sx);  // refinement factors are powers of two
            for (int rr = 0; rr < 32; ++rr) {
                const int r = warp * 32 + rr;
                const int v = r0 + r;           // virtual row
                const int ex = slice_row(pd.xr, (int64_t)(v >> lsx), v < L1, d, d_pad, A.inc_mode, lsx,
                                         ablk + (int64_t)r * d_pad, (int64_t)kTcRows * d_pad, lane);
                if (lane == 0) aexp[r] = ex;
            }
        }
        group_sync(gr);
        // ---- phase 1b: the coefficients, 32 columns at a time --------------------
        // step n of the block: chunk n / KS, dimensions 16 (n % KS); its digit
        // tiles are copied one step ahead into stage (step + n) & 1
        const int lsy = 31 - __clz(pd.sy);
        const uint16_t* yc = T.ycache + (int64_t)pd.yslot * T.max_len * kTcDigits * d_pad;
        const int32_t* ye = T.yexp + (int64_t)pd.yslot * T.max_len;
        float2* cw = cblk + (int64_t)warp * T.cst_stride;
        const int nch = (L2 + kTcN - 1) / kTcN;
        const int nst = ok ? nch * KS : 0;
        auto issue = [&](int n) {
            const int c0 = (n / KS) * kTcN, kk = n % KS;
            unsigned char* sa = st0 + ((step + n) & 1) * Sm::stage;
            unsigned char* sb = sa + kTcDigits * Sm::a_tile;
            if (kk == 0 && tid < kTcN) {
                const int j = c0 + tid;
                yexp_s[(n / KS) & 1][tid] = j < L2 ? ye[j >> lsy] - lsy : 0;
            }
            // A: 4 digits x 128 rows x 2 halves of 8 dims; B: 4 digits x 32 columns x 2 halves
            for (int idx = tid; idx < kTcDigits * kTcRows * 2; idx += 128) {
                const int h = idx & 1, r = (idx >> 1) & 127, k = idx >> 8;
                cp_async16(smem_u32(sa + k * Sm::a_tile + (r >> 3) * kTcSbo + h * kTcLbo + (r & 7) * 16),
                           ablk + ((int64_t)k * kTcRows + r) * d_pad + kk * kTcK + 8 * h, 16u);
            }
            for (int idx = tid; idx < kTcDigits * kTcN * 2; idx += 128) {
                const int h = idx & 1, jj = (idx >> 1) & 31, k = idx >> 6;
                const int j = c0 + jj;
                const bool in = j < L2;
                cp_async16(smem_u32(sb + k * Sm::b_tile + (jj >> 3) * kTcSbo + h * kTcLbo + (jj & 7) * 16),
                           yc + ((int64_t)(in ? (j >> lsy) : 0) * kTcDigits + k) * d_pad + kk * kTcK + 8 * h,
                           in ? 16u : 0u);
            }
        };
        if (nst > 0) issue(0);
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int n = 0; n < nst; ++n) {
            const uint32_t g = step + n;  // this step's global index
            if (n + 1 < nst) {
                // stage (g + 1) & 1 was last read by the MMAs of step g - 1
                if (g >= 1 && !mbar_wait(&mbar[(g + 1) & 1], ((g - 1) >> 1) & 1, A.status)) ok = false;
                issue(n + 1);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");  // step n's tiles have landed
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            ok = group_and(gr, ok);
            if (!ok) break;
            const int kk = n % KS;
            if (tid == 0) {
                tc_fence_after();
                unsigned char* sa = st0 + (g & 1) * Sm::stage;
                unsigned char* sb = sa + kTcDigits * Sm::a_tile;
                // group q = k + l accumulates at TMEM columns 32 q
#pragma unroll
                for (int q = 0; q < 4; ++q) {
#pragma unroll
                    for (int k = 0; k <= q; ++k) {
                        const uint64_t da = tc_desc(smem_u32(sa + k * Sm::a_tile), kTcLbo, kTcSbo);
                        const uint64_t db = tc_desc(smem_u32(sb + (q - k) * Sm::b_tile), kTcLbo, kTcSbo);
                        tc_mma(tbase + 32 * q, da, db, (kk > 0 || k > 0) ? 1u : 0u);
                    }
                }
                tc_commit(&mbar[g & 1]);
            }
            issued = g;
            if (kk == KS - 1) {
                // the chunk's MMAs are done (the last commit covers all before it)
                if (!mbar_wait(&mbar[g & 1], (g >> 1) & 1, A.status)) ok = false;
                ok = group_and(gr, ok);
                if (!ok) break;
                waited = g;
                tc_fence_after();
                {
                    const int c0 = (n / KS) * kTcN;
                    const int32_t* yx = yexp_s[(n / KS) & 1];
                    const int row = warp * 32 + lane;
                    const int ea = aexp[row];
                    const uint32_t tl = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        uint32_t g0[16], g1[16], g2[16], g3[16];
                        tmem_ld16<16>(tl + 0 * 32 + 16 * half, g0);
                        tmem_ld16<16>(tl + 1 * 32 + 16 * half, g1);
                        tmem_ld16<16>(tl + 2 * 32 + 16 * half, g2);
                        tmem_ld16<16>(tl + 3 * 32 + 16 * half, g3);
                        tmem_ld_wait();
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int jj = 16 * half + q;
                            const int j = c0 + jj;
                            // c = 2^(ea + eb) (G0 + G1 2^-8 + G2 2^-16 + G3 2^-24), rounded once to (hi, lo)
                            const float s0 = __uint_as_float(g0[q]);
                            const float t1 = __uint_as_float(g1[q]) * 0.00390625f;
                            const float sh = s0 + t1;
                            const float bv = sh - s0;
                            float e = (s0 - (sh - bv)) + (t1 - bv);
                            e += fmaf(__uint_as_float(g2[q]), 1.52587890625e-05f,
                                      __uint_as_float(g3[q]) * 5.9604644775390625e-08f);
                            const float hi = sh + e;
                            const float lo = e - (hi - sh);
                            const int ex = ea + yx[jj];
                            if (j < L2)
                                cw[(int64_t)(j + lane) * 32 + lane] = make_float2(ldexpf(hi, ex), ldexpf(lo, ex));
                        }
                    }
                }
                tc_fence_before();
                group_sync(gr);  // TMEM is free for the next chunk
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        step += nst;  // (after an early exit the loop below ends the kernel)
        // ---- phase 2: warp w sweeps strip w of the block -------------------------
        group_sync(gr);
        if (ok) {
            if (ir.next >= 0) ok = wait_slot_free(A.sched, A.pairs, item, A.nslot, A.done, A.status);
            if (ok)
                ok = sweep_strip_tc<P, NR>(A, pd, lo_p, s, item, ir.prev, ir.next, cw, seam_w,
                                           seam_w + kG * S, tiles_done, lane_tiles, rhist);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            st_release_s64(&A.done[item % A.nslot], (long long)item);
        }
        if (!ok && lane == 0) atomicExch(&stop_s, 1);
        group_sync(gr);
        if (stop_s) break;
    }
    // in-flight MMAs (after an early exit) complete before TMEM is freed
    if (issued > waited) mbar_wait(&mbar[issued & 1], (uint32_t)(issued >> 1) & 1, A.status);
    tc_fence_before();
    __syncthreads();  // every group is done with TMEM
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s), "r"(128 * kTcGroups));
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
        for (int q = 0; q < 4; ++q) {
            unsigned v = rhist[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
            if (lane == 0 && v) atomicAdd(&A.ring_hist[q], v);
        }
    }
}

}  // namespace sigk
