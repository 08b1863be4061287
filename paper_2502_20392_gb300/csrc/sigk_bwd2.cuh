// sigk_bwd2.cuh -- reverse-mode (adjoint) sweep of the wavefront solver for
// any dimension d, with the chain to the increments as a contraction.
//
// One work item = (pair, 32-row strip, one row per lane), the strips of a pair
// in DECREASING order (the schedule's k-th item of a pair is strip
// n_strips - 1 - k).  Per item the warp runs four phases over a per-warp
// strip area cs of (L2 + 32 + kB2PF) x 32 floats, skewed so that the 32 values the
// lanes touch in one sweep step are contiguous: entry t * 32 + l belongs to
// row l and column t - l.
//
//   phase 0  the strip's coefficients c_ij = <dx_i, dy_j>: a register-blocked
//            FMA micro-GEMM (lane = column, 32 row accumulators, the
//            contraction staged through shared memory 32 dimensions at a time,
//            two-level sums), written into cs through a shared-memory
//            transpose;
//   pass A   (only when the training forward did not store the tile records)
//            the strip's forward replayed from its stored input seam, every
//            tile's record written to a per-warp scratch area;
//   pass B   the reverse sweep (mirrored skew, lane 31 first): each tile's
//            inputs rebuilt from its record by inverting the bottom-to-top
//            update, the adjoint of the tile map applied (tile_adjoint), and
//            g_ij = dk/dc_ij times the pair's upstream weight written over c_ij
//            in cs;
//   phase C  the chain to the increments, two contractions over the strip:
//            dL/ddx_i = sum_j g_ij dy_j (lane = row, summed over the whole
//            strip before one atomic add per row and dimension) and
//            dL/ddy_j += sum_i g_ij dx_i (lane = column, added with atomics
//            per column block), in chunks of 8, 16 or 32 dimensions.
// Neither pass A nor pass B holds an increment: their registers go to the
// edge polynomials and the tile adjoint, and the kernel serves every d.
#pragma once
#include "sigk_device.cuh"
#include "sigk_fwd.cuh"
#include "sigk_fwd_cm.cuh"
#include "sigk_bwd.cuh"

namespace sigk {

constexpr int kB2KC = 32;   // contraction chunk of phase 0
constexpr int kB2Blk = 32 * 34;        // a 32 x 32 block of c or g (row stride 34)
// the strip rows' and a column block's points or increments, [33][up to 32
// dimensions + 4] each (33 points give 32 increments)
constexpr int kB2XS = 33 * 36;
constexpr int kB2YS = 33 * 36;

template <int P>
struct Bwd2Smem {
    static constexpr int S = P + 4;
    static constexpr int RS = rec_floats(P);
    static constexpr int RB = 32 * (S > RS ? S : RS);   // record block / seam-in block
    static constexpr int SA = adj_seam_floats(P);
    static constexpr int sweep = 2 * RB + 2 * 32 * SA;  // passes A and B
    // phases 0 and C: one 32 x 32 block (c, then g and the transposed
    // gradients), the strip rows' increments and one column block's
    static constexpr int gemm = kB2Blk + kB2XS + kB2YS;
    static constexpr int per_warp = (sweep > gemm ? sweep : gemm);
};

// Async copy (cp.async, one wait for all of them) of the skewed entries of
// columns [j0, j0 + 32) into blk[r * 34 + col] = entry (row r, column
// j0 + col); each step tt reads one contiguous 128-byte line of cs (entry
// t * 32 + l = row l, column t - l) and the lanes write distinct banks.
// Columns at or past L2 are zeros.
__device__ __forceinline__ void skew_to_block_async(const float* cs, float* blk, int j0, int L2, int lane) {
#pragma unroll 7
    for (int tt = 0; tt < 63; ++tt) {
        const int col = tt - lane;
        if (col >= 0 && col < 32) {
            if (j0 + col < L2) cp_async4(blk + lane * 34 + col, cs + (int64_t)(j0 + tt) * 32 + lane);
            else blk[lane * 34 + col] = 0.0f;
        }
    }
}

// The reverse: blk[r * 34 + col] -> skewed entries of cs (columns < L2).
__device__ __forceinline__ void block_to_skew(float* cs, const float* blk, int j0, int L2, int lane) {
#pragma unroll 7
    for (int tt = 0; tt < 63; ++tt) {
        const int col = tt - lane;
        if (col >= 0 && col < 32 && j0 + col < L2) cs[(int64_t)(j0 + tt) * 32 + lane] = blk[lane * 34 + col];
    }
}

// Staging of 32 increments (rows v0 .. v0 + 31 of a path with Lv segments,
// dimensions k0 .. k0 + DC - 1, zero past the path or past d) into
// dst[r * ds + e'].  Unrefined paths with d a multiple of 4 and 16-byte
// aligned rows are copied with 16-byte cp.async (points: 33 rows, differenced
// by finish_rows after the wait; the caller commits and waits); otherwise the
// rows are loaded and differenced at once (stage_increments: refined paths,
// odd d).  Returns true when finish_rows is needed.
template <int DC>
__device__ __forceinline__ bool stage_rows(float* dst, int ds, const float* z, int v0, int Lv, int d, int k0,
                                           int inc_mode, int s, int lane) {
    const bool async = s == 1 && (d & 3) == 0 && ((reinterpret_cast<uintptr_t>(z) & 15) == 0);
    if (!async) {
        if (lane < DC) stage_increments(dst + lane, ds, z, v0, Lv, d, k0 + lane, inc_mode, s);
        return false;
    }
    const int dn = min(DC, d - k0);  // a multiple of 4
    const int nq = dn >> 2;
    const int nrow = inc_mode ? 32 : 33;
    const int vend = inc_mode ? Lv : Lv + 1;  // rows of z that exist
    for (int idx = lane; idx < nrow * nq; idx += 32) {
        const int r = idx / nq, q = idx - r * nq;
        const int v = v0 + r;
        const bool in = v < vend;
        cp_async16z(dst + r * ds + 4 * q, z + (int64_t)(in ? v : v0) * d + k0 + 4 * q, in ? 16 : 0);
    }
    if (dn < DC) {  // dimensions past d
        for (int idx = lane; idx < nrow * (DC - dn); idx += 32) {
            const int r = idx / (DC - dn);
            dst[r * ds + dn + (idx - r * (DC - dn))] = 0.0f;
        }
    }
    return inc_mode == 0;
}

// After the copies of stage_rows (points) have landed: increments
// dst[r] = dst[r + 1] - dst[r] in place (zero for rows past the path).
template <int DC>
__device__ __forceinline__ void finish_rows(float* dst, int ds, int v0, int Lv, int lane) {
    if (lane < DC) {
        float p = dst[lane];
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const float q = dst[(r + 1) * ds + lane];
            dst[r * ds + lane] = v0 + r < Lv ? q - p : 0.0f;
            p = q;
        }
    }
}

// Phase 0 of the adjoint: the strip's coefficients c_ij = <dx_i, dy_j> for all
// columns, by 32-column blocks: a register-blocked FMA micro-GEMM (lane =
// column, 32 row accumulators; the rows' increments broadcast from shared
// memory, four dimensions per 128-bit load; chunks of 32 dimensions summed in
// two levels, as in the two-phase forward), written into the skewed area cs
// through the block blk.  The strip's rows are staged once when d <= 32.
// ONE: d <= 32, a single chunk: the products are summed straight into the
// accumulators (the two-level sum would only add zero, and its second set of
// 32 accumulators costs registers).
template <bool ONE>
__device__ __forceinline__ void strip_coefficients(float* cs, float* wsm, const float* xr, const float* yr,
                                                   int i0, int L1, int L2, int d, int inc_mode, int sx,
                                                   int sy, int lane) {
    float* blk = wsm;
    float* xs = blk + kB2Blk;  // [33][36]
    float* ys = xs + kB2XS;    // [33][36]
    for (int j0 = 0; j0 < L2; j0 += 32) {
        float acc[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) acc[r] = 0.0f;
        for (int k0 = 0; k0 < d; k0 += kB2KC) {
            __syncwarp();
            const bool rows = j0 == 0 || d > kB2KC;
            bool fx = false;
            if (rows) fx = stage_rows<kB2KC>(xs, 36, xr, i0, L1, d, k0, inc_mode, sx, lane);
            const bool fy = stage_rows<kB2KC>(ys, 36, yr, j0, L2, d, k0, inc_mode, sy, lane);
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp();
            if (fx) finish_rows<kB2KC>(xs, 36, i0, L1, lane);
            if (fy) finish_rows<kB2KC>(ys, 36, j0, L2, lane);
            __syncwarp();
            const int kn = min(kB2KC, d - k0);
            if constexpr (ONE) {
                for (int e = 0; e < kn; e += 4) {
                    const float4 y = *reinterpret_cast<const float4*>(ys + lane * 36 + e);
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        const float4 x = *reinterpret_cast<const float4*>(xs + r * 36 + e);
                        acc[r] = fmaf(x.x, y.x, acc[r]);
                        acc[r] = fmaf(x.y, y.y, acc[r]);
                        acc[r] = fmaf(x.z, y.z, acc[r]);
                        acc[r] = fmaf(x.w, y.w, acc[r]);
                    }
                }
            } else {
                float part[32];
#pragma unroll
                for (int r = 0; r < 32; ++r) part[r] = 0.0f;
                for (int e = 0; e < kn; e += 4) {
                    const float4 y = *reinterpret_cast<const float4*>(ys + lane * 36 + e);
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        const float4 x = *reinterpret_cast<const float4*>(xs + r * 36 + e);
                        part[r] = fmaf(x.x, y.x, part[r]);
                        part[r] = fmaf(x.y, y.y, part[r]);
                        part[r] = fmaf(x.z, y.z, part[r]);
                        part[r] = fmaf(x.w, y.w, part[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < 32; ++r) acc[r] += part[r];
            }
        }
        __syncwarp();
        // lane = column: blk[r][col] = c(row r, column j0 + col), then skewed into cs
#pragma unroll
        for (int r = 0; r < 32; ++r) blk[r * 34 + lane] = acc[r];
        __syncwarp();
        block_to_skew(cs, blk, j0, L2, lane);
    }
    __syncwarp();
}

// Gradient of one strip's rows or of one column block, added to the path's
// gradient rows with atomics, 32 consecutive floats per warp instruction:
// tb[r * (DC + 1) + e'] holds the gradient of increment v0 + r, dimension
// k0 + e'.  With increments (inc_mode 1) it is added to the increment's row
// (a refined path's increment v to its segment v / s, scaled by 1/s).  With
// points, increment v = point v + 1 - point v: for unrefined paths the
// point gradients of the block are formed first (point v0 + r gets
// tb[r - 1] - tb[r], one atomic per point and dimension; the block's two end
// points get one term each, the other comes from the neighbouring block),
// otherwise each increment adds to its two end points.
template <int DC>
__device__ __forceinline__ void add_gradient_rows(float* g, const float* tb, int v0, int Lv, int s,
                                                  int k0, int d, int inc_mode, int lane) {
    if (!inc_mode && s == 1) {
#pragma unroll 4
        for (int idx = lane; idx < 33 * DC; idx += 32) {
            const int r = idx / DC, ee = idx - r * DC;
            const int e = k0 + ee, v = v0 + r;  // point v
            float val = 0.0f;
            if (r >= 1 && v - 1 < Lv) val += tb[(r - 1) * (DC + 1) + ee];
            if (r < 32 && v < Lv) val -= tb[r * (DC + 1) + ee];
            if (e < d && v <= Lv && val != 0.0f) atomicAdd(g + (int64_t)v * d + e, val);
        }
        return;
    }
    const float rs = 1.0f / (float)s;
#pragma unroll 4
    for (int idx = lane; idx < 32 * DC; idx += 32) {
        const int r = idx / DC, ee = idx - r * DC;
        const int v = v0 + r, e = k0 + ee;
        const float val = tb[r * (DC + 1) + ee];
        if (v < Lv && e < d && val != 0.0f) {
            const int64_t seg = v / s;
            const float w = s == 1 ? val : val * rs;
            if (inc_mode) {
                atomicAdd(g + seg * d + e, w);
            } else {
                atomicAdd(g + (seg + 1) * d + e, w);
                atomicAdd(g + seg * d + e, -w);
            }
        }
    }
}

// Phase C of the adjoint: the chain from g_ij = w dk/dc_ij (the strip's
// skewed area cs) to the increments, in chunks of DC dimensions:
//   dL/ddx_i = sum_j g_ij dy_j   (lane = row i; the strip's sum over all
//                                 column blocks, in two levels)
//   dL/ddy_j += sum_i g_ij dx_i  (lane = column j of the block)
// Each lane accumulates DC dimensions in registers; the other operand's row
// is read from shared memory with 128-bit broadcast loads, so every lane does
// useful work for any d (an FMA per 1.25 instructions).  Each column block's
// g and increments arrive by cp.async with one wait.  Shared memory of the
// warp: blk [32][34] (the block of g, later the transposed gradients), xs
// and ys [33][DC + 4] (the increments of the strip's rows and of
// the block's columns).
template <int DC>
__device__ __forceinline__ void chain_strip(const float* cs, float* wsm, const float* xr, const float* yr,
                                            float* gxr, float* gyr, int i0, int L1, int L2, int d,
                                            int inc_mode, int sx, int sy, int lane) {
    constexpr int DS = DC + 4;
    float* blk = wsm;
    float* xs = blk + kB2Blk;
    float* ys = xs + kB2XS;
    for (int k0 = 0; k0 < d; k0 += DC) {
        __syncwarp();
        const bool fx = stage_rows<DC>(xs, DS, xr, i0, L1, d, k0, inc_mode, sx, lane);
        float gx[DC];
#pragma unroll
        for (int e = 0; e < DC; ++e) gx[e] = 0.0f;
        for (int j0 = 0; j0 < L2; j0 += 32) {
            __syncwarp();
            skew_to_block_async(cs, blk, j0, L2, lane);  // blk[r * 34 + col] = g(row r, column j0 + col)
            const bool fy = stage_rows<DC>(ys, DS, yr, j0, L2, d, k0, inc_mode, sy, lane);
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp();
            if (fx && j0 == 0) finish_rows<DC>(xs, DS, i0, L1, lane);
            if (fy) finish_rows<DC>(ys, DS, j0, L2, lane);
            __syncwarp();
            if (gxr) {
                float gb[DC];
#pragma unroll
                for (int e = 0; e < DC; ++e) gb[e] = 0.0f;
#pragma unroll 4
                for (int c = 0; c < 32; ++c) {
                    const float gv = blk[lane * 34 + c];
                    const float4* y4 = reinterpret_cast<const float4*>(ys + c * DS);
#pragma unroll
                    for (int q = 0; q < DC / 4; ++q) {
                        const float4 y = y4[q];
                        gb[4 * q + 0] = fmaf(gv, y.x, gb[4 * q + 0]);
                        gb[4 * q + 1] = fmaf(gv, y.y, gb[4 * q + 1]);
                        gb[4 * q + 2] = fmaf(gv, y.z, gb[4 * q + 2]);
                        gb[4 * q + 3] = fmaf(gv, y.w, gb[4 * q + 3]);
                    }
                }
#pragma unroll
                for (int e = 0; e < DC; ++e) gx[e] += gb[e];
            }
            if (gyr) {
                float gy[DC];
#pragma unroll
                for (int e = 0; e < DC; ++e) gy[e] = 0.0f;
#pragma unroll 4
                for (int r = 0; r < 32; ++r) {
                    const float gv = blk[r * 34 + lane];
                    const float4* x4 = reinterpret_cast<const float4*>(xs + r * DS);
#pragma unroll
                    for (int q = 0; q < DC / 4; ++q) {
                        const float4 x = x4[q];
                        gy[4 * q + 0] = fmaf(gv, x.x, gy[4 * q + 0]);
                        gy[4 * q + 1] = fmaf(gv, x.y, gy[4 * q + 1]);
                        gy[4 * q + 2] = fmaf(gv, x.z, gy[4 * q + 2]);
                        gy[4 * q + 3] = fmaf(gv, x.w, gy[4 * q + 3]);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int e = 0; e < DC; ++e) blk[lane * (DC + 1) + e] = gy[e];
                __syncwarp();
                add_gradient_rows<DC>(gyr, blk, j0, L2, sy, k0, d, inc_mode, lane);
            }
        }
        if (gxr) {
            __syncwarp();
#pragma unroll
            for (int e = 0; e < DC; ++e) blk[lane * (DC + 1) + e] = gx[e];
            __syncwarp();
            add_gradient_rows<DC>(gxr, blk, i0, L1, sx, k0, d, inc_mode, lane);
        }
    }
    __syncwarp();
}

// 168 registers at three CTAs per SM: measured 80.9 ms on the 64-path Gram
// against 93.0 ms at four CTAs per SM and 128 registers (which spill) at order
// 8, and 70.8 against 72.0 ms at order 6 with three rings (60 bytes spilled).
template <int P, int NR>
__global__ void __launch_bounds__(128, 3) bwd2_kernel(BwdArgs A, float* cscratch, int64_t cstride) {
    constexpr int S = P + 4;
    constexpr int SA = adj_seam_floats(P);
    using Sm = Bwd2Smem<P>;
    constexpr int RS = Sm::RS;
    extern __shared__ float4 smem_f4[];
    float* smem = reinterpret_cast<float*>(smem_f4);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    float* wsm = smem + warp * Sm::per_warp;
    // passes A and B
    float* sin_ = wsm;                      // forward seam-in block / record buffer 0
    float* rbuf1 = sin_ + Sm::RB;           // record buffer 1
    float* ain = rbuf1 + Sm::RB;            // adjoint seam-in block
    float* aout = ain + 32 * SA;            // adjoint seam-out block
    // phases 0 and C use the same memory (strip_coefficients, chain_strip)
    float* rec = A.rec + (size_t)gwarp * A.rec_stride;
    float* cs = cscratch + (size_t)gwarp * cstride;
    const int n_items = A.sched.hdr[2];
    const int d = A.d;
    unsigned long long tiles = 0, replayed = 0;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.item_counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_items) break;
        if (ld_volatile_s32(A.status) != 0) break;
        const ItemRef ir = decode_item(A.sched, A.pairs, item);
        const int lo_p = ir.pair;
        const PairDesc pd = A.pairs[lo_p];
        const int nst = pd.n_strips;
        const int s = nst - 1 - ir.k;  // reverse strip order
        const int L1 = pd.L1, L2 = pd.L2;
        const int i0 = s * 32;
        const int row = i0 + lane;
        const bool has_row = row < L1;
        const float* st_base = A.store + A.store_off[lo_p];
        bool ok = true;
#ifdef SIGK_DEBUG
        {
            const int RRd = A.rec_off != nullptr ? A.rec_rows : 1;
            bool in = dbg_in(A.status, 21, lo_p, A.n_pairs - 1) &&
                      dbg_in(A.status, 22, item % A.nslot, A.nslot - 1) &&
                      dbg_in(A.status, 23, ir.prev >= 0 ? ir.prev % A.nslot : 0, A.nslot - 1) &&
                      dbg_in(A.status, 24, s > 0 ? A.store_off[lo_p] + (int64_t)s * L2 * S : 0, A.store_cap) &&
                      dbg_in(A.status, 28, (int64_t)(L2 + 32 + kB2PF) * 32, cstride);
            if (in && A.rec_off != nullptr)
                in = dbg_in(A.status, 25, A.rec_off[lo_p] + (int64_t)(s / RRd + 1) * (L2 + 32) * 32 * RRd * RS,
                            A.rec_cap);
            if (in && A.rec_off == nullptr)
                in = dbg_in(A.status, 26, (int64_t)(L2 + 31) * 32 * RS, A.rec_stride) &&
                     dbg_in(A.status, 27, (int64_t)(gwarp + 1) * A.rec_stride, A.rec_total);
            if (!__all_sync(kFull, in)) break;
        }
#endif

        // ------------------------- phase 0: coefficients -------------------------
        if (d <= kB2KC) strip_coefficients<true>(cs, wsm, pd.xr, pd.yr, i0, L1, L2, d, A.inc_mode, pd.sx, pd.sy, lane);
        else strip_coefficients<false>(cs, wsm, pd.xr, pd.yr, i0, L1, L2, d, A.inc_mode, pd.sx, pd.sy, lane);

        // ------------------------- pass A: forward replay ------------------------
        float a[P + 1], a1lo = 0.0f;
#pragma unroll
        for (int p = 0; p <= P; ++p) a[p] = 0.0f;
        int E = 0;
        float ohi = 1.0f, olo = 0.0f, ob1lo = 0.0f, ob[P + 1];
#pragma unroll
        for (int q = 0; q <= P; ++q) ob[q] = 0.0f;
        int oE = 0;
        const int T = L2 + 31;
        const bool stored = A.rec_off != nullptr;
        const int RR = stored ? A.rec_rows : 1;
        const int rw = (s % RR) * 32 + lane;
        const float* rbase = stored ? A.rec_store + A.rec_off[lo_p] + (int64_t)(s / RR) * (L2 + 32) * 32 * RR * RS
                                    : rec;
        if (stored) rec_get_state<P>(rbase + ((int64_t)T * 32 * RR + rw) * RS, a1lo, a);
        // BULK: records of a multiple of 4 floats leave the replay as one
        // bulk copy per step (staged in the two buffers that the replay does
        // not use, the second record buffer and the adjoint seam-in block);
        // pass B then reads them past L1 (16-byte cp.async.cg), which does
        // not see the bulk copies' writes
        constexpr bool BULK = (RS % 4) == 0;
        static_assert(2 * Sm::RB + 32 * RS <= Sm::per_warp, "the second staging block fits the warp's area");
        float* const stg0 = rbuf1;
        float* const stg1 = ain;
        if (!stored) {
            float cq[kB2PF];
#pragma unroll
            for (int k = 0; k < kB2PF; ++k) cq[k] = cs[k * 32 + lane];
            for (int t = 0; t < T; ++t) {
                const float c = cq[0];
#pragma unroll
                for (int k = 0; k + 1 < kB2PF; ++k) cq[k] = cq[k + 1];
                cq[kB2PF - 1] = cs[(int64_t)(t + kB2PF) * 32 + lane];
                if ((t & 31) == 0 && t < L2) {
                    const int nb = min(32, L2 - t);
                    if (s > 0) warp_copy_cg<S>(sin_, st_base + ((size_t)(s - 1) * L2 + t) * S, nb * S, lane);
                    __syncwarp();
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
                    if (s > 0 && t < L2) {
                        float v[S];
                        seam_entry_load<S>(sin_ + (t & 31) * S, v);
                        seam_unpack<P>(v, hi, lo, b1lo, b, F);
                    } else {
                        hi = 1.0f; lo = 0.0f; b1lo = 0.0f; F = 0;
#pragma unroll
                        for (int q = 1; q <= P; ++q) b[q] = 0.0f;
                    }
                }
                if constexpr (BULK) {
                    // the bulk copy of step t - 2 has read this step's staging block
                    if (lane == 0) bulk_wait_read<1>();
                    __syncwarp();
                }
                const int j = t - lane;
                if (j >= 0 && j < L2) {
                    float* rslot = BULK ? ((t & 1) ? stg1 : stg0) + lane * RS : rec + (size_t)t * RS * 32 + lane * RS;
                    rec_put_head<P>(rslot, hi, b1lo, b);
                    const float rbP = b[P];
                    const int Eb = E;
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
                    tile_update<P, NR>(c, a, a1lo, hi, lo, b, b1lo, NR);
                    int bump = 0;
                    if (fabsf(hi) > 1.8446744e19f) {
                        const float sc = 5.421011e-20f;
                        a1lo *= sc;
#pragma unroll
                        for (int p = 1; p <= P; ++p) a[p] *= sc;
                        hi *= sc; lo *= sc; b1lo *= sc;
#pragma unroll
                        for (int q = 1; q <= P; ++q) b[q] *= sc;
                        E += 64;
                        bump = 1;
                    }
                    rec_put_tail<P>(rslot, rbP, pack_exp(F, Eb, bump, bump));
                    ohi = hi; olo = lo; ob1lo = b1lo; oE = E;
#pragma unroll
                    for (int q = 1; q <= P; ++q) ob[q] = b[q];
                    replayed += has_row ? 1ull : 0ull;
                }
                if constexpr (BULK) {
                    // the step's 32 records (slots of lanes outside the grid
                    // carry stale values that no reader asks for)
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        bulk_store(rec + (size_t)t * RS * 32, (t & 1) ? stg1 : stg0, 32 * RS * (uint32_t)sizeof(float));
                        bulk_commit();
                    }
                }
            }
            if constexpr (BULK) {
                // every record is in global memory and visible to the generic
                // proxy before pass B reads it (and the staging blocks are free)
                if (lane == 0) {
                    bulk_wait_all();
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
            }
        }
        __syncwarp();

        // ------------------------- pass B: reverse sweep -------------------------
        const double wsc_d = A.pair_w[lo_p] * ldexp(1.0, A.pair_exp[lo_p]);
        const float wsc = (float)wsc_d;
        const bool last_strip = (s == nst - 1);
        const bool has_ain = ir.prev >= 0;   // adjoint seam of strip s + 1
        const bool has_aout = ir.next >= 0;  // consumed by strip s - 1
        const int slot_in = has_ain ? ir.prev % A.nslot : 0;
        const int slot_out = item % A.nslot;
        if (has_aout) ok = wait_slot_free(A.sched, A.pairs, item, A.nslot, A.done, A.status);
        a[1] += a1lo;  // the reverse sweep carries the first-order term as one float
        float Ab[P + 1];
#pragma unroll
        for (int p = 0; p <= P; ++p) Ab[p] = 0.0f;
        float oB0 = 0.0f, oBb[P + 1];
#pragma unroll
        for (int q = 0; q <= P; ++q) oBb[q] = 0.0f;
        const int lp = 31 - lane;
        __threadfence_block();
        __syncwarp();
        auto rbuf = [&](int tpp) { return (tpp & 1) ? rbuf1 : sin_; };
        auto rec_fetch = [&](int tpp) {
            const int j = L2 + 30 - tpp - lane;
            if (j >= 0 && j < L2) {
                const float* src = rbase + ((int64_t)(j + rw / RR) * 32 * RR + rw) * RS;
                float* dst = rbuf(tpp) + lane * RS;
                if constexpr (BULK) {
#pragma unroll
                    for (int g = 0; g < RS / 4; ++g) cp_async16z(dst + 4 * g, src + 4 * g, 16);
                } else {
#pragma unroll
                    for (int g = 0; g < RS / 2; ++g) cp_async8(dst + 2 * g, src + 2 * g);
                }
            }
            cp_async_commit();
        };
        // the coefficient of reverse step tp sits at entry (L2 + 30 - tp) * 32 + lane
        auto cidx = [&](int tpp) { return (int64_t)(L2 + 30 - tpp) * 32 + lane; };
        float cq[kB2PF];
#pragma unroll
        for (int k = 0; k < kB2PF; ++k) cq[k] = (k < T) ? cs[cidx(k)] : 0.0f;
        if (ok) {
            rec_fetch(0);
            rec_fetch(1);
        }
        for (int tp = 0; tp < T && ok; ++tp) {
            const float c = cq[0];
#pragma unroll
            for (int k = 0; k + 1 < kB2PF; ++k) cq[k] = cq[k + 1];
            cq[kB2PF - 1] = (tp + kB2PF < T) ? cs[cidx(tp + kB2PF)] : 0.0f;
            if ((tp & 31) == 0 && tp < L2) {
                const int nb = min(32, L2 - tp);
                if (has_ain) {
                    const unsigned long long need =
                        ((unsigned long long)ir.prev << 32) | (unsigned)(tp + nb);
                    bool okl = true;
                    if (lane == 0) okl = wait_ge_u64(&A.prod[slot_in], need, A.status);
                    ok = __shfl_sync(kFull, okl, 0);
                    if (ok) {
                        const float* src = A.aseam + ((size_t)slot_in * A.wcols + (tp % A.wcols)) * SA;
                        warp_copy_cg<SA>(ain, src, nb * SA, lane);
                        __syncwarp();
                        if (lane == 0)
                            st_release_u64(&A.cons[slot_in],
                                           ((unsigned long long)item << 32) | (unsigned)(tp + nb));
                    }
                }
                __syncwarp();
                if (!ok) break;
            }
            float rhi, rb[P + 1];
            int rexp;
            {
                cp_async_wait<1>();
                rec_get<P>(rbuf(tp) + lane * RS, rhi, rb, rexp);
                rec_fetch(tp + 2);
            }
            float B0 = __shfl_down_sync(kFull, oB0, 1);
            float Bb[P + 1];
            Bb[0] = 0.0f;
#pragma unroll
            for (int q = 1; q <= P; ++q) Bb[q] = __shfl_down_sync(kFull, oBb[q], 1);
            if (lane == 31) {
                if (has_ain && tp < L2) {
                    const float* e_ = ain + (tp & 31) * SA;
                    if constexpr (SA % 4 == 0) {
                        float v[SA];
#pragma unroll
                        for (int g4 = 0; g4 < SA / 4; ++g4) {
                            const float4 w = reinterpret_cast<const float4*>(e_)[g4];
                            v[4 * g4] = w.x; v[4 * g4 + 1] = w.y; v[4 * g4 + 2] = w.z; v[4 * g4 + 3] = w.w;
                        }
                        B0 = v[0];
#pragma unroll
                        for (int q = 1; q <= P; ++q) Bb[q] = v[q];
                    } else {
                        B0 = e_[0];
#pragma unroll
                        for (int q = 1; q <= P; ++q) Bb[q] = e_[q];
                    }
                } else {
                    const bool seed = last_strip && tp == 0;  // k = b0 + sum_q bh_q / q!
                    B0 = seed ? 1.0f : 0.0f;
#pragma unroll
                    for (int q = 1; q <= P; ++q) Bb[q] = seed ? c_inv_fact[q] : 0.0f;
                }
            }
            const int jr = tp - lp;
            if (jr >= 0 && jr < L2) {
                float hi = rhi;
                float b[P + 1];
                b[0] = 0.0f;
#pragma unroll
                for (int q = 1; q <= P; ++q) b[q] = rb[q];
                const bool plain = exp_plain(rexp);
                int F = 0, Eb = 0, Em = 0;
                if (!plain) {
                    int abump, bbump;
                    unpack_exp(rexp, F, Eb, abump, bbump);
                    Em = F > Eb ? F : Eb;
                    if (abump) {
#pragma unroll
                        for (int p = 1; p <= P; ++p) { a[p] *= 1.8446744e19f; Ab[p] *= 5.421011e-20f; }
                    }
                    if (bbump) {
                        B0 *= 5.421011e-20f;
#pragma unroll
                        for (int q = 1; q <= P; ++q) Bb[q] *= 5.421011e-20f;
                    }
                    if (F < Em) {
                        const float sc = exp2_nonpos(F - Em);
                        hi *= sc;
#pragma unroll
                        for (int q = 1; q <= P; ++q) b[q] *= sc;
                    }
                }
                float ain_[P + 1], ha[P + 1];
                tile_inverse_a<P, NR>(c, a, hi, b, NR, ain_, ha);
                const float cbar = tile_adjoint<P, NR>(c, ain_, hi, b, ha, Ab, B0, Bb, NR);
#pragma unroll
                for (int p = 1; p <= P; ++p) a[p] = ain_[p];
                if (!plain) {
                    if (Eb < Em) {
                        const float dn = exp2_nonpos(Eb - Em), up = exp2_nonneg(Em - Eb);
#pragma unroll
                        for (int p = 1; p <= P; ++p) { a[p] *= up; Ab[p] *= dn; }
                    }
                    if (F < Em) {
                        const float sc = exp2_nonpos(F - Em);
                        B0 *= sc;
#pragma unroll
                        for (int q = 1; q <= P; ++q) Bb[q] *= sc;
                    }
                }
                // g = dk/dc times the pair's upstream weight, over c (rows past
                // the path contribute nothing)
                cs[cidx(tp)] = has_row ? cbar * wsc : 0.0f;
                oB0 = B0;
#pragma unroll
                for (int q = 1; q <= P; ++q) oBb[q] = Bb[q];
                if (lane == 0 && has_aout) {
                    float* e_ = aout + (jr & 31) * SA;
                    if constexpr (SA % 4 == 0) {
                        float v[SA];
                        v[0] = B0;
#pragma unroll
                        for (int q = 1; q <= P; ++q) v[q] = Bb[q];
#pragma unroll
                        for (int q = P + 1; q < SA; ++q) v[q] = 0.0f;
#pragma unroll
                        for (int g4 = 0; g4 < SA / 4; ++g4)
                            reinterpret_cast<float4*>(e_)[g4] =
                                make_float4(v[4 * g4], v[4 * g4 + 1], v[4 * g4 + 2], v[4 * g4 + 3]);
                    } else {
                        e_[0] = B0;
#pragma unroll
                        for (int q = 1; q <= P; ++q) e_[q] = Bb[q];
                    }
                }
                tiles += has_row ? 1ull : 0ull;
            }
            __syncwarp();
            // lane 0 closed a block of 32 reverse columns: flush the adjoint seam
            const int jj = tp - 31;
            if (has_aout && jj >= 0 && jj < L2 && (((jj & 31) == 31) || jj == L2 - 1)) {
                const int start = jj & ~31;
                const int nb = jj - start + 1;
                if (start + nb > A.wcols) {
                    const unsigned long long need = ((unsigned long long)ir.next << 32) |
                                                    (unsigned)(start + nb - A.wcols);
                    bool okl = true;
                    if (lane == 0) okl = wait_ge_u64(&A.cons[slot_out], need, A.status);
                    ok = __shfl_sync(kFull, okl, 0);
                }
                if (ok) {
                    float* dst = A.aseam + ((size_t)slot_out * A.wcols + (start % A.wcols)) * SA;
                    for (int idx = lane; idx < nb * SA; idx += 32) __stcg(dst + idx, aout[idx]);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0)
                        st_release_u64(&A.prod[slot_out],
                                       ((unsigned long long)item << 32) | (unsigned)(start + nb));
                }
                __syncwarp();
            }
        }
        // record copies still in flight (the last steps', or after an early
        // exit) complete before the buffers are used again
        cp_async_wait<0>();
        __syncwarp();
        // the adjoint seam of this strip is published: the next strip may start
        if (lane == 0) {
            __threadfence();
            st_release_s64(&A.done[item % A.nslot], (long long)item);
        }

        // ------------------------- phase C: chain to the increments ----------------
        if (ok) {
            if (d <= 8)
                chain_strip<8>(cs, wsm, pd.xr, pd.yr, pd.gxr, pd.gyr, i0, L1, L2, d, A.inc_mode, pd.sx, pd.sy, lane);
            else if (d <= 16)
                chain_strip<16>(cs, wsm, pd.xr, pd.yr, pd.gxr, pd.gyr, i0, L1, L2, d, A.inc_mode, pd.sx, pd.sy, lane);
            else
                chain_strip<32>(cs, wsm, pd.xr, pd.yr, pd.gxr, pd.gyr, i0, L1, L2, d, A.inc_mode, pd.sx, pd.sy, lane);
        }
        __syncwarp();
        if (!ok) break;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tiles += __shfl_down_sync(kFull, tiles, o);
        replayed += __shfl_down_sync(kFull, replayed, o);
    }
    if (lane == 0) {
        atomicAdd(&A.counters[2], tiles);
        atomicAdd(&A.counters[3], replayed);
    }
}

}  // namespace sigk
