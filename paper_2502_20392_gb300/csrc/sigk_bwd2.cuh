// sigk_bwd2.cuh -- reverse-mode (adjoint) sweep of the wavefront solver for
// any dimension d, with the chain to the increments as a contraction.
//
// One work item = (pair, 32-row strip, one row per lane), the strips of a pair
// in DECREASING order (the schedule's k-th item of a pair is strip
// n_strips - 1 - k).  Per item the warp runs four phases over a per-warp
// strip area cs of (L2 + 34) x 32 floats, skewed so that the 32 values the
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
//            dL/ddx_i = sum_j g_ij dy_j and dL/ddy_j += sum_i g_ij dx_i, again
//            as FMA micro-GEMMs (lane = dimension), the first summed over the
//            whole strip before one atomic add per row and dimension, the
//            second added with atomics per column block.
// Neither pass A nor pass B holds an increment: their registers go to the
// edge polynomials and the tile adjoint, and the kernel serves every d.
#pragma once
#include "sigk_device.cuh"
#include "sigk_fwd.cuh"
#include "sigk_fwd_cm.cuh"
#include "sigk_bwd.cuh"

namespace sigk {

constexpr int kB2KC = 32;   // contraction chunk of phases 0 and C
constexpr int kB2PF = 2;    // coefficient loads in flight per lane in passes A and B

template <int P>
struct Bwd2Smem {
    static constexpr int S = P + 4;
    static constexpr int RS = rec_floats(P);
    static constexpr int RB = 32 * (S > RS ? S : RS);   // record block / seam-in block
    static constexpr int SA = adj_seam_floats(P);
    static constexpr int sweep = 2 * RB + 2 * 32 * SA;  // passes A and B
    // phases 0 and C: the row increments (phase 0: [dim][row], stride 36 for
    // 16-byte reads; phase C: [row][dim], stride 33), the column increments
    // ([column][dim], stride 33) and a 32 x 34 block of coefficients or of g
    // (row stride 34: the skewed reads and the row-wise writes hit distinct
    // banks)
    static constexpr int gemm = kB2KC * 36 + 32 * 33 + 32 * 34;
    static constexpr int per_warp = (sweep > gemm ? sweep : gemm);
};

// Copy the 32 x 32 block of skewed entries of columns [j0, j0 + 32) (all
// rows) between cs and blk[r * 34 + col]; to_blk: cs -> blk.  Columns at or
// past L2 are zero in blk and untouched in cs.
__device__ __forceinline__ void skew_block(float* cs, float* blk, int j0, int L2, bool to_blk, int lane) {
    for (int tt = 0; tt < 63; ++tt) {
        const int col = tt - lane;
        if (col >= 0 && col < 32) {
            const int j = j0 + col;
            float* e = cs + (int64_t)(j0 + tt) * 32 + lane;
            if (to_blk) blk[lane * 34 + col] = j < L2 ? *e : 0.0f;
            else if (j < L2) *e = blk[lane * 34 + col];
        }
    }
}

template <int P, int NR>
__global__ void __launch_bounds__(128, 4) bwd2_kernel(BwdArgs A, float* cscratch, int64_t cstride) {
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
    // phases 0 and C (the same memory)
    float* opa = wsm;                       // [32][36] or [32][33]
    float* opb = opa + kB2KC * 36;          // [32][33]
    float* blk = opb + 32 * 33;             // [32][34]
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
        for (int j0 = 0; j0 < L2; j0 += 32) {
            float acc[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) acc[r] = 0.0f;
            for (int k0 = 0; k0 < d; k0 += kB2KC) {
                __syncwarp();
                const int e = k0 + lane;
                // rows transposed to [dim][row], columns to [column][dim]
                stage_increments(opa + lane * 36, 1, pd.xr, i0, L1, d, e, A.inc_mode, pd.sx);
                stage_increments(opb + lane, 33, pd.yr, j0, L2, d, e, A.inc_mode, pd.sy);
                __syncwarp();
                const int kn = min(kB2KC, d - k0);
                float part[32];
#pragma unroll
                for (int r = 0; r < 32; ++r) part[r] = 0.0f;
                for (int ee = 0; ee < kn; ++ee) {
                    const float y = opb[lane * 33 + ee];
                    const float4* xr = reinterpret_cast<const float4*>(opa + ee * 36);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 x = xr[q];
                        part[4 * q + 0] = fmaf(x.x, y, part[4 * q + 0]);
                        part[4 * q + 1] = fmaf(x.y, y, part[4 * q + 1]);
                        part[4 * q + 2] = fmaf(x.z, y, part[4 * q + 2]);
                        part[4 * q + 3] = fmaf(x.w, y, part[4 * q + 3]);
                    }
                }
#pragma unroll
                for (int r = 0; r < 32; ++r) acc[r] += part[r];
            }
            __syncwarp();
            // lane = column: blk[r][col] = c(row r, column j0 + col), then skewed into cs
#pragma unroll
            for (int r = 0; r < 32; ++r) blk[r * 34 + lane] = acc[r];
            __syncwarp();
            skew_block(cs, blk, j0, L2, false, lane);
        }
        __syncwarp();

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
                if (j >= 0 && j < L2) {
                    float* rslot = rec + (size_t)t * RS * 32 + lane * RS;
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
                    tile_update<P>(c, a, a1lo, hi, lo, b, b1lo, NR);
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
#pragma unroll
                for (int g = 0; g < RS / 2; ++g) cp_async8(dst + 2 * g, src + 2 * g);
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
                tile_inverse_a<P>(c, a, hi, b, NR, ain_, ha);
                const float cbar = tile_adjoint<P>(c, ain_, hi, b, ha, Ab, B0, Bb, NR);
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
        // dL/ddx (rows of this strip) and dL/ddy (every column), by dimension
        // chunks of 32 with lane = dimension
        if (ok) {
            const float rsx = 1.0f / (float)pd.sx, rsy = 1.0f / (float)pd.sy;
            for (int k0 = 0; k0 < d; k0 += kB2KC) {
                const int e = k0 + lane;
                __syncwarp();
                // this chunk's row increments, [row][dim] (refined rows scaled)
                stage_increments(opa + lane, 33, pd.xr, i0, L1, d, e, A.inc_mode, pd.sx);
                float gxt[32];  // dL/ddx of the strip's rows, this dimension (lane)
#pragma unroll
                for (int r = 0; r < 32; ++r) gxt[r] = 0.0f;
                for (int j0 = 0; j0 < L2; j0 += 32) {
                    __syncwarp();
                    skew_block(cs, blk, j0, L2, true, lane);  // blk[r][col] = g(row r, column j0 + col)
                    // columns' increments, [column][dim]
                    stage_increments(opb + lane, 33, pd.yr, j0, L2, d, e, A.inc_mode, pd.sy);
                    __syncwarp();
                    // dL/ddy_j (lane = dimension e): sum over the strip's rows
                    if (pd.gyr) {
                        float gy[32];
#pragma unroll
                        for (int c = 0; c < 32; ++c) gy[c] = 0.0f;
                        for (int r = 0; r < 32; ++r) {
                            const float x = opa[r * 33 + lane];
#pragma unroll
                            for (int c = 0; c < 32; ++c) gy[c] = fmaf(blk[r * 34 + c], x, gy[c]);
                        }
                        if (e < d) {
                            for (int c = 0; c < 32; ++c) {
                                const int j = j0 + c;
                                if (j < L2 && gy[c] != 0.0f) {
                                    const int64_t jcol = j / pd.sy;
                                    const float w = gy[c] * rsy;
                                    if (A.inc_mode) {
                                        atomicAdd(pd.gyr + jcol * d + e, w);
                                    } else {
                                        atomicAdd(pd.gyr + (jcol + 1) * d + e, w);
                                        atomicAdd(pd.gyr + jcol * d + e, -w);
                                    }
                                }
                            }
                        }
                    }
                    // dL/ddx_i (lane = dimension e): this block's sum, added to the
                    // strip's total (two-level sums)
                    if (pd.gxr) {
                        float gx[32];
#pragma unroll
                        for (int r = 0; r < 32; ++r) gx[r] = 0.0f;
                        for (int c = 0; c < 32; ++c) {
                            const float y = opb[c * 33 + lane];
#pragma unroll
                            for (int r = 0; r < 32; ++r) gx[r] = fmaf(blk[r * 34 + c], y, gx[r]);
                        }
#pragma unroll
                        for (int r = 0; r < 32; ++r) gxt[r] += gx[r];
                    }
                }
                if (pd.gxr && e < d) {
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        const int v = i0 + r;
                        const float g = gxt[r];
                        if (v < L1 && g != 0.0f) {
                            const int64_t seg = v / pd.sx;
                            const float w = g * rsx;
                            if (A.inc_mode) {
                                atomicAdd(pd.gxr + seg * d + e, w);
                            } else {
                                atomicAdd(pd.gxr + (seg + 1) * d + e, w);
                                atomicAdd(pd.gxr + seg * d + e, -w);
                            }
                        }
                    }
                }
            }
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
