// sigk_fwd.cuh -- persistent wavefront solver for k(x,y) = K(1,1) (forward).
//
// Schedule (the anti-diagonal sweep of App. C.1, re-blocked for a warp):
//   * the row path's segments are cut into strips of 32*R rows; a work item is
//     one (pair, strip); items of a pair are consecutive and in strip order;
//   * a warp owns an item: lane l holds rows i0 + l*R + k (k < R) with their
//     bottom-edge states a in registers and sweeps the columns j of the swept
//     path with a skew of one column per lane: at step t lane l updates tiles
//     (i0+l*R+k, t-l) for k = 0..R-1, taking the left edge b from lane l-1's
//     previous step through a warp shuffle (so every tile's two inputs are
//     ready: its left neighbour was done one step earlier, its lower neighbour
//     by the same lane one step earlier);
//   * lane 0 takes its left edges from the seam written by the previous strip
//     (strip 0 uses the boundary K = 1); lane 31 writes its right edges to the
//     seam of the next strip.  Seams live in a ring of global slots, staged 32
//     columns at a time through shared memory, with progress words published
//     by release stores and read by acquire loads.  Every wait is bounded.
//   * Rows past the end of the path are given zero increments: such tiles have
//     c = 0 and map their edges through unchanged, so lane 31 of the last
//     strip always carries the right edge of the pair's last tile.
//   * Each lane keeps one power-of-two exponent E for its edge data; incoming
//     edges are aligned to it, and both are rescaled by 2^-64 when the corner
//     value passes 2^64 (log-scale renormalisation of boundary data).
#pragma once
#include "sigk_device.cuh"

namespace sigk {

template <int D>
struct DyStride {
    // shared-memory row stride (floats) for the dy ring: an odd number of
    // 16-byte chunks, so the 8 lanes of a 128-bit load phase hit distinct banks.
    static constexpr int value = ((D / 4) % 2 == 1) ? D : D + 4;
};

template <int P, int D, int R = 1, bool REC = false>
struct FwdSmem {
    static constexpr int S = P + 4;  // seam entry: hi, lo, b1lo, b1..bP, exponent
    static constexpr int DS = DyStride<D>::value;
    // record-storing forward: two staging blocks of a step's 32 * R records
    static constexpr int stage = REC ? 2 * 32 * R * rec_floats(P) : 0;
    static constexpr int per_warp = 64 * DS + 2 * kG * S + stage;  // floats
};

// Increment of row `row` of path base z (points or increments), coordinate e.
__device__ __forceinline__ float inc_at(const float* z, int64_t row, int d, int e, int inc_mode) {
    if (inc_mode) return z[row * d + e];
    return z[(row + 1) * d + e] - z[row * d + e];
}

// Increment of VIRTUAL row v of a path whose every segment is split into s
// equal collinear pieces: segment v / s, scaled by 1/s.  Splitting leaves the
// kernel unchanged (reparametrisation / collinear-insertion invariance) and
// divides every tile coefficient c by the product of the two factors.
__device__ __forceinline__ float inc_ref(const float* z, int64_t v, int d, int e, int inc_mode,
                                         int s) {
    if (s == 1) return inc_at(z, v, d, e, inc_mode);
    return inc_at(z, v / s, d, e, inc_mode) * (1.0f / (float)s);
}

// The next 32 columns of the swept path's increments into the 64-column
// shared ring (slot (t0 + col) & 63, row stride DS): column t0 + col, or
// L2 - 1 - (t0 + col) with REV (the adjoint's reverse sweep), nb <= 32 valid.
// Every global load of a chunk is issued before its shared stores: a loop
// that interleaves them waits for each load in turn (the two pointers may
// alias as far as the compiler knows).
template <int D, int DS, bool REV>
__device__ __forceinline__ void fill_dy(float* dyw, const float* z, int t0, int nb, int L2, int d,
                                        int inc_mode, int s, int lane) {
    constexpr int CH = D < 8 ? D : 8;  // loads in flight per chunk and lane
    const float rs = 1.0f / (float)s;
#pragma unroll
    for (int q0 = 0; q0 < D; q0 += CH) {
        float v[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int idx = lane + 32 * (q0 + q);
            const int col = idx / D, e = idx % D;
            float x = 0.0f;
            if (col < nb && e < d) {
                const int64_t vr = REV ? (int64_t)(L2 - 1 - (t0 + col)) : (int64_t)(t0 + col);
                const float* p = z + (s == 1 ? vr : vr / s) * d + e;
                x = inc_mode ? __ldg(p) : __ldg(p + d) - __ldg(p);
                if (s != 1) x *= rs;
            }
            v[q] = x;
        }
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int idx = lane + 32 * (q0 + q);
            const int col = idx / D, e = idx % D;
            dyw[((t0 + col) & 63) * DS + e] = v[q];
        }
    }
}

// dst[i] = src[i] for i < n (n <= 32 * NQ) by a warp, L2-coherent loads
// (the data was written by other warps), all loads of a chunk before its
// stores (see fill_dy).
template <int NQ>
__device__ __forceinline__ void warp_copy_cg(float* dst, const float* src, int n, int lane) {
    constexpr int CH = NQ < 8 ? NQ : 8;
#pragma unroll
    for (int q0 = 0; q0 < NQ; q0 += CH) {
        float v[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int i = lane + 32 * (q0 + q);
            v[q] = (q0 + q < NQ && i < n) ? __ldcg(src + i) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int i = lane + 32 * (q0 + q);
            if (q0 + q < NQ && i < n) dst[i] = v[q];
        }
    }
}

// CTAs per SM the register allocation must allow (128 threads each): the
// largest count that ptxas meets without spilling more than a few words for
// that instantiation.  Two rows per lane at orders 10-12 with up to six rings
// take four CTAs at 128 registers (12-20 bytes spilled): the order-12,
// six-ring Gram forward took 24.9 against 26.0 ms at three CTAs and 162
// registers; seven rings would spill 220 bytes and keep three.
constexpr int fwd_min_blocks(int P, int D, int R, int NR, bool REC) {
    return REC ? ((R == 1 && !(P >= 14 && D >= 16)) || P <= 8 ? 4 : 3)
               : (R == 1 ? 4 : (R == 2 ? ((P <= 8 || (P <= 12 && NR <= 6)) ? 4 : 3) : (P <= 4 ? 4 : 3)));
}

// REC: training forward that also stores every tile's record (SolverArgs::rec).
template <int P, int D, int R, int NR, bool REC = false>
__global__ void __launch_bounds__(128, fwd_min_blocks(P, D, R, NR, REC)) fwd_kernel(SolverArgs A) {
    constexpr int S = P + 4;
    constexpr int DS = DyStride<D>::value;
    constexpr int RS = rec_floats(P);
    extern __shared__ float4 smem_f4[];
    float* smem = reinterpret_cast<float*>(smem_f4);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float* dyw = smem + warp * FwdSmem<P, D, R, REC>::per_warp;  // 64-column ring of dy
    float* sin_ = dyw + 64 * DS;                        // seam-in block
    float* sout = sin_ + kG * S;                        // seam-out block
    // record-storing forward: a step's 32*R records are staged in shared
    // memory (two blocks, step t uses t & 1) and stored by one bulk copy,
    // which the seam flushes' fences do not wait for
    float* stg = sout + kG * S;
    constexpr int kStage = 32 * R * RS;  // floats per staged block
    const int n_items = A.sched.hdr[2];
    unsigned long long tiles_done = 0, lane_tiles = 0;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.item_counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_items) break;
        if (ld_volatile_s32(A.status) != 0) break;
        const ItemRef ir = decode_item(A.sched, A.pairs, item);
        const int lo_p = ir.pair;
        const PairDesc pd = A.pairs[lo_p];
        const int s = ir.k;
        const int L1 = pd.L1, L2 = pd.L2;
        const bool has_in = ir.prev >= 0;
        const bool has_out = ir.next >= 0;
        const int slot_in = has_in ? ir.prev % A.nslot : 0;
        const int slot_out = item % A.nslot;
        const int i0 = s * 32 * R;
        const bool train = A.store != nullptr;
        float* st_pair = train ? A.store + A.store_off[lo_p] : nullptr;
        // training: the store keeps the seam after every 32-row strip (the
        // adjoint's checkpoints).  This item covers 32-row strips s*R ..
        // s*R + R - 1; lane l = 32m/R - 1 ends strip s*R + m - 1, so lanes
        // 32/R - 1, 2*32/R - 1, ... write the seams inside the item directly,
        // lane 31 the item's last one through the seam-out block.
        const int n32 = pd.n_strips;  // table strips (32 rows) in training mode
        const int mid_m = (lane + 1) * R / 32;  // m for a mid-item seam lane, else 0
        const bool mid_writer = train && R > 1 && lane != 31 && ((lane + 1) * R) % 32 == 0 &&
                                s * R + mid_m < n32;
        float* mid_dst = mid_writer ? st_pair + (size_t)(s * R + mid_m - 1) * L2 * S : nullptr;
        // stored tile records: this item's region, (L2 + 32) blocks of 32*R
        // records; block t holds the records of step t in the order of the
        // item's rows (row lane*R + k), block L2 + 31 the rows' final states
        float* rec_item = nullptr;
        if constexpr (REC) rec_item = A.rec + A.rec_off[lo_p] + (int64_t)s * (L2 + 32) * 32 * R * RS;
        bool ok = true;

        // row increments of this lane (zero past the end of the path)
        float dx[R][D];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int row = i0 + lane * R + k;
#pragma unroll
            for (int e = 0; e < D; ++e)
                dx[k][e] = (row < L1 && e < A.d) ? inc_ref(pd.xr, row, A.d, e, A.inc_mode, pd.sx) : 0.0f;
        }
        float a[R][P + 1], a1lo[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            a1lo[k] = 0.0f;
#pragma unroll
            for (int p = 0; p <= P; ++p) a[k][p] = 0.0f;
        }
        int E = 0;
        // outgoing right edge of the previous step (what lane+1 receives)
        float ohi = 1.0f, olo = 0.0f, ob1lo = 0.0f, ob[P + 1];
#pragma unroll
        for (int q = 0; q <= P; ++q) ob[q] = 0.0f;
        int oE = 0;

        // progress words: per slot (inference) or per item (training, where
        // the seams are not reused and a slot's word could be overtaken)
        const int pw_in = train ? ir.prev : slot_in;
        const int pw_out = train ? item : slot_out;
#ifdef SIGK_DEBUG
        // the regions this item touches lie inside their buffers
        ok = dbg_in(A.status, 1, lo_p, A.n_pairs - 1) && dbg_in(A.status, 2, slot_out, A.nslot - 1) &&
             dbg_in(A.status, 3, slot_in, A.nslot - 1) && dbg_in(A.status, 4, pw_out, A.nwords - 1) &&
             dbg_in(A.status, 5, has_in ? pw_in : 0, A.nwords - 1) &&
             dbg_in(A.status, 6, pd.out0, A.out_cap - 1) && dbg_in(A.status, 7, pd.out1 < 0 ? 0 : pd.out1, A.out_cap - 1);
        if (ok && train) {
            // seams of strips s*R - 1 (read) .. min(s*R + R - 1, n32 - 2) (written)
            const int last = min(s * R + R - 1, n32 - 2);
            const int64_t base = st_pair - A.store;
            if (has_out || R > 1) ok = dbg_in(A.status, 8, base + (int64_t)(last + 1) * L2 * S, A.store_cap);
            if (ok && has_in) ok = dbg_in(A.status, 9, base + (int64_t)(s * R) * L2 * S, A.store_cap);
        }
        if constexpr (REC)
            if (ok) ok = dbg_in(A.status, 10, (rec_item - A.rec) + (int64_t)(L2 + 32) * 32 * R * RS, A.rec_cap);
        ok = __all_sync(kFull, ok);
#endif
        // the slot we write must have been read by its previous consumer
        if (ok && has_out && !train) ok = wait_slot_free(A.sched, A.pairs, item, A.nslot, A.done, A.status);
        const int T = L2 + 31;
        for (int t = 0; t < T && ok; ++t) {
            if ((t & 31) == 0 && t < L2) {
                // next 32 columns of dy into the ring
                const int nb = min(32, L2 - t);
                fill_dy<D, DS, false>(dyw, pd.yr, t, nb, L2, A.d, A.inc_mode, pd.sy, lane);
                if (has_in) {
                    const unsigned long long need =
                        ((unsigned long long)ir.prev << 32) | (unsigned)(t + nb);
                    bool okl = true;
                    if (lane == 0) okl = wait_ge_u64(&A.prod[pw_in], need, A.status);
                    ok = __shfl_sync(kFull, okl, 0);
                    if (ok) {
                        const float* src =
                            train ? st_pair + ((size_t)(s * R - 1) * L2 + t) * S
                                  : A.seam + ((size_t)slot_in * A.wcols + (t % A.wcols)) * S;
                        warp_copy_cg<S>(sin_, src, nb * S, lane);
                        __syncwarp();
                        if (lane == 0 && !train)
                            st_release_u64(&A.cons[slot_in],
                                           ((unsigned long long)item << 32) | (unsigned)(t + nb));
                    }
                }
                __syncwarp();
                if (!ok) break;
            }
            // left edge: from lane-1 (previous step), or the seam / boundary for lane 0
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
            if constexpr (REC) {
                // the bulk store of step t - 2 has read this step's staging block
                if (lane == 0) bulk_wait_read<1>();
                __syncwarp();
            }
            const int j = t - lane;
            if (j >= 0 && j < L2) {
                // records of the rows' incoming left edges (the adjoint rebuilds
                // each tile's inputs from them): row k = 0 as received, before
                // the alignment; row k > 0 the previous row's outgoing edge.
                // The first groups are stored before the tile, the group with
                // the exponent word after the step's renormalisation.
                float* rslot[R];
                float rbP[R];
                int Frec[R];
                const int Eb = E;
                auto rec_head = [&](int k, int Fv) {
                    rslot[k] = stg + (t & 1) * kStage + (lane * R + k) * RS;
                    rec_put_head<P>(rslot[k], hi, b1lo, b);
                    rbP[k] = b[P];
                    Frec[k] = Fv;
                };
                if constexpr (REC) rec_head(0, F);
                // align exponents of the incoming edge and the lane's states
                if (F != E) {
                    if (F > E) {
                        const float sc = exp2_nonpos(E - F);
#pragma unroll
                        for (int k = 0; k < R; ++k) {
                            a1lo[k] *= sc;
#pragma unroll
                            for (int p = 1; p <= P; ++p) a[k][p] *= sc;
                        }
                        E = F;
                    } else {
                        const float sc = exp2_nonpos(F - E);
                        hi *= sc; lo *= sc; b1lo *= sc;
#pragma unroll
                        for (int q = 1; q <= P; ++q) b[q] *= sc;
                    }
                }
                float dy[D];
                const float4* rowp = reinterpret_cast<const float4*>(dyw + (j & 63) * DS);
#pragma unroll
                for (int e4 = 0; e4 < D / 4; ++e4) {
                    const float4 v = rowp[e4];
                    dy[4 * e4 + 0] = v.x; dy[4 * e4 + 1] = v.y;
                    dy[4 * e4 + 2] = v.z; dy[4 * e4 + 3] = v.w;
                }
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    if constexpr (REC)
                        if (k > 0) rec_head(k, E);
                    float c = 0.0f;
#pragma unroll
                    for (int e = 0; e < D; ++e) c = fmaf(dx[k][e], dy[e], c);
                    tile_update<P, NR>(c, a[k], a1lo[k], hi, lo, b, b1lo, NR);
                }
                // renormalise when the corner value grows past 2^64
                int bump = 0;
                if (fabsf(hi) > 1.8446744e19f) {
                    bump = 1;
                    const float sc = 5.421011e-20f;  // 2^-64
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        a1lo[k] *= sc;
#pragma unroll
                        for (int p = 1; p <= P; ++p) a[k][p] *= sc;
                    }
                    hi *= sc; lo *= sc; b1lo *= sc;
#pragma unroll
                    for (int q = 1; q <= P; ++q) b[q] *= sc;
                    E += 64;
                }
                if constexpr (REC) {
#pragma unroll
                    for (int k = 0; k < R; ++k)  // only the last row's outgoing edge leaves the lane
                        rec_put_tail<P>(rslot[k], rbP[k], pack_exp(Frec[k], Eb, bump, k == R - 1 ? bump : 0));
                }
                ohi = hi; olo = lo; ob1lo = b1lo; oE = E;
#pragma unroll
                for (int q = 1; q <= P; ++q) ob[q] = b[q];
                tiles_done += (unsigned long long)max(0, min(R, L1 - (i0 + lane * R)));
                lane_tiles += R;
                if (mid_writer) {
                    float* e_ = mid_dst + (size_t)j * S;
                    e_[0] = hi; e_[1] = lo; e_[2] = b1lo;
#pragma unroll
                    for (int q = 1; q <= P; ++q) e_[2 + q] = b[q];
                    e_[P + 3] = __int_as_float(E);
                }
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
                        if (A.pair_exp) A.pair_exp[lo_p] = E;
                    }
                }
            }
            if constexpr (REC) {
                // the step's records, staged by every lane, leave in one bulk store
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    bulk_store(rec_item + (int64_t)t * kStage, stg + (t & 1) * kStage,
                               kStage * (uint32_t)sizeof(float));
                    bulk_commit();
                }
            }
            // flush a completed 32-column block of the outgoing seam
            const int jj = t - 31;
            if (has_out && jj >= 0 && jj < L2 && (((jj & 31) == 31) || jj == L2 - 1)) {
                __syncwarp();
                const int start = jj & ~31;
                const int nb = jj - start + 1;
                if (!train && start + nb > A.wcols) {
                    const unsigned long long need = ((unsigned long long)ir.next << 32) |
                                                    (unsigned)(start + nb - A.wcols);
                    bool okl = true;
                    if (lane == 0) okl = wait_ge_u64(&A.cons[slot_out], need, A.status);
                    ok = __shfl_sync(kFull, okl, 0);
                }
                if (ok) {
                    float* dst = train ? st_pair + ((size_t)(s * R + R - 1) * L2 + start) * S
                                       : A.seam + ((size_t)slot_out * A.wcols + (start % A.wcols)) * S;
                    for (int idx = lane; idx < nb * S; idx += 32) __stcg(dst + idx, sout[idx]);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0 && !(A.withhold_first_seam && item == 0))
                        st_release_u64(&A.prod[pw_out],
                                       ((unsigned long long)item << 32) | (unsigned)(start + nb));
                }
                __syncwarp();
            }
        }
        // stored records: each row's bottom-edge state after the last column
        // (where the adjoint's reverse sweep starts), block L2 + 31
        if constexpr (REC) {
            // the staging blocks are free for the next item
            if (lane == 0) bulk_wait_read<0>();
            __syncwarp();
            if (ok) {
#pragma unroll
                for (int k = 0; k < R; ++k)
                    rec_put_state<P>(rec_item + ((int64_t)(L2 + 31) * 32 * R + lane * R + k) * RS, a1lo[k], a[k]);
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            st_release_s64(&A.done[item % A.nslot], (long long)item);
        }
        if (!ok) break;
    }
    if constexpr (REC) {
        if (lane == 0) bulk_wait_all();  // the record stores are complete
    }
    // counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tiles_done += __shfl_down_sync(kFull, tiles_done, o);
        lane_tiles += __shfl_down_sync(kFull, lane_tiles, o);
    }
    if (lane == 0) {
        atomicAdd(&A.counters[0], tiles_done);
        atomicAdd(&A.counters[1], lane_tiles);
    }
}

}  // namespace sigk
