// sigk_bwd.cuh -- reverse-mode (adjoint) sweep of the wavefront solver.
//
// Runs after a training forward that stored the right-edge seam after every
// 32-row strip (the checkpointed wavefront boundaries).  One work item =
// (pair, strip of 32 rows, one row per lane), strips of a pair in DECREASING
// order (the schedule's k-th item of a pair is strip n_strips - 1 - k).
//
// Every tile's record -- the row's incoming left edge and the exponent
// decisions, P + 2 floats -- comes either from the training forward, which
// writes all of them (with each row's final bottom-edge state) when they fit
// the device memory budget, or from pass A: a replay of the strip's forward
// from its stored input seam into a per-warp scratch area, ending with each
// lane's bottom-edge state after the last column in registers.
//
// Pass B sweeps the columns in reverse with the mirrored skew (lane 31 first).
// At each tile it rebuilds the tile's bottom-edge input by inverting the
// bottom-to-top update (tile_inverse_a) from the known top edge and the stored
// left edge, then applies the adjoint of the tile map (tile_adjoint): the
// adjoint of the right edge arrives from lane+1 (or, for lane 31, from the
// next strip's adjoint seam or the seed at the last tile), the adjoint of the
// top edge is the lane's own state from the column above.  dk/dc_ij is
// chained at once to the increments: dk/ddx_i += g dy_j (registers),
// dk/ddy_j += g dx_i (a shared-memory column accumulator flushed with
// atomics), g = dk/dc_ij times the pair's upstream weight.
#pragma once
#include "sigk_device.cuh"
#include "sigk_fwd.cuh"

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

template <int P, int D>
struct BwdSmem {
    static constexpr int S = P + 4;   // forward seam entry
    static constexpr int RS = rec_floats(P);  // record per lane
    static constexpr int RB = 32 * (S > RS ? S : RS);  // one record block / seam-in block
    static constexpr int SA = adj_seam_floats(P);  // adjoint seam entry: corner, b1..bP (padded)
    static constexpr int DS = DyStride<D>::value;
    // dy ring, two record blocks (the first doubles as pass A's seam-in
    // block), adjoint seam in/out blocks, column gradients (every part a
    // multiple of 4 floats: 16-byte aligned)
    static constexpr int per_warp = 64 * DS + 2 * RB + 2 * 32 * SA + 64 * D;
};

// gradient v of virtual row `vrow` (refinement s) -> its segment vrow / s
// (scaled 1/s), then points (+ at segment+1, - at segment) or increments
template <int D>
__device__ __forceinline__ void add_inc_grad(float* g, int64_t vrow, int d, int inc_mode, int s,
                                             const float (&v)[D]) {
    if (!g) return;
    const int64_t row = vrow / s;
    const float sc = 1.0f / (float)s;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        if (e < d && v[e] != 0.0f) {
            const float w = v[e] * sc;
            if (inc_mode) {
                atomicAdd(g + row * d + e, w);
            } else {
                atomicAdd(g + (row + 1) * d + e, w);
                atomicAdd(g + row * d + e, -w);
            }
        }
    }
}

constexpr int bwd_min_blocks(int P, int D) { return (P <= 8 && D <= 8) ? 4 : 3; }

template <int P, int D, int NR>
__global__ void __launch_bounds__(128, bwd_min_blocks(P, D)) bwd_kernel(BwdArgs A) {
    constexpr int S = P + 4;
    constexpr int SA = adj_seam_floats(P);
    constexpr int DS = DyStride<D>::value;
    extern __shared__ float4 smem_f4[];
    float* smem = reinterpret_cast<float*>(smem_f4);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    float* dyw = smem + warp * BwdSmem<P, D>::per_warp;  // 64-column ring of dy
    constexpr int RS = BwdSmem<P, D>::RS;
    float* sin_ = dyw + 64 * DS;                        // forward seam-in block
    float* rbuf1 = sin_ + BwdSmem<P, D>::RB;            // second record block
    float* ain = rbuf1 + BwdSmem<P, D>::RB;             // adjoint seam-in block
    float* aout = ain + 32 * SA;                        // adjoint seam-out block
    float* colacc = aout + 32 * SA;  // column gradient, float4 [D/4][64]: (e, col) at ((e/4)*64+col)*4 + e%4
    float* rec = A.rec + (size_t)gwarp * A.rec_stride;
    const int n_items = A.sched.hdr[2];
    unsigned long long tiles = 0, replayed = 0;
    // pass B reads every lane's record of one step per step, prefetched two
    // steps ahead by each lane with cp.async into its slot of sin_ / rbuf1
    // (step tp uses buffer tp & 1)
    // records: rec_put_head / rec_put_tail / rec_get (pairs of floats; the
    // last pair, with the exponent word, is stored after the tile)

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
        const int row = s * 32 + lane;
        const bool has_row = row < L1;
        const float* st_base = A.store + A.store_off[lo_p];
        bool ok = true;
#ifdef SIGK_DEBUG
        {
            // the regions this item touches lie inside their buffers
            const int RRd = A.rec_off != nullptr ? A.rec_rows : 1;
            bool in = dbg_in(A.status, 21, lo_p, A.n_pairs - 1) &&
                      dbg_in(A.status, 22, item % A.nslot, A.nslot - 1) &&
                      dbg_in(A.status, 23, ir.prev >= 0 ? ir.prev % A.nslot : 0, A.nslot - 1) &&
                      dbg_in(A.status, 24, s > 0 ? A.store_off[lo_p] + (int64_t)s * L2 * S : 0, A.store_cap);
            if (in && A.rec_off != nullptr)
                in = dbg_in(A.status, 25, A.rec_off[lo_p] + (int64_t)(s / RRd + 1) * (L2 + 32) * 32 * RRd * rec_floats(P),
                            A.rec_cap);
            if (in && A.rec_off == nullptr)
                in = dbg_in(A.status, 26, (int64_t)(L2 + 31) * 32 * rec_floats(P), A.rec_stride) &&
                     dbg_in(A.status, 27, (int64_t)(gwarp + 1) * A.rec_stride, A.rec_total);
            if (!__all_sync(kFull, in)) break;
        }
#endif

        float dx[D];
#pragma unroll
        for (int e = 0; e < D; ++e)
            dx[e] = (has_row && e < A.d) ? inc_ref(pd.xr, row, A.d, e, A.inc_mode, pd.sx) : 0.0f;

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
        // records stored by the training forward (no replay) in regions of
        // items of RR strips: this lane's row is row rw of item s / RR, its
        // record for column j in block j + rw / RR; the final bottom-edge
        // state is block L2 + 31.  Replayed records: the one-row layout of the
        // warp's scratch.
        const bool stored = A.rec_off != nullptr;
        const int RR = stored ? A.rec_rows : 1;
        const int rw = (s % RR) * 32 + lane;
        const float* rbase = stored ? A.rec_store + A.rec_off[lo_p] + (int64_t)(s / RR) * (L2 + 32) * 32 * RR * RS
                                    : rec;
        if (stored) rec_get_state<P>(rbase + ((int64_t)T * 32 * RR + rw) * RS, a1lo, a);
        for (int t = 0; t < T && !stored; ++t) {
            if ((t & 31) == 0 && t < L2) {
                const int nb = min(32, L2 - t);
                fill_dy<D, DS, false>(dyw, pd.yr, t, nb, L2, A.d, A.inc_mode, pd.sy, lane);
                if (s > 0) {
                    const float* src = st_base + ((size_t)(s - 1) * L2 + t) * S;
                    warp_copy_cg<S>(sin_, src, nb * S, lane);
                }
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
                // record of the incoming left edge, before alignment
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
                const float4* rowp = reinterpret_cast<const float4*>(dyw + (j & 63) * DS);
                float c = 0.0f;
#pragma unroll
                for (int e4 = 0; e4 < D / 4; ++e4) {
                    const float4 v = rowp[e4];
                    c = fmaf(dx[4 * e4 + 0], v.x, c);
                    c = fmaf(dx[4 * e4 + 1], v.y, c);
                    c = fmaf(dx[4 * e4 + 2], v.z, c);
                    c = fmaf(dx[4 * e4 + 3], v.w, c);
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
        float gx[D];
#pragma unroll
        for (int e = 0; e < D; ++e) gx[e] = 0.0f;
        for (int idx = lane; idx < 64 * D; idx += 32) colacc[idx] = 0.0f;
        float oB0 = 0.0f, oBb[P + 1];
#pragma unroll
        for (int q = 0; q <= P; ++q) oBb[q] = 0.0f;
        const int lp = 31 - lane;
        // pass A's records and its use of sin_ come before pass B's copies
        __threadfence_block();
        __syncwarp();
        auto rbuf = [&](int tpp) { return (tpp & 1) ? rbuf1 : sin_; };
        // the record of reverse step tpp, if this lane has a tile there (column
        // j = L2 + 30 - tpp - lane), into its slot of the step's buffer; one
        // commit group per step
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
        if (ok) {
            rec_fetch(0);
            rec_fetch(1);
        }
        for (int tp = 0; tp < T && ok; ++tp) {
            if ((tp & 31) == 0 && tp < L2) {
                const int nb = min(32, L2 - tp);
                // dy for reverse columns jr in [tp, tp+nb): j = L2-1-jr
                fill_dy<D, DS, true>(dyw, pd.yr, tp, nb, L2, A.d, A.inc_mode, pd.sy, lane);
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
            // this step's record (groups in flight: this step's and the next)
            float rhi, rb[P + 1];
            int rexp;
            {
                cp_async_wait<1>();
                rec_get<P>(rbuf(tp) + lane * RS, rhi, rb, rexp);
                rec_fetch(tp + 2);  // into the buffer just read (an empty group past the end)
            }
            // adjoint of the right edge: from lane+1, or seam / seed for lane 31
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
                for (int q = 1; q <= P; ++q) b[q] = rb[q];  // b[1]: first-order term as one float
                // exponent handling of this tile (none in the common case)
                const bool plain = exp_plain(rexp);
                int F = 0, Eb = 0, Em = 0;
                if (!plain) {
                    int abump, bbump;
                    unpack_exp(rexp, F, Eb, abump, bbump);
                    Em = F > Eb ? F : Eb;
                    // undo the renormalisations after this tile
                    if (abump) {  // of the bottom-edge state
#pragma unroll
                        for (int p = 1; p <= P; ++p) { a[p] *= 1.8446744e19f; Ab[p] *= 5.421011e-20f; }
                    }
                    if (bbump) {  // of the outgoing right edge
                        B0 *= 5.421011e-20f;
#pragma unroll
                        for (int q = 1; q <= P; ++q) Bb[q] *= 5.421011e-20f;
                    }
                    if (F < Em) {  // the incoming edge was scaled to the lane exponent
                        const float sc = exp2_nonpos(F - Em);
                        hi *= sc;
#pragma unroll
                        for (int q = 1; q <= P; ++q) b[q] *= sc;
                    }
                }
                const float4* rowp = reinterpret_cast<const float4*>(dyw + (jr & 63) * DS);
                float dy[D];
#pragma unroll
                for (int e4 = 0; e4 < D / 4; ++e4) {
                    const float4 v = rowp[e4];
                    dy[4 * e4 + 0] = v.x; dy[4 * e4 + 1] = v.y;
                    dy[4 * e4 + 2] = v.z; dy[4 * e4 + 3] = v.w;
                }
                float c = 0.0f;
#pragma unroll
                for (int e = 0; e < D; ++e) c = fmaf(dx[e], dy[e], c);
                float ain_[P + 1], ha[P + 1];
                tile_inverse_a<P>(c, a, hi, b, NR, ain_, ha);
                const float cbar = tile_adjoint<P>(c, ain_, hi, b, ha, Ab, B0, Bb, NR);
                // undo the alignment of this step
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
                const float g = cbar * wsc;
                // float4 [D/4][64] layout: the 32 lanes (consecutive columns)
                // read and write 512 contiguous bytes, free of bank conflicts
                float4* ca = reinterpret_cast<float4*>(colacc) + (jr & 63);
#pragma unroll
                for (int e4 = 0; e4 < D / 4; ++e4) {
                    float4 v = ca[e4 * 64];
                    v.x = fmaf(g, dx[4 * e4 + 0], v.x);
                    v.y = fmaf(g, dx[4 * e4 + 1], v.y);
                    v.z = fmaf(g, dx[4 * e4 + 2], v.z);
                    v.w = fmaf(g, dx[4 * e4 + 3], v.w);
                    ca[e4 * 64] = v;
                }
#pragma unroll
                for (int e = 0; e < D; ++e) gx[e] = fmaf(g, dy[e], gx[e]);
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
            // lane 0 closed a block of 32 reverse columns: flush gradients and seam
            const int jj = tp - 31;
            if (jj >= 0 && jj < L2 && (((jj & 31) == 31) || jj == L2 - 1)) {
                const int start = jj & ~31;
                const int nb = jj - start + 1;
                if (pd.gyr) {
                    // dimension fastest: a warp's atomics hit whole rows of dL/dy
                    for (int idx = lane; idx < nb * D; idx += 32) {
                        const int col = idx / D, e = idx % D;
                        float* cell = colacc + ((e >> 2) * 64 + ((start + col) & 63)) * 4 + (e & 3);
                        const float v = *cell;
                        *cell = 0.0f;
                        if (e < A.d && v != 0.0f) {
                            const int64_t jcol = (L2 - 1 - (start + col)) / pd.sy;
                            const float w = v * (1.0f / (float)pd.sy);
                            if (A.inc_mode) {
                                atomicAdd(pd.gyr + jcol * A.d + e, w);
                            } else {
                                atomicAdd(pd.gyr + (jcol + 1) * A.d + e, w);
                                atomicAdd(pd.gyr + jcol * A.d + e, -w);
                            }
                        }
                    }
                } else {
                    for (int idx = lane; idx < nb * D; idx += 32)
                        colacc[(((idx / nb) >> 2) * 64 + ((start + idx % nb) & 63)) * 4 + ((idx / nb) & 3)] = 0.0f;
                }
                if (has_aout) {
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
                }
                __syncwarp();
            }
        }
        // record copies still in flight (the last steps', or after an early
        // exit) complete before the buffers are used again
        cp_async_wait<0>();
        __syncwarp();
        if (has_row) add_inc_grad<D>(pd.gxr, row, A.d, A.inc_mode, pd.sx, gx);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            st_release_s64(&A.done[item % A.nslot], (long long)item);
        }
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
