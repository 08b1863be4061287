// sigk_fwd_cm.cuh -- forward solver for paths of large dimension d (d > 16),
// and the FP64 solver for any d.
//
// The increment Gram c_ij = <dx_i, dy_j> is a dense contraction over d.  For a
// work item (pair, 32-row strip) the warp first computes the strip's
// coefficients for every column (phase 1: a register-blocked FMA micro-GEMM,
// lane = column, 32 row accumulators per lane, the contraction dimension
// staged through shared memory in chunks of 32) into a per-warp scratch
// strip, column-major [L2][32].  Only one strip per warp exists at a time: the
// L1 x L2 coefficient matrix is never materialised.  Phase 2 is the wavefront
// sweep of fwd_kernel with one row per lane, reading c from a 64-column
// shared-memory ring filled 32 columns at a time from the strip.
//
// T = float: the FP32 solver (float-float corner, compensated first-order
// terms, two-level sums in phase 1).  T = double: every step in FP64 --
// point differences, the contraction, the refinement scaling and the tile map.
#pragma once
#include "sigk_device.cuh"
#include "sigk_f64.cuh"
#include "sigk_fwd.cuh"

namespace sigk {

constexpr int kCmKC = 32;  // contraction chunk

template <int P, typename T>
struct CmSmem {
    static constexpr int S = P + 4;
    // phase 1 staging (dx chunk [KC][36], dy chunk [32][KC+1]) and the phase 2
    // coefficient ring [64][32] share one region; sizes in elements of T
    static constexpr int stage = kCmKC * 36 + 32 * (kCmKC + 1);
    static constexpr int ring = 64 * 32;
    static constexpr int uni = stage > ring ? stage : ring;
    static constexpr int per_warp = uni + 2 * kG * S;
    static constexpr int bytes = 4 * per_warp * (int)sizeof(T);  // 4 warps per CTA
};

// Segment increment in FP64: exact for FP32 points (their difference has at
// most 25 significant bits).
__device__ __forceinline__ double inc_at_d(const float* z, int64_t row, int d, int e, int inc_mode) {
    if (inc_mode) return (double)z[row * d + e];
    return (double)z[(row + 1) * d + e] - (double)z[row * d + e];
}

// stage_increments for s = 2^LS and v0 a multiple of 32: virtual row v0 + r
// lies on segment (v0 >> LS) + (r >> LS), so all loads are independent and
// issued back to back (ceil(32/s) + 1 points, or ceil(32/s) increments).
template <int LS>
__device__ __forceinline__ void stage_pow2(float* dst, int stride, const float* z, int v0, int Lv,
                                           int d, int e, int inc_mode) {
    constexpr int S = 1 << LS;
    constexpr int NQ = (32 + S - 1) / S;   // segments under the 32 rows
    constexpr int G = NQ < 16 ? NQ : 16;   // segments per batch of loads
    const int q0 = v0 >> LS;
    const int Lseg = Lv >> LS;
#pragma unroll
    for (int g0 = 0; g0 < NQ; g0 += G) {
        float inc[G];
        if (inc_mode) {
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int q = q0 + g0 + k;
                inc[k] = q < Lseg ? z[(int64_t)q * d + e] : 0.0f;
            }
        } else {
            float pt[G + 1];
#pragma unroll
            for (int k = 0; k <= G; ++k) {
                const int q = q0 + g0 + k;
                pt[k] = q <= Lseg ? z[(int64_t)q * d + e] : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < G; ++k) inc[k] = q0 + g0 + k < Lseg ? pt[k + 1] - pt[k] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < G; ++k) {
#pragma unroll
            for (int u = 0; u < S && (g0 + k) * S + u < 32; ++u)
                dst[((g0 + k) * S + u) * stride] = S == 1 ? inc[k] : inc[k] * (1.0f / S);
        }
    }
}

// Increments of the 32 consecutive virtual rows v0 .. v0+31 of a path (each
// segment refined into s pieces) at dimension e, one value per row into
// dst[r * stride]; rows at or past Lv (virtual rows of the path) give 0.
// Points: consecutive virtual rows share their end points, so each point is
// loaded once (one new load per segment instead of two per row).  Values are
// those of inc_ref: (z[q+1] - z[q]) * (1/s), or z[q] * (1/s).
__device__ __forceinline__ void stage_increments(float* dst, int stride, const float* z, int v0,
                                                 int Lv, int d, int e, int inc_mode, int s) {
    if (e < d && (v0 & 31) == 0) {
        switch (s) {
            case 1: stage_pow2<0>(dst, stride, z, v0, Lv, d, e, inc_mode); return;
            case 2: stage_pow2<1>(dst, stride, z, v0, Lv, d, e, inc_mode); return;
            case 4: stage_pow2<2>(dst, stride, z, v0, Lv, d, e, inc_mode); return;
            case 8: stage_pow2<3>(dst, stride, z, v0, Lv, d, e, inc_mode); return;
            case 16: stage_pow2<4>(dst, stride, z, v0, Lv, d, e, inc_mode); return;
            case 32: stage_pow2<5>(dst, stride, z, v0, Lv, d, e, inc_mode); return;
            case 64: stage_pow2<6>(dst, stride, z, v0, Lv, d, e, inc_mode); return;
            default: break;
        }
    }
    if (e >= d) {
#pragma unroll 8
        for (int r = 0; r < 32; ++r) dst[r * stride] = 0.0f;
        return;
    }
    const float inv = 1.0f / (float)s;
    if (inc_mode) {
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const int v = v0 + r;
            dst[r * stride] = v < Lv ? (s == 1 ? z[(int64_t)(v / s) * d + e]
                                               : z[(int64_t)(v / s) * d + e] * inv)
                                     : 0.0f;
        }
        return;
    }
    const int Lseg = Lv / s;  // segments of the unrefined path
    int qc = v0 / s;
    float p0 = 0.0f, p1 = 0.0f;
    if (qc < Lseg) {
        p0 = z[(int64_t)qc * d + e];
        p1 = z[(int64_t)(qc + 1) * d + e];
    }
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const int q = (v0 + r) / s;
        if (q != qc) {  // the same for every lane: no divergence
            qc = q;
            p0 = p1;
            p1 = q < Lseg ? z[(int64_t)(q + 1) * d + e] : p0;
        }
        const float inc = p1 - p0;
        dst[r * stride] = q < Lseg ? (s == 1 ? inc : inc * inv) : 0.0f;
    }
}

// The wavefront sweep of one 32-row strip with one row per lane, c read
// from the strip scratch `cst` ([L2][32], column-major) through the shared
// ring `cring`.  In the seam protocol the strip is `item`, fed by `prev` and
// feeding `next` (-1: none); the caller has already made sure that slot
// item % nslot is free.  Returns false when a bounded wait failed.
template <int P, typename T, int NR>
__device__ __forceinline__ bool sweep_strip(const SolverArgs& A, const PairDesc& pd, int lo_p,
                                            int s, int item, int prev, int next, const T* cst,
                                            T* cring, T* sin_, T* sout, T* seam,
                                            unsigned long long& tiles_done,
                                            unsigned long long& lane_tiles) {
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int S = P + 4;
    const int lane = threadIdx.x & 31;
    const int L1 = pd.L1, L2 = pd.L2;
    const bool has_in = prev >= 0;
    const bool has_out = next >= 0;
    const int slot_in = has_in ? prev % A.nslot : 0;
    const int slot_out = item % A.nslot;
    const int i0 = s * 32;
    bool ok = true;
    T a[P + 1];
    float a1lo = 0.0f;  // FP32 only: compensation of the first-order terms
#pragma unroll
    for (int p = 0; p <= P; ++p) a[p] = T(0);
    int E = 0;
    T ohi = T(1), ob[P + 1];
    float olo = 0.0f, ob1lo = 0.0f;
#pragma unroll
    for (int q = 0; q <= P; ++q) ob[q] = T(0);
    int oE = 0;
    // training forward (FP32; A.store set): every strip's right-edge seam goes
    // to the per-pair store (the adjoint's checkpoints) instead of the ring,
    // with one progress word per item
    const bool train = F32 && A.store != nullptr;
    float* st_pair = train ? A.store + A.store_off[lo_p] : nullptr;
    const int pw_in = train ? prev : slot_in;
    const int pw_out = train ? item : slot_out;
    constexpr int NV = 32 * (int)sizeof(T) / 16;  // 16-byte vectors per strip column
    const int Tn = L2 + 31;
    const bool has_row = i0 + lane < L1;
    for (int t = 0; t < Tn && ok; ++t) {
        if ((t & 31) == 0 && t < L2) {
            const int nb = min(32, L2 - t);
            // coefficients of columns [t, t+nb) into the ring (contiguous)
            const int4* src = reinterpret_cast<const int4*>(cst + (size_t)t * 32);
            for (int idx = lane; idx < nb * NV; idx += 32) {
                const int col = idx / NV, q = idx % NV;
                reinterpret_cast<int4*>(cring + ((t + col) & 63) * 32)[q] = src[idx];
            }
            if (has_in) {
                const unsigned long long need =
                    ((unsigned long long)prev << 32) | (unsigned)(t + nb);
                bool okl = true;
                if (lane == 0) okl = wait_ge_u64(&A.prod[pw_in], need, A.status);
                ok = __shfl_sync(kFull, okl, 0);
                if (ok) {
                    const T* src2 = train ? reinterpret_cast<const T*>(st_pair + ((size_t)(s - 1) * L2 + t) * S)
                                          : seam + ((size_t)slot_in * A.wcols + (t % A.wcols)) * S;
                    for (int idx = lane; idx < nb * S; idx += 32) sin_[idx] = __ldcg(src2 + idx);
                    __syncwarp();
                    if (lane == 0 && !train)
                        st_release_u64(&A.cons[slot_in],
                                       ((unsigned long long)item << 32) | (unsigned)(t + nb));
                }
            }
            __syncwarp();
            if (!ok) break;
        }
        T hi = __shfl_up_sync(kFull, ohi, 1);
        float lo = 0.0f, b1lo = 0.0f;
        if constexpr (F32) {
            lo = __shfl_up_sync(kFull, olo, 1);
            b1lo = __shfl_up_sync(kFull, ob1lo, 1);
        }
        T b[P + 1];
        b[0] = T(0);
#pragma unroll
        for (int q = 1; q <= P; ++q) b[q] = __shfl_up_sync(kFull, ob[q], 1);
        int F = __shfl_up_sync(kFull, oE, 1);
        if (lane == 0) {
            if (has_in && t < L2) {
                const T* e_ = sin_ + (t & 31) * S;
                if constexpr (F32) {
                    float v[S];
                    seam_entry_load<S>(e_, v);
                    seam_unpack<P>(v, hi, lo, b1lo, b, F);
                } else {
                    hi = e_[0];
#pragma unroll
                    for (int q = 1; q <= P; ++q) b[q] = e_[2 + q];
                    F = (int)e_[P + 3];
                }
            } else {
                hi = T(1); lo = 0.0f; b1lo = 0.0f; F = 0;
#pragma unroll
                for (int q = 1; q <= P; ++q) b[q] = T(0);
            }
        }
        const int j = t - lane;
        if (j >= 0 && j < L2) {
            if (F != E) {
                if (F > E) {
                    const T sc = F32 ? (T)exp2_nonpos(E - F) : (T)exp2_nonpos_d(E - F);
                    a1lo *= (float)sc;
#pragma unroll
                    for (int p = 1; p <= P; ++p) a[p] *= sc;
                    E = F;
                } else {
                    const T sc = F32 ? (T)exp2_nonpos(F - E) : (T)exp2_nonpos_d(F - E);
                    hi *= sc; lo *= (float)sc; b1lo *= (float)sc;
#pragma unroll
                    for (int q = 1; q <= P; ++q) b[q] *= sc;
                }
            }
            const T c = cring[(j & 63) * 32 + lane];
            if constexpr (F32) {
                tile_update<P, NR>(c, a, a1lo, hi, lo, b, b1lo, NR);
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
            } else {
                tile_update_f64<P>(c, a, hi, b, NR);
                if (fabs(hi) > 0x1p512) {
                    const double sc = 0x1p-512;
#pragma unroll
                    for (int p = 1; p <= P; ++p) a[p] *= sc;
                    hi *= sc;
#pragma unroll
                    for (int q = 1; q <= P; ++q) b[q] *= sc;
                    E += 512;
                }
            }
            ohi = hi; olo = lo; ob1lo = b1lo; oE = E;
#pragma unroll
            for (int q = 1; q <= P; ++q) ob[q] = b[q];
            tiles_done += has_row ? 1ull : 0ull;
            lane_tiles += 1;
            if (lane == 31) {
                if (has_out) {
                    T* e_ = sout + (j & 31) * S;
                    if constexpr (F32) {
                        float v[S];
                        seam_pack<P>(v, hi, lo, b1lo, b, E);
                        seam_entry_store<S>(e_, v);
                    } else {
                        e_[0] = hi;
                        e_[1] = (T)lo;
                        e_[2] = (T)b1lo;
#pragma unroll
                        for (int q = 1; q <= P; ++q) e_[2 + q] = b[q];
                        e_[P + 3] = (double)E;
                    }
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
        const int jj = t - 31;
        if (has_out && jj >= 0 && jj < L2 && (((jj & 31) == 31) || jj == L2 - 1)) {
            __syncwarp();
            const int start = jj & ~31;
            const int nb = jj - start + 1;
            if (!train && start + nb > A.wcols) {
                const unsigned long long need = ((unsigned long long)next << 32) |
                                                (unsigned)(start + nb - A.wcols);
                bool okl = true;
                if (lane == 0) okl = wait_ge_u64(&A.cons[slot_out], need, A.status);
                ok = __shfl_sync(kFull, okl, 0);
            }
            if (ok) {
                T* dst = train ? reinterpret_cast<T*>(st_pair + ((size_t)s * L2 + start) * S)
                               : seam + ((size_t)slot_out * A.wcols + (start % A.wcols)) * S;
                for (int idx = lane; idx < nb * S; idx += 32) __stcg(dst + idx, sout[idx]);
                __threadfence();
                __syncwarp();
                if (lane == 0)
                    st_release_u64(&A.prod[pw_out],
                                   ((unsigned long long)item << 32) | (unsigned)(start + nb));
            }
            __syncwarp();
        }
    }
    return ok;
}

// COMP (FP32 only): add the chunk partials with TwoSum compensation.  Needed
// for very long dot products (d beyond ~1000); it costs 32 registers, which
// the shorter ones spend on keeping more loads in flight.
template <int P, typename T, int NR, bool COMP>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2)
    fwd_cm_kernel(SolverArgs A, T* cscratch, int64_t cstride) {
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int S = P + 4;
    using Sm = CmSmem<P, T>;
    extern __shared__ float4 smem_f4[];
    T* smem = reinterpret_cast<T*>(smem_f4);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    T* uni = smem + warp * Sm::per_warp;
    T* dxs = uni;                    // [KC][36]: dims x rows
    T* dys = uni + kCmKC * 36;       // [32][KC+1]: columns x dims
    T* cring = uni;                  // [64][32]: columns x rows (phase 2)
    T* sin_ = uni + Sm::uni;         // seam-in block
    T* sout = sin_ + kG * S;         // seam-out block
    T* cst = cscratch + (size_t)gwarp * cstride;  // this warp's strip [L2][32]
    T* seam = reinterpret_cast<T*>(A.seam);
    const int n_items = A.sched.hdr[2];
    const int d = A.d;
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
        const int i0 = s * 32;
        bool ok = true;
#ifdef SIGK_DEBUG
        {
            // the strip scratch, seam slots and outputs of this item lie inside
            // their buffers
            const bool in = dbg_in(A.status, 31, lo_p, A.n_pairs - 1) &&
                            dbg_in(A.status, 32, (int64_t)L2 * 32, cstride) &&
                            dbg_in(A.status, 33, item % A.nslot, A.nslot - 1) &&
                            dbg_in(A.status, 34, pd.out0, A.out_cap - 1) &&
                            dbg_in(A.status, 35, pd.out1 < 0 ? 0 : pd.out1, A.out_cap - 1);
            if (!__all_sync(kFull, in)) break;
        }
#endif

        // ---- phase 1: c[i0 + r][j] for r < 32, all j, into the scratch strip ----
        // FP64: the increments are staged unscaled and the refinement factor
        // 1/(sx*sy) is applied to the finished dot product
        const double cscale = 1.0 / ((double)pd.sx * (double)pd.sy);
        for (int j0 = 0; j0 < L2; j0 += 32) {
            T acc[32];
            float comp[32];  // FP32: compensation of the sum of chunk partials
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                acc[r] = T(0);
                comp[r] = 0.0f;
            }
            const int jl = j0 + lane;
            for (int k0 = 0; k0 < d; k0 += kCmKC) {
                __syncwarp();
                const int e = k0 + lane;
                // dx chunk, transposed to [dim][row]; dy chunk [column][dim]
                if constexpr (F32) {
                    stage_increments(dxs + lane * 36, 1, pd.xr, i0, L1, d, e, A.inc_mode, pd.sx);
                    stage_increments(dys + lane, kCmKC + 1, pd.yr, j0, L2, d, e, A.inc_mode, pd.sy);
                } else {
#pragma unroll 4
                for (int r = 0; r < 32; ++r) {
                    const int row = i0 + r;
                    const int col = j0 + r;
                    {
                        dxs[lane * 36 + r] =
                            (row < L1 && e < d) ? inc_at_d(pd.xr, row / pd.sx, d, e, A.inc_mode) : 0.0;
                        dys[r * (kCmKC + 1) + lane] =
                            (col < L2 && e < d) ? inc_at_d(pd.yr, col / pd.sy, d, e, A.inc_mode) : 0.0;
                    }
                }
                }
                __syncwarp();
                const int kn = min(kCmKC, d - k0);
                if constexpr (F32) {
                    // two-level sum: a chunk's products are accumulated from
                    // zero, then added to the total (with TwoSum compensation
                    // under COMP, so the error is that of 32-term sums whatever
                    // d; one running sum of 256 products had ~2.5x, of 8192
                    // ~10x more error than the plain two-level sum)
                    float part[32];
#pragma unroll
                    for (int r = 0; r < 32; ++r) part[r] = 0.0f;
                    for (int ee = 0; ee < kn; ++ee) {
                        const float y = dys[lane * (kCmKC + 1) + ee];
                        const float4* xr = reinterpret_cast<const float4*>(dxs + ee * 36);
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
                    for (int r = 0; r < 32; ++r) {
                        if constexpr (COMP) {
                            const float t = acc[r] + part[r];
                            const float bp = t - acc[r];
                            comp[r] += (acc[r] - (t - bp)) + (part[r] - bp);
                            acc[r] = t;
                        } else {
                            acc[r] += part[r];
                        }
                    }
                } else {
                    for (int ee = 0; ee < kn; ++ee) {
                        const double y = dys[lane * (kCmKC + 1) + ee];
                        const double2* xr = reinterpret_cast<const double2*>(dxs + ee * 36);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const double2 x = xr[q];
                            acc[2 * q + 0] = fma(x.x, y, acc[2 * q + 0]);
                            acc[2 * q + 1] = fma(x.y, y, acc[2 * q + 1]);
                        }
                    }
                }
            }
            if (jl < L2) {
                if constexpr (F32) {
                    float4* dst = reinterpret_cast<float4*>(cst + (size_t)jl * 32);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        dst[q] = make_float4(acc[4 * q] + comp[4 * q], acc[4 * q + 1] + comp[4 * q + 1],
                                             acc[4 * q + 2] + comp[4 * q + 2],
                                             acc[4 * q + 3] + comp[4 * q + 3]);
                } else {
                    double2* dst = reinterpret_cast<double2*>(cst + (size_t)jl * 32);
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        dst[q] = make_double2(acc[2 * q] * cscale, acc[2 * q + 1] * cscale);
                }
            }
        }
        __syncwarp();

        // ---- phase 2: the wavefront sweep (one row per lane) -------------------
        // (training: the seams are not reused, no slot to wait for)
        if (has_out && A.store == nullptr) ok = wait_slot_free(A.sched, A.pairs, item, A.nslot, A.done, A.status);
        if (ok)
            ok = sweep_strip<P, T, NR>(A, pd, lo_p, s, item, has_in ? ir.prev : -1,
                                       has_out ? ir.next : -1, cst, cring, sin_, sout, seam,
                                       tiles_done, lane_tiles);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            st_release_s64(&A.done[item % A.nslot], (long long)item);
        }
        if (!ok) break;
    }
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
