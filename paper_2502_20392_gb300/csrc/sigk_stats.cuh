// sigk_stats.cuh -- exact a-priori statistics of the tile coefficients for the
// order choice (App. C.3: the truncation order is chosen from the size of the
// coefficients and of the accumulated coupling over the grid).
//
// For every pair of the pair table (refined as it will be solved) and every
// tile coefficient c_ij = <dx_i, dy_j>:
//   M     = max_ij |c_ij|                              (largest tile)
//   R_m   = sum_ij |c_ij|^m, m = 2..9                  (size of a dropped ring m)
//   C_a   = max_{i,J} |<dx_i, y_J - y_0>| = max |sum_{j<J} c_ij|   (row coupling)
//   C_b   = max_{I,j} |<x_I - x_0, dy_j>| = max |sum_{i<I} c_ij|   (column coupling)
// computed exactly (in FP32) rather than bounded: a warp takes a 32-row strip
// of a pair and forms its coefficients 32 columns at a time with the FMA
// micro-GEMM of the large-d solver; C_a comes from a warp prefix scan along
// each row with a carry across column blocks, C_b from the column prefix down
// the strip started from <x_{i0} - x_0, dy_j> (one extra row of the product).
// The coefficient matrix is never stored.  Results are combined per pair with
// atomics: maxima as the bit patterns of non-negative doubles, sums as adds.
#pragma once
#include "sigk_device.cuh"
#include "sigk_fwd.cuh"

namespace sigk {

// per-pair record: [0] L1, [1] L2 (segments as solved), [2] C_a, [3] C_b,
// [4 + m - 2] R_m for m = 2..9, [12] M, [13] unused
constexpr int kStatFields = 14;
constexpr int kStKC = 32;  // contraction chunk

struct StatArgs {
    const PairDesc* pairs;
    Schedule sched;             // items of rows_per_strip rows (any order)
    int32_t n_pairs;
    int32_t rows_per_strip;
    int32_t d;
    int32_t inc_mode;
    int* item_counter;          // zero before the launch
    double* stats;              // [n_pairs][kStatFields], zero before the launch
    float* base;                // [warps][d]: x_{i0} - x_0 of the warp's strip
};

struct StSmem {
    static constexpr int per_warp = kStKC * 36 + 32 * (kStKC + 1) + kStKC;
};

__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(128) pair_stats_kernel(StatArgs A) {
    extern __shared__ float4 smem_f4[];
    float* smem = reinterpret_cast<float*>(smem_f4);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    float* dxs = smem + warp * StSmem::per_warp;  // [KC][36]: dims x rows
    float* dys = dxs + kStKC * 36;                // [32][KC+1]: columns x dims
    float* bs = dys + 32 * (kStKC + 1);           // [KC]: x_{i0} - x_0, this chunk
    float* base = A.base + (size_t)gwarp * A.d;
    const int n_items = A.sched.hdr[2];
    const int d = A.d;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.item_counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_items) break;
        const ItemRef ir = decode_item(A.sched, A.pairs, item);
        const int lo_p = ir.pair;
        const PairDesc pd = A.pairs[lo_p];
        const int L1 = pd.L1, L2 = pd.L2;
        const int s = ir.k;
        float mloc = 0.0f, ca = 0.0f, cb = 0.0f;
        float rs[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) rs[m] = 0.0f;
        for (int i0 = s * A.rows_per_strip; i0 < min(L1, (s + 1) * A.rows_per_strip); i0 += 32) {
            // x_{i0} - x_0 of the (refined) row path, one dimension per lane
            // (virtual point i0 = original point q plus (i0 - q*sx) pieces of
            // segment q, each a 1/sx of it)
            {
                const int q = i0 / pd.sx, rem = i0 - q * pd.sx;
                for (int e = lane; e < d; e += 32) {
                    float v = 0.0f;
                    if (!A.inc_mode) {
                        v = pd.xr[(int64_t)q * d + e] - pd.xr[e];
                    } else {
                        for (int i = 0; i < q; ++i) v += pd.xr[(int64_t)i * d + e];
                    }
                    if (rem > 0) v = fmaf((float)rem, inc_ref(pd.xr, i0, d, e, A.inc_mode, pd.sx), v);
                    base[e] = v;
                }
            }
            __syncwarp();
            float carry[32];  // row prefix sums up to the current column block
#pragma unroll
            for (int r = 0; r < 32; ++r) carry[r] = 0.0f;
            for (int j0 = 0; j0 < L2; j0 += 32) {
                float acc[32], g = 0.0f;
#pragma unroll
                for (int r = 0; r < 32; ++r) acc[r] = 0.0f;
                for (int k0 = 0; k0 < d; k0 += kStKC) {
                    __syncwarp();
                    const int e = k0 + lane;
#pragma unroll 4
                    for (int r = 0; r < 32; ++r) {
                        const int row = i0 + r, col = j0 + r;
                        dxs[lane * 36 + r] =
                            (row < L1 && e < d) ? inc_ref(pd.xr, row, d, e, A.inc_mode, pd.sx) : 0.0f;
                        dys[r * (kStKC + 1) + lane] =
                            (col < L2 && e < d) ? inc_ref(pd.yr, col, d, e, A.inc_mode, pd.sy) : 0.0f;
                    }
                    bs[lane] = e < d ? base[e] : 0.0f;
                    __syncwarp();
                    const int kn = min(kStKC, d - k0);
                    for (int ee = 0; ee < kn; ++ee) {
                        const float y = dys[lane * (kStKC + 1) + ee];
                        const float4* xr = reinterpret_cast<const float4*>(dxs + ee * 36);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 x = xr[q];
                            acc[4 * q + 0] = fmaf(x.x, y, acc[4 * q + 0]);
                            acc[4 * q + 1] = fmaf(x.y, y, acc[4 * q + 1]);
                            acc[4 * q + 2] = fmaf(x.z, y, acc[4 * q + 2]);
                            acc[4 * q + 3] = fmaf(x.w, y, acc[4 * q + 3]);
                        }
                        g = fmaf(bs[ee], y, g);
                    }
                }
                // rows past L1 and columns past L2 hold zeros: they change no
                // maximum and no sum
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const float v = acc[r];
                    const float av = fabsf(v);
                    mloc = fmaxf(mloc, av);
                    float pw = av * av;
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        rs[m] += pw;
                        pw *= av;
                    }
                    // column prefix: <x_{i0+r+1} - x_0, dy_j>
                    g += v;
                    cb = fmaxf(cb, fabsf(g));
                    // row prefix over the columns: inclusive warp scan + carry
                    float w = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const float u = __shfl_up_sync(kFull, w, o);
                        if (lane >= o) w += u;
                    }
                    w += carry[r];
                    ca = fmaxf(ca, fabsf(w));
                    carry[r] = __shfl_sync(kFull, w, 31);
                }
            }
        }
        // combine the warp's values, then the pair's record
        double rsd[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) rsd[m] = (double)rs[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mloc = fmaxf(mloc, __shfl_xor_sync(kFull, mloc, o));
            ca = fmaxf(ca, __shfl_xor_sync(kFull, ca, o));
            cb = fmaxf(cb, __shfl_xor_sync(kFull, cb, o));
#pragma unroll
            for (int m = 0; m < 8; ++m) rsd[m] += __shfl_xor_sync(kFull, rsd[m], o);
        }
        if (lane == 0) {
            double* o = A.stats + (size_t)lo_p * kStatFields;
            o[0] = (double)L1;
            o[1] = (double)L2;
            atomic_max_nonneg(&o[2], (double)ca);
            atomic_max_nonneg(&o[3], (double)cb);
#pragma unroll
            for (int m = 0; m < 8; ++m) atomicAdd(&o[4 + m], rsd[m]);
            atomic_max_nonneg(&o[12], (double)mloc);
        }
    }
}

}  // namespace sigk
