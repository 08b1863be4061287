// sigk_f64.cuh -- the tile map of sigk_device.cuh in FP64.
//
// Same expansion and factorial scaling as tile_update (Sec. 2.3, App. A.6),
// with every coefficient, edge value and the corner held in double.  FP64
// needs no float-float corner or compensated first-order terms: its 53-bit
// significand leaves the rounding error of a whole sweep far below the
// truncation error.  Used for pairs whose FP32 result is too ill-conditioned
// (strong coupling over long paths, oscillating signs) to meet a tight
// tolerance: the solve is then FP64 end to end, increments included.
#pragma once
#include "sigk_device.cuh"

namespace sigk {

// 1/k! for k = 0..33, correctly rounded to double
static __constant__ double c_inv_fact_d[34] = {
    1.0, 1.0, 0.5, 0.16666666666666666, 0.041666666666666664, 0.008333333333333333,
    0.001388888888888889, 0.0001984126984126984, 2.48015873015873e-05, 2.7557319223985893e-06,
    2.755731922398589e-07, 2.505210838544172e-08, 2.08767569878681e-09, 1.6059043836821613e-10,
    1.1470745597729725e-11, 7.647163731819816e-13, 4.779477332387385e-14, 2.8114572543455206e-15,
    1.5619206968586225e-16, 8.22063524662433e-18, 4.110317623312165e-19, 1.9572941063391263e-20,
    8.896791392450574e-22, 3.868170170630684e-23, 1.6117375710961184e-24, 6.446950284384474e-26,
    2.4795962632247976e-27, 9.183689863795546e-29, 3.279889237069838e-30, 1.1309962886447716e-31,
    3.7699876288159054e-33, 1.216125041553518e-34, 3.8003907548547434e-36, 1.151633562077195e-37};

// 2^n as a double for n <= 0 (0 below the normal range).
__device__ __forceinline__ double exp2_nonpos_d(int n) {
    return n < -1022 ? 0.0 : __longlong_as_double((long long)(1023 + n) << 52);
}

// One tile in FP64.  a[1..P]: scaled bottom edge (overwritten by the top
// edge); b0: corner (overwritten by the new corner); b[1..P]: scaled left edge
// (overwritten by the right edge).  a[0] and b[0] are not read.
template <int P>
__device__ __forceinline__ void tile_update_f64(double c, double (&a)[P + 1], double& b0,
                                                double (&b)[P + 1], int nr) {
    constexpr int NRM = P < kMaxRings ? P : kMaxRings;
    double cp[NRM + 1], ch[NRM + 1];
    cp[1] = c;
    ch[1] = c;
#pragma unroll
    for (int m = 2; m <= NRM; ++m) {
        cp[m] = cp[m - 1] * c;
        ch[m] = cp[m] * c_inv_fact_d[m];
    }
    // ring-p Hankel sums of the incoming edges (a_0 = b_0 := corner)
    double ha[NRM + 1], hb[NRM + 1];
#pragma unroll
    for (int p = 1; p <= NRM; ++p) {
        ha[p] = 0.0;
        hb[p] = 0.0;
        if (p <= nr) {
            double sa = b0 * c_inv_fact_d[p];
            double sb = sa;
#pragma unroll
            for (int r = 1; r <= P - p; ++r) {
                sa = fma(b[r], c_inv_fact_d[p + r], sa);
                sb = fma(a[r], c_inv_fact_d[p + r], sb);
            }
            ha[p] = sa;
            hb[p] = sb;
        }
    }
    // bottom edge at u = 1 without its constant term
    double S = 0.0;
#pragma unroll
    for (int p = P; p >= 1; --p) S = fma(a[p], c_inv_fact_d[p], S);
    // top and right edges in place, high degree first
#pragma unroll
    for (int p = P; p >= 1; --p) {
        double v = a[p];
#pragma unroll
        for (int m = 1; m < p && m <= NRM; ++m)
            if (m <= nr) v = fma(ch[m], a[p - m], v);
        if (p <= NRM && p <= nr) v = fma(cp[p], ha[p], v);
        a[p] = v;
    }
#pragma unroll
    for (int q = P; q >= 1; --q) {
        double v = b[q];
#pragma unroll
        for (int m = 1; m < q && m <= NRM; ++m)
            if (m <= nr) v = fma(ch[m], b[q - m], v);
        if (q <= NRM && q <= nr) v = fma(cp[q], hb[q], v);
        b[q] = v;
    }
    b0 += S;
}

}  // namespace sigk
