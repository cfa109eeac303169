// pparams.cuh -- the p-shift filters of one column (Sec. 3, Eqs. splinegen, splinecoeffs, findif):
// the foot split of the column's displacement and its ten filter weights, written in the forms
// the p-shift kernels read.  Shared by the filter launches and the ring force kernel, which forms
// the filters of the columns it has just computed.
#pragma once
#include "emul.cuh"
#include "fixed_point.cuh"
#include "vlasov_internal.cuh"

namespace vl {

// ============================================================================ p-shift parameters
// Column i moves by sigma_i = F_i dt/dp cells (FP64).  For FP64-class storage the split of the
// foot (n0 = floor(-sigma), beta = -sigma - n0) and the ten filter weights are computed in 62-bit
// fixed point; for FP32 storage the split is FP64 and the weights FP32.
// FD coefficients of Eq. (findif) as round(c * 2^60): -205/72, 8/5, -1/5, 8/315, -1/560.
constexpr long long FD60_C0 = -3282623728394494862ll;
constexpr long long FD60_C1 = 1844674407370955162ll;
constexpr long long FD60_C2 = -230584300921369395ll;
constexpr long long FD60_C3 = 29280546148745320ll;
constexpr long long FD60_C4 = -2058788401083655ll;

// x * c for x on the 2^-62 grid and c on the 2^-60 grid, rounded onto the 2^-62 grid.
__device__ __forceinline__ long long mul_fd60(long long x, long long c)
{
    return (long long)(((i128)x * (i128)c + ((i128)1 << 59)) >> 60);
}

// (x^3 - x) / 6 for x in [0, 1] on the 2^-62 grid (the spline's f'' coefficients).
__device__ __forceinline__ long long spline_cubic62(uint64_t x)
{
    const uint64_t x2 = (uint64_t)(((u128)x * x) >> 62);
    const uint64_t x3 = (uint64_t)(((u128)x2 * x) >> 62);
    return ((long long)x3 - (long long)x) / 6;
}

// The split of the foot and the ten weights for FP64-class storage, in 62-bit fixed point.  Only
// the force and sigma = F dt/dp are FP64 operations: dependent FP64 operations have a latency of
// hundreds of cycles on this GPU, integer ones a few.  The weights are exact to 2^-61 (FP64
// arithmetic: 2^-53 relative).
__device__ __forceinline__ void pparams_fixed(const PParamsArgs& a, int i, double sigma)
{
    const i128 V = fx128_from_f64(-sigma, 62);                     // -sigma 2^62
    const int n0 = (int)(long long)(V >> 62);                      // floor(-sigma)
    const uint64_t be = (uint64_t)(V & (((i128)1 << 62) - 1));   // beta 2^62 in [0, 2^62)
    const uint64_t al = (1ull << 62) - be;                         // alpha = 1 - beta
    const long long g = spline_cubic62(al), d = spline_cubic62(be);
    if (a.beta) a.beta[i] = fx128_to_f64((i128)be, 62);
    // W = the alpha/beta taps + g D_k (taps 0..8) + d D_{k+1} (taps 1..9), each exact on the 2^-62 grid
    const long long C[5] = {FD60_C0, FD60_C1, FD60_C2, FD60_C3, FD60_C4};
    long long Wg[NTAP], Wd[NTAP], W[NTAP];
#pragma unroll
    for (int t = 0; t < NTAP; ++t) {
        const int m0 = t - 4, m1 = t - 5;
        Wg[t] = (m0 >= -4 && m0 <= 4) ? mul_fd60(g, C[m0 < 0 ? -m0 : m0]) : 0;
        Wd[t] = (m1 >= -4 && m1 <= 4) ? mul_fd60(d, C[m1 < 0 ? -m1 : m1]) : 0;
        const long long base = t == 4 ? (long long)al : t == 5 ? (long long)be : 0;
        W[t] = base + Wg[t] + Wd[t];
    }
    const size_t n = (size_t)a.Nx;
    double* w = static_cast<double*>(a.w);
    double* gd = static_cast<double*>(a.gd);
    a.n0[i] = n0;
#pragma unroll
    for (int t = 0; t < NTAP; ++t) w[(size_t)t * n + i] = fx128_to_f64((i128)W[t], 62);
    gd[i] = fx128_to_f64((i128)g, 62);
    gd[n + i] = fx128_to_f64((i128)d, 62);
    if (a.Wh) {
        // Wh = round(w 2^30); wl = (w 2^30 - Wh) 2^-EMUL_RS; wf = w 2^30 2^-EMUL_RS (emul.cuh)
        const float sc = EMUL_WSCALE * 0.25f;   // 2^-(32 + EMUL_RS): W is on the 2^-62 grid
        auto split = [&](long long Wt, int* Wh, float* wl, float* wf, size_t idx) {
            const long long h = (Wt + (1ll << 31)) >> 32;
            const long long l = Wt - (h << 32);                                     // |l| <= 2^31
            const float lf = 2.f * __int2float_rn((int)(l >> 1)) + (float)(int)(l & 1);
            const float wfull = fmaf(__int2float_rn((int)(Wt >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)Wt));
            Wh[idx] = (int)h;
            wl[idx] = lf * sc;
            wf[idx] = wfull * sc;
        };
#pragma unroll
        for (int t = 0; t < NTAP; ++t) split(W[t], a.Wh, a.wl, a.wf, (size_t)t * n + i);
        if (a.Whe) {
            // zero-outside columns: the filters without g D_k (foot cell k = -1) and without
            // d D_{k+1} (k = Np - 1), [2][NTAP][n]
            const long long base4 = (long long)al, base5 = (long long)be;
#pragma unroll
            for (int t = 0; t < NTAP; ++t) {
                const long long base = t == 4 ? base4 : t == 5 ? base5 : 0;
                split(base + Wd[t], a.Whe, a.wle, a.wfe, (size_t)t * n + i);
                split(base + Wg[t], a.Whe, a.wle, a.wfe, (size_t)(NTAP + t) * n + i);
            }
        }
    }
}

// FP32-class storage: the foot split in FP64, the ten weights in FP32.
__device__ __forceinline__ void pparams_f32(const PParamsArgs& a, int i, double sigma)
{
    using T = float;
    const double ms = -sigma;
    const double fl = floor(ms);
    const double beta = ms - fl;
    if (a.beta) a.beta[i] = beta;
    T* w = static_cast<T*>(a.w);
    T* gd = static_cast<T*>(a.gd);
    a.n0[i] = (int)fl;
    const T b = (T)beta;
    const T al = (T)(1.0 - beta);
    const T g = (al * al * al - al) * (T)(1.0 / 6.0);
    const T d = (b * b * b - b) * (T)(1.0 / 6.0);
    const T c0 = T(VL_FD_C0), c1 = T(VL_FD_C1), c2 = T(VL_FD_C2), c3 = T(VL_FD_C3), c4 = T(VL_FD_C4);
    const size_t n = (size_t)a.Nx;
    w[0 * n + i] = g * c4;
    w[1 * n + i] = g * c3 + d * c4;
    w[2 * n + i] = g * c2 + d * c3;
    w[3 * n + i] = g * c1 + d * c2;
    w[4 * n + i] = al + g * c0 + d * c1;
    w[5 * n + i] = b + g * c1 + d * c0;
    w[6 * n + i] = g * c2 + d * c1;
    w[7 * n + i] = g * c3 + d * c2;
    w[8 * n + i] = g * c4 + d * c3;
    w[9 * n + i] = d * c4;
    gd[i] = g;
    gd[n + i] = d;
}

}  // namespace vl
