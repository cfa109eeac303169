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
// The FP32 filter of a column moving by sigma cells: foot offset n0 = floor(-sigma) and fraction beta
// in FP64, the ten weights of Eqs. (splinegen, splinecoeffs, findif) and g, d (the f'' factors of the
// two spline nodes) in FP32.  One routine for the filter launch and the p-shift that forms its
// tiles' filters itself, so both give the same values.
struct FiltF32 {
    int n0;
    double beta;
    float w[NTAP];
    float g, d;
};
__device__ __forceinline__ FiltF32 filt_f32(double sigma)
{
    using T = float;
    FiltF32 o;
    const double ms = -sigma;
    const double fl = floor(ms);
    o.beta = ms - fl;
    o.n0 = (int)fl;
    const T b = (T)o.beta;
    const T al = (T)(1.0 - o.beta);
    const T g = (al * al * al - al) * (T)(1.0 / 6.0);
    const T d = (b * b * b - b) * (T)(1.0 / 6.0);
    const T c0 = T(VL_FD_C0), c1 = T(VL_FD_C1), c2 = T(VL_FD_C2), c3 = T(VL_FD_C3), c4 = T(VL_FD_C4);
    o.w[0] = g * c4;
    o.w[1] = g * c3 + d * c4;
    o.w[2] = g * c2 + d * c3;
    o.w[3] = g * c1 + d * c2;
    o.w[4] = al + g * c0 + d * c1;
    o.w[5] = b + g * c1 + d * c0;
    o.w[6] = g * c2 + d * c1;
    o.w[7] = g * c3 + d * c2;
    o.w[8] = g * c4 + d * c3;
    o.w[9] = d * c4;
    o.g = g;
    o.d = d;
    return o;
}

__device__ __forceinline__ void pparams_f32(const PParamsArgs& a, int i, double sigma)
{
    const FiltF32 o = filt_f32(sigma);
    if (a.beta) a.beta[i] = o.beta;
    float* w = static_cast<float*>(a.w);
    float* gd = static_cast<float*>(a.gd);
    a.n0[i] = o.n0;
    const size_t n = (size_t)a.Nx;
#pragma unroll
    for (int t = 0; t < NTAP; ++t) w[t * n + i] = o.w[t];
    gd[i] = o.g;
    gd[n + i] = o.d;
}

// The HMF force of Eq. (hmfmeanforce) at a node with sin x_i = s, cos x_i = c.
__device__ __forceinline__ double hmf_force(double Mx, double My, double s, double c) { return -Mx * s + My * c; }

// HMF mean field from the x-shift's per-CTA numbers ([ctas][3] int128: mass, cos- and sin-weighted
// column sums, units 2^(Ef-51) and 2^(Ef-101)), summed exactly by one warp: Mx, My of Eq. (mxmydef),
// the same values as the filter launch's block sums give.
__device__ __forceinline__ void hmf_mxmy_warp(const HmfFiltArgs& h, double& Mx, double& My)
{
    const int lane = threadIdx.x & 31;
    const i128* p = static_cast<const i128*>(h.ctapart);
    i128 x = 0, y = 0;
    for (int b = lane; b < h.ctas; b += 32) {
        x += p[(size_t)b * 3 + 1];
        y += p[(size_t)b * 3 + 2];
    }
    x = warp_sum_i128(x);
    y = warp_sum_i128(y);
    Mx = h.dxdp * fx128_to_f64(x, 101 - h.Ef);
    My = h.dxdp * fx128_to_f64(y, 101 - h.Ef);
}

}  // namespace vl
