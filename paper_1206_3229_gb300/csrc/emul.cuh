// emul.cuh -- FP64-accurate spline filter without FP64 instructions.
//
// GB300 executes FP64 arithmetic at ~1.6 operations per clock per SM (and float<->double
// conversions at the same rate), far below what a 10-tap filter on FP64 data needs to keep up with
// HBM.  For FP64 storage the sweeps therefore compute
//
//     out = sum_t w_t x_t
//
// with integer and FP32 units only, on a fixed-point grid set by a bound 2^Ef >= |f| (four times
// the largest |f| uploaded):
//   x_t * 2^(31-Ef) = kx_t + r_t,  kx_t = floor (int32), r_t in (-1, 1) (float, 24 bits)
//   w_t * 2^30      = Wh_t + wl_t, Wh_t = round (int32), |wl_t| <= 1/2 (float)
//   out * 2^(61-Ef) = sum_t Wh_t kx_t                      exact, int64 (IMAD.WIDE)
//                   + sum_t (wl_t kx_t + w_t 2^30 r_t)      FP32 FMAs, rounded onto the int64 sum
// and the int64 total is turned back into an FP64 value with integer instructions.  The error is
// about 2^-49 of 2^Ef per sweep, the size of the rounding noise of an FP64 evaluation.  All
// conversions read and build IEEE bit patterns directly.
#pragma once
#include <stdint.h>

namespace vl {

struct EmulElem {
    int kx;     // floor part on the 2^(Ef-31) grid
    float r;    // remainder in grid units
};

// Split x on the grid 2^(Ef-31).  s_base = 1044 + Ef.  |x| must be below 2^(Ef+1) (otherwise
// `out_of_range` is set and the value is clamped to that); values below 2^(Ef-77) become zero.
// 32-bit funnel shifts on the two halves of the mantissa; no 64-bit variable shifts.
__device__ __forceinline__ EmulElem emul_split(double x, int s_base, bool& out_of_range)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int e = (int)((hi >> 20) & 0x7FFu);
    int s = s_base - e;                             // value = m * 2^-s in grid units
    if (s < 22) {
        out_of_range = true;
        s = 22;
    }
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;   // mantissa m = mh:lo (53 bits)
    // integer part k = m >> s (s >= 22, so k < 2^31)
    uint32_t k;
    if (s < 32) k = __funnelshift_r(lo, mh, s);
    else k = s < 53 ? (mh >> (s - 32)) : 0u;
    // 24 bits right below the binary point: (m >> (s - 24)) mod 2^24
    const int a = s - 24;
    uint32_t t;
    if (a <= 0) t = lo << (-a);
    else if (a < 32) t = __funnelshift_r(lo, mh, a);
    else t = a < 53 ? (mh >> (a - 32)) : 0u;
    t &= 0xFFFFFFu;
    float r = __uint2float_rn(t) * 5.9604644775390625e-08f;   // * 2^-24
    int kx = (int)k;
    if (e == 0 || s > 77) {
        kx = 0;
        r = 0.f;
    }
    if (hi >> 31) {
        kx = -kx;
        r = -r;
    }
    EmulElem o;
    o.kx = kx;
    o.r = r;
    return o;
}

// acc + a * b (32 x 32 -> 64 multiply-add).  On this GPU the 64-bit accumulate costs two integer
// additions besides the IMAD.WIDE; where two products go into the same sum, mul_wide + one
// three-input add is cheaper.
__device__ __forceinline__ long long mad_wide(int a, int b, long long acc)
{
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(acc));
    return d;
}

// a * b as int64 (one IMAD.WIDE).
__device__ __forceinline__ long long mul_wide(int a, int b)
{
    long long d;
    asm("mul.wide.s32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
    return d;
}

// The FP32 part of the sum enters the int64 total without a conversion instruction (the hardware
// float->int64 conversion issues on the FP64 pipe on this GPU).  The weights that feed the FP32
// sums carry an extra factor 2^-EMUL_RS, so the FP32 sum S' = S 2^-EMUL_RS satisfies |S'| < 2^22
// (|S| < 2^33.5 for any |x| < 2^Ef: ten |wl kx| <= 2^30 terms plus |w| 2^30 |r| summed over the
// taps, sum |w| < 2).  Adding 1.5 * 2^23 then leaves round(S') in the low mantissa bits:
//     bits(S' + 1.5 * 2^23) = 0x4B400000 + round(S')            (round to nearest even)
// and one IMAD.WIDE adds 2^EMUL_RS * bits to an integer sum that started at EMUL_M0, which cancels
// the constant.  The rounding step 2^EMUL_RS on the 2^(Ef-61) grid is below the FP32 rounding of S.
constexpr int EMUL_RS = 12;
constexpr float EMUL_MAGIC = 12582912.0f;                        // 1.5 * 2^23
constexpr long long EMUL_M0 = -(1ll << EMUL_RS) * 0x4B400000ll;
constexpr float EMUL_WSCALE = 2.2737367544323206e-13f;           // 2^-(30 + EMUL_RS)

__device__ __forceinline__ long long emul_finish(long long M, float Sp)
{
    return mad_wide(__float_as_int(Sp + EMUL_MAGIC), 1 << EMUL_RS, M);
}

// Value of an element in FP64 (for the rare boundary corrections).
__device__ __forceinline__ double emul_value(EmulElem v, double grid)
{
    return ((double)v.kx + (double)v.r) * grid;
}

// T * 2^(Ef-61) as an FP64 value, round to nearest even, integer instructions only.
__device__ __forceinline__ double emul_to_f64(long long T, int Ef)
{
    if (T == 0) return 0.0;
    const uint64_t sgn = (uint64_t)T >> 63;
    const uint64_t a = sgn ? (uint64_t)(-T) : (uint64_t)T;
    const int lz = __clzll((long long)a);
    const uint64_t n = a << lz;                     // leading one at bit 63
    uint64_t mant = n >> 11;                        // 53 bits including the hidden one
    const uint64_t rem = n & 0x7FFull;
    mant += (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
    // biased exponent of a value in [2^(63-lz), 2^(64-lz)) times 2^(Ef-61); the hidden bit of
    // mant adds one to the exponent field (and a rounding carry into bit 53 adds one more).
    const int64_t E = (int64_t)(63 - lz + Ef - 61 + 1023 - 1);
    const uint64_t bits = (sgn << 63) + ((uint64_t)E << 52) + mant;
    return __longlong_as_double((long long)bits);
}

// Filter weights in the emulated form.  Wh = round(w 2^30), wl = (w 2^30 - Wh) 2^-EMUL_RS as
// float, wf = w 2^30 2^-EMUL_RS as float.  Integer instructions only.
__host__ __device__ __forceinline__ void emul_weight(double w, int& Wh, float& wl, float& wf)
{
#ifdef __CUDA_ARCH__
    const uint64_t b = (uint64_t)__double_as_longlong(w);
#else
    uint64_t b;
    __builtin_memcpy(&b, &w, 8);
#endif
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0) {
        Wh = 0;
        wl = 0.f;
        wf = 0.f;
        return;
    }
    const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    // w * 2^60 = m * 2^(e - 1075 + 60); |w| < 4 so the shift is <= 3 to the left
    const int sh = e - 1015;
    long long fx;   // round(w * 2^60)
    if (sh >= 0) fx = (long long)(m << sh);
    else if (sh > -64) fx = (long long)((m >> (-sh)) + ((m >> (-sh - 1)) & 1ull));
    else fx = 0;
    if (b >> 63) fx = -fx;
    // Wh = round(fx / 2^30), remainder in [-2^29, 2^29]
    const long long h = (fx + (1ll << 29)) >> 30;
    const long long l = fx - (h << 30);
    Wh = (int)h;
#ifdef __CUDA_ARCH__
    wl = __ll2float_rn(l) * EMUL_WSCALE;               // * 2^-30 * 2^-EMUL_RS
    wf = __ll2float_rn(fx) * EMUL_WSCALE;              // round(w 2^60) rounded to float, same scale
#else
    wl = (float)l * EMUL_WSCALE;
    wf = (float)fx * EMUL_WSCALE;
#endif
}

}  // namespace vl
