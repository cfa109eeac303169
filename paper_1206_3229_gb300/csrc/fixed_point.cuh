// fixed_point.cuh -- exact integer fixed-point accumulation for the moment reductions.
//
// On GB300 an FP64 add or multiply has a throughput of ~1.6 per clock per SM and a dependent-issue
// latency of hundreds of cycles, so a reduction written as a chain of FP64 adds (a compensated
// running sum, a shuffle tree) takes tens of microseconds.  Every cross-thread sum of the solver is
// therefore done in integers: a double x becomes round(x * 2^k) in int64/int128 with integer
// instructions only, sums are exact and independent of order (so any tree, any atomics order gives
// the same bits), and the total is converted back to double with round-to-nearest-even, again with
// integer instructions.  Scales k are chosen on the host from bounds of |f| so nothing overflows.
#pragma once
#include <stdint.h>

namespace vl {

typedef __int128 i128;
typedef unsigned __int128 u128;

__host__ __device__ __forceinline__ int clz64(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

__host__ __device__ __forceinline__ uint64_t f64_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    __builtin_memcpy(&b, &x, 8);
    return b;
#endif
}

__host__ __device__ __forceinline__ double f64_from_bits(uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    __builtin_memcpy(&x, &b, 8);
    return x;
#endif
}

// round(x * 2^k) as int128 (ties away from zero); |x| * 2^k must stay below 2^126 (saturates).
// Zero, subnormal, infinite and NaN inputs give 0.
__host__ __device__ __forceinline__ i128 fx128_from_f64(double x, int k)
{
    const uint64_t b = f64_bits(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0 || e == 0x7FF) return 0;
    const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;   // 53 significant bits
    const int sh = e - 1075 + k;                                           // x * 2^k = m * 2^sh
    u128 v;
    if (sh >= 0) {
        v = sh > 73 ? (((u128)1 << 126) - 1) : ((u128)m << sh);
    } else if (sh > -64) {
        const int r = -sh;
        v = (u128)((m >> r) + ((m >> (r - 1)) & 1ull));
    } else {
        v = 0;
    }
    return (b >> 63) ? -(i128)v : (i128)v;
}

// v * 2^-k rounded to the nearest double (ties to even); assumes the result is a normal double.
__host__ __device__ __forceinline__ double fx128_to_f64(i128 v, int k)
{
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    const u128 a = neg ? (u128)(-v) : (u128)v;
    const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
    const int lz = hi ? clz64(hi) : 64 + clz64(lo);
    const u128 n = a << lz;                         // leading one at bit 127
    const uint64_t top = (uint64_t)(n >> 64), low = (uint64_t)n;
    uint64_t mant = top >> 11;                      // 53 bits
    const uint64_t rem = top & 0x7FFull;
    int E = 127 - lz - k;
    if (rem > 0x400ull || (rem == 0x400ull && (low != 0 || (mant & 1ull)))) {
        ++mant;
        if (mant >> 53) {
            mant >>= 1;
            ++E;
        }
    }
    const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)(E + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
    return f64_from_bits(bits);
}

// round(x * 2^k) for a float (integer instructions only); |x| * 2^k < 2^126.
__host__ __device__ __forceinline__ i128 fx128_from_f32(float x, int k)
{
#ifdef __CUDA_ARCH__
    const uint32_t b = (uint32_t)__float_as_int(x);
#else
    uint32_t b;
    __builtin_memcpy(&b, &x, 4);
#endif
    const int e = (int)((b >> 23) & 0xFF);
    if (e == 0 || e == 0xFF) return 0;
    const uint64_t m = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = e - 150 + k;
    u128 v;
    if (sh >= 0) v = sh > 102 ? (((u128)1 << 126) - 1) : ((u128)m << sh);
    else if (sh > -64) v = (u128)((m >> (-sh)) + ((m >> (-sh - 1)) & 1ull));
    else v = 0;
    return (b >> 31) ? -(i128)v : (i128)v;
}

__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int o)
{
    const uint64_t lo = (uint64_t)v, hi = (uint64_t)((u128)v >> 64);
    const uint64_t l2 = (uint64_t)__shfl_xor_sync(0xffffffffu, (long long)lo, o);
    const uint64_t h2 = (uint64_t)__shfl_xor_sync(0xffffffffu, (long long)hi, o);
    return (i128)(((u128)h2 << 64) | (u128)l2);
}

__device__ __forceinline__ i128 warp_sum_i128(i128 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_i128(v, o);
    return v;
}

// Exact sum of products c_i t_i (|c| <= 2^51, |t| < 2^57) without 128-bit multiplies: each factor
// splits at 2^26 into a high part and a low part in [0, 2^26), and the four partial products are
// added in int64 (each below 2^57 in magnitude, so up to 64 terms fit) until fold() forms the int128
// value.  Exact: the same integer as summing (int128) c_i * t_i.
struct Mac26 {
    long long hh = 0, mid = 0, ll = 0;
    __device__ __forceinline__ void add(long long c, long long t)
    {
        const int ch = (int)(c >> 26), cl = (int)(c & 0x3FFFFFFll);
        const int th = (int)(t >> 26), tl = (int)(t & 0x3FFFFFFll);
        hh += (long long)ch * th;
        mid += (long long)ch * tl + (long long)cl * th;
        ll += (long long)cl * tl;
    }
    __device__ __forceinline__ i128 fold() const { return ((i128)hh << 52) + ((i128)mid << 26) + (i128)ll; }
};

// Exact block-wide sum (any order gives the same value); `sh` holds >= 32 entries.
__device__ __forceinline__ i128 block_sum_i128(i128 v, i128* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_i128(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        i128 r = lane < nw ? sh[lane] : (i128)0;
        r = warp_sum_i128(r);
        if (lane == 0) sh[0] = r;
    }
    __syncthreads();
    const i128 r = sh[0];
    __syncthreads();
    return r;
}

// Exact block-wide sums of four values in one pass (one set of barriers); `sh` holds >= 128 entries.
__device__ __forceinline__ void block_sum4_i128(i128& a, i128& b, i128& c, i128& d, i128* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += shfl_xor_i128(a, o);
        b += shfl_xor_i128(b, o);
        c += shfl_xor_i128(c, o);
        d += shfl_xor_i128(d, o);
    }
    __syncthreads();
    if (lane == 0) {
        sh[wid] = a;
        sh[32 + wid] = b;
        sh[64 + wid] = c;
        sh[96 + wid] = d;
    }
    __syncthreads();
    if (wid == 0) {
        i128 ra = lane < nw ? sh[lane] : (i128)0, rb = lane < nw ? sh[32 + lane] : (i128)0;
        i128 rc = lane < nw ? sh[64 + lane] : (i128)0, rd = lane < nw ? sh[96 + lane] : (i128)0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ra += shfl_xor_i128(ra, o);
            rb += shfl_xor_i128(rb, o);
            rc += shfl_xor_i128(rc, o);
            rd += shfl_xor_i128(rd, o);
        }
        if (lane == 0) {
            sh[0] = ra;
            sh[32] = rb;
            sh[64] = rc;
            sh[96] = rd;
        }
    }
    __syncthreads();
    a = sh[0];
    b = sh[32];
    c = sh[64];
    d = sh[96];
    __syncthreads();
}

}  // namespace vl
