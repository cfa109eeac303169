// ring.cu -- the ring model's mean force and potential energy, Eq. (ringpot) into Eq. (meanforce)
// (Sec. 2), as a circulant convolution on the theta nodes:
//
//   F_i   = -dx sum_k V'((i-k) dx) rho_k        (after each first x half-shift)
//   Phi_i =  dx sum_k V ((i-k) dx) rho_k,  U = 1/2 dx sum_i rho_i Phi_i   (after the step)
//
// Two methods besides the direct FMA loop of aux_kernels.cu (ring_kernel):
//
//  * FIXED: an exact fixed-point sum.  The density arrives as exact int64 column sums t_k
//    (rho_k = dp t_k 2^-k_col, from the x-shift's partial sums), the kernel tables as round(V'(m dx)
//    2^sK) and round(V(m dx) 2^sV) with |table| <= 2^(64 - log2 N); every product t_k * table is an
//    exact int128 and so is every sum.  The only roundings are the table entries (relative 2^-52, the
//    FP64 representation of V') and the final conversion, so the force is FP64-accurate in every
//    storage mode, deterministic, and independent of the launch shape.  The multiply-adds run on
//    the integer pipe (64-bit mad.lo/madc.hi pairs), which on this GPU is many times faster than the
//    FP64 pipe.
//  * FFT: a Stockham radix-2 FFT (Govindaraju et al., SC 2008) in shared memory, one CTA per
//    grid, in FP64 or FP32: F = -dx/N Re IFFT(FFT(V') FFT(rho)); the potential by Parseval,
//    sum_i rho_i Phi_i = dx/N sum_k |FFT(rho)_k|^2 FFT(V)_k (V even, so FFT(V) is real).  N a power
//    of two.  The spectra of the kernel tables are computed once on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cstring>

#include "fixed_point.cuh"
#include "pparams.cuh"
#include "ptx.cuh"
#include "vlasov_internal.cuh"

namespace vl {

// ============================================================================ FIXED
// acc (hi:lo, two's complement int128) += a * b, a and b signed int64.
__device__ __forceinline__ void mac128(unsigned long long& lo, long long& hi, long long a, long long b)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.s64 %1, %2, %3, %1;"
        : "+l"(lo), "+l"(hi)
        : "l"(a), "l"(b));
}

__device__ __forceinline__ i128 ld_i128_cg(const void* p)
{
    const longlong2 v = __ldcg(static_cast<const longlong2*>(p));
    return (i128)(((u128)(unsigned long long)v.y << 64) | (u128)(unsigned long long)v.x);
}

int ringfx_ksplit(int N, int nsm)
{
    const int ngrp = (N + 31) / 32;
    const int ks = (int)std::lround(2.0 * (double)nsm / (double)ngrp);
    return std::max(1, std::min(ks, std::max(1, N / 256)));
}

size_t ringfx_smem_bytes(int N, int ksplit)
{
    const int len = (N + ksplit - 1) / ksplit;
    return (size_t)(2 * len + 32) * sizeof(long long);
}

// Block (g, q): outputs i = 32 g + lane, inputs k in the q-th of ksplit slices [kb, ke) of [0, N).
// Warp w adds the w-th eighth of the slice.  Warp sums and slice sums are exact int128 additions,
// so the result does not depend on the split; the last slice block of a group (ticket) finishes it.
template <bool POT, bool FILT = false>
__device__ __forceinline__ void ringfx_body(const RingArgs& a, int bx)
{
    constexpr int NW = RINGFX_THREADS / 32;
    extern __shared__ __align__(16) long long rfx_smem[];
    __shared__ i128 wsum[NW][32];
    const int N = a.N, ngrp = (N + 31) >> 5;
    const int g = bx % ngrp, q = bx / ngrp;
    if (q >= a.ksplit) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int kb = (int)(((long long)N * q) / a.ksplit), ke = (int)(((long long)N * (q + 1)) / a.ksplit);
    const int len = ke - kb;
    const int i0 = g << 5;
    long long* ts = rfx_smem;          // t_k, k = kb .. ke - 1
    long long* kk = rfx_smem + len;    // table entries at m = (base + r) mod N, r = 0 .. len + 30
    const long long* __restrict__ tab = POT ? a.Vq : a.Kq;
    for (int r = threadIdx.x; r < len; r += RINGFX_THREADS) ts[r] = __ldcg(a.colfx + kb + r);
    const int base = i0 - ke + 1;      // > -N
    for (int r = threadIdx.x; r < len + 31; r += RINGFX_THREADS) {
        int m = (base + r) % N;
        if (m < 0) m += N;
        kk[r] = __ldg(tab + m);
    }
    __syncthreads();
    // output i = i0 + lane, input k = kb + j: the table entry at i - k is kk[len - 1 + lane - j].
    // Four independent accumulators (j mod 4) keep four carry chains in flight per lane.
    constexpr int NACC = 4;
    unsigned long long lo[NACC];
    long long hi[NACC];
#pragma unroll
    for (int u = 0; u < NACC; ++u) {
        lo[u] = 0;
        hi[u] = 0;
    }
    const int jb = (len * w) / NW, je = (len * (w + 1)) / NW;
    const long long* kp = kk + (len - 1 + lane);
    int j = jb;
    for (; j + NACC <= je; j += NACC) {
#pragma unroll
        for (int u = 0; u < NACC; ++u) mac128(lo[u], hi[u], kp[-(j + u)], ts[j + u]);
    }
    for (; j < je; ++j) mac128(lo[0], hi[0], kp[-j], ts[j]);
    i128 ws = 0;
#pragma unroll
    for (int u = 0; u < NACC; ++u) ws += (i128)(((u128)(unsigned long long)hi[u] << 64) | (u128)lo[u]);
    wsum[w][lane] = ws;
    __syncthreads();
    if (w != 0) return;

    i128 s = 0;
#pragma unroll
    for (int v = 0; v < NW; ++v) s += wsum[v][lane];
    const int i = i0 + lane;
    if (a.ksplit > 1) {
        i128* gp = static_cast<i128*>(a.gpart);
        if (i < N) gp[(size_t)q * N + i] = s;
        __threadfence();
        __syncwarp();
        unsigned int tk = 0;
        if (lane == 0) tk = atomicAdd(&a.gticket[g], 1u);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk != (unsigned int)a.ksplit - 1) return;
        __threadfence();
        s = 0;
        if (i < N)
            for (int r = 0; r < a.ksplit; ++r) s += ld_i128_cg(gp + (size_t)r * N + i);
        if (lane == 0) a.gticket[g] = 0u;   // ready for the next launch
    }
    if constexpr (!POT) {
        if (i < N) {
            const double F = fx128_to_f64(s, a.k_col + a.sK) * (-a.dx * a.dp);
            a.F[i] = F;
            if (FILT && a.pp_on) {   // this column's p-shift filters, as the filter launch would write them
                if (a.pp_fixed) pparams_fixed(a.pp, i, F * a.pp.cp);
                else pparams_f32(a.pp, i, F * a.pp.cp);
            }
        }
    } else {
        // rho_i * Phi_i with Phi_i = dx dp 2^-(k_col+sV) S_i, summed exactly (scale 2^k_pot)
        i128 u = 0;
        if (i < N) u = fx128_from_f64(a.rho[i] * (a.dx * a.dp * fx128_to_f64(s, a.k_col + a.sV)), a.k_pot);
        u = warp_sum_i128(u);
        i128* up = static_cast<i128*>(a.upart);
        unsigned int tk = 0;
        if (lane == 0) {
            up[g] = u;
            __threadfence();
            tk = atomicAdd(a.ticket, 1u);
        }
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk != (unsigned int)ngrp - 1) return;
        __threadfence();
        i128 t = 0;
        for (int r = lane; r < ngrp; r += 32) t += ld_i128_cg(up + r);
        t = warp_sum_i128(t);
        if (lane != 0) return;
        *a.ticket = 0u;
        const double U = a.pot_scale * fx128_to_f64(t, a.k_pot);
        const Scalars sc = *a.sc;
        const long long st = *a.step;
        MomentRec rec;
        rec.t = (double)(st + 1) * a.dt;
        rec.mass = sc.mass;
        rec.Mx = sc.Mx;
        rec.My = sc.My;
        rec.kinetic = sc.kinetic;
        rec.potential = U;
        rec.energy = sc.kinetic + U;
        rec.step = st + 1;
        a.hist[st % HIST_CAP] = rec;
        *a.step = st + 1;
        a.sc->potential = U;
    }
}

template <bool POT>
__global__ void __launch_bounds__(RINGFX_THREADS) ringfx_kernel(RingArgs a)
{
    ringfx_body<POT, true>(a, blockIdx.x);
}

// The force of one state (f) and the potential of another (p) in one launch: blocks [0, nf) take
// the force, the rest the potential; each keeps its own scratch and tickets.
__global__ void __launch_bounds__(RINGFX_THREADS) ringfx_dual_kernel(RingArgs f, RingArgs p)
{
    const int nf = ((f.N + 31) / 32) * f.ksplit;
    if ((int)blockIdx.x < nf) ringfx_body<false, true>(f, blockIdx.x);
    else ringfx_body<true>(p, (int)blockIdx.x - nf);
}

cudaError_t launch_ring_fixed_dual(const RingArgs& f, const RingArgs& p, cudaStream_t st)
{
    const int nf = ((f.N + 31) / 32) * f.ksplit;
    ringfx_dual_kernel<<<2 * nf, RINGFX_THREADS, ringfx_smem_bytes(f.N, f.ksplit), st>>>(f, p);
    return cudaGetLastError();
}

// Batched form: blockIdx.y = slot (N = 0: not a ring slot); each slot keeps its own split.
template <bool POT>
__global__ void __launch_bounds__(RINGFX_THREADS) ringfx_batch_kernel(const RingArgs* __restrict__ args)
{
    const RingArgs a = args[blockIdx.y];
    if (a.N <= 0) return;
    ringfx_body<POT>(a, blockIdx.x);
}

// Blocks and shared memory a batched launch needs to cover every slot size N <= max_n (a smaller N
// can take a few more blocks than max_n itself, as the split is rounded).
static void ringfx_batch_shape(int max_n, int nsm, int* blocks, size_t* smem)
{
    *blocks = 1;
    *smem = 0;
    for (int N = 16; N <= max_n; N += 8) {
        const int ks = ringfx_ksplit(N, nsm);
        *blocks = std::max(*blocks, ((N + 31) / 32) * ks);
        *smem = std::max(*smem, ringfx_smem_bytes(N, ks));
    }
}

cudaError_t launch_ring_fixed_batch(bool pot, int slots, int max_n, int nsm, const RingArgs* args, cudaStream_t st)
{
    int blocks = 0;
    size_t smem = 0;
    ringfx_batch_shape(max_n, nsm, &blocks, &smem);
    const dim3 grid(blocks, slots);
    if (pot) ringfx_batch_kernel<true><<<grid, RINGFX_THREADS, smem, st>>>(args);
    else ringfx_batch_kernel<false><<<grid, RINGFX_THREADS, smem, st>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_ring_fixed(const RingArgs& a, cudaStream_t st)
{
    const int ngrp = (a.N + 31) / 32;
    const size_t smem = ringfx_smem_bytes(a.N, a.ksplit);
    if (a.final_moments) ringfx_kernel<true><<<ngrp * a.ksplit, RINGFX_THREADS, smem, st>>>(a);
    else ringfx_kernel<false><<<ngrp * a.ksplit, RINGFX_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

static int ceil_log2_host(double v)
{
    int e = 0;
    const double m = std::frexp(v, &e);   // v = m 2^e, m in [0.5, 1)
    return m == 0.5 ? e - 1 : e;
}

void ring_fixed_tables(int N, double dx, double eps, long long* Kq, long long* Vq, int* sK, int* sV)
{
    // |entry| <= 2^(64 - ceil log2 N): N products with |t_k| < 2^62 stay inside int128
    const int bits = 64 - ceil_log2_host((double)N);
    std::vector<double> dV(N), V(N);
    double mK = 0, mV = 0;
    for (int i = 0; i < N; ++i) {
        const double u = (double)i * dx;
        const double q = 1.0 - std::cos(u) + eps;
        dV[i] = std::sin(u) / (2.0 * std::sqrt(2.0) * q * std::sqrt(q));   // V'(u), Eq. (ringpot)
        V[i] = -1.0 / (std::sqrt(2.0) * std::sqrt(q));                      // V(u)
        mK = std::max(mK, std::fabs(dV[i]));
        mV = std::max(mV, std::fabs(V[i]));
    }
    *sK = bits - ceil_log2_host(mK);
    *sV = bits - ceil_log2_host(mV);
    for (int i = 0; i < N; ++i) {
        Kq[i] = std::llround(std::ldexp(dV[i], *sK));
        Vq[i] = std::llround(std::ldexp(V[i], *sV));
    }
}

// ============================================================================ TENSOR
// The circulant product as a GEMM on the tensor cores.  With N = N1 * 128, output i = a*128 + b and
// input k = c*128 + d, and e = (a - c) mod N1:
//   y[a*128 + b] = sum_e sum_d T_e[b, d] R_e[d, a],   T_e[b, d] = K((e*128 + b - d) mod N),
//                                                      R_e[d, a] = rho[((a - e) mod N1)*128 + d],
// i.e. Y (128 x N1) = [T_0 .. T_{N1-1}] (128 x N) [R_0; ..; R_{N1-1}] (N x N1).  CTA e forms
// T_e R_e with tcgen05.mma (kind::tf32, M = 128, N = N1 padded to 16 or 32, K = 128 in 16 steps of
// 8) on TF32 operands split in high and low parts (3xTF32: hi x hi + hi x lo + lo x hi, accumulated in
// FP32 in tensor memory); the last CTA adds the N1 partial results in a fixed order.  T_e is constant for a
// handle: its TF32 high and low parts are built once on the host as shared-memory images and
// arrive by bulk copy; R_e is gathered from rho by the CTA.  Operands are K-major without swizzle:
// 8-row x 16-byte core matrices, the cores of one 4-element K column contiguous.
__host__ __device__ __forceinline__ uint32_t tc_off(int r, int k, int rows)
{
    return (uint32_t)((k >> 2) * (rows / 8) * 128 + (r >> 3) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

bool ring_tc_ok(int N) { return N % RING_TC_M == 0 && N >= 2 * RING_TC_M && N / RING_TC_M <= RING_TC_N; }

// operand images (T_e high/low, R_e high/low), 1024 bytes of alignment slack, and 4 KB past the last
// operand so that every read a descriptor could address stays inside the allocation
size_t ring_tc_smem_bytes() { return 2 * RING_TC_IMG + 2 * (size_t)RING_TC_N * RING_TC_M * 4 + 1024 + 4096; }

static float tf32_rna_host(float x)
{
    uint32_t b;
    std::memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) != 0x7f800000u) b = (b + 0x1000u) & 0xffffe000u;   // nearest, ties away
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

void ring_tc_tables(const double* table, int N, float* images)
{
    const int N1 = N / RING_TC_M;
    const size_t img = RING_TC_IMG / 4;
    for (int e = 0; e < N1; ++e) {
        float* hi = images + (size_t)(2 * e) * img;
        float* lo = hi + img;
        for (int m = 0; m < RING_TC_M; ++m)
            for (int k = 0; k < RING_TC_M; ++k) {
                int q = (e * RING_TC_M + m - k) % N;
                if (q < 0) q += N;
                const double v = table[q];
                const float h = tf32_rna_host((float)v);
                const uint32_t o = tc_off(m, k, RING_TC_M) / 4;
                hi[o] = h;
                // the low part rounded to TF32 here: the tensor cores would otherwise drop its low
                // 13 bits by truncation, a bias that adds up step after step
                lo[o] = tf32_rna_host((float)(v - (double)h));
            }
    }
}

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor: start, leading-dimension (K) and stride-dimension (M/N) byte
// offsets between core matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

template <bool POT>
__global__ void __launch_bounds__(128, 1) ring_tc_kernel(RingArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_dyn[];
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ int tc_fail;
    __shared__ bool is_last;
    __shared__ i128 red[33];
    const uint32_t raw = smem_u32(tc_smem_dyn);
    unsigned char* sm = tc_smem_dyn + ((1024u - (raw & 1023u)) & 1023u);
    const int N = a.N, N1 = N / RING_TC_M, e = blockIdx.x;
    const int nmma = N1 <= 16 ? 16 : 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* Ahi = reinterpret_cast<float*>(sm);
    float* Bhi = reinterpret_cast<float*>(sm + 2 * RING_TC_IMG);
    float* Blo = Bhi + RING_TC_N * RING_TC_M;

    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        tc_fail = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(32u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned char* src = static_cast<const unsigned char*>(POT ? a.tcV : a.tcK) + (size_t)e * 2 * RING_TC_IMG;
        mbar_arrive_expect_tx(&bar_load, (uint32_t)(2 * RING_TC_IMG));
        bulk_g2s(sm, src, (uint32_t)RING_TC_IMG, &bar_load);
        bulk_g2s(sm + RING_TC_IMG, src + RING_TC_IMG, (uint32_t)RING_TC_IMG, &bar_load);
    }
    // R_e[d, n] for d = tid (this thread's K row), n < nmma (columns past N1 are zero)
#pragma unroll 4
    for (int n = 0; n < nmma; ++n) {
        float h = 0.f, l = 0.f;
        if (n < N1) {
            int c = n - e;
            c += (c < 0) ? N1 : 0;
            const double r = a.rho[c * RING_TC_M + tid];
            h = tf32_rna((float)r);
            l = tf32_rna((float)(r - (double)h));
        }
        const uint32_t o = tc_off(n, tid, nmma) / 4;
        Bhi[o] = h;
        Blo[o] = l;
    }
    fence_proxy_async_smem();   // the generic-proxy writes of R_e, before the tensor cores read them
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (tid == 0) {
        if (mbar_wait_bounded(&bar_load, 0u, WAIT_LIMIT_NS)) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) |
                                   ((uint32_t)(RING_TC_M >> 4) << 24);
            const uint32_t a_hi = smem_u32(Ahi), a_lo = a_hi + (uint32_t)RING_TC_IMG;
            const uint32_t b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
            const uint32_t a_lbo = (RING_TC_M / 8) * 128, b_lbo = (uint32_t)(nmma / 8) * 128;
            // three products of the split operands (lo x lo, 2^-22 of each term, measured to change
            // nothing: the FP32 accumulation in the tensor cores sets the accuracy)
            const uint32_t as[3] = {a_hi, a_hi, a_lo}, bs[3] = {b_hi, b_lo, b_hi};
            for (int p = 0; p < 3; ++p)
                for (int s = 0; s < RING_TC_M / 8; ++s)
                    tc_mma(tmem, tc_desc(as[p] + 2u * s * a_lbo, a_lbo, 128u), tc_desc(bs[p] + 2u * s * b_lbo, b_lbo, 128u),
                           idesc, (p | s) != 0 ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar_mma))
                         : "memory");
        } else {
            tc_fail = 1;
            atomicCAS(a.err, DEV_ERR_NONE, DEV_ERR_RING_WAIT);
            mbar_wait_bounded(&bar_load, 0u, WAIT_LIMIT_NS);   // the copies must land before exit
            mbar_arrive(&bar_mma);
        }
    }
    const bool done = mbar_wait_bounded(&bar_mma, 0u, WAIT_LIMIT_NS);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (done && !tc_fail) {
        uint32_t y[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]), "=r"(y[7]),
              "=r"(y[8]), "=r"(y[9]), "=r"(y[10]), "=r"(y[11]), "=r"(y[12]), "=r"(y[13]), "=r"(y[14]), "=r"(y[15])
            : "r"(taddr));
        if (nmma > 16)
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(y[16]), "=r"(y[17]), "=r"(y[18]), "=r"(y[19]), "=r"(y[20]), "=r"(y[21]), "=r"(y[22]),
                  "=r"(y[23]), "=r"(y[24]), "=r"(y[25]), "=r"(y[26]), "=r"(y[27]), "=r"(y[28]), "=r"(y[29]),
                  "=r"(y[30]), "=r"(y[31])
                : "r"(taddr + 16u));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // this block's partial results into the exact fixed-point sums (order-free, so deterministic)
        const int m = warp * 32 + lane;   // output row b of this block
        const float sc = __int_as_float((127 + a.tcq) << 23);   // 2^tcq
        for (int n = 0; n < N1; ++n)
            atomicAdd(reinterpret_cast<unsigned long long*>(a.tcacc) + n * RING_TC_M + m,
                      (unsigned long long)__float2ll_rn(__uint_as_float(y[n]) * sc));
    } else if (tid == 0 && !done) {
        atomicCAS(a.err, DEV_ERR_NONE, DEV_ERR_RING_WAIT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u) : "memory");

    // the last CTA adds the N1 partial results in block order
    if (tid == 0) {
        __threadfence();
        is_last = atomicAdd(a.tcticket, 1u) == (unsigned int)N1 - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // every block has added its partial results: convert, and clear the sums for the next launch
    i128 u = 0;
    const double unit = ldexp(1.0, -a.tcq);
    for (int i = tid; i < N; i += blockDim.x) {
        const double sum = (double)__ldcg(a.tcacc + i) * unit;
        a.tcacc[i] = 0;
        if constexpr (!POT) a.F[i] = -a.dx * sum;
        else u += fx128_from_f64(a.rho[i] * (a.dx * sum), a.k_pot);
    }
    if constexpr (POT) u = block_sum_i128(u, red);
    if (tid != 0) return;
    *a.tcticket = 0u;
    if constexpr (POT) {
        const double U = a.pot_scale * fx128_to_f64(u, a.k_pot);
        const Scalars sc = *a.sc;
        const long long st = *a.step;
        MomentRec rec;
        rec.t = (double)(st + 1) * a.dt;
        rec.mass = sc.mass;
        rec.Mx = sc.Mx;
        rec.My = sc.My;
        rec.kinetic = sc.kinetic;
        rec.potential = U;
        rec.energy = sc.kinetic + U;
        rec.step = st + 1;
        a.hist[st % HIST_CAP] = rec;
        *a.step = st + 1;
        a.sc->potential = U;
    }
}

cudaError_t launch_ring_tc(const RingArgs& a, cudaStream_t st)
{
    const int grid = a.N / RING_TC_M;
    if (a.final_moments) ring_tc_kernel<true><<<grid, 128, ring_tc_smem_bytes(), st>>>(a);
    else ring_tc_kernel<false><<<grid, 128, ring_tc_smem_bytes(), st>>>(a);
    return cudaGetLastError();
}

// ============================================================================ FFT
bool ring_fft_ok(int N) { return N >= 16 && N <= 4096 && (N & (N - 1)) == 0; }

size_t ring_fft_smem_bytes(int N, bool f64) { return (size_t)2 * N * (f64 ? 16 : 8); }

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// Stockham radix-2 transform of the N points in `a` (N a power of two), using `b` as the other
// buffer; returns the buffer that holds the result (natural order).  Unnormalised; inverse = the
// conjugate twiddles.  tw[m] = exp(-2 pi i m / N), m < N/2.
template <typename T2>
__device__ T2* stockham(T2* a, T2* b, int N, const T2* __restrict__ tw, bool inverse)
{
    const int half = N >> 1;
    for (int Ns = 1; Ns < N; Ns <<= 1) {
        const int stride = half / Ns;
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int k = j & (Ns - 1);
            T2 w = tw[k * stride];
            if (inverse) w.y = -w.y;
            const T2 u = a[j];
            const T2 v = cmul(a[j + half], w);
            const int o = ((j - k) << 1) + k;   // (j / Ns) * 2 Ns + k
            T2 p, m;
            p.x = u.x + v.x;
            p.y = u.y + v.y;
            m.x = u.x - v.x;
            m.y = u.y - v.y;
            b[o] = p;
            b[o + Ns] = m;
        }
        __syncthreads();
        T2* t = a;
        a = b;
        b = t;
    }
    return a;
}

// One CTA: FFT of rho; the force by the inverse transform of FFT(V') FFT(rho), or the potential by
// Parseval with FFT(V) (then the moment record, as the other methods write it).
template <typename T, typename T2>
__global__ void __launch_bounds__(RING_FFT_THREADS) ring_fft_kernel(RingArgs a)
{
    extern __shared__ __align__(16) unsigned char rfft_smem[];
    __shared__ i128 red[33];
    T2* A = reinterpret_cast<T2*>(rfft_smem);
    T2* B = A + a.N;
    const int N = a.N;
    const T2* __restrict__ tw = static_cast<const T2*>(a.twid);
    for (int i = threadIdx.x; i < N; i += RING_FFT_THREADS) {
        T2 z;
        z.x = (T)a.rho[i];
        z.y = T(0);
        A[i] = z;
    }
    __syncthreads();
    T2* R = stockham(A, B, N, tw, false);
    T2* S = (R == A) ? B : A;
    if (!a.final_moments) {
        const T2* __restrict__ kh = static_cast<const T2*>(a.khat);
        for (int k = threadIdx.x; k < N; k += RING_FFT_THREADS) R[k] = cmul(R[k], kh[k]);
        __syncthreads();
        const T2* out = stockham(R, S, N, tw, true);
        const double scale = -a.dx / (double)N;
        for (int i = threadIdx.x; i < N; i += RING_FFT_THREADS) a.F[i] = scale * (double)out[i].x;
        return;
    }
    // the terms rho_i (dx sum_k V_{i-k} rho_k) the other methods add, by Parseval:
    // sum_i rho_i dx (V * rho)_i = dx / N sum_k |R_k|^2 Vhat_k; summed exactly at scale 2^k_pot
    const T2* __restrict__ vh = static_cast<const T2*>(a.vhat);
    const double c = a.dx / (double)N;
    i128 u = 0;
    for (int k = threadIdx.x; k < N; k += RING_FFT_THREADS) {
        const double re = (double)R[k].x, im = (double)R[k].y;
        u += fx128_from_f64((re * re + im * im) * (double)vh[k].x * c, a.k_pot);
    }
    u = block_sum_i128(u, red);
    if (threadIdx.x != 0) return;
    const double U = a.pot_scale * fx128_to_f64(u, a.k_pot);
    const Scalars sc = *a.sc;
    const long long st = *a.step;
    MomentRec rec;
    rec.t = (double)(st + 1) * a.dt;
    rec.mass = sc.mass;
    rec.Mx = sc.Mx;
    rec.My = sc.My;
    rec.kinetic = sc.kinetic;
    rec.potential = U;
    rec.energy = sc.kinetic + U;
    rec.step = st + 1;
    a.hist[st % HIST_CAP] = rec;
    *a.step = st + 1;
    a.sc->potential = U;
}

cudaError_t launch_ring_fft(bool f64, const RingArgs& a, cudaStream_t st)
{
    const size_t smem = ring_fft_smem_bytes(a.N, f64);
    if (f64) ring_fft_kernel<double, double2><<<1, RING_FFT_THREADS, smem, st>>>(a);
    else ring_fft_kernel<float, float2><<<1, RING_FFT_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t set_ringfx_attributes(int max_smem)
{
    cudaError_t e = allow_dynamic_smem(ringfx_kernel<false>, max_smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(ringfx_kernel<true>, max_smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(ringfx_dual_kernel, max_smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(ringfx_batch_kernel<false>, max_smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(ringfx_batch_kernel<true>, max_smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(ring_fft_kernel<double, double2>, max_smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(ring_fft_kernel<float, float2>, max_smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(ring_tc_kernel<false>, max_smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(ring_tc_kernel<true>, max_smem);
    return e;
}

// Host DFT of a real table: out[2k] + i out[2k+1] = sum_m v_m exp(-2 pi i m k / N), with an FP64
// twiddle table and Neumaier-compensated sums (used once per handle for the FFT method's spectra).
void ring_dft_host(const double* v, int N, double* out)
{
    std::vector<double> c(N), s(N);
    for (int r = 0; r < N; ++r) {
        const double ang = 2.0 * 3.14159265358979323846 * (double)r / (double)N;
        c[r] = std::cos(ang);
        s[r] = -std::sin(ang);
    }
    auto add = [](double& sum, double& comp, double x) {
        const double t = sum + x;
        if (std::fabs(sum) >= std::fabs(x)) comp += (sum - t) + x;
        else comp += (x - t) + sum;
        sum = t;
    };
    for (int k = 0; k < N; ++k) {
        double re = 0, rc = 0, im = 0, ic = 0;
        long long r = 0;
        for (int m = 0; m < N; ++m) {
            add(re, rc, v[m] * c[r]);
            add(im, ic, v[m] * s[r]);
            r += k;
            if (r >= N) r -= N;
        }
        out[2 * k] = re + rc;
        out[2 * k + 1] = im + ic;
    }
}

}  // namespace vl
