// aux_kernels.cu -- density and moment reductions, the three mean-field forces, the p-shift
// line parameters, and small utility kernels.
//
// Density (Sec. 2): rho_i = dp sum_j f[j,i], assembled from the per-CTA column partials written
// by the x-shift epilogue.  Moments: mass = dx sum rho, Mx, My = dx sum cos/sin(x_i) rho_i
// (Eq. mxmydef), kinetic = dx dp sum_j p_j^2/2 sum_i f.  Forces, Eq. (meanforce) by the rectangle
// rule:
//   HMF   (Eq. hmfmeanforce): F_i = -Mx sin x_i + My cos x_i
//   ring  (Eq. ringpot):      F_i = -dx sum_k V'((i-k) dx) rho_k   (circulant)
//   sheet (V = 2 pi G |x|):   F_i = -2 pi G dx (sum_{k<i} rho_k - sum_{k>i} rho_k)  (prefix scan)
// Every sum across threads is an exact integer fixed-point sum (fixed_point.cuh): deterministic,
// order-free, and without the long dependent FP64 chains that are slow on this GPU.
#include "emul.cuh"
#include "fixed_point.cuh"
#include "pparams.cuh"
#include "ptx.cuh"
#include <cuda_bf16.h>
#include "vlasov_internal.cuh"

namespace vl {

constexpr int CR_COLS = 32;      // columns per colreduce block
constexpr int CR_GROUPS = 8;     // partial-row groups per block (blockDim = 256)
constexpr int CR_ACC_THREADS = 1024;   // single-CTA reduction of exact column sums

__device__ __forceinline__ i128 shfl_up_i128(i128 v, int o)
{
    const uint64_t lo = (uint64_t)v, hi = (uint64_t)((u128)v >> 64);
    const uint64_t l2 = (uint64_t)__shfl_up_sync(0xffffffffu, (long long)lo, o);
    const uint64_t h2 = (uint64_t)__shfl_up_sync(0xffffffffu, (long long)hi, o);
    return (i128)(((u128)h2 << 64) | (u128)l2);
}

// Exclusive scan of one int128 per thread across the block (blockDim <= 1024); returns the prefix
// and writes the block total to *total.  `sh` holds >= 33 entries.
__device__ i128 block_exclusive_scan_i128(i128 v, i128* sh, i128* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    i128 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const i128 t = shfl_up_i128(inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        i128 run = 0;
        for (int w = 0; w < nw; ++w) {
            const i128 t = sh[w];
            sh[w] = run;
            run += t;
        }
        sh[32] = run;
    }
    __syncthreads();
    const i128 r = sh[wid] + inc - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// Totals of one sweep in one CTA: per-thread partials m, x, y (mass, cos-, sin-weighted column
// sums) are added exactly across the block, with the kinetic partials; then the sheet prefix scan,
// the scalars and (after the second x-shift) the moment record.
__device__ __forceinline__ void colreduce_final(const ColReduceArgs& a, i128 m, i128 x, i128 y, i128* red)
{
    const long long step0 = (threadIdx.x == 0 && a.final_moments) ? __ldcg(a.step) : 0;   // read early
    i128 k = 0;
    if (a.kinpart) {
        double kv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = threadIdx.x + u * blockDim.x;
            kv[u] = b < a.B ? __ldcg(&a.kinpart[b]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) k += fx128_from_f64(kv[u], a.k_kin);
        for (int b = threadIdx.x + 4 * blockDim.x; b < a.B; b += blockDim.x) k += fx128_from_f64(__ldcg(&a.kinpart[b]), a.k_kin);
    } else if (a.kin128) {
        const i128* kp = static_cast<const i128*>(a.kin128);
        for (int b = threadIdx.x; b < a.B; b += blockDim.x) k += kp[b];
    }
    {
        __shared__ i128 red4[128];
        block_sum4_i128(m, x, y, k, red4);
    }

    i128 U_acc = 0;
    if (a.model == 2) {
        // Sheet: C_i = sum_{k<i} s_k (exact); Q_i = 2 C_i + s_i - S gives F_i = -2 pi G dx dp Q_i.
        const int nt = blockDim.x;
        const int per = (a.Nx + nt - 1) / nt;
        const int lo = min(a.Nx, (int)threadIdx.x * per), hi = min(a.Nx, lo + per);
        i128 ls = 0, lx = 0;
        for (int q = lo; q < hi; ++q) {
            const long long v = __ldcg(&a.colfx[q]);
            ls += v;
            lx += (i128)q * v;
        }
        i128 S = 0, XS = 0;
        i128 C = block_exclusive_scan_i128(ls, red, &S);
        i128 X = block_exclusive_scan_i128(lx, red, &XS);
        for (int q = lo; q < hi; ++q) {
            const long long v = __ldcg(&a.colfx[q]);
            a.Qd[q] = fx128_to_f64(2 * C + (i128)v - S, a.k_col);
            if (a.final_moments) {
                // U = 2 pi G dx^3 sum_i rho_i sum_{k<i} (i-k) rho_k
                const double r = fx128_to_f64((i128)v, a.k_col);
                const double wgt = fx128_to_f64((i128)q * C - X, a.k_col);
                U_acc += fx128_from_f64(r * wgt, a.k_pot);
            }
            C += v;
            X += (i128)q * v;
        }
        if (a.final_moments) U_acc = block_sum_i128(U_acc, red);
    }

    if (threadIdx.x == 0) {
        const double mass = a.dxdp * fx128_to_f64(m, a.k_col);
        const double Mx = a.dxdp * fx128_to_f64(x, a.k_col + 30);
        const double My = a.dxdp * fx128_to_f64(y, a.k_col + 30);
        const double kin = a.dxdp * fx128_to_f64(k, a.kinpart ? a.k_kin : a.kin_frac);
        double U = 0.0;
        if (a.model == 0) U = 0.5 * (mass * mass - Mx * Mx - My * My);
        else if (a.model == 2 && a.final_moments) U = a.pot_scale * fx128_to_f64(U_acc, a.k_pot);
        a.sc->mass = mass;
        a.sc->Mx = Mx;
        a.sc->My = My;
        a.sc->kinetic = kin;
        a.sc->potential = U;
        if (a.final_moments && a.model != 1) {
            const long long st = step0;
            MomentRec rec;
            rec.t = (double)(st + 1) * a.dt;
            rec.mass = mass;
            rec.Mx = Mx;
            rec.My = My;
            rec.kinetic = kin;
            rec.potential = U;
            rec.energy = kin + U;
            rec.step = st + 1;
            a.hist[st % HIST_CAP] = rec;
            *a.step = st + 1;
        }
        *a.ticket = 0u;   // ready for the next launch
    }
}


// ============================================================================ colreduce
// Block: 32 columns x 8 groups over the B partial rows.  Each partial becomes an int64 on the
// column scale, so the column sum is exact; then int128 block partials of mass, Mx, My.  The last
// block to finish (ticket) adds those, the kinetic partials, runs the sheet prefix scan, and writes
// the scalars and (after the second x-shift) the moment record.
__device__ __forceinline__ void colreduce_body(const ColReduceArgs& a)
{
    __shared__ long long shc[CR_GROUPS][CR_COLS];
    __shared__ i128 red[33];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int i = blockIdx.x * CR_COLS + lane;
    const int nblk = (a.Nx + CR_COLS - 1) / CR_COLS;   // blocks that take part (the grid may be larger)
    if ((int)blockIdx.x >= nblk) return;

    // all loads of a thread are independent: issue them in batches of eight
    long long s = 0;
    if (a.colacc) {
        // exact column sums were added by the x-shift CTAs; take them and clear for the next sweep
        if (grp == 0 && i < a.Nx) {
            s = (long long)a.colacc[i];
            a.colacc[i] = 0ull;
        }
    } else if (a.colpart64) {
        // exact per-CTA partial rows (already on the column scale): plain int64 sums
        if (i < a.Nx) {
            const long long* __restrict__ cp = a.colpart64 + i;
            int b = grp;
            for (; b + 7 * CR_GROUPS < a.B; b += 8 * CR_GROUPS) {
                long long v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcs(cp + (size_t)(b + u * CR_GROUPS) * a.Nx);
#pragma unroll
                for (int u = 0; u < 8; ++u) s += v[u];
            }
            for (; b < a.B; b += CR_GROUPS) s += __ldcs(cp + (size_t)b * a.Nx);
        }
    } else if (i < a.Nx) {
        const double* __restrict__ cp = a.colpart + i;
        const size_t st = (size_t)a.Nx * CR_GROUPS;
        int b = grp;
        for (; b + 7 * CR_GROUPS < a.B; b += 8 * CR_GROUPS) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcs(cp + (size_t)b * a.Nx + u * st);
#pragma unroll
            for (int u = 0; u < 8; ++u) s += (long long)fx128_from_f64(v[u], a.k_col);
        }
        for (; b < a.B; b += CR_GROUPS) s += (long long)fx128_from_f64(__ldcs(cp + (size_t)b * a.Nx), a.k_col);
    }
    shc[grp][lane] = s;
    __syncthreads();
    i128 cm = 0, cx = 0, cy = 0;
    if (grp == 0 && i < a.Nx) {
        long long t = 0;
#pragma unroll
        for (int q = 0; q < CR_GROUPS; ++q) t += shc[q][lane];
        a.colfx[i] = t;
        a.rho[i] = a.dp * fx128_to_f64((i128)t, a.k_col);
        cm = (i128)t;
        const i128 half = (i128)1 << 31;
        cx = ((i128)a.cosfx[i] * (i128)t + half) >> 32;   // scale 2^-(k_col + 30)
        cy = ((i128)a.sinfx[i] * (i128)t + half) >> 32;
    }
    cm = block_sum_i128(cm, red);
    cx = block_sum_i128(cx, red);
    cy = block_sum_i128(cy, red);
    i128* bp = static_cast<i128*>(a.blockpart);
    if (threadIdx.x == 0) {
        bp[blockIdx.x * 3 + 0] = cm;
        bp[blockIdx.x * 3 + 1] = cx;
        bp[blockIdx.x * 3 + 2] = cy;
        __threadfence();
        const unsigned int tk = atomicAdd(a.ticket, 1u);
        is_last = (tk == (unsigned int)nblk - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    // ---- last block: totals (exact, any order)
    i128 m = 0, x = 0, y = 0;
    const volatile i128* vb = bp;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        m += vb[b * 3 + 0];
        x += vb[b * 3 + 1];
        y += vb[b * 3 + 2];
    }
    colreduce_final(a, m, x, y, red);
}

// Single-CTA form for the exact int64 column sums the 8-byte x-shifts add with atomics: one pass
// over the Nx columns (take, clear, density, cos/sin-weighted sums) and the totals, with no
// second round of blocks.
__device__ __forceinline__ void colreduce_acc_body(const ColReduceArgs& a)
{
    __shared__ i128 red[33];
    i128 m = 0, x = 0, y = 0;
    const i128 half = (i128)1 << 31;
    constexpr int U = 4;   // all loads of a round are issued before any store (no aliasing stalls)
    for (int i0 = threadIdx.x; i0 < a.Nx; i0 += U * blockDim.x) {
        long long t[U], c[U], sn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            const bool in = i < a.Nx;
            t[u] = in ? (long long)__ldcg(a.colacc + i) : 0ll;
            c[u] = in ? __ldg(a.cosfx + i) : 0ll;
            sn[u] = in ? __ldg(a.sinfx + i) : 0ll;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < a.Nx) {
                a.colacc[i] = 0ull;
                if (a.model == 2 || a.model == 1) a.colfx[i] = t[u];                   // sheet scan / ring fixed-point input
                if (a.model == 1) a.rho[i] = a.dp * fx128_to_f64((i128)t[u], a.k_col);   // ring: convolution input
            }
            m += (i128)t[u];
            x += ((i128)c[u] * (i128)t[u] + half) >> 32;   // scale 2^-(k_col + 30)
            y += ((i128)sn[u] * (i128)t[u] + half) >> 32;
        }
    }
    colreduce_final(a, m, x, y, red);
}

__global__ void __launch_bounds__(256) colreduce_kernel(ColReduceArgs a)
{
    colreduce_body(a);
}

__global__ void __launch_bounds__(256) colreduce_batch_kernel(const ColReduceArgs* __restrict__ args)
{
    const ColReduceArgs a = args[blockIdx.y];
    if (a.Nx <= 0) return;
    colreduce_body(a);
}

__global__ void __launch_bounds__(CR_ACC_THREADS) colreduce_acc_kernel(ColReduceArgs a)
{
    colreduce_acc_body(a);
}

// Exact per-CTA partial rows (int64, column scale): 32 columns x 32 row groups per block, so each
// thread adds only about B/32 partials; warp 0 forms the block's mass and cos/sin-weighted sums with
// shuffles, and the last block to finish computes the totals (colreduce_final).
constexpr int CRP_THREADS = 1024;
__device__ __forceinline__ void colreduce_p64_body(const ColReduceArgs& a, int bx)
{
    __shared__ long long shc[32][33];
    __shared__ i128 red[33];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int i = bx * 32 + lane;
    const int nblk = (a.Nx + 31) / 32;
    if (bx >= nblk) return;
    long long s = 0;
    if (i < a.Nx) {
        const long long* __restrict__ cp = a.colpart64 + i;
        int b = grp;
        for (; b + 3 * 32 < a.B; b += 4 * 32) {
            long long v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcs(cp + (size_t)(b + u * 32) * a.Nx);
#pragma unroll
            for (int u = 0; u < 4; ++u) s += v[u];
        }
        for (; b < a.B; b += 32) s += __ldcs(cp + (size_t)b * a.Nx);
    }
    shc[grp][lane] = s;
    __syncthreads();
    i128* bp = static_cast<i128*>(a.blockpart);
    if (grp == 0) {
        i128 cm = 0, cx = 0, cy = 0;
        if (i < a.Nx) {
            long long t = 0;
#pragma unroll 8
            for (int q = 0; q < 32; ++q) t += shc[q][lane];
            a.colfx[i] = t;
            a.rho[i] = a.dp * fx128_to_f64((i128)t, a.k_col);
            const i128 half = (i128)1 << 31;
            cm = (i128)t;
            cx = ((i128)a.cosfx[i] * (i128)t + half) >> 32;   // scale 2^-(k_col + 30)
            cy = ((i128)a.sinfx[i] * (i128)t + half) >> 32;
        }
        cm = warp_sum_i128(cm);
        cx = warp_sum_i128(cx);
        cy = warp_sum_i128(cy);
        if (lane == 0) {
            bp[bx * 3 + 0] = cm;
            bp[bx * 3 + 1] = cx;
            bp[bx * 3 + 2] = cy;
            __threadfence();
            is_last = atomicAdd(a.ticket, 1u) == (unsigned int)nblk - 1;
        }
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    i128 m = 0, x = 0, y = 0;
    const volatile i128* vb = bp;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        m += vb[b * 3 + 0];
        x += vb[b * 3 + 1];
        y += vb[b * 3 + 2];
    }
    colreduce_final(a, m, x, y, red);
}

__global__ void __launch_bounds__(CRP_THREADS) colreduce_p64_kernel(ColReduceArgs a)
{
    colreduce_p64_body(a, blockIdx.x);
}

// Two independent reductions of exact per-CTA partial rows in one launch (blocks [0, nblk) take a,
// the rest b); each keeps its own outputs, scratch and ticket.
__global__ void __launch_bounds__(CRP_THREADS) colreduce_p64_dual_kernel(ColReduceArgs a, ColReduceArgs b)
{
    const int nblk = (a.Nx + 31) / 32;
    if ((int)blockIdx.x < nblk) colreduce_p64_body(a, blockIdx.x);
    else colreduce_p64_body(b, (int)blockIdx.x - nblk);
}

cudaError_t launch_colreduce_p64_dual(const ColReduceArgs& a, const ColReduceArgs& b, cudaStream_t st)
{
    const int nblk = (a.Nx + 31) / 32;
    colreduce_p64_dual_kernel<<<2 * nblk, CRP_THREADS, 0, st>>>(a, b);
    return cudaGetLastError();
}

cudaError_t launch_colreduce(const ColReduceArgs& a, int grid, cudaStream_t st)
{
    if (a.colacc) colreduce_acc_kernel<<<1, CR_ACC_THREADS, 0, st>>>(a);
    else if (a.colpart64) colreduce_p64_kernel<<<(a.Nx + 31) / 32, CRP_THREADS, 0, st>>>(a);
    else colreduce_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_colreduce_batch(int slots, int blocks_per_slot, const ColReduceArgs* args, cudaStream_t st)
{
    colreduce_batch_kernel<<<dim3(blocks_per_slot, slots), 256, 0, st>>>(args);
    return cudaGetLastError();
}

// ============================================================================ ring force
// F_i = -dx sum_k V'(((i-k) mod N) dx) rho_k, or after the last x-shift Phi_i = dx sum_k V(...) rho_k
// and U = 1/2 dx sum_i rho_i Phi_i (exact int128 sum).  A block stages rho in shared memory in the
// arithmetic type T (double for FP64 storage, float for FP32 storage), with the kernel table beside
// it, and produces RING_OUT outputs, RING_OUT / 8 per warp, lanes striding over k.  Few outputs
// per block spread the N^2 multiply-adds over every SM (FP64 ones run on the slow FP64 pipe).
constexpr int RING_OUT = 16;
constexpr int RING_OPW = RING_OUT / 8;

template <typename T>
__device__ __forceinline__ void ring_body(const RingArgs& a)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    T* rs = reinterpret_cast<T*>(ring_smem);
    __shared__ i128 red[33];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int N = a.N;
    const int nblk = (N + RING_OUT - 1) / RING_OUT;
    if ((int)blockIdx.x >= nblk) return;
    T* ks = rs + N;   // the kernel table V' (force) or V (potential) by index difference
    const T* __restrict__ ker = static_cast<const T*>(a.final_moments ? a.V : a.dV);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        rs[k] = (T)a.rho[k];
        ks[k] = ker[k];
    }
    __syncthreads();
    const int i0 = blockIdx.x * RING_OUT + wid * RING_OPW;
    T acc[RING_OPW];
#pragma unroll
    for (int q = 0; q < RING_OPW; ++q) acc[q] = T(0);
    int iq[RING_OPW];
#pragma unroll
    for (int q = 0; q < RING_OPW; ++q) iq[q] = (i0 + q < N) ? i0 + q : 0;   // outputs past N: dummy, unused
    for (int k = lane; k < N; k += 32) {
        const T r = rs[k];
#pragma unroll
        for (int q = 0; q < RING_OPW; ++q) {
            int m = iq[q] - k;          // in (-N, N)
            m += (m < 0) ? N : 0;
            acc[q] = fma(ks[m], r, acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < RING_OPW; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    i128 up = 0;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < RING_OPW; ++q) {
            const int i = i0 + q;
            if (i < N) {
                if (a.final_moments) up += fx128_from_f64(a.rho[i] * (a.dx * (double)acc[q]), a.k_pot);
                else a.F[i] = -a.dx * (double)acc[q];
            }
        }
    }
    if (!a.final_moments) return;
    up = block_sum_i128(up, red);
    i128* bp = static_cast<i128*>(a.blockpart);
    if (threadIdx.x == 0) {
        bp[blockIdx.x] = up;
        __threadfence();
        const unsigned int tk = atomicAdd(a.ticket, 1u);
        is_last = (tk == (unsigned int)nblk - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    i128 u = 0;
    const volatile i128* vb = bp;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) u += vb[b];
    u = block_sum_i128(u, red);
    if (threadIdx.x != 0) return;
    *a.ticket = 0u;
    const double U = a.pot_scale * fx128_to_f64(u, a.k_pot);
    const Scalars s = *a.sc;
    const long long st = *a.step;
    MomentRec rec;
    rec.t = (double)(st + 1) * a.dt;
    rec.mass = s.mass;
    rec.Mx = s.Mx;
    rec.My = s.My;
    rec.kinetic = s.kinetic;
    rec.potential = U;
    rec.energy = s.kinetic + U;
    rec.step = st + 1;
    a.hist[st % HIST_CAP] = rec;
    *a.step = st + 1;
    a.sc->potential = U;
}

template <typename T>
__global__ void __launch_bounds__(256) ring_kernel(RingArgs a)
{
    ring_body<T>(a);
}

int ring_blocks(int N) { return (N + RING_OUT - 1) / RING_OUT; }

// The ring kernels stage rho and the kernel table: 2 N elements of shared memory (64 KB at N = 4096
// in FP64).
cudaError_t set_ring_attributes(int max_smem)
{
    cudaError_t e = cudaFuncSetAttribute(ring_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ring_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
}

cudaError_t launch_ring(int elem_bytes, const RingArgs& a, cudaStream_t st)
{
    const int grid = ring_blocks(a.N);
    if (elem_bytes == 8) ring_kernel<double><<<grid, 256, (size_t)a.N * 16, st>>>(a);
    else ring_kernel<float><<<grid, 256, (size_t)a.N * 8, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
__device__ __forceinline__ void pparams_body(const PParamsArgs& a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.Nx) return;
    double F;
    if (a.model == 0) F = -a.sc->Mx * a.sintab[i] + a.sc->My * a.costab[i];
    else if (a.model == 3) F = 0.0;
    else if (a.model == 2) F = a.Fscale * a.Fin[i];
    else F = a.Fin[i];
    if (a.Fout) a.Fout[i] = F;
    const double sigma = F * a.cp;
    if constexpr (sizeof(T) == 8) pparams_fixed(a, i, sigma);
    else pparams_f32(a, i, sigma);
}

template <typename T>
__global__ void __launch_bounds__(64) pparams_kernel(PParamsArgs a)
{
    pparams_body<T>(a);
}

template <typename T>
__global__ void __launch_bounds__(64) pparams_batch_kernel(const PParamsArgs* __restrict__ args)
{
    const PParamsArgs a = args[blockIdx.y];
    pparams_body<T>(a);
}

cudaError_t launch_pparams_batch(int elem_bytes, int slots, int max_n, const PParamsArgs* args, cudaStream_t st)
{
    const dim3 grid((max_n + 63) / 64, slots);
    if (elem_bytes == 8) pparams_batch_kernel<double><<<grid, 64, 0, st>>>(args);
    else pparams_batch_kernel<float><<<grid, 64, 0, st>>>(args);
    return cudaGetLastError();
}

// Exact totals of the x-shift's per-CTA HMF partials, in every thread of the block.
__device__ __forceinline__ void sum_ctaparts(const void* parts, int ctas, i128& m, i128& x, i128& y, i128* red4)
{
    const i128* p = static_cast<const i128*>(parts);
    m = 0;
    x = 0;
    y = 0;
    i128 z = 0;
    for (int b = threadIdx.x; b < ctas; b += blockDim.x) {
        m += p[(size_t)b * 3 + 0];
        x += p[(size_t)b * 3 + 1];
        y += p[(size_t)b * 3 + 2];
    }
    block_sum4_i128(m, x, y, z, red4);
}

// HMF after the first x-shift: Mx, My from the per-CTA partials (the same exact integers in every
// block), then F_i = -Mx sin x_i + My cos x_i and the p-shift parameters of the block's columns.
constexpr int PPC_THREADS = 256;
template <typename T>
__global__ void __launch_bounds__(PPC_THREADS) pparams_hmf_cta_kernel(PParamsArgs a)
{
    __shared__ i128 red4[128];
    i128 m, x, y;
    sum_ctaparts(a.ctapart, a.ctas, m, x, y, red4);
    const int i = blockIdx.x * PPC_THREADS + threadIdx.x;
    if (i >= a.Nx) return;
    const double Mx = a.dxdp * fx128_to_f64(x, 101 - a.Ef);
    const double My = a.dxdp * fx128_to_f64(y, 101 - a.Ef);
    const double F = hmf_force(Mx, My, a.sintab[i], a.costab[i]);
    if (a.Fout) a.Fout[i] = F;
    if constexpr (sizeof(T) == 8) pparams_fixed(a, i, F * a.cp);
    else pparams_f32(a, i, F * a.cp);
}

cudaError_t launch_pparams_hmf_cta(int elem_bytes, const PParamsArgs& a, cudaStream_t st)
{
    const int grid = (a.Nx + PPC_THREADS - 1) / PPC_THREADS;
    if (elem_bytes == 8) pparams_hmf_cta_kernel<double><<<grid, PPC_THREADS, 0, st>>>(a);
    else pparams_hmf_cta_kernel<float><<<grid, PPC_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

// x * 2^s rounded (s < 0: round half up), exact in int128.
__device__ __forceinline__ i128 shift_round(i128 x, int s)
{
    if (s >= 0) return x << s;
    return (x + ((i128)1 << (-s - 1))) >> (-s);
}

// HMF moments after the second x-shift: totals of the per-CTA partials on the scales of
// colreduce_final (2^-k_col and 2^-(k_col+30)), then the kinetic partials, U and the record.
__global__ void __launch_bounds__(256) colreduce_cta_kernel(ColReduceArgs a)
{
    __shared__ i128 red4[128];
    __shared__ i128 red[33];
    i128 m, x, y;
    sum_ctaparts(a.ctapart, a.B, m, x, y, red4);
    m = shift_round(m, a.k_col + a.Ef - 51);
    x = shift_round(x, a.k_col + a.Ef - 71);
    y = shift_round(y, a.k_col + a.Ef - 71);
    if (threadIdx.x != 0) {   // colreduce_final adds the block's values: hand them to one thread
        m = 0;
        x = 0;
        y = 0;
    }
    colreduce_final(a, m, x, y, red);
}

cudaError_t launch_colreduce_cta(const ColReduceArgs& a, cudaStream_t st)
{
    colreduce_cta_kernel<<<1, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pparams(int elem_bytes, const PParamsArgs& a, cudaStream_t st)
{
    const int grid = (a.Nx + 63) / 64;
    if (elem_bytes == 8) pparams_kernel<double><<<grid, 64, 0, st>>>(a);
    else pparams_kernel<float><<<grid, 64, 0, st>>>(a);
    return cudaGetLastError();
}

// ============================================================================ Casimirs
// Eq. (casimirs) for s(f) = -f log f (the entropy of Secs. 4.1-4.2) and s(f) = f^2, on the stored f:
// per-thread FP64 sums over a fixed grid-stride set of cells, fixed-order block sums, one partial
// pair per block; casimir_final_kernel adds the partials in block order.  Deterministic.
// kind 0: FX64 cells (unit = 2^(Ef-61)), 1: double, 2: float, 3: bf16.
constexpr int CAS_THREADS = 256;

template <int KIND>
__global__ void __launch_bounds__(CAS_THREADS) casimir_kernel(const void* __restrict__ f, size_t n, double unit,
                                                               double* __restrict__ part)
{
    double s = 0.0, q = 0.0;
    for (size_t k = blockIdx.x * (size_t)CAS_THREADS + threadIdx.x; k < n; k += (size_t)gridDim.x * CAS_THREADS) {
        double v;
        if constexpr (KIND == 0) v = (double)__ldg(static_cast<const long long*>(f) + k) * unit;
        else if constexpr (KIND == 1) v = __ldg(static_cast<const double*>(f) + k);
        else if constexpr (KIND == 2) v = (double)__ldg(static_cast<const float*>(f) + k);
        else v = (double)__bfloat162float(static_cast<const __nv_bfloat16*>(f)[k]);
        if (v > 0.0) s -= v * log(v);
        q = fma(v, v, q);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    __shared__ double sh[2][CAS_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = s;
        sh[1][wid] = q;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < CAS_THREADS / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// One block of CAS_FINAL_THREADS: thread t adds the partials t, t + CAS_FINAL_THREADS, ..., then a
// fixed shared-memory tree (a dependent chain of FP64 additions costs microseconds per hundred
// on this GPU, so the partials are not added one after another by one thread).
constexpr int CAS_FINAL_THREADS = 512;
__global__ void __launch_bounds__(CAS_FINAL_THREADS) casimir_final_kernel(const double* __restrict__ part, int nb,
                                                                         double dxdp, double* __restrict__ out)
{
    __shared__ double sa[CAS_FINAL_THREADS], sb[CAS_FINAL_THREADS];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nb; k += CAS_FINAL_THREADS) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int h = CAS_FINAL_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sa[threadIdx.x] += sa[threadIdx.x + h];
            sb[threadIdx.x] += sb[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = dxdp * sa[0];
        out[1] = dxdp * sb[0];
    }
}

// part: 2 * CAS_BLOCKS doubles, out: 2 doubles (entropy, l2).
cudaError_t launch_casimirs(int kind, const void* f, size_t n, double unit, double dxdp, double* part, double* out,
                            cudaStream_t st)
{
    if (kind == 0) casimir_kernel<0><<<CAS_BLOCKS, CAS_THREADS, 0, st>>>(f, n, unit, part);
    else if (kind == 1) casimir_kernel<1><<<CAS_BLOCKS, CAS_THREADS, 0, st>>>(f, n, unit, part);
    else if (kind == 2) casimir_kernel<2><<<CAS_BLOCKS, CAS_THREADS, 0, st>>>(f, n, unit, part);
    else casimir_kernel<3><<<CAS_BLOCKS, CAS_THREADS, 0, st>>>(f, n, unit, part);
    casimir_final_kernel<<<1, CAS_FINAL_THREADS, 0, st>>>(part, CAS_BLOCKS, dxdp, out);
    return cudaGetLastError();
}

// ============================================================================ utilities
// Column sums of f into one partial row (used by the density/force test hook).
template <typename T>
__global__ void __launch_bounds__(256) colsum_kernel(const T* __restrict__ f, int Nx, int Np, double* colpart)
{
    __shared__ double sh[8][32];
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (i < Nx)
        for (int j = grp; j < Np; j += 8) s += (double)f[(size_t)j * Nx + i];
    sh[grp][lane] = s;
    __syncthreads();
    if (grp == 0 && i < Nx) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += sh[q][lane];
        colpart[i] = t;
    }
}

cudaError_t launch_colsum(int elem_bytes, const void* f, int Nx, int Np, double* colpart, int B, cudaStream_t st)
{
    (void)B;
    const int grid = (Nx + 31) / 32;
    if (elem_bytes == 8) colsum_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(f), Nx, Np, colpart);
    else if (elem_bytes == 2)
        colsum_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(f), Nx, Np, colpart);
    else colsum_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(f), Nx, Np, colpart);
    return cudaGetLastError();
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ s, D* __restrict__ d, size_t n)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        d[k] = (D)s[k];
}

cudaError_t launch_convert(const void* src, int src_bytes, void* dst, int dst_bytes, size_t n, cudaStream_t st)
{
    const int grid = 1024;
    if (src_bytes == 8 && dst_bytes == 2)
        convert_kernel<double, __nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const double*>(src),
                                                                     static_cast<__nv_bfloat16*>(dst), n);
    else if (src_bytes == 2 && dst_bytes == 8)
        convert_kernel<__nv_bfloat16, double><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(src),
                                                                     static_cast<double*>(dst), n);
    else if (src_bytes == 8 && dst_bytes == 4)
        convert_kernel<double, float><<<grid, 256, 0, st>>>(static_cast<const double*>(src), static_cast<float*>(dst), n);
    else if (src_bytes == 4 && dst_bytes == 8)
        convert_kernel<float, double><<<grid, 256, 0, st>>>(static_cast<const float*>(src), static_cast<double*>(dst), n);
    else if (src_bytes == 8 && dst_bytes == 8)
        return cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, st);
    else
        return cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

// Largest |f| of a device array (for the fixed-point scales after a device-side upload).  The bit
// pattern of a non-negative double orders like the value, so an integer atomicMax works.
template <typename T>
__global__ void maxabs_kernel(const T* __restrict__ f, size_t n, unsigned long long* out)
{
    double m = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs((double)f[k]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_maxabs(int elem_bytes, const void* f, size_t n, unsigned long long* out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (elem_bytes == 8) maxabs_kernel<double><<<608, 256, 0, st>>>(static_cast<const double*>(f), n, out);
    else maxabs_kernel<float><<<608, 256, 0, st>>>(static_cast<const float*>(f), n, out);
    return cudaGetLastError();
}

// ============================================================================ waterbag initial states
// The initial states of Sec. 4 written on the device: f0_ij = rowv[j] * colv[i] * (1 + noise xi_ij)
// with the profile tables computed on the host (box or homogeneous cos-mode waterbag), and xi_ij =
// 2u - 1, u the top 53 bits of the (j*Nx + i + 1)-th SplitMix64 output of `seed` (Steele, Lea &
// Flood 2014; a counter-based draw, so every cell is generated independently).  The products are
// rounded one by one (no FMA contraction), as the FP64 host generator rounds them.  Pass 1 sums the
// unnormalised f exactly in int128 fixed point (deterministic); pass 2 regenerates each cell,
// divides it by the mass and stores it in the storage type, keeping the largest |f| for the
// fixed-point scales.
__device__ __forceinline__ unsigned long long wb_splitmix64(unsigned long long seed, unsigned long long k)
{
    unsigned long long z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double wb_value(const WaterbagArgs& a, size_t k)
{
    const int j = (int)(k / (size_t)a.Nx), i = (int)(k - (size_t)j * a.Nx);
    double v = __dmul_rn(__ldg(a.rowv + j), __ldg(a.colv + i));
    if (v != 0.0 && a.noise != 0.0) {
        const unsigned long long z = wb_splitmix64(a.seed, (unsigned long long)k + 1ull);
        const double u = __dmul_rn((double)(z >> 11), 1.1102230246251565e-16);   // top 53 bits / 2^53
        const double xi = __dadd_rn(__dmul_rn(2.0, u), -1.0);
        v = __dmul_rn(v, __dadd_rn(1.0, __dmul_rn(a.noise, xi)));
    }
    return v;
}

__global__ void __launch_bounds__(WB_THREADS) waterbag_mass_kernel(WaterbagArgs a)
{
    __shared__ i128 red[33];
    __shared__ bool is_last;
    const size_t n = (size_t)a.Nx * a.Np;
    i128 acc = 0;
    for (size_t k = blockIdx.x * (size_t)WB_THREADS + threadIdx.x; k < n; k += (size_t)gridDim.x * WB_THREADS)
        acc += fx128_from_f64(wb_value(a, k), a.k_m);
    acc = block_sum_i128(acc, red);
    i128* part = static_cast<i128*>(a.part);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = acc;
        __threadfence();
        is_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    i128 t = 0;
    const volatile i128* vp = part;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += WB_THREADS) t += vp[b];
    t = block_sum_i128(t, red);
    if (threadIdx.x == 0) *a.mass = __dmul_rn(a.dxdp, fx128_to_f64(t, a.k_m));
}

template <typename D>
__global__ void __launch_bounds__(WB_THREADS) waterbag_write_kernel(WaterbagArgs a, D* __restrict__ f)
{
    const size_t n = (size_t)a.Nx * a.Np;
    const double mass = *a.mass;
    double m = 0.0;
    for (size_t k = blockIdx.x * (size_t)WB_THREADS + threadIdx.x; k < n; k += (size_t)gridDim.x * WB_THREADS) {
        const double v = __ddiv_rn(wb_value(a, k), mass);
        m = fmax(m, fabs(v));
        f[k] = (D)v;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(a.maxbits, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_waterbag(const WaterbagArgs& a, int elem_bytes, void* f, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.maxbits, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    waterbag_mass_kernel<<<WB_BLOCKS, WB_THREADS, 0, st>>>(a);
    if (elem_bytes == 8) waterbag_write_kernel<double><<<WB_BLOCKS, WB_THREADS, 0, st>>>(a, static_cast<double*>(f));
    else if (elem_bytes == 4) waterbag_write_kernel<float><<<WB_BLOCKS, WB_THREADS, 0, st>>>(a, static_cast<float*>(f));
    else waterbag_write_kernel<__nv_bfloat16><<<WB_BLOCKS, WB_THREADS, 0, st>>>(a, static_cast<__nv_bfloat16*>(f));
    return cudaGetLastError();
}

// ============================================================================ failure path
// A wait that must expire: the barrier expects one arrival that no thread makes and no copy
// completes, so mbar_wait_bounded gives up after limit_ns of %globaltimer time.  Every thread of
// the CTA waits, as a sweep's threads wait for a staged row; on expiry the CTA records the error
// code the sweeps record and returns.  Nothing is in flight, so the context stays usable.
__global__ void __launch_bounds__(128) expire_wait_kernel(int* err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    __syncthreads();
    if (!ok && threadIdx.x == 0) atomicCAS(err, DEV_ERR_NONE, DEV_ERR_TEST_WAIT);
}

cudaError_t launch_expire_wait(int* err, unsigned long long limit_ns, cudaStream_t st)
{
    expire_wait_kernel<<<1, 128, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

}  // namespace vl
