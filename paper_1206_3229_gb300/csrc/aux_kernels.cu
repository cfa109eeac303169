// aux_kernels.cu -- density and moment reductions, the three mean-field forces, the p-shift
// line parameters, and small utility kernels.
//
// Density (Sec. 2): rho_i = dp sum_j f[j,i], assembled from the per-CTA column partials written
// by the x-shift epilogue, in a fixed order (deterministic).  Moments: mass = dx sum rho,
// Mx, My = dx sum cos/sin(x_i) rho_i (Eq. mxmydef), kinetic = dx dp sum_j p_j^2/2 sum_i f.
// Forces, Eq. (meanforce) by the rectangle rule:
//   HMF   (Eq. hmfmeanforce): F_i = -Mx sin x_i + My cos x_i
//   ring  (Eq. ringpot):      F_i = -dx sum_k V'((i-k) dx) rho_k   (circulant)
//   sheet (V = 2 pi G |x|):   F_i = -2 pi G dx (sum_{k<i} rho_k - sum_{k>i} rho_k)  (prefix scan)
// All reductions are FP64 with Neumaier compensation in the final stages.
#include "vlasov_internal.cuh"

namespace vl {

struct NSum {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double x)
    {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double val() const { return s + c; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum in a fixed order (warp trees, then warp 0 over the warp results).
__device__ double block_sum(double v, double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

constexpr int CR_COLS = 32;      // columns per colreduce block
constexpr int CR_GROUPS = 8;     // partial groups per block (blockDim = 256)

// ============================================================================ colreduce
// Block: 32 columns x 8 groups over the B partials; then block partials of (mass, Mx, My); the
// last block to finish (ticket) reduces those in block order, adds the kinetic partials, and runs
// the model-specific tail (sheet scan, moment record).
__global__ void __launch_bounds__(256) colreduce_kernel(ColReduceArgs a)
{
    __shared__ double sh[CR_GROUPS][CR_COLS];
    __shared__ double red[32];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int i = blockIdx.x * CR_COLS + lane;

    double s = 0.0;
    if (i < a.Nx)
        for (int b = grp; b < a.B; b += CR_GROUPS) s += a.colpart[(size_t)b * a.Nx + i];
    sh[grp][lane] = s;
    __syncthreads();
    double rho = 0.0, cm = 0.0, cx = 0.0, cy = 0.0;
    if (grp == 0) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < CR_GROUPS; ++q) t += sh[q][lane];
        if (i < a.Nx) {
            rho = a.dp * t;
            a.rho[i] = rho;
            cm = rho;
            cx = a.costab[i] * rho;
            cy = a.sintab[i] * rho;
        }
    }
    cm = block_sum(cm, red);
    cx = block_sum(cx, red);
    cy = block_sum(cy, red);
    if (threadIdx.x == 0) {
        a.blockpart[blockIdx.x * 4 + 0] = cm;
        a.blockpart[blockIdx.x * 4 + 1] = cx;
        a.blockpart[blockIdx.x * 4 + 2] = cy;
        __threadfence();
        const unsigned int tk = atomicAdd(a.ticket, 1u);
        is_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    // ---- last block: totals in block order (thread 0, compensated)
    __shared__ double tot[4];
    if (threadIdx.x == 0) {
        NSum m, x, y, k;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            m.add(__ldcg(&a.blockpart[b * 4 + 0]));
            x.add(__ldcg(&a.blockpart[b * 4 + 1]));
            y.add(__ldcg(&a.blockpart[b * 4 + 2]));
        }
        if (a.kinpart)
            for (int b = 0; b < a.B; ++b) k.add(a.kinpart[b]);
        tot[0] = a.dx * m.val();
        tot[1] = a.dx * x.val();
        tot[2] = a.dx * y.val();
        tot[3] = a.dx * a.dp * k.val();
        *a.ticket = 0u;   // ready for the next launch
    }
    __syncthreads();
    const double mass = tot[0], Mx = tot[1], My = tot[2], kin = tot[3];
    double U = 0.0;

    if (a.model == 2) {
        // Sheet: exclusive prefix C_i = sum_{k<i} rho_k (compensated, fixed order), then
        // F_i = -2 pi G dx (2 C_i + rho_i - S), S = sum rho; U = 2 pi G dx^3 sum_i rho_i (i C_i - X_i),
        // X_i = sum_{k<i} k rho_k.
        __shared__ double offs[256][2];
        __shared__ double offx[256][2];
        const int nt = blockDim.x;
        const int per = (a.Nx + nt - 1) / nt;
        const int lo = threadIdx.x * per, hi = min(a.Nx, lo + per);
        NSum ls, lx;
        for (int q = lo; q < hi; ++q) {
            const double r = __ldcg(&a.rho[q]);
            ls.add(r);
            lx.add((double)q * r);
        }
        offs[threadIdx.x][0] = ls.s;
        offs[threadIdx.x][1] = ls.c;
        offx[threadIdx.x][0] = lx.s;
        offx[threadIdx.x][1] = lx.c;
        __syncthreads();
        if (threadIdx.x == 0) {
            NSum run, runx;
            for (int t = 0; t < nt; ++t) {
                const double s0 = offs[t][0], c0 = offs[t][1], s1 = offx[t][0], c1 = offx[t][1];
                offs[t][0] = run.s;
                offs[t][1] = run.c;
                offx[t][0] = runx.s;
                offx[t][1] = runx.c;
                run.add(s0);
                run.add(c0);
                runx.add(s1);
                runx.add(c1);
            }
            tot[0] = run.val();
        }
        __syncthreads();
        const double S = tot[0];
        const double k2 = 2.0 * 3.14159265358979323846 * a.G;
        NSum c, xx;
        c.s = offs[threadIdx.x][0];
        c.c = offs[threadIdx.x][1];
        xx.s = offx[threadIdx.x][0];
        xx.c = offx[threadIdx.x][1];
        double up = 0.0;
        for (int q = lo; q < hi; ++q) {
            const double r = __ldcg(&a.rho[q]);
            const double C = c.val();
            a.F[q] = -k2 * a.dx * (2.0 * C + r - S);
            if (a.final_moments) up += r * ((double)q * C - xx.val());
            c.add(r);
            xx.add((double)q * r);
        }
        if (a.final_moments) {
            up = block_sum(up, red);
            U = k2 * a.dx * a.dx * a.dx * up;
        }
    } else if (a.model == 0) {
        U = 0.5 * (mass * mass - Mx * Mx - My * My);
    }

    if (threadIdx.x == 0) {
        a.sc->mass = mass;
        a.sc->Mx = Mx;
        a.sc->My = My;
        a.sc->kinetic = kin;
        a.sc->potential = U;
        if (a.final_moments && a.model != 1) {
            const long long st = *a.step;
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
    }
}

cudaError_t launch_colreduce(const ColReduceArgs& a, int grid, cudaStream_t st)
{
    colreduce_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ============================================================================ ring force
// One warp per output node i: F_i = -dx sum_k V'(((i-k) mod N) dx) rho_k (and, for the moments,
// Phi_i = dx sum_k V(...) rho_k).  The last block forms U = 1/2 dx sum_i rho_i Phi_i.
__global__ void __launch_bounds__(256) ring_kernel(RingArgs a)
{
    __shared__ double red[32];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = blockIdx.x * 8 + wid;
    const int N = a.N;
    double up = 0.0;
    if (i < N) {
        double f = 0.0;
        // after the last x-shift only the potential is needed; otherwise only the force
        const double* __restrict__ ker = a.final_moments ? a.V : a.dV;
        for (int k = lane; k < N; k += 32) {
            int m = i - k;
            if (m < 0) m += N;
            f = fma(ker[m], a.rho[k], f);
        }
        f = warp_sum(f);
        if (lane == 0) {
            if (a.final_moments) up = a.rho[i] * a.dx * f;
            else a.F[i] = -a.dx * f;
        }
    }
    if (!a.final_moments) return;
    up = block_sum(up, red);
    if (threadIdx.x == 0) {
        a.blockpart[blockIdx.x] = up;
        __threadfence();
        const unsigned int tk = atomicAdd(a.ticket, 1u);
        is_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last || threadIdx.x != 0) return;
    __threadfence();
    NSum u;
    for (int b = 0; b < (int)gridDim.x; ++b) u.add(__ldcg(&a.blockpart[b]));
    *a.ticket = 0u;
    const double U = 0.5 * a.dx * u.val();
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

cudaError_t launch_ring(const RingArgs& a, cudaStream_t st)
{
    ring_kernel<<<(a.N + 7) / 8, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ============================================================================ p-shift parameters
template <typename T>
__global__ void __launch_bounds__(64) pparams_kernel(PParamsArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.Nx) return;
    double F;
    if (a.model == 0) F = -a.sc->Mx * a.sintab[i] + a.sc->My * a.costab[i];
    else if (a.model == 3) F = 0.0;
    else F = a.Fin[i];
    if (a.Fout) a.Fout[i] = F;
    const double sigma = F * a.cp;
    LineSplit L;
    line_split(sigma, L);
    T* w = static_cast<T*>(a.w);
    T* gd = static_cast<T*>(a.gd);
    a.n0[i] = L.n0;
#pragma unroll
    for (int t = 0; t < NTAP; ++t) w[(size_t)t * a.Nx + i] = (T)L.w[t];
    gd[i] = (T)L.g;
    gd[a.Nx + i] = (T)L.d;
}

cudaError_t launch_pparams(int elem_bytes, const PParamsArgs& a, cudaStream_t st)
{
    const int grid = (a.Nx + 63) / 64;
    if (elem_bytes == 8) pparams_kernel<double><<<grid, 64, 0, st>>>(a);
    else pparams_kernel<float><<<grid, 64, 0, st>>>(a);
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
    if (src_bytes == 8 && dst_bytes == 4)
        convert_kernel<double, float><<<grid, 256, 0, st>>>(static_cast<const double*>(src), static_cast<float*>(dst), n);
    else if (src_bytes == 4 && dst_bytes == 8)
        convert_kernel<float, double><<<grid, 256, 0, st>>>(static_cast<const float*>(src), static_cast<double*>(dst), n);
    else if (src_bytes == 8 && dst_bytes == 8)
        return cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, st);
    else
        return cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

}  // namespace vl
