// shift_kernels.cu -- the two sweeps of the Strang split (Sec. 3 of arXiv:1206.3229).
//
//  x-shift (Eqs. step1/step4): every p row j moves by s_j = p_j dt/(2 dx) cells.  Row-constant
//  spline weights (one 10-tap filter per row), so a CTA stages whole rows in shared memory with
//  1-D bulk (TMA) copies, a few rows in flight, and each thread produces V = 16/sizeof(T)
//  consecutive outputs from a register window loaded with 16-byte shared-memory reads; the output
//  is one coalesced 16-byte store per thread.  Optional epilogue: per-column sums (density) and
//  the p^2/2-weighted row sums (kinetic energy) of the produced rows.
//
//  p-shift (Eq. step3): every x column i moves by sigma_i = F_i dt/dp cells.  Done in the natural
//  layout (no global transpose): a tile of 32 columns x 128 output rows stages the union window
//  of input rows it needs with 2-D TMA boxes (out-of-range rows come back as zeros, which is the
//  f = 0 outside reading of the p axis), each thread walks 16 rows of one column with a sliding
//  register window.
#include "fixed_point.cuh"
#include "pparams.cuh"
#include "ptx.cuh"
#include "shift_common.cuh"
#include "vlasov_internal.cuh"

#include <cuda_bf16.h>
#include <cstddef>
#include <type_traits>

namespace vl {

using bf16 = __nv_bfloat16;

// Storage type S of f (double, float, or bf16 for the BF16 storage experiment), the type T the
// filter computes in, and the 16-byte vector of V cells the x-shift loads and stores.
template <typename S>
struct VecOf;
template <>
struct VecOf<double> {
    static constexpr int V = 2;
    static constexpr int W = 12;   // window: V + 9 taps + alignment slack, rounded to V
    using vec = double2;
    using T = double;
    using acc = double;
};
template <>
struct VecOf<float> {
    static constexpr int V = 4;
    static constexpr int W = 16;
    using vec = float4;
    using T = float;
    using acc = float;
};
template <>
struct VecOf<bf16> {
    static constexpr int V = 8;
    static constexpr int W = 24;
    using vec = uint4;             // 8 bf16, element 2q in the low half of word q
    using T = float;
    using acc = float;
};

__device__ __forceinline__ float to_math(bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_math(float v) { return v; }
__device__ __forceinline__ double to_math(double v) { return v; }
template <typename S>
__device__ __forceinline__ S from_math(typename VecOf<S>::T v)
{
    if constexpr (std::is_same<S, bf16>::value) return __float2bfloat16_rn(v);   // round to nearest even
    else return v;
}

// The V cells of a loaded vector as math values, and V results as a vector to store.
template <typename S>
__device__ __forceinline__ void unpack(const typename VecOf<S>::vec& v, typename VecOf<S>::T* x)
{
    if constexpr (std::is_same<S, double>::value) {
        x[0] = v.x;
        x[1] = v.y;
    } else if constexpr (std::is_same<S, float>::value) {
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    } else {
        const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wd[q]));
            x[2 * q] = f2.x;
            x[2 * q + 1] = f2.y;
        }
    }
}
template <typename S>
__device__ __forceinline__ typename VecOf<S>::vec pack(const typename VecOf<S>::T* x)
{
    typename VecOf<S>::vec v;
    if constexpr (std::is_same<S, double>::value) {
        v.x = x[0];
        v.y = x[1];
    } else if constexpr (std::is_same<S, float>::value) {
        v.x = x[0];
        v.y = x[1];
        v.z = x[2];
        v.w = x[3];
    } else {
        uint32_t wd[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
            wd[q] = *reinterpret_cast<const uint32_t*>(&h);
        }
        v.x = wd[0];
        v.y = wd[1];
        v.z = wd[2];
        v.w = wd[3];
    }
    return v;
}

constexpr int XS_MAXCH = 8;   // chunks of V*threads outputs per row handled by one thread
// BF16 storage: 8-cell chunks, so 2 chunks per thread cover 4096 columns (fewer accumulator registers)
template <typename S>
__host__ __device__ constexpr int maxch_of() { return std::is_same<S, bf16>::value ? 2 : XS_MAXCH; }

// ============================================================================ x-shift
template <typename S, int A, bool PERIODIC, typename T = typename VecOf<S>::T>
__device__ __forceinline__ void xshift_chunk(const S* __restrict__ rowbuf, int e, const T (&w)[NTAP],
                                             int i, int k, int Nx, T g, T d, T (&out)[VecOf<S>::V])
{
    constexpr int V = VecOf<S>::V, W = VecOf<S>::W;
    using vec = typename VecOf<S>::vec;
    T x[W];
    const vec* p = reinterpret_cast<const vec*>(rowbuf + e);
#pragma unroll
    for (int q = 0; q < W / V; ++q) unpack<S>(p[q], x + q * V);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T acc = w[0] * x[A + v];
#pragma unroll
        for (int t = 1; t < NTAP; ++t) acc = fma(w[t], x[A + v + t], acc);
        out[v] = acc;
    }
    if constexpr (!PERIODIC) {
        if (k < 0 || k + V - 1 >= Nx - 1) {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = edge_fix(out[v], &x[A + v], k + v, Nx, g, d);
        }
    }
    (void)i;
}

// One row: chunks of V outputs at columns V (tid + c nthreads), c < CH, written to orow (global or
// shared memory; with WRAP the chunks below column 16 also at orow + Nx, the wrap copy a periodic
// second pass reads).
template <typename S, int A, bool PERIODIC, int CH = maxch_of<S>(), bool WRAP = false,
          typename T = typename VecOf<S>::T>
__device__ __forceinline__ void xshift_row(const S* __restrict__ rowbuf, S* __restrict__ orow,
                                           const T (&w)[NTAP], int n0, int Nx, T g, T d, int nthreads,
                                           typename VecOf<S>::acc (&colacc)[CH][VecOf<S>::V],
                                           typename VecOf<S>::acc& rowsum)
{
    constexpr int V = VecOf<S>::V;
    using vec = typename VecOf<S>::vec;
    const int tid = threadIdx.x;
    int base;   // window start of output 0 (aligned down by A)
    if constexpr (PERIODIC) {
        base = (n0 - 4 - A) % Nx;
        if (base < 0) base += Nx;
    } else {
        base = n0 - 4 - A;
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int i = V * (tid + c * nthreads);
        if (i < Nx) {
            int e = i + base;
            if constexpr (PERIODIC) {
                if (e >= Nx) e -= Nx;
            }
            T out[V];
            xshift_chunk<S, A, PERIODIC>(rowbuf, e, w, i, i + n0, Nx, g, d, out);
            const vec o = pack<S>(out);
            *reinterpret_cast<vec*>(orow + i) = o;
            if constexpr (WRAP) {
                if (i < 16) *reinterpret_cast<vec*>(orow + Nx + i) = o;
            }
            T stored[V];   // the column sums are those of the stored values
            unpack<S>(o, stored);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                colacc[c][v] += stored[v];
                rowsum += stored[v];
            }
        }
    }
}

// End of a sweep: hand over this CTA's column sums acc[c][v] (column V (tid + c blockDim) + v) in
// the form the arguments ask for.  Every thread calls it; `scratch` (>= 2 KB of shared memory no
// warp still reads) serves the block reduction.
template <typename S, int CH, int VW = VecOf<S>::V>
__device__ __forceinline__ void colsum_epilogue(const XShiftArgs& a, const typename VecOf<S>::acc (&colacc)[CH][VW],
                                                i128* scratch)
{
    using acc_t = typename VecOf<S>::acc;
    constexpr int V = VW;   // columns V (tid + c nthreads) + v, v < V
    const int Nx = a.Nx, tid = threadIdx.x, nthreads = blockDim.x;
    if (a.colacc) {
        // exact fixed-point column sums, added across CTAs (order-free)
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    long long q;
                    if constexpr (sizeof(acc_t) == 8) q = (long long)fx128_from_f64((double)colacc[c][v], a.k_col);
                    else q = (long long)fx128_from_f32((float)colacc[c][v], a.k_col);
                    atomicAdd(a.colacc + i + v, (unsigned long long)q);
                }
            }
        }
    } else if (a.ctapart) {
        // HMF: this CTA's column sums t_i as integers in units 2^(Ef-51), then sum t_i and the
        // 50-bit cos/sin-weighted sums (exact int128), three numbers per CTA instead of a row
        i128 pm = 0, px = 0, py = 0, pz = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    long long t;
                    if constexpr (sizeof(acc_t) == 8) t = (long long)fx128_from_f64((double)colacc[c][v], 51 - a.Ef);
                    else t = (long long)fx128_from_f32((float)colacc[c][v], 51 - a.Ef);
                    pm += (i128)t;
                    px += (i128)__ldg(a.cos50 + i + v) * (i128)t;
                    py += (i128)__ldg(a.sin50 + i + v) * (i128)t;
                }
            }
        }
        block_sum4_i128(pm, px, py, pz, scratch);
        if (tid == 0) {
            i128* cp = static_cast<i128*>(a.ctapart) + (size_t)blockIdx.x * 3;
            cp[0] = pm;
            cp[1] = px;
            cp[2] = py;
        }
    } else if (a.colpart64) {
        // exact fixed-point partial rows (units 2^-k_col): the reduction adds them with integer
        // instructions, not a chain of FP64 additions per column
        long long* cp = a.colpart64 + (size_t)blockIdx.x * Nx;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if constexpr (sizeof(acc_t) == 8) cp[i + v] = (long long)fx128_from_f64((double)colacc[c][v], a.k_col);
                    else cp[i + v] = (long long)fx128_from_f32((float)colacc[c][v], a.k_col);
                }
            }
        }
    } else if (a.colpart) {
        double* cp = a.colpart + (size_t)blockIdx.x * Nx;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < V; ++v) cp[i + v] = (double)colacc[c][v];
            }
        }
    }
}

// The CTA's kinetic sum (per-thread FP64 partial kin) into a.kinpart[blockIdx.x]; red: 32 doubles.
__device__ __forceinline__ void kin_epilogue(const XShiftArgs& a, double kin, double* red)
{
    const int tid = threadIdx.x, nthreads = blockDim.x;
    double v = kin;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int q = 0; q < (nthreads + 31) / 32; ++q) sum += red[q];
        a.kinpart[blockIdx.x] = sum;
    }
}

// Shared memory the fused HMF epilogue needs: six int128 and one double per thread.
constexpr size_t XX_HMF_EPI_BYTES = (size_t)XXS_THREADS * (6 * 16 + 8);
static_assert(XXS_THREADS >= 7 * 32, "seven warps share the fused HMF epilogue");

// End of the fused x-shifts, HMF: both passes' per-CTA sums (mass, cos- and sin-weighted column sums,
// exact) and the first pass's kinetic sum in one pass over shared memory.  Every thread stores its
// seven partials in slot-major order; then warp w (w < 6) adds slot w's partials with a lane-strided
// loop and one warp reduction, and warp 6 the kinetic partials: seven short warp reductions instead
// of a block-wide shuffle tree per value.  The weighted sums use split 32-bit products (Mac26).
template <typename S, int CH>
__device__ __forceinline__ void xx_hmf_epilogue(const XShiftArgs& a, const XShiftArgs& b,
                                                const typename VecOf<S>::acc (&acc1)[CH][VecOf<S>::V],
                                                const typename VecOf<S>::acc (&acc2)[CH][VecOf<S>::V], float kinf,
                                                unsigned char* smem)
{
    constexpr int V = VecOf<S>::V;
    const int Nx = a.Nx, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    i128* sm = reinterpret_cast<i128*>(smem);   // [6][XXS_THREADS]
    double* kd = reinterpret_cast<double*>(sm + 6 * XXS_THREADS);
    // one pass at a time (fewer live registers): slots 3q .. 3q + 2 for pass q
    auto part = [&](const typename VecOf<S>::acc (&acc)[CH][V], int Ef, int q) {
        long long m = 0;
        Mac26 x, y;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = V * (tid + c * XXS_THREADS);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const long long t = (long long)fx128_from_f32((float)acc[c][v], 51 - Ef);
                    m += t;
                    x.add(__ldg(a.cos50 + i + v), t);
                    y.add(__ldg(a.sin50 + i + v), t);
                }
            }
        }
        sm[(3 * q + 0) * XXS_THREADS + tid] = (i128)m;
        sm[(3 * q + 1) * XXS_THREADS + tid] = x.fold();
        sm[(3 * q + 2) * XXS_THREADS + tid] = y.fold();
    };
    part(acc1, a.Ef, 0);
    part(acc2, b.Ef, 1);
    kd[tid] = (double)kinf;
    __syncthreads();
    if (wid < 6) {
        i128 t = 0;
#pragma unroll 4
        for (int k = lane; k < XXS_THREADS; k += 32) t += sm[wid * XXS_THREADS + k];
        t = warp_sum_i128(t);
        if (lane == 0) {
            const XShiftArgs& o = wid < 3 ? a : b;
            static_cast<i128*>(o.ctapart)[(size_t)blockIdx.x * 3 + wid % 3] = t;
        }
    } else if (wid == 6) {
        double t = 0.0;
#pragma unroll 4
        for (int k = lane; k < XXS_THREADS; k += 32) t += kd[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) a.kinpart[blockIdx.x] = t;
    }
}

template <typename S, bool PERIODIC, bool KIN>
__device__ __forceinline__ void xshift_body(const XShiftArgs& a)
{
    using T = typename VecOf<S>::T;
    constexpr int V = VecOf<S>::V;
    using acc_t = typename VecOf<S>::acc;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    S* bufs = reinterpret_cast<S*>(smem_raw + 128);
    __shared__ double red[32];

    const S* __restrict__ fin = static_cast<const S*>(a.fin);
    S* __restrict__ fout = static_cast<S*>(a.fout);
    const int Nx = a.Nx, Np = a.Np, PAD = a.pad, NS = a.stages;
    const int stride = Nx + 2 * PAD;
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int G = a.ctas > 0 ? a.ctas : (int)gridDim.x;
    const T* __restrict__ wrow = static_cast<const T*>(a.w);
    const T* __restrict__ gdrow = static_cast<const T*>(a.gd);
    const uint32_t row_bytes = (uint32_t)(Nx * sizeof(S));
    const bool use_rec = a.rec != nullptr;
    const uint32_t tx_bytes = row_bytes + (PERIODIC ? 16u * (uint32_t)sizeof(S) : 0u) + (use_rec ? XREC_BYTES : 0u);
    unsigned char* recs = reinterpret_cast<unsigned char*>(bufs + (size_t)NS * stride);

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    if constexpr (!PERIODIC) {
        // zero halos of every stage (never touched by the copies)
        for (int s = 0; s < NS; ++s) {
            S* b = bufs + (size_t)s * stride;
            for (int e = tid; e < PAD; e += nthreads) {
                b[e] = from_math<S>(T(0));
                b[PAD + Nx + e] = from_math<S>(T(0));
            }
        }
    }
    __syncthreads();

    auto issue = [&](int s, int r) {
        S* dst = bufs + (size_t)s * stride + PAD;
        const S* src = fin + (size_t)r * Nx;
        mbar_arrive_expect_tx(&bars[s], tx_bytes);
        bulk_g2s(dst, src, row_bytes, &bars[s]);
        if constexpr (PERIODIC) bulk_g2s(dst + Nx, src, 16u * (uint32_t)sizeof(S), &bars[s]);
        if (use_rec)
            bulk_g2s(recs + (size_t)s * XREC_BYTES, static_cast<const unsigned char*>(a.rec) + (size_t)r * XREC_BYTES,
                     XREC_BYTES, &bars[s]);
    };

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            const int r = blockIdx.x + s * G;
            if (r < Np) issue(s, r);
        }
    }

    acc_t colacc[maxch_of<S>()][V];
#pragma unroll
    for (int c = 0; c < maxch_of<S>(); ++c)
#pragma unroll
        for (int v = 0; v < V; ++v) colacc[c][v] = acc_t(0);
    // kinetic sum of this thread's rows: FP64 for FP64 storage; for FP32-class storage the row sums
    // are FP32 already, and an FP32 fused multiply-add per row keeps the slow FP64 pipe out of the
    // row loop (the sum becomes FP64 in the per-CTA epilogue)
    double kin = 0.0;
    float kinf = 0.f;

    int it = 0;
    int r = blockIdx.x;
    bool failed = false;
    for (; r < Np; r += G, ++it) {
        const int s = it % NS;
        const uint32_t parity = (uint32_t)((it / NS) & 1);
        const bool ok = mbar_wait_bounded(&bars[s], parity, WAIT_LIMIT_NS);
        acc_t rowsum = acc_t(0);
        if (ok) {
            int n0;
            T w[NTAP];
            T g = T(0), d = T(0);
            float p2h = 0.f;
            if (use_rec) {
                const XRec* rc = reinterpret_cast<const XRec*>(recs + (size_t)s * XREC_BYTES);
                n0 = rc->n0;
                p2h = rc->p2h;
#pragma unroll
                for (int t = 0; t < NTAP; ++t) w[t] = sizeof(T) == 8 ? (T)rc->w64[t] : (T)rc->w32[t];
                if constexpr (!PERIODIC) {
                    g = sizeof(T) == 8 ? (T)rc->g64 : (T)rc->g32;
                    d = sizeof(T) == 8 ? (T)rc->d64 : (T)rc->d32;
                }
            } else {
                n0 = a.n0[r];
#pragma unroll
                for (int t = 0; t < NTAP; ++t) w[t] = wrow[(size_t)t * Np + r];
                if constexpr (!PERIODIC) {
                    g = gdrow[r];
                    d = gdrow[Np + r];
                }
            }
            const S* rowbuf = bufs + (size_t)s * stride + PAD;
            S* orow = fout + (size_t)r * Nx;
            const int A = (n0 - 4) & (V - 1);
#define VL_ROW(AA) xshift_row<S, AA, PERIODIC>(rowbuf, orow, w, n0, Nx, g, d, nthreads, colacc, rowsum)
            if constexpr (V == 2) {
                if (A == 0) VL_ROW(0);
                else VL_ROW(1);
            } else if constexpr (V == 4) {
                switch (A) {
                    case 0: VL_ROW(0); break;
                    case 1: VL_ROW(1); break;
                    case 2: VL_ROW(2); break;
                    default: VL_ROW(3); break;
                }
            } else {
                switch (A) {
                    case 0: VL_ROW(0); break;
                    case 1: VL_ROW(1); break;
                    case 2: VL_ROW(2); break;
                    case 3: VL_ROW(3); break;
                    case 4: VL_ROW(4); break;
                    case 5: VL_ROW(5); break;
                    case 6: VL_ROW(6); break;
                    default: VL_ROW(7); break;
                }
            }
#undef VL_ROW
            if constexpr (KIN) {
                if constexpr (sizeof(T) == 4) {
                    if (!use_rec) {
                        const double pj = a.pmin + (double)r * a.dp;
                        p2h = (float)(0.5 * pj * pj);
                    }
                    kinf = fmaf(p2h, (float)rowsum, kinf);
                } else {
                    const double pj = a.pmin + (double)r * a.dp;
                    kin += 0.5 * pj * pj * (double)rowsum;
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            const int rn = r + NS * G;
            if (rn < Np) {
                fence_proxy_async_smem();
                issue(s, rn);
            }
        }
    }

    if (failed) {
        // Record the failure and wait (bounded) for this CTA's copies still in flight.
        if (tid == 0) {
            atomicCAS(a.err, 0, DEV_ERR_XSHIFT_WAIT);
            for (int k = 0; k < NS; ++k) {
                const int rr = r + k * G;
                if (rr >= Np) break;
                const int itk = it + k;
                mbar_wait_bounded(&bars[itk % NS], (uint32_t)((itk / NS) & 1), WAIT_LIMIT_NS);
            }
        }
        __syncthreads();
        return;
    }

    colsum_epilogue<S, maxch_of<S>()>(a, colacc, reinterpret_cast<i128*>(bufs));
    if constexpr (KIN) kin_epilogue(a, sizeof(T) == 4 ? (double)kinf : kin, red);
}

template <typename S, bool PERIODIC, bool KIN>
__global__ void __launch_bounds__(XS_THREADS_MAX, 1) xshift_kernel(XShiftArgs a)
{
    xshift_body<S, PERIODIC, KIN>(a);
}

// Batched form: blockIdx.y selects the grid (slot); args[slot * 2 + ver[slot]] are its arguments
// for the buffer parity it is at.  Slots with Np = 0 (free, or another boundary kind) exit.
template <typename T, bool PERIODIC, bool KIN>
__global__ void __launch_bounds__(XS_THREADS_MIN, 1) xshift_batch_kernel(const XShiftArgs* __restrict__ args,
                                                                          const int* __restrict__ ver)
{
    const int slot = blockIdx.y;
    const XShiftArgs a = args[slot * 2 + ver[slot]];
    if (a.Np <= 0 || (int)blockIdx.x >= a.Np || (a.ctas > 0 && (int)blockIdx.x >= a.ctas)) return;
    xshift_body<T, PERIODIC, KIN>(a);
}

// ============================================================================ fused x-shifts
// FP32-class storage: the second x half-shift of step n and the first of step n+1 in one launch,
// as xxshift_fx_body does for FX64 — each row staged once, the first pass written to a shared-memory
// row (its column sums and kinetic sum: step n's moments), the second read from there and written
// to HBM (its column sums: the next density).  Same arithmetic as two launches.  512 threads,
// 8 / V chunks of V columns each (Nx <= 4096); two intermediate rows alternate (one barrier per row).
//   a: input, records, shape, first-pass outputs; b: output buffer and second-pass column sums.
// One pass over a fused row: chunks of V columns at V (tid + c XXS_THREADS), c < CH, from the row
// staged at `src` whose window for output 0 starts at `base` (periodic rows: base in [0, Nx), the
// wrap copy at src + Nx serves windows that cross the end), written to `dst`: the intermediate row
// in shared memory (TO_SMEM; periodic rows also get the wrap copy of its first 16 columns) or the
// output row in HBM.  The row constants come in from the caller, computed once for both passes.
template <typename S, int A, bool PERIODIC, int CH, bool TO_SMEM, typename T = typename VecOf<S>::T>
__device__ __forceinline__ void xx_pass(const S* __restrict__ src, S* __restrict__ dst, const T (&w)[NTAP],
                                        int base, int n0, int Nx, T g, T d,
                                        typename VecOf<S>::acc (&acc)[CH][VecOf<S>::V],
                                        typename VecOf<S>::acc& rowsum)
{
    constexpr int V = VecOf<S>::V;
    using vec = typename VecOf<S>::vec;
    const int i0 = V * (int)threadIdx.x;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int i = i0 + c * V * XXS_THREADS;
        if (i < Nx) {
            int e = i + base;
            if constexpr (PERIODIC) e = e >= Nx ? e - Nx : e;
            T out[V];
            xshift_chunk<S, A, PERIODIC>(src, e, w, i, i + n0, Nx, g, d, out);
            const vec o = pack<S>(out);
            *reinterpret_cast<vec*>(dst + i) = o;
            if constexpr (TO_SMEM && PERIODIC) {
                if (i < 16) *reinterpret_cast<vec*>(dst + Nx + i) = o;
            }
            T stored[V];   // the column sums are those of the stored values
            unpack<S>(o, stored);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                acc[c][v] += stored[v];
                rowsum += stored[v];
            }
        }
    }
}

template <typename S, bool PERIODIC>
__device__ __forceinline__ void xxshift_body(const XShiftArgs& a, const XShiftArgs& b)
{
    using T = typename VecOf<S>::T;
    using acc_t = typename VecOf<S>::acc;
    constexpr int V = VecOf<S>::V;
    constexpr int CH = XXS_MAX_NX / (V * XXS_THREADS);
    static_assert(CH * V * XXS_THREADS == XXS_MAX_NX && sizeof(T) == 4, "FP32-class storage");
    static_assert(offsetof(XRec, w32) % 16 == 0 && XREC_BYTES % 16 == 0, "16-byte weight loads");
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    S* bufs = reinterpret_cast<S*>(smem_raw + 128);
    __shared__ double red[32];
    __shared__ unsigned int issued[8];

    const S* __restrict__ fin = static_cast<const S*>(a.fin);
    S* __restrict__ fout = static_cast<S*>(b.fout);
    const int Nx = a.Nx, Np = a.Np, PAD = a.pad, NS = a.stages;
    const int stride = Nx + 2 * PAD;
    const int tid = threadIdx.x;
    const int G = a.ctas > 0 ? a.ctas : (int)gridDim.x;
    S* ibufs = bufs + (size_t)NS * stride;   // two intermediate rows
    unsigned char* recs = reinterpret_cast<unsigned char*>(ibufs + 2 * (size_t)stride);
    const uint32_t row_bytes = (uint32_t)(Nx * sizeof(S));
    const uint32_t tx_bytes = row_bytes + (PERIODIC ? 16u * (uint32_t)sizeof(S) : 0u) + XREC_BYTES;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&bars[s], 1);
            issued[s] = 0;
        }
        fence_barrier_init();
    }
    for (int e = tid; e < 2 * stride; e += XXS_THREADS) ibufs[e] = from_math<S>(T(0));
    if constexpr (!PERIODIC) {
        for (int s = 0; s < NS; ++s) {
            S* q = bufs + (size_t)s * stride;
            for (int e = tid; e < PAD; e += XXS_THREADS) {
                q[e] = from_math<S>(T(0));
                q[PAD + Nx + e] = from_math<S>(T(0));
            }
        }
    }
    __syncthreads();

    auto issue = [&](int s, int r) {
        S* dst = bufs + (size_t)s * stride + PAD;
        const S* src = fin + (size_t)r * Nx;
        issued[s] += 1;
        mbar_arrive_expect_tx(&bars[s], tx_bytes);
        bulk_g2s(dst, src, row_bytes, &bars[s]);
        if constexpr (PERIODIC) bulk_g2s(dst + Nx, src, 16u * (uint32_t)sizeof(S), &bars[s]);
        bulk_g2s(recs + (size_t)s * XREC_BYTES, static_cast<const unsigned char*>(a.rec) + (size_t)r * XREC_BYTES,
                 XREC_BYTES, &bars[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            const int r = blockIdx.x + s * G;
            if (r < Np) issue(s, r);
        }
    }

    acc_t acc1[CH][V], acc2[CH][V];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            acc1[c][v] = acc_t(0);
            acc2[c][v] = acc_t(0);
        }
    float kinf = 0.f;   // FP32 kinetic sum of this thread's rows (FP64 in the epilogue)

    int s = 0;          // stage of row r, and the parity of its barrier phase
    uint32_t ph = 0;
    int it = 0;
    bool failed = false;
    for (int r = blockIdx.x; r < Np; r += G, ++it) {
        const bool ok = mbar_wait_bounded(&bars[s], ph, WAIT_LIMIT_NS);
        S* ib = ibufs + ((it & 1) ? stride : 0) + PAD;
        // row constants, shared by both passes (the same displacement and weights)
        int n0 = 0, A = 0, base = 0;
        T w[NTAP];
        T g = T(0), d = T(0);
        float p2h = 0.f;
        acc_t rowsum = acc_t(0);
        if (ok) {
            const XRec* rc = reinterpret_cast<const XRec*>(recs + (size_t)s * XREC_BYTES);
            n0 = rc->n0;
            p2h = rc->p2h;
            const float4 w03 = *reinterpret_cast<const float4*>(rc->w32);
            const float4 w47 = *reinterpret_cast<const float4*>(rc->w32 + 4);
            const float2 w89 = *reinterpret_cast<const float2*>(rc->w32 + 8);
            w[0] = w03.x;
            w[1] = w03.y;
            w[2] = w03.z;
            w[3] = w03.w;
            w[4] = w47.x;
            w[5] = w47.y;
            w[6] = w47.z;
            w[7] = w47.w;
            w[8] = w89.x;
            w[9] = w89.y;
            if constexpr (PERIODIC) {
                const int m4 = rc->m4;   // (n0 - 4) mod Nx; Nx is a multiple of V
                A = m4 & (V - 1);
                base = m4 - A;
            } else {
                A = (n0 - 4) & (V - 1);
                base = n0 - 4 - A;
                g = rc->g32;
                d = rc->d32;
            }
            const S* rowbuf = bufs + (size_t)s * stride + PAD;
#define VL_PASS1(AA) xx_pass<S, AA, PERIODIC, CH, true>(rowbuf, ib, w, base, n0, Nx, g, d, acc1, rowsum)
            if constexpr (V == 4) {
                switch (A) {
                    case 0: VL_PASS1(0); break;
                    case 1: VL_PASS1(1); break;
                    case 2: VL_PASS1(2); break;
                    default: VL_PASS1(3); break;
                }
            } else {
                switch (A) {
                    case 0: VL_PASS1(0); break;
                    case 1: VL_PASS1(1); break;
                    case 2: VL_PASS1(2); break;
                    case 3: VL_PASS1(3); break;
                    case 4: VL_PASS1(4); break;
                    case 5: VL_PASS1(5); break;
                    case 6: VL_PASS1(6); break;
                    default: VL_PASS1(7); break;
                }
            }
#undef VL_PASS1
        }
        // every warp's first pass is done: the intermediate row is complete and stage s is free
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            const int rn = r + NS * G;
            if (rn < Np) {
                fence_proxy_async_smem();
                issue(s, rn);
            }
        }
        kinf = fmaf(p2h, (float)rowsum, kinf);
        acc_t rowsum2 = acc_t(0);
        S* orow = fout + (size_t)r * Nx;
#define VL_PASS2(AA) xx_pass<S, AA, PERIODIC, CH, false>(ib, orow, w, base, n0, Nx, g, d, acc2, rowsum2)
        if constexpr (V == 4) {
            switch (A) {
                case 0: VL_PASS2(0); break;
                case 1: VL_PASS2(1); break;
                case 2: VL_PASS2(2); break;
                default: VL_PASS2(3); break;
            }
        } else {
            switch (A) {
                case 0: VL_PASS2(0); break;
                case 1: VL_PASS2(1); break;
                case 2: VL_PASS2(2); break;
                case 3: VL_PASS2(3); break;
                case 4: VL_PASS2(4); break;
                case 5: VL_PASS2(5); break;
                case 6: VL_PASS2(6); break;
                default: VL_PASS2(7); break;
            }
        }
#undef VL_PASS2
        if (++s == NS) {
            s = 0;
            ph ^= 1u;
        }
    }
    __syncthreads();   // every warp is done with the stages and intermediate rows

    if (failed) {
        if (tid == 0) {
            atomicCAS(a.err, 0, DEV_ERR_XSHIFT_WAIT);
            for (int k = 0; k < NS; ++k)   // the last copy issued into each stage must land before exit
                if (issued[k] > 0) mbar_wait_bounded(&bars[k], (uint32_t)((issued[k] - 1) & 1), WAIT_LIMIT_NS);
        }
        __syncthreads();
        return;
    }
    if (a.ctapart && b.ctapart && a.kinpart) {
        xx_hmf_epilogue<S, CH>(a, b, acc1, acc2, kinf, reinterpret_cast<unsigned char*>(bufs));
        return;
    }
    i128* scratch = reinterpret_cast<i128*>(bufs);
    colsum_epilogue<S, CH>(a, acc1, scratch);
    kin_epilogue(a, (double)kinf, red);
    colsum_epilogue<S, CH>(b, acc2, scratch);
}

template <typename S, bool PERIODIC>
__global__ void __launch_bounds__(XXS_THREADS, XXS_CTAS_PER_SM) xxshift_kernel(XShiftArgs a, XShiftArgs b)
{
    xxshift_body<S, PERIODIC>(a, b);
}

size_t xxshift_smem_bytes(int Nx, int pad, int stages, int elem_bytes)
{
    const size_t row = (size_t)(Nx + 2 * pad) * (size_t)elem_bytes;
    const size_t rows = (size_t)stages * (row + XREC_BYTES) + 2 * row;
    return 256 + (rows > XX_HMF_EPI_BYTES ? rows : XX_HMF_EPI_BYTES);
}

cudaError_t launch_xxshift(int elem_bytes, bool periodic, int grid, const XShiftArgs& a, const XShiftArgs& b,
                           cudaStream_t st)
{
    if (a.rec == nullptr || a.Nx > XXS_MAX_NX || a.stages < 1 || a.stages > 8) return cudaErrorInvalidValue;
    const size_t smem = xxshift_smem_bytes(a.Nx, a.pad, a.stages, elem_bytes);
    if (elem_bytes == 2) {
        if (periodic) xxshift_kernel<bf16, true><<<grid, XXS_THREADS, smem, st>>>(a, b);
        else xxshift_kernel<bf16, false><<<grid, XXS_THREADS, smem, st>>>(a, b);
    } else {
        if (periodic) xxshift_kernel<float, true><<<grid, XXS_THREADS, smem, st>>>(a, b);
        else xxshift_kernel<float, false><<<grid, XXS_THREADS, smem, st>>>(a, b);
    }
    return cudaGetLastError();
}

cudaError_t xxshift_occupancy(int elem_bytes, bool periodic, size_t smem, int* blocks)
{
    if (elem_bytes == 2)
        return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xxshift_kernel<bf16, true>, XXS_THREADS, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xxshift_kernel<bf16, false>, XXS_THREADS, smem);
    return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xxshift_kernel<float, true>, XXS_THREADS, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xxshift_kernel<float, false>, XXS_THREADS, smem);
}

int xshift_max_cols(int elem_bytes, int threads)
{
    const int V = 16 / elem_bytes;
    return V * threads * (elem_bytes == 2 ? maxch_of<bf16>() : XS_MAXCH);
}

size_t xshift_smem_bytes(int Nx, int pad, int stages, int elem_bytes)
{
    return 256 + (size_t)stages * ((size_t)(Nx + 2 * pad) * (size_t)elem_bytes + XREC_BYTES);
}

template <typename S, bool P, bool K>
static cudaError_t launch_x(int grid, int threads, const XShiftArgs& a, cudaStream_t st)
{
    const size_t smem = xshift_smem_bytes(a.Nx, a.pad, a.stages, (int)sizeof(S));
    xshift_kernel<S, P, K><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_xshift(int elem_bytes, bool periodic, bool kin, int grid, int threads, const XShiftArgs& a,
                          cudaStream_t st)
{
    if (elem_bytes == 8) {
        if (periodic) return kin ? launch_x<double, true, true>(grid, threads, a, st)
                                 : launch_x<double, true, false>(grid, threads, a, st);
        return kin ? launch_x<double, false, true>(grid, threads, a, st)
                   : launch_x<double, false, false>(grid, threads, a, st);
    }
    if (elem_bytes == 2) {
        if (periodic) return kin ? launch_x<bf16, true, true>(grid, threads, a, st)
                                 : launch_x<bf16, true, false>(grid, threads, a, st);
        return kin ? launch_x<bf16, false, true>(grid, threads, a, st)
                   : launch_x<bf16, false, false>(grid, threads, a, st);
    }
    if (periodic) return kin ? launch_x<float, true, true>(grid, threads, a, st)
                             : launch_x<float, true, false>(grid, threads, a, st);
    return kin ? launch_x<float, false, true>(grid, threads, a, st)
               : launch_x<float, false, false>(grid, threads, a, st);
}

// ============================================================================ global spline
// The comparison method of the paper's Tables 1-2 (Eq. tridiagsys): the spline whose f'' solves
// the tridiagonal system instead of Eq. findif, as a filter of GS_TAPS taps over the line extended
// periodically or oddly about the nodes -1 and n (the constants' header gives the derivation).
// IEEE arithmetic in the storage type S (double or float); the filter taps are formed in FP64.

// Tap t < GS_TAPS of a line with foot fraction beta.
__device__ __forceinline__ double gs_tap(double beta, const double* __restrict__ h, int t)
{
    const double alpha = 1.0 - beta;
    const double gm = (alpha * alpha * alpha - alpha) / 6.0, dl = (beta * beta * beta - beta) / 6.0;
    const int u = t - GS_R - 1;
    double w = (u == 0 ? alpha : 0.0) + (u == 1 ? beta : 0.0);
    if (u <= GS_R + 1) w += gm * h[u + GS_R + 1];
    if (u - 1 >= -GS_R - 1) w += dl * h[u + GS_R];
    return w;
}

// Value of the extended line at node q (|q| within one halo of the grid): periodic wrap, or the odd
// extension about -1 and n of a zero-outside line (0 where the reflection leaves the grid: such
// nodes feed only outputs whose foot lies outside, which are 0).
template <typename S, bool PER>
__device__ __forceinline__ S gs_ext(const S* __restrict__ line, long long stride, int q, int n)
{
    if (q >= 0 && q < n) return line[(long long)q * stride];
    if constexpr (PER) {
        int r = q % n;
        if (r < 0) r += n;
        return line[(long long)r * stride];
    } else {
        if (q == -1 || q == n) return S(0);
        const int m = q < 0 ? -2 - q : 2 * n - q;
        return (m >= 0 && m < n) ? S(-line[(long long)m * stride]) : S(0);
    }
}

// x: rows strided over the CTAs; a row and its GS_HALO extended nodes each side in shared memory,
// thread t owns columns t + c blockDim (c < GS_XCH: coalesced, conflict-free window reads), with the
// density (and kinetic) partials of the same forms as the spline x-shift.
template <typename S, bool PERIODIC, bool KIN>
__global__ void __launch_bounds__(GS_XTHREADS) gs_xshift_kernel(XShiftArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    const int Nx = a.Nx, Np = a.Np, tid = threadIdx.x, nthreads = blockDim.x;
    S* ext = reinterpret_cast<S*>(smem_dyn);
    S* W = ext + Nx + 2 * GS_HALO;
    __shared__ double red[32];
    const S* __restrict__ fin = static_cast<const S*>(a.fin);
    S* __restrict__ fout = static_cast<S*>(a.fout);
    S colacc[GS_XCH];
#pragma unroll
    for (int c = 0; c < GS_XCH; ++c) colacc[c] = S(0);
    double kin = 0.0;
    for (int r = blockIdx.x; r < Np; r += gridDim.x) {
        const S* row = fin + (size_t)r * Nx;
        for (int q = tid; q < Nx + 2 * GS_HALO; q += nthreads) ext[q] = gs_ext<S, PERIODIC>(row, 1, q - GS_HALO, Nx);
        if (tid < GS_TAPS) W[tid] = (S)gs_tap(a.beta[r], a.gs_h, tid);
        const int n0 = a.n0[r];
        __syncthreads();
        // FP32: the row's taps in registers (one shared-memory read per multiply-add); FP64 taps
        // would take 128 registers and stay in shared memory
        constexpr int WR = sizeof(S) == 4 ? GS_TAPS : 1;
        S wr[WR];
        if constexpr (sizeof(S) == 4) {
#pragma unroll
            for (int t = 0; t < GS_TAPS; ++t) wr[t] = W[t];
        }
        S rowsum = S(0);
        S* orow = fout + (size_t)r * Nx;
#pragma unroll
        for (int c = 0; c < GS_XCH; ++c) {
            const int i = tid + c * nthreads;
            if (i < Nx) {
                int k = i + n0;
                S out = S(0);
                if constexpr (PERIODIC) {
                    k %= Nx;
                    if (k < 0) k += Nx;
                }
                if (PERIODIC || (k >= -1 && k < Nx)) {
                    const S* e = ext + k + 1;   // extended node k - GS_R - 1
                    S acc = S(0);
                    if constexpr (sizeof(S) == 4) {
#pragma unroll
                        for (int t = 0; t < GS_TAPS; ++t) acc = fma(wr[t], e[t], acc);
                    } else {
#pragma unroll 16
                        for (int t = 0; t < GS_TAPS; ++t) acc = fma(W[t], e[t], acc);
                    }
                    out = acc;
                }
                orow[i] = out;
                colacc[c] += out;
                rowsum += out;
            }
        }
        if constexpr (KIN) {
            const double pj = a.pmin + (double)r * a.dp;
            kin += 0.5 * pj * pj * (double)rowsum;
        }
        __syncthreads();   // every thread done with this row's nodes and taps
    }
    // column sums in the forms of the spline x-shift: exact int64 atomics, int64 or FP64 CTA rows
#pragma unroll
    for (int c = 0; c < GS_XCH; ++c) {
        const int i = tid + c * nthreads;
        if (i >= Nx) continue;
        long long q;
        if constexpr (sizeof(S) == 8) q = (long long)fx128_from_f64((double)colacc[c], a.k_col);
        else q = (long long)fx128_from_f32((float)colacc[c], a.k_col);
        if (a.colacc) atomicAdd(a.colacc + i, (unsigned long long)q);
        else if (a.colpart64) a.colpart64[(size_t)blockIdx.x * Nx + i] = q;
        else if (a.colpart) a.colpart[(size_t)blockIdx.x * Nx + i] = (double)colacc[c];
    }
    if constexpr (KIN) kin_epilogue(a, kin, red);
}

// p: tiles of 32 columns x GS_PTH rows; the union of the columns' windows (GS_PROWS rows at most,
// else straight from global memory) and each column's taps in shared memory; lane = column.
template <typename S, bool PPER>
__global__ void __launch_bounds__(256) gs_pshift_kernel(PShiftArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    S* stage = reinterpret_cast<S*>(smem_dyn);   // [GS_PROWS][32]
    S* W = stage + GS_PROWS * 32;                 // [GS_TAPS][32]
    const S* __restrict__ fin = static_cast<const S*>(a.fin);
    S* __restrict__ fout = static_cast<S*>(a.fout);
    const int Nx = a.Nx, Np = a.Np, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntx = (Nx + 31) / 32, nty = (Np + GS_PTH - 1) / GS_PTH;
    for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
        const int i = (tile % ntx) * 32 + lane, j0 = (tile / ntx) * GS_PTH;
        const bool colok = i < Nx;
        const int n0 = colok ? a.n0[i] : 0;
        int kmin = colok ? n0 : 0x7fffffff, kmax = colok ? n0 : (int)0x80000000;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        const int r0 = j0 + kmin - GS_R - 1;
        const long long rows = (long long)GS_PTH + GS_TAPS + ((long long)kmax - kmin);
        const bool staged = rows <= GS_PROWS;
        if (staged) {
            for (int q = warp; q < (int)rows; q += 8)
                stage[q * 32 + lane] = colok ? gs_ext<S, PPER>(fin + i, Nx, r0 + q, Np) : S(0);
        }
        const double be = colok ? a.beta[i] : 0.0;
        for (int t = warp; t < GS_TAPS; t += 8) W[t * 32 + lane] = (S)gs_tap(be, a.gs_h, t);
        __syncthreads();
        constexpr int RQ = GS_PTH / 8;   // output rows per thread (consecutive feet)
        bool done = false;
        if constexpr (sizeof(S) == 4) {
            if (staged && colok) {
                // FP32: the column's taps in registers and each staged node read once for the
                // thread's RQ outputs (input-stationary: RQ + GS_TAPS - 1 reads, not RQ * GS_TAPS)
                S wr[GS_TAPS], acc[RQ];
#pragma unroll
                for (int t = 0; t < GS_TAPS; ++t) wr[t] = W[t * 32 + lane];
#pragma unroll
                for (int q = 0; q < RQ; ++q) acc[q] = S(0);
                const int jb = j0 + warp * RQ;
                const S* e = stage + (jb + n0 - GS_R - 1 - r0) * 32 + lane;
#pragma unroll
                for (int u = 0; u < RQ + GS_TAPS - 1; ++u) {
                    const S v = e[u * 32];
#pragma unroll
                    for (int q = 0; q < RQ; ++q) {
                        const int t = u - q;
                        if (t >= 0 && t < GS_TAPS) acc[q] = fma(wr[t], v, acc[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < RQ; ++q) {
                    const int j = jb + q, k = j + n0;
                    if (j < Np) fout[(size_t)j * Nx + i] = (PPER || (k >= -1 && k < Np)) ? acc[q] : S(0);
                }
                done = true;
            }
        }
#pragma unroll 1
        for (int q = 0; q < (done ? 0 : RQ); ++q) {
            const int j = j0 + warp * RQ + q;
            if (!colok || j >= Np) continue;
            const int k = j + n0;
            S out = S(0);
            if (PPER || (k >= -1 && k < Np)) {
                S acc = S(0);
                if (staged) {
                    const S* e = stage + (k - GS_R - 1 - r0) * 32 + lane;
#pragma unroll 16
                    for (int t = 0; t < GS_TAPS; ++t) acc = fma(W[t * 32 + lane], e[t * 32], acc);
                } else {
#pragma unroll 4
                    for (int t = 0; t < GS_TAPS; ++t)
                        acc = fma(W[t * 32 + lane], gs_ext<S, PPER>(fin + i, Nx, k - GS_R - 1 + t, Np), acc);
                }
                out = acc;
            }
            fout[(size_t)j * Nx + i] = out;
        }
        __syncthreads();   // before the next tile's rows and taps
    }
}

size_t gs_xshift_smem_bytes(int Nx, int elem_bytes)
{
    return (size_t)(Nx + 2 * GS_HALO + GS_TAPS) * (size_t)elem_bytes;
}

size_t gs_pshift_smem_bytes(int elem_bytes) { return (size_t)(GS_PROWS + GS_TAPS) * 32 * (size_t)elem_bytes; }

cudaError_t launch_gs_xshift(int elem_bytes, bool periodic, bool kin, int grid, const XShiftArgs& a, cudaStream_t st)
{
    if (a.beta == nullptr || a.gs_h == nullptr || a.Nx > GS_XTHREADS * GS_XCH || a.Nx < GS_MIN_N)
        return cudaErrorInvalidValue;
    const size_t smem = gs_xshift_smem_bytes(a.Nx, elem_bytes);
    const int T = GS_XTHREADS;
    if (elem_bytes == 8) {
        if (periodic) kin ? gs_xshift_kernel<double, true, true><<<grid, T, smem, st>>>(a)
                          : gs_xshift_kernel<double, true, false><<<grid, T, smem, st>>>(a);
        else kin ? gs_xshift_kernel<double, false, true><<<grid, T, smem, st>>>(a)
                 : gs_xshift_kernel<double, false, false><<<grid, T, smem, st>>>(a);
    } else if (elem_bytes == 4) {
        if (periodic) kin ? gs_xshift_kernel<float, true, true><<<grid, T, smem, st>>>(a)
                          : gs_xshift_kernel<float, true, false><<<grid, T, smem, st>>>(a);
        else kin ? gs_xshift_kernel<float, false, true><<<grid, T, smem, st>>>(a)
                 : gs_xshift_kernel<float, false, false><<<grid, T, smem, st>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_gs_pshift(int elem_bytes, bool p_periodic, int grid, const PShiftArgs& a, cudaStream_t st)
{
    if (a.beta == nullptr || a.gs_h == nullptr || a.Np < GS_MIN_N) return cudaErrorInvalidValue;
    const size_t smem = gs_pshift_smem_bytes(elem_bytes);
    if (elem_bytes == 8) {
        if (p_periodic) gs_pshift_kernel<double, true><<<grid, 256, smem, st>>>(a);
        else gs_pshift_kernel<double, false><<<grid, 256, smem, st>>>(a);
    } else if (elem_bytes == 4) {
        if (p_periodic) gs_pshift_kernel<float, true><<<grid, 256, smem, st>>>(a);
        else gs_pshift_kernel<float, false><<<grid, 256, smem, st>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t gs_occupancy(int elem_bytes, bool xdir, size_t smem, int* blocks)
{
    if (xdir)
        return elem_bytes == 8
                   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, gs_xshift_kernel<double, true, true>, GS_XTHREADS, smem)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, gs_xshift_kernel<float, true, true>, GS_XTHREADS, smem);
    return elem_bytes == 8 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, gs_pshift_kernel<double, false>, 256, smem)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, gs_pshift_kernel<float, false>, 256, smem);
}

// ============================================================================ p-shift
// Warp-specialised: PS_RG compute warps (16 output rows each) and one producer warp per CTA.  The
// producer works out each tile's window, stages its columns' foot offsets (and, for partial column
// tiles, filters) in the slot info[b] and issues the copies of its rows and filters into buffer b
// (full[b]); the compute warps take the tiles in the same order and hand each buffer back through
// empty[b].  No CTA-wide barrier per tile: a warp waits only for the data it reads.
template <typename S, bool PPER>
__device__ __forceinline__ void pshift_body(const CUtensorMap* tmap_ptr, const PShiftArgs& a,
                                            const HmfFiltArgs* hf = nullptr)
{
    using T = typename VecOf<S>::T;
    constexpr int NB = PS_NB;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + NB;
    S* bufs = reinterpret_cast<S*>(smem_raw + 128);
    constexpr int BUF = PS_RB * PS_TW;
    static_assert(2 * NB * 8 <= 128, "barriers fit in front of the buffers");

    const S* __restrict__ fin = static_cast<const S*>(a.fin);
    S* __restrict__ fout = static_cast<S*>(a.fout);
    const T* __restrict__ wcol = static_cast<const T*>(a.w);
    const T* __restrict__ gdcol = static_cast<const T*>(a.gd);
    const int Nx = a.Nx, Np = a.Np;
    const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 5;
    const int ntx = (Nx + PS_TW - 1) / PS_TW, nty = (Np + PS_TH - 1) / PS_TH;
    const int ntiles = ntx * nty;
    const int G = gridDim.x;

    struct __align__(16) TileInfo {
        T w[NTAP][PS_TW];
        T gd[2][PS_TW];
        int n0[PS_TW];
        TileWin t;
    };
    __shared__ TileInfo info[NB];

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], PS_RG);
        }
        fence_barrier_init();
        prefetch_tensormap(tmap_ptr);
    }
    __syncthreads();   // the last CTA-wide barrier: the roles part here

    if (grp == PS_RG) {
        // ---- producer.  Filters of a tile with all 32 columns inside the grid arrive by bulk copies
        // on the tile's barrier; BF16 storage loads them (measured faster there, its tiles being half
        // the bytes), as does the last, partial column tile.
        // HMF with hf->on: the filters of the tile's columns are formed here from Mx, My (Eq.
        // hmfmeanforce) instead of being loaded, and no filter launch precedes this one.
        constexpr uint32_t ROWB = PS_TW * (uint32_t)sizeof(T);
        constexpr uint32_t WBYTES = (NTAP + (PPER ? 0 : 2)) * ROWB;
        const bool hfilt = hf != nullptr && hf->on != 0;
        double hMx = 0.0, hMy = 0.0;
        if (hfilt) hmf_mxmy_warp(*hf, hMx, hMy);
        int k = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles; tile += G, ++k) {
            const int b = k % NB;
            // the tile's window, offsets and (loaded or formed) filters first: their global loads
            // overlap the wait for the slot
            int n0l;
            bool cv;
            TileWin t;
            T wr[NTAP], gr[2];
            bool wbulk;
            if (hfilt) {
                const int icol = (tile % ntx) * PS_TW + lane;
                cv = icol < Nx;
                FiltF32 o{};
                if (cv) o = filt_f32(hmf_force(hMx, hMy, hf->sintab[icol], hf->costab[icol]) * hf->cp);
                n0l = o.n0;
                t = tile_window_of<PPER>(tile, ntx, cv, n0l);
#pragma unroll
                for (int q = 0; q < NTAP; ++q) wr[q] = cv ? T(o.w[q]) : T(0);
                gr[0] = cv ? T(o.g) : T(0);
                gr[1] = cv ? T(o.d) : T(0);
                wbulk = false;
            } else {
                t = tile_window<PPER>(tile, ntx, a.n0, Nx, lane, n0l, cv);
                wbulk = sizeof(S) >= 4 && t.i0 + PS_TW <= Nx;
            }
            const int ic = t.i0 + lane;
            if (!wbulk && !hfilt) {
#pragma unroll
                for (int q = 0; q < NTAP; ++q) wr[q] = cv ? wcol[(size_t)q * Nx + ic] : T(0);
                if constexpr (!PPER) {
                    gr[0] = cv ? gdcol[ic] : T(0);
                    gr[1] = cv ? gdcol[Nx + ic] : T(0);
                }
            }
            if (k >= NB) ok = mbar_wait_bounded(&empty[b], (uint32_t)(((k / NB) - 1) & 1), WAIT_LIMIT_NS);
            if (!__all_sync(0xffffffffu, ok)) break;
            if (!wbulk) {
#pragma unroll
                for (int q = 0; q < NTAP; ++q) info[b].w[q][lane] = wr[q];
                if constexpr (!PPER) {
                    info[b].gd[0][lane] = gr[0];
                    info[b].gd[1][lane] = gr[1];
                }
            }
            info[b].n0[lane] = n0l;
            __syncwarp();
            if (lane == 0) {
                info[b].t = t;
                fence_proxy_async_smem();   // the compute warps' reads of buffer b before its refill
                const uint32_t tile_bytes = t.smem_ok ? (uint32_t)(t.nb * PS_BH * PS_TW * sizeof(S)) : 0u;
                mbar_arrive_expect_tx(&full[b], tile_bytes + (wbulk ? WBYTES : 0u));   // releases info[b]
                if (t.smem_ok)
                    for (int q = 0; q < t.nb; ++q)
                        tma_load_2d(bufs + (size_t)b * BUF + (size_t)q * PS_BH * PS_TW, tmap_ptr, t.i0, t.r0 + q * PS_BH, &full[b]);
                if (wbulk) {
                    for (int q = 0; q < NTAP; ++q) bulk_g2s(info[b].w[q], wcol + (size_t)q * Nx + t.i0, ROWB, &full[b]);
                    if constexpr (!PPER) {
                        bulk_g2s(info[b].gd[0], gdcol + t.i0, ROWB, &full[b]);
                        bulk_g2s(info[b].gd[1], gdcol + Nx + t.i0, ROWB, &full[b]);
                    }
                }
            }
        }
        if (lane == 0) {
            if (!ok) atomicCAS(a.err, 0, DEV_ERR_PSHIFT_WAIT);
            // stay until every copy issued has landed (the CTA's shared memory must outlive them)
            for (int j = k - 1; j >= 0 && j >= k - NB; --j)
                mbar_wait_bounded(&full[j % NB], (uint32_t)((j / NB) & 1), WAIT_LIMIT_NS);
        }
        return;
    }

    // ---- compute warps
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, ++k) {
        const int b = k % NB;
        if (!mbar_wait_bounded(&full[b], (uint32_t)((k / NB) & 1), WAIT_LIMIT_NS)) {
            if (lane == 0) atomicCAS(a.err, 0, DEV_ERR_PSHIFT_WAIT);
            break;
        }
        const TileWin t = info[b].t;
        const int n0_i = info[b].n0[lane];
        const int i = t.i0 + lane;
        const bool colvalid = i < Nx;
        T w[NTAP];
#pragma unroll
        for (int q = 0; q < NTAP; ++q) w[q] = info[b].w[q][lane];
        T g = T(0), d = T(0);
        if constexpr (!PPER) {
            g = info[b].gd[0][lane];
            d = info[b].gd[1][lane];
        }
        const int jb = t.j0 + grp * PS_RPT;     // first output row of this thread
        T x[PS_RPT + 9];
        if (t.smem_ok) {
            const S* buf = bufs + (size_t)b * BUF;
            const int base = jb + n0_i - 4 - t.r0;
#pragma unroll
            for (int u = 0; u < PS_RPT + 9; ++u) x[u] = to_math(buf[(base + u) * PS_TW + lane]);
        } else {
#pragma unroll
            for (int u = 0; u < PS_RPT + 9; ++u)
                x[u] = colvalid ? to_math(gload_p<S, PPER>(fin, jb + n0_i - 4 + u, i, Nx, Np)) : T(0);
        }
        // the staged window and slot are read: hand buffer b back (stores below need neither)
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
        // A tile whose columns and rows all lie inside the grid, with every foot cell inside
        // too (the common case), takes the rows without per-row checks.
        const bool interior = t.i0 + PS_TW <= Nx && t.j0 + PS_TH <= Np &&
                              (PPER || (t.j0 + t.kmin >= 0 && t.j0 + PS_TH - 1 + t.kmax < Np - 1));
        if (interior) {
            S* __restrict__ op = fout + (size_t)jb * Nx + i;
#pragma unroll
            for (int rr = 0; rr < PS_RPT; ++rr) {
                T acc = w[0] * x[rr];
#pragma unroll
                for (int q = 1; q < NTAP; ++q) acc = fma(w[q], x[rr + q], acc);
                *op = from_math<S>(acc);
                op += Nx;
            }
        } else {
#pragma unroll
            for (int rr = 0; rr < PS_RPT; ++rr) {
                const int j = jb + rr;
                T acc = w[0] * x[rr];
#pragma unroll
                for (int q = 1; q < NTAP; ++q) acc = fma(w[q], x[rr + q], acc);
                if constexpr (!PPER) {
                    const int kk = j + n0_i;
                    if (kk < 0 || kk >= Np - 1) acc = edge_fix(acc, &x[rr], kk, Np, g, d);
                }
                if (colvalid && j < Np) fout[(size_t)j * Nx + i] = from_math<S>(acc);
            }
        }
    }
}

template <typename S, bool PPER>
__global__ void __launch_bounds__(PS_THREADS, sizeof(S) == 8 ? 1 : PS_MINB) pshift_kernel(const __grid_constant__ CUtensorMap tmap, PShiftArgs a,
                                                                                          const __grid_constant__ HmfFiltArgs hf)
{
    pshift_body<S, PPER>(&tmap, a, &hf);
}

// Batched form: tensor maps and arguments of each slot, per buffer parity, in global memory.
template <typename T, bool PPER>
__global__ void __launch_bounds__(PS_THREADS, PS_MINB) pshift_batch_kernel(const CUtensorMap* __restrict__ tmaps,
                                                                         const PShiftArgs* __restrict__ args,
                                                                         const int* __restrict__ ver)
{
    const int slot = blockIdx.y;
    const int k = slot * 2 + ver[slot];
    const PShiftArgs a = args[k];
    if (a.Np <= 0) return;
    pshift_body<T, PPER>(tmaps + k, a);
}

size_t pshift_smem_bytes(int elem_bytes)
{
    return 256 + (size_t)PS_NB * PS_RB * PS_TW * (size_t)elem_bytes;
}

template <typename S, bool PPER>
static cudaError_t launch_p(int grid, const CUtensorMap* tmap, const PShiftArgs& a, const HmfFiltArgs& hf, cudaStream_t st)
{
    const size_t smem = pshift_smem_bytes((int)sizeof(S));
    pshift_kernel<S, PPER><<<grid, PS_THREADS, smem, st>>>(*tmap, a, hf);
    return cudaGetLastError();
}

cudaError_t launch_pshift(int elem_bytes, bool p_periodic, int grid, const CUtensorMap* tmap, const PShiftArgs& a,
                          const HmfFiltArgs* hfp, cudaStream_t st)
{
    HmfFiltArgs hf{};
    if (hfp && elem_bytes <= 4) hf = *hfp;
    if (elem_bytes == 8) return p_periodic ? launch_p<double, true>(grid, tmap, a, hf, st) : launch_p<double, false>(grid, tmap, a, hf, st);
    if (elem_bytes == 2) return p_periodic ? launch_p<bf16, true>(grid, tmap, a, hf, st) : launch_p<bf16, false>(grid, tmap, a, hf, st);
    return p_periodic ? launch_p<float, true>(grid, tmap, a, hf, st) : launch_p<float, false>(grid, tmap, a, hf, st);
}

cudaError_t launch_xshift_batch(bool periodic, bool kin, int slots, int ctas_per_slot, size_t smem,
                                const XShiftArgs* args, const int* ver, cudaStream_t st)
{
    const dim3 grid(ctas_per_slot, slots);
    if (periodic) {
        if (kin) xshift_batch_kernel<float, true, true><<<grid, XS_THREADS_MIN, smem, st>>>(args, ver);
        else xshift_batch_kernel<float, true, false><<<grid, XS_THREADS_MIN, smem, st>>>(args, ver);
    } else {
        if (kin) xshift_batch_kernel<float, false, true><<<grid, XS_THREADS_MIN, smem, st>>>(args, ver);
        else xshift_batch_kernel<float, false, false><<<grid, XS_THREADS_MIN, smem, st>>>(args, ver);
    }
    return cudaGetLastError();
}

cudaError_t launch_pshift_batch(int slots, int ctas_per_slot, const CUtensorMap* tmaps, const PShiftArgs* args,
                                const int* ver, cudaStream_t st)
{
    const dim3 grid(ctas_per_slot, slots);
    pshift_batch_kernel<float, false><<<grid, PS_THREADS, pshift_smem_bytes(4), st>>>(tmaps, args, ver);
    return cudaGetLastError();
}

// Opt every shift kernel into the shared memory it may use (called once per device, before any
// launch or stream capture).  Also reports the resident CTAs per SM of the two sweeps.
cudaError_t set_kernel_attributes(int max_smem)
{
    cudaError_t e = cudaSuccess;
#define VL_ATTR(fn) \
    if (e == cudaSuccess) e = allow_dynamic_smem(fn, max_smem)
    VL_ATTR((xshift_kernel<double, true, true>));
    VL_ATTR((xshift_kernel<double, true, false>));
    VL_ATTR((xshift_kernel<double, false, true>));
    VL_ATTR((xshift_kernel<double, false, false>));
    VL_ATTR((xshift_kernel<float, true, true>));
    VL_ATTR((xshift_kernel<float, true, false>));
    VL_ATTR((xshift_kernel<float, false, true>));
    VL_ATTR((xshift_kernel<float, false, false>));
    VL_ATTR((pshift_kernel<double, true>));
    VL_ATTR((pshift_kernel<double, false>));
    VL_ATTR((pshift_kernel<float, true>));
    VL_ATTR((pshift_kernel<float, false>));
    VL_ATTR((xshift_batch_kernel<float, true, true>));
    VL_ATTR((xshift_batch_kernel<float, true, false>));
    VL_ATTR((xshift_batch_kernel<float, false, true>));
    VL_ATTR((xshift_batch_kernel<float, false, false>));
    VL_ATTR((pshift_batch_kernel<float, false>));
    VL_ATTR((xshift_kernel<bf16, true, true>));
    VL_ATTR((xshift_kernel<bf16, true, false>));
    VL_ATTR((xshift_kernel<bf16, false, true>));
    VL_ATTR((xshift_kernel<bf16, false, false>));
    VL_ATTR((pshift_kernel<bf16, true>));
    VL_ATTR((pshift_kernel<bf16, false>));
    VL_ATTR((gs_xshift_kernel<double, true, true>));
    VL_ATTR((gs_xshift_kernel<double, true, false>));
    VL_ATTR((gs_xshift_kernel<double, false, true>));
    VL_ATTR((gs_xshift_kernel<double, false, false>));
    VL_ATTR((gs_xshift_kernel<float, true, true>));
    VL_ATTR((gs_xshift_kernel<float, true, false>));
    VL_ATTR((gs_xshift_kernel<float, false, true>));
    VL_ATTR((gs_xshift_kernel<float, false, false>));
    VL_ATTR((gs_pshift_kernel<double, true>));
    VL_ATTR((gs_pshift_kernel<double, false>));
    VL_ATTR((gs_pshift_kernel<float, true>));
    VL_ATTR((gs_pshift_kernel<float, false>));
    VL_ATTR((xxshift_kernel<float, true>));
    VL_ATTR((xxshift_kernel<float, false>));
    VL_ATTR((xxshift_kernel<bf16, true>));
    VL_ATTR((xxshift_kernel<bf16, false>));
#undef VL_ATTR
    return e;
}

cudaError_t xshift_occupancy(int elem_bytes, bool periodic, int threads, size_t smem, int* blocks)
{
    if (elem_bytes == 8)
        return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_kernel<double, true, true>, threads, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_kernel<double, false, true>, threads, smem);
    if (elem_bytes == 2)
        return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_kernel<bf16, true, true>, threads, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_kernel<bf16, false, true>, threads, smem);
    return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_kernel<float, true, true>, threads, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_kernel<float, false, true>, threads, smem);
}

cudaError_t pshift_occupancy(int elem_bytes, int* blocks)
{
    const size_t smem = pshift_smem_bytes(elem_bytes);
    if (elem_bytes == 8)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pshift_kernel<double, false>, PS_THREADS, smem);
    if (elem_bytes == 2)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pshift_kernel<bf16, false>, PS_THREADS, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pshift_kernel<float, false>, PS_THREADS, smem);
}

}  // namespace vl
