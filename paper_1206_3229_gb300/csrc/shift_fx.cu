// shift_fx.cu -- the two sweeps for 64-bit fixed-point storage (VLASOV_FX64).
//
// f is stored as X = round(f * 2^(61-Ef)) in int64 (|f| < 2^Ef, Ef = a bound four times the largest
// uploaded |f|): the same 8 bytes per cell as FP64, an absolute resolution of 2^-59 of max|f|, and no
// IEEE decoding.  Each staged element splits with two integer instructions into
//   X = kx * 2^30 + rem,  kx = X >> 30 (int32), rem in [0, 2^30)
// and the filter runs as in the emulated-FP64 sweeps (emul.cuh): 10 IMAD.WIDE on kx and 10 paired
// FMAs (FFMA2) on ((float)kx, (float)rem); the int64 result T is already in storage units.  Data
// movement is that of shift_kernels.cu: whole rows by 1-D bulk copies (x-shift), 2-D TMA column
// tiles with zero fill (p-shift).
#include "emul.cuh"
#include "fixed_point.cuh"
#include "ptx.cuh"
#include "shift_common.cuh"
#include "vlasov_internal.cuh"

namespace vl {

namespace {

constexpr int XF_V = 8;       // consecutive outputs per thread and chunk
constexpr int XF_W = 18;      // window elements: V + 9 + alignment slack (even)
constexpr int XF_MAXCH = 2;   // chunks per row per thread (Nx <= 8 * 256 * 2 = 4096)
constexpr int PSF_RB = 192;   // staged rows per p-shift buffer (two CTAs per SM)

struct FxW {
    int Wh[NTAP];
    float2 wlr[NTAP];   // (wl, w 2^30 2^-30): one paired FMA with (kf, (float)rem)
};

__device__ __forceinline__ void fx_split(long long X, int& kx, float& kf, float& rf)
{
    const uint32_t lo = (uint32_t)X, hi = (uint32_t)((unsigned long long)X >> 32);
    kx = (int)__funnelshift_r(lo, hi, 30);
    kf = __int2float_rn(kx);
    rf = __uint2float_rn(lo & 0x3FFFFFFFu);
}

// Stored value of a filter result T (storage units).  Results outside |f| < 2^Ef (|T| >= 2^61) are
// caught from the high word: hi + 2^29 < 2^30 for every valid T, so the OR of these over a CTA
// stays below 2^30 unless one result was out of range.
__device__ __forceinline__ long long fx_store(long long T, uint32_t& rng)
{
    rng |= (uint32_t)((unsigned long long)T >> 32) + (1u << 29);
    return T;
}

// The rare boundary outputs of non-periodic axes, recomputed in FP64 from the fixed values.
__device__ __forceinline__ long long fx_edge(const long long* X, const double* w64, size_t wstride, int k, int n,
                                             double g, double d, double unit, int Ef)
{
    double xv[NTAP];
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < NTAP; ++t) {
        xv[t] = (double)X[t] * unit;
        acc = fma(w64[(size_t)t * wstride], xv[t], acc);
    }
    const double out = edge_fix(acc, xv, k, n, g, d);
    return (long long)fx128_from_f64(out, FX_FRAC - Ef);
}

// XF_V consecutive outputs of one x row from the staged fixed-point values starting at `src`
// (f_{k-4-A} .. ): input-stationary, each element split once and fed to the outputs it touches.
// The two FP32 residual products of a tap go through one paired FMA (FFMA2).
template <int A>
__device__ __forceinline__ void fx_chunk(const long long* src, const FxW& w, long long (&out)[XF_V], uint32_t& rng)
{
    long long M[XF_V];
    float2 S[XF_V];
#pragma unroll
    for (int v = 0; v < XF_V; ++v) {
        M[v] = EMUL_M0;
        S[v] = make_float2(0.f, 0.f);
    }
    const longlong2* q = reinterpret_cast<const longlong2*>(src);
#pragma unroll
    for (int h = 0; h < XF_W / 2; ++h) {
        const longlong2 pr = q[h];
        int kx0, kx1;
        float kf0, rf0, kf1, rf1;
        fx_split(pr.x, kx0, kf0, rf0);
        fx_split(pr.y, kx1, kf1, rf1);
        const float2 xa = make_float2(kf0, rf0), xb = make_float2(kf1, rf1);
#pragma unroll
        for (int v = 0; v < XF_V; ++v) {
            const int t0 = 2 * h - A - v, t1 = t0 + 1;   // taps of the two elements for output v
            const bool v0 = t0 >= 0 && t0 < NTAP, v1 = t1 >= 0 && t1 < NTAP;
            // products first, then one three-input 64-bit sum (IADD3 + IADD3.X) per pair
            if (v0 && v1) M[v] = M[v] + (long long)w.Wh[t0] * (long long)kx0 + (long long)w.Wh[t1] * (long long)kx1;
            else if (v0) M[v] += (long long)w.Wh[t0] * (long long)kx0;
            else if (v1) M[v] += (long long)w.Wh[t1] * (long long)kx1;
            if (v0) S[v] = __ffma2_rn(w.wlr[t0], xa, S[v]);
            if (v1) S[v] = __ffma2_rn(w.wlr[t1], xb, S[v]);
        }
    }
#pragma unroll
    for (int v = 0; v < XF_V; ++v) out[v] = fx_store(emul_finish(M[v], S[v].x + S[v].y), rng);
}

}  // namespace

// ============================================================================ x-shift (FX64)
template <bool PERIODIC, bool KIN>
__device__ __forceinline__ void xshift_fx_body(const XShiftArgs& a, const EmulArgs& em)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    long long* bufs = reinterpret_cast<long long*>(smem_raw + 128);
    __shared__ unsigned int done_cnt[8];   // warps finished with each stage's current row
    __shared__ unsigned int issued[8];     // copies issued into each stage
    unsigned char* recs = reinterpret_cast<unsigned char*>(bufs + (size_t)a.stages * (a.Nx + 2 * a.pad));

    const long long* __restrict__ fin = static_cast<const long long*>(a.fin);
    long long* __restrict__ fout = static_cast<long long*>(a.fout);
    const int Nx = a.Nx, Np = a.Np, PAD = a.pad, S = a.stages;
    const int stride = Nx + 2 * PAD;
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int G = a.ctas > 0 ? a.ctas : (int)gridDim.x;
    const uint32_t row_bytes = (uint32_t)(Nx * 8);
    const uint32_t tx_bytes = row_bytes + (PERIODIC ? 128u : 0u) + XREC_BYTES;   // row + wrap + record
    const double unit = ldexp(1.0, em.Ef - FX_FRAC);
    bool bad = false;
    uint32_t rng = 0;   // OR of (high word + 2^29) of every stored result

    const int lane = tid & 31, nwarps = nthreads >> 5;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&bars[s], 1);
            done_cnt[s] = 0;
            issued[s] = 0;
        }
        fence_barrier_init();
    }
    if constexpr (!PERIODIC) {
        for (int s = 0; s < S; ++s) {
            long long* b = bufs + (size_t)s * stride;
            for (int e = tid; e < PAD; e += nthreads) {
                b[e] = 0;
                b[PAD + Nx + e] = 0;
            }
        }
    }
    __syncthreads();

    auto issue = [&](int s, int r) {
        long long* dst = bufs + (size_t)s * stride + PAD;
        const long long* src = fin + (size_t)r * Nx;
        issued[s] += 1;
        mbar_arrive_expect_tx(&bars[s], tx_bytes);
        bulk_g2s(dst, src, row_bytes, &bars[s]);
        if constexpr (PERIODIC) bulk_g2s(dst + Nx, src, 128u, &bars[s]);
        bulk_g2s(recs + (size_t)s * XREC_BYTES, static_cast<const unsigned char*>(a.rec) + (size_t)r * XREC_BYTES,
                     XREC_BYTES, &bars[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            const int r = blockIdx.x + s * G;
            if (r < Np) issue(s, r);
        }
    }

    long long colacc[XF_MAXCH][XF_V];
#pragma unroll
    for (int c = 0; c < XF_MAXCH; ++c)
#pragma unroll
        for (int v = 0; v < XF_V; ++v) colacc[c][v] = 0;
    i128 kin = 0;   // units 2^(Ef-51-KIN_Q)

    int it = 0;
    int r = blockIdx.x;
    bool failed = false;
    for (; r < Np; r += G, ++it) {
        const int s = it % S;
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[s], (uint32_t)((it / S) & 1), WAIT_LIMIT_NS));
        long long rowsum = 0;
        if (ok) {
            const long long* rowbuf = bufs + (size_t)s * stride + PAD;
            const XRec* rc = reinterpret_cast<const XRec*>(recs + (size_t)s * XREC_BYTES);
            const int n0 = rc->n0;
            FxW w;
#pragma unroll
            for (int t = 0; t < NTAP; ++t) {
                w.Wh[t] = rc->Wh[t];
                w.wlr[t] = make_float2(rc->wl[t], rc->wf[t] * 9.313225746154785e-10f);   // * 2^-30
            }
            const int A = (n0 - 4) & 1;
            int base;
            if constexpr (PERIODIC) {
                base = (n0 - 4 - A) % Nx;
                if (base < 0) base += Nx;
            } else {
                base = n0 - 4 - A;
            }
            long long* orow = fout + (size_t)r * Nx;
#pragma unroll
            for (int c = 0; c < XF_MAXCH; ++c) {
                const int i = XF_V * (tid + c * nthreads);
                if (i < Nx) {
                    int e = i + base;
                    if constexpr (PERIODIC) {
                        if (e >= Nx) e -= Nx;
                    }
                    long long out[XF_V];
                    if (A == 0) fx_chunk<0>(rowbuf + e, w, out, rng);
                    else fx_chunk<1>(rowbuf + e, w, out, rng);
                    if constexpr (!PERIODIC) {
                        const int k = i + n0;
                        if (k < 0 || k + XF_V - 1 >= Nx - 1) {
                            const double g = rc->g64, d = rc->d64;
                            const double* w64 = rc->w64;
                            const size_t wst = 1;
#pragma unroll
                            for (int v = 0; v < XF_V; ++v)
                                out[v] = fx_edge(rowbuf + e + A + v, w64, wst, k + v, Nx, g, d, unit, em.Ef);
                        }
                    }
#pragma unroll
                    for (int v = 0; v < XF_V; ++v) {
                        const long long Tc = out[v] >> 10;   // units 2^(Ef-51), rounded down
                        colacc[c][v] += Tc;
                        rowsum += Tc;
                    }
#pragma unroll
                    for (int v = 0; v < XF_V; v += 4)   // full 32-byte sectors per instruction
                        st_global_v4_b64(orow + i + v, out[v], out[v + 1], out[v + 2], out[v + 3]);
                }
            }
            if constexpr (KIN) kin += (i128)rowsum * (i128)rc->p2q;   // exact: sum_i f * p_j^2/2
        }
        if (!ok) {
            failed = true;
            break;
        }
        // No CTA-wide barrier per row: the last warp done with stage s refills it.
        __syncwarp();
        if (lane == 0) {
            unsigned int prev;
            asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(prev) : "r"(smem_u32(&done_cnt[s])) : "memory");
            if (prev == (unsigned int)nwarps - 1) {
                done_cnt[s] = 0;
                const int rn = r + S * G;
                if (rn < Np) {
                    fence_proxy_async_smem();
                    issue(s, rn);
                }
            }
        }
    }
    failed = __syncthreads_or(failed);   // also: every warp is done with the stage buffers
    if (bad || rng >= (1u << 30)) atomicCAS(a.err, 0, DEV_ERR_RANGE);
    i128* scratch = reinterpret_cast<i128*>(bufs);   // block-sum scratch (128 entries) in the free stages

    if (failed) {
        if (tid == 0) {
            atomicCAS(a.err, 0, DEV_ERR_XSHIFT_WAIT);
            for (int k = 0; k < S; ++k)   // the last copy issued into each stage must land before exit
                if (issued[k] > 0) mbar_wait_bounded(&bars[k], (uint32_t)((issued[k] - 1) & 1), WAIT_LIMIT_NS);
        }
        __syncthreads();
        return;
    }

    if (a.colacc) {
        // exact fixed-point column sums, added across CTAs: units 2^(Ef-51) -> 2^-k_col
        const int sh = a.k_col + em.Ef - 51;
#pragma unroll
        for (int c = 0; c < XF_MAXCH; ++c) {
            const int i = XF_V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < XF_V; ++v) {
                    const long long x = colacc[c][v];
                    const long long q = sh >= 0 ? (long long)((unsigned long long)x << sh) : ((x + (1ll << (-sh - 1))) >> (-sh));
                    atomicAdd(a.colacc + i + v, (unsigned long long)q);
                }
            }
        }
    } else if (a.ctapart) {
        // HMF: only sum_i rho_i and the cos/sin-weighted sums are needed; form them for this CTA's
        // column sums here (exact int128) and write three numbers instead of a partial row
        i128 pm = 0, px = 0, py = 0, pz = 0;
#pragma unroll
        for (int c = 0; c < XF_MAXCH; ++c) {
            const int i = XF_V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < XF_V; ++v) {
                    const long long t = colacc[c][v];
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
        // exact per-CTA column sums, one partial row per CTA (plain 32-byte stores, no atomics)
        const int sh = a.k_col + em.Ef - 51;
        long long* cp = a.colpart64 + (size_t)blockIdx.x * Nx;
#pragma unroll
        for (int c = 0; c < XF_MAXCH; ++c) {
            const int i = XF_V * (tid + c * nthreads);
            if (i < Nx) {
                long long q[XF_V];
#pragma unroll
                for (int v = 0; v < XF_V; ++v) {
                    const long long x = colacc[c][v];
                    q[v] = sh >= 0 ? (long long)((unsigned long long)x << sh) : ((x + (1ll << (-sh - 1))) >> (-sh));
                }
#pragma unroll
                for (int v = 0; v < XF_V; v += 4) st_global_v4_b64(cp + i + v, q[v], q[v + 1], q[v + 2], q[v + 3]);
            }
        }
    } else if (a.colpart) {
        double* cp = a.colpart + (size_t)blockIdx.x * Nx;
#pragma unroll
        for (int c = 0; c < XF_MAXCH; ++c) {
            const int i = XF_V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < XF_V; ++v) cp[i + v] = fx128_to_f64((i128)colacc[c][v], 51 - em.Ef);
            }
        }
    }
    if constexpr (KIN) {
        const i128 t = block_sum_i128(kin, scratch);
        if (tid == 0) a.kinpart[blockIdx.x] = fx128_to_f64(t, 51 + KIN_Q - em.Ef);
    }
}

template <bool PERIODIC, bool KIN>
__global__ void __launch_bounds__(XS_THREADS_MIN, 2) xshift_fx_kernel(XShiftArgs a, EmulArgs em)
{
    xshift_fx_body<PERIODIC, KIN>(a, em);
}

// Batched form: blockIdx.y selects the slot; args[slot * 2 + ver[slot]] and ems[slot] are its
// arguments (free slots carry Np = 0).
template <bool PERIODIC, bool KIN>
__global__ void __launch_bounds__(XS_THREADS_MIN, 2) xshift_fx_batch_kernel(const XShiftArgs* __restrict__ args,
                                                                            const EmulArgs* __restrict__ ems,
                                                                            const int* __restrict__ ver)
{
    const int slot = blockIdx.y;
    const XShiftArgs a = args[slot * 2 + ver[slot]];
    if (a.Np <= 0 || (int)blockIdx.x >= a.Np || (a.ctas > 0 && (int)blockIdx.x >= a.ctas)) return;
    const EmulArgs em = ems[slot];
    xshift_fx_body<PERIODIC, KIN>(a, em);
}

// ============================================================================ p-shift (FX64)
template <bool PPER>
__device__ __forceinline__ void pshift_fx_body(const CUtensorMap* tmap, const PShiftArgs& a, const EmulArgs& em)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    long long* bufs = reinterpret_cast<long long*>(smem_raw + 128);
    constexpr int BUF = PSF_RB * PS_TW;

    const long long* __restrict__ fin = static_cast<const long long*>(a.fin);
    long long* __restrict__ fout = static_cast<long long*>(a.fout);
    const int Nx = a.Nx, Np = a.Np;
    const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 5;
    const int ntx = (Nx + PS_TW - 1) / PS_TW, nty = (Np + PS_TH - 1) / PS_TH;
    const int ntiles = ntx * nty;
    const int G = gridDim.x;
    const double unit = ldexp(1.0, em.Ef - FX_FRAC);
    bool bad = false;
    uint32_t rng = 0;   // OR of (high word + 2^29) of every stored result

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        prefetch_tensormap(tmap);
    }
    __syncthreads();

    auto issue = [&](int b, const TileWin& t) {
        if (t.smem_ok) {
            mbar_arrive_expect_tx(&bars[b], (uint32_t)(t.nb * PS_BH * PS_TW * 8));
            for (int q = 0; q < t.nb; ++q)
                tma_load_2d(bufs + (size_t)b * BUF + (size_t)q * PS_BH * PS_TW, tmap, t.i0, t.r0 + q * PS_BH, &bars[b]);
        } else {
            mbar_arrive_expect_tx(&bars[b], 0u);
        }
    };

    int tile = blockIdx.x;
    if (grp == 0 && tile < ntiles) {
        int n0l;
        bool cv;
        TileWin t = tile_window<PPER, PSF_RB>(tile, ntx, em.n0, Nx, lane, n0l, cv);
        if (lane == 0) issue(0, t);
    }

    int q = 0;
    bool failed = false;
    for (; tile < ntiles; tile += G, ++q) {
        const int b = q & 1;
        const int nt = tile + G;
        if (grp == 0 && nt < ntiles) {
            int n0l;
            bool cv;
            TileWin tn = tile_window<PPER, PSF_RB>(nt, ntx, em.n0, Nx, lane, n0l, cv);
            if (lane == 0) {
                fence_proxy_async_smem();
                issue(b ^ 1, tn);
            }
        }
        int n0_i;
        bool colvalid;
        const TileWin t = tile_window<PPER, PSF_RB>(tile, ntx, em.n0, Nx, lane, n0_i, colvalid);
        const int i = t.i0 + lane;
        FxW w;
#pragma unroll
        for (int k = 0; k < NTAP; ++k) {
            w.Wh[k] = colvalid ? em.Wh[(size_t)k * Nx + i] : 0;
            w.wlr[k] = colvalid ? make_float2(em.wl[(size_t)k * Nx + i], em.wf[(size_t)k * Nx + i] * 9.313225746154785e-10f)
                                : make_float2(0.f, 0.f);
        }
        const bool ok = mbar_wait_bounded(&bars[b], (uint32_t)((q >> 1) & 1), WAIT_LIMIT_NS);
        if (ok) {
            const long long* buf = bufs + (size_t)b * BUF;
            const int jb = t.j0 + grp * PS_RPT;
            const int base = jb + n0_i - 4 - t.r0;
            long long M[PS_RPT];
            float2 Sacc[PS_RPT];
#pragma unroll
            for (int rw = 0; rw < PS_RPT; ++rw) {
                M[rw] = EMUL_M0;
                Sacc[rw] = make_float2(0.f, 0.f);
            }
            // Elements u and u+1 together: their two products for an output enter its int64 sum in
            // one three-input add (two IMAD.WIDE + IADD3 + IADD3.X) instead of two 64-bit
            // multiply-adds (three instructions each on this GPU).
            auto feed2 = [&](int u, long long X0, long long X1, bool second) {
                int kx0, kx1;
                float kf0, rf0, kf1, rf1;
                fx_split(X0, kx0, kf0, rf0);
                fx_split(X1, kx1, kf1, rf1);
                const float2 xa = make_float2(kf0, rf0), xb = make_float2(kf1, rf1);
#pragma unroll
                for (int rw = 0; rw < PS_RPT; ++rw) {
                    const int t0 = u - rw, t1 = t0 + 1;
                    const bool v0 = t0 >= 0 && t0 < NTAP, v1 = second && t1 >= 0 && t1 < NTAP;
                    if (v0 && v1) M[rw] = M[rw] + mul_wide(w.Wh[t0], kx0) + mul_wide(w.Wh[t1], kx1);
                    else if (v0) M[rw] += mul_wide(w.Wh[t0], kx0);
                    else if (v1) M[rw] += mul_wide(w.Wh[t1], kx1);
                    if (v0) Sacc[rw] = __ffma2_rn(w.wlr[t0], xa, Sacc[rw]);
                    if (v1) Sacc[rw] = __ffma2_rn(w.wlr[t1], xb, Sacc[rw]);
                }
            };
            constexpr int NU = PS_RPT + 9;
            if (t.smem_ok) {
#pragma unroll
                for (int u = 0; u < NU; u += 2)
                    feed2(u, buf[(base + u) * PS_TW + lane], u + 1 < NU ? buf[(base + u + 1) * PS_TW + lane] : 0ll, u + 1 < NU);
            } else {
#pragma unroll
                for (int u = 0; u < NU; u += 2) {
                    const long long X0 = colvalid ? gload_p<long long, PPER>(fin, jb + n0_i - 4 + u, i, Nx, Np) : 0ll;
                    const long long X1 = (colvalid && u + 1 < NU) ? gload_p<long long, PPER>(fin, jb + n0_i - 3 + u, i, Nx, Np) : 0ll;
                    feed2(u, X0, X1, u + 1 < NU);
                }
            }
            bool any_edge = false;
#pragma unroll
            for (int rw = 0; rw < PS_RPT; ++rw) {
                const int j = jb + rw;
                const long long out = fx_store(emul_finish(M[rw], Sacc[rw].x + Sacc[rw].y), rng);
                bool edge = false;
                if constexpr (!PPER) {
                    const int kk = j + n0_i;
                    edge = kk < 0 || kk >= Np - 1;
                }
                any_edge |= edge;
                if (colvalid && j < Np && !edge) fout[(size_t)j * Nx + i] = out;
            }
            if constexpr (!PPER) {
                if (any_edge && colvalid) {
                    const double g = em.gd[i], d = em.gd[Nx + i];
                    for (int rw = 0; rw < PS_RPT; ++rw) {
                        const int j = jb + rw, kk = j + n0_i;
                        if (j >= Np || !(kk < 0 || kk >= Np - 1)) continue;
                        long long X[NTAP];
                        for (int u = 0; u < NTAP; ++u)
                            X[u] = t.smem_ok ? buf[(base + rw + u) * PS_TW + lane]
                                             : gload_p<long long, PPER>(fin, j + n0_i - 4 + u, i, Nx, Np);
                        fout[(size_t)j * Nx + i] = fx_edge(X, em.w64 + i, Nx, kk, Np, g, d, unit, em.Ef);
                    }
                }
            }
        }
        if (__syncthreads_or(!ok)) {   // also: every thread done with buffer b before it is refilled
            failed = true;
            break;
        }
    }
    if (bad || rng >= (1u << 30)) atomicCAS(a.err, 0, DEV_ERR_RANGE);
    if (failed && tid == 0) {
        atomicCAS(a.err, 0, DEV_ERR_PSHIFT_WAIT);
        if (tile + G < ntiles) mbar_wait_bounded(&bars[(q + 1) & 1], (uint32_t)(((q + 1) >> 1) & 1), WAIT_LIMIT_NS);
        mbar_wait_bounded(&bars[q & 1], (uint32_t)((q >> 1) & 1), WAIT_LIMIT_NS);
    }
}

template <bool PPER>
__global__ void __launch_bounds__(PS_TW * PS_RG, 2) pshift_fx_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                     PShiftArgs a, EmulArgs em)
{
    pshift_fx_body<PPER>(&tmap, a, em);
}

// Batched form: the slot's tensor map sits in global memory next to its arguments.
template <bool PPER>
__global__ void __launch_bounds__(PS_TW * PS_RG, 2) pshift_fx_batch_kernel(const CUtensorMap* __restrict__ tmaps,
                                                                           const PShiftArgs* __restrict__ args,
                                                                           const EmulArgs* __restrict__ ems,
                                                                           const int* __restrict__ ver)
{
    const int slot = blockIdx.y;
    const int k = slot * 2 + ver[slot];
    const PShiftArgs a = args[k];
    if (a.Nx <= 0) return;
    const EmulArgs em = ems[slot];
    pshift_fx_body<PPER>(tmaps + k, a, em);
}

int xshift_fx_max_cols(int threads) { return XF_V * threads * XF_MAXCH; }

size_t pshift_fx_smem_bytes() { return 256 + 2 * (size_t)PSF_RB * PS_TW * 8; }

cudaError_t launch_xshift_fx(bool periodic, bool kin, int grid, int threads, const XShiftArgs& a, const EmulArgs& em,
                             cudaStream_t st)
{
    if (a.rec == nullptr) return cudaErrorInvalidValue;   // the per-row record is staged with each row
    const size_t smem = xshift_smem_bytes(a.Nx, a.pad, a.stages, 8);
    if (periodic) {
        if (kin) xshift_fx_kernel<true, true><<<grid, threads, smem, st>>>(a, em);
        else xshift_fx_kernel<true, false><<<grid, threads, smem, st>>>(a, em);
    } else {
        if (kin) xshift_fx_kernel<false, true><<<grid, threads, smem, st>>>(a, em);
        else xshift_fx_kernel<false, false><<<grid, threads, smem, st>>>(a, em);
    }
    return cudaGetLastError();
}

cudaError_t launch_pshift_fx(bool p_periodic, int grid, const CUtensorMap* tmap, const PShiftArgs& a,
                             const EmulArgs& em, cudaStream_t st)
{
    const size_t smem = pshift_fx_smem_bytes();
    if (p_periodic) pshift_fx_kernel<true><<<grid, PS_TW * PS_RG, smem, st>>>(*tmap, a, em);
    else pshift_fx_kernel<false><<<grid, PS_TW * PS_RG, smem, st>>>(*tmap, a, em);
    return cudaGetLastError();
}

cudaError_t launch_xshift_fx_batch(bool periodic, bool kin, int slots, int ctas_per_slot, size_t smem,
                                   const XShiftArgs* args, const EmulArgs* ems, const int* ver, cudaStream_t st)
{
    const dim3 grid(ctas_per_slot, slots);
    if (periodic) {
        if (kin) xshift_fx_batch_kernel<true, true><<<grid, XS_THREADS_MIN, smem, st>>>(args, ems, ver);
        else xshift_fx_batch_kernel<true, false><<<grid, XS_THREADS_MIN, smem, st>>>(args, ems, ver);
    } else {
        if (kin) xshift_fx_batch_kernel<false, true><<<grid, XS_THREADS_MIN, smem, st>>>(args, ems, ver);
        else xshift_fx_batch_kernel<false, false><<<grid, XS_THREADS_MIN, smem, st>>>(args, ems, ver);
    }
    return cudaGetLastError();
}

cudaError_t launch_pshift_fx_batch(int slots, int ctas_per_slot, const CUtensorMap* tmaps, const PShiftArgs* args,
                                   const EmulArgs* ems, const int* ver, cudaStream_t st)
{
    const dim3 grid(ctas_per_slot, slots);
    pshift_fx_batch_kernel<false><<<grid, PS_TW * PS_RG, pshift_fx_smem_bytes(), st>>>(tmaps, args, ems, ver);
    return cudaGetLastError();
}

cudaError_t set_kernel_attributes_fx(int max_smem)
{
    cudaError_t e = cudaSuccess;
#define VL_ATTR(fn) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)
    VL_ATTR((xshift_fx_kernel<true, true>));
    VL_ATTR((xshift_fx_kernel<true, false>));
    VL_ATTR((xshift_fx_kernel<false, true>));
    VL_ATTR((xshift_fx_kernel<false, false>));
    VL_ATTR((pshift_fx_kernel<true>));
    VL_ATTR((pshift_fx_kernel<false>));
    VL_ATTR((xshift_fx_batch_kernel<true, true>));
    VL_ATTR((xshift_fx_batch_kernel<true, false>));
    VL_ATTR((xshift_fx_batch_kernel<false, true>));
    VL_ATTR((xshift_fx_batch_kernel<false, false>));
    VL_ATTR((pshift_fx_batch_kernel<false>));
#undef VL_ATTR
    return e;
}

cudaError_t xshift_fx_occupancy(bool periodic, size_t smem, int* blocks)
{
    return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_fx_kernel<true, true>, XS_THREADS_MIN, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_fx_kernel<false, true>, XS_THREADS_MIN, smem);
}

cudaError_t pshift_fx_occupancy(int* blocks)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pshift_fx_kernel<false>, PS_TW * PS_RG,
                                                         pshift_fx_smem_bytes());
}

// ============================================================================ conversions, column sums
__global__ void f64_to_fx_kernel(const double* __restrict__ s, long long* __restrict__ d, size_t n, int k)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        d[q] = (long long)fx128_from_f64(s[q], k);
}

__global__ void fx_to_f64_kernel(const long long* __restrict__ s, double* __restrict__ d, size_t n, int k)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        d[q] = fx128_to_f64((i128)s[q], k);
}

cudaError_t launch_f64_to_fx(const double* s, long long* d, size_t n, int Ef, cudaStream_t st)
{
    f64_to_fx_kernel<<<1024, 256, 0, st>>>(s, d, n, FX_FRAC - Ef);
    return cudaGetLastError();
}

cudaError_t launch_fx_to_f64(const long long* s, double* d, size_t n, int Ef, cudaStream_t st)
{
    fx_to_f64_kernel<<<1024, 256, 0, st>>>(s, d, n, FX_FRAC - Ef);
    return cudaGetLastError();
}

// Column sums of a fixed-point f into one partial row (density test hook): exact in int64 at
// 2^-10 of the storage resolution (units 2^(Ef-51)).
__global__ void __launch_bounds__(256) colsum_fx_kernel(const long long* __restrict__ f, int Nx, int Np, int Ef,
                                                        double* colpart)
{
    __shared__ long long sh[8][32];
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    long long s = 0;
    if (i < Nx)
        for (int j = grp; j < Np; j += 8) s += (f[(size_t)j * Nx + i] + 512) >> 10;
    sh[grp][lane] = s;
    __syncthreads();
    if (grp == 0 && i < Nx) {
        long long t = 0;
        for (int q = 0; q < 8; ++q) t += sh[q][lane];
        colpart[i] = fx128_to_f64((i128)t, 51 - Ef);
    }
}

cudaError_t launch_colsum_fx(const long long* f, int Nx, int Np, int Ef, double* colpart, cudaStream_t st)
{
    colsum_fx_kernel<<<(Nx + 31) / 32, 256, 0, st>>>(f, Nx, Np, Ef, colpart);
    return cudaGetLastError();
}

}  // namespace vl
