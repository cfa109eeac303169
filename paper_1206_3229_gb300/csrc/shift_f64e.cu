// shift_f64e.cu -- the two sweeps for FP64 storage, computed without FP64 instructions.
//
// Same data movement as shift_kernels.cu (rows staged by 1-D bulk copies for the x-shift, 2-D TMA
// column tiles for the p-shift), plus one pass over the staged values that rewrites every FP64
// element in place as (kx, r) on the 2^(Ef-31) grid (emul.cuh).  The filter then runs on integer
// and FP32 pipes: 10 IMAD.WIDE + 20 FFMA per output, the result is rebuilt as an FP64 bit pattern
// with integer instructions.  Boundary corrections of non-periodic axes (f'' = 0 outside the grid)
// are rare and done in FP64.
#include "emul.cuh"
#include "fixed_point.cuh"
#include "ptx.cuh"
#include "shift_common.cuh"
#include "vlasov_internal.cuh"

namespace vl {

// Rewrite n doubles at p (shared memory) as EmulElem, block-strided.
__device__ __forceinline__ void convert_range(double* p, int n, int s_base, bool& bad)
{
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const EmulElem v = emul_split(p[e], s_base, bad);
        reinterpret_cast<int2*>(p)[e] = make_int2(v.kx, __float_as_int(v.r));
    }
}

struct EmulW {
    int Wh[NTAP];
    float wl[NTAP];
    float wf[NTAP];
};


constexpr int XE_V = 4;      // consecutive outputs per thread and chunk
constexpr int PSE_RB = 192;  // staged rows per buffer of the emulated p-shift (two CTAs per SM)
static_assert(PSE_RB % PS_BH == 0, "a staged window is whole TMA boxes: the slot must hold nb * PS_BH rows");
constexpr int XE_W = 14;     // window elements: V + 9 + alignment slack (even)
constexpr int XE_MAXCH = 4;  // chunks per row per thread (Nx <= 4 * 4 * 256 = 4096)

// XE_V consecutive outputs from the converted (kx, r) pairs starting at `src` (f_{k-4-A} ..):
// input-stationary with separate chains for the integer part and the two FP32 residual sums.
template <int A>
__device__ __forceinline__ void emul_chunk(const int2* src, const EmulW& w, long long (&T)[XE_V])
{
    long long M[XE_V];
    float Sa[XE_V], Sb[XE_V];
#pragma unroll
    for (int v = 0; v < XE_V; ++v) {
        M[v] = EMUL_M0;
        Sa[v] = 0.f;
        Sb[v] = 0.f;
    }
    const int4* q = reinterpret_cast<const int4*>(src);
#pragma unroll
    for (int h = 0; h < XE_W / 2; ++h) {
        const int4 pr = q[h];
#pragma unroll
        for (int z = 0; z < 2; ++z) {
            const int u = 2 * h + z;
            const int kx = z ? pr.z : pr.x;
            const float rr = __int_as_float(z ? pr.w : pr.y);
            const float kf = __int2float_rn(kx);
#pragma unroll
            for (int v = 0; v < XE_V; ++v) {
                const int t = u - A - v;
                if (t >= 0 && t < NTAP) {
                    M[v] = mad_wide(w.Wh[t], kx, M[v]);
                    Sa[v] = fmaf(w.wl[t], kf, Sa[v]);
                    Sb[v] = fmaf(w.wf[t], rr, Sb[v]);
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < XE_V; ++v) T[v] = emul_finish(M[v], Sa[v] + Sb[v]);
}

// FP64 boundary correction (non-periodic axes): value of the zero-extended filter minus the
// f'' terms at nodes outside [0, n).  x points at the ten window values (as doubles).
__device__ __forceinline__ double emul_edge(double out, const double* x, int k, int n, double g, double d)
{
    return edge_fix(out, x, k, n, g, d);
}

// ============================================================================ x-shift (emulated FP64)
template <bool PERIODIC, bool KIN>
__global__ void __launch_bounds__(XS_THREADS_MAX, 1) xshift_e_kernel(XShiftArgs a, EmulArgs em)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    double* bufs = reinterpret_cast<double*>(smem_raw + 128);
    __shared__ double red[32];
    unsigned char* recs = reinterpret_cast<unsigned char*>(bufs + (size_t)a.stages * (a.Nx + 2 * a.pad));

    const double* __restrict__ fin = static_cast<const double*>(a.fin);
    double* __restrict__ fout = static_cast<double*>(a.fout);
    const int Nx = a.Nx, Np = a.Np, PAD = a.pad, S = a.stages;
    const int stride = Nx + 2 * PAD;
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int G = gridDim.x;
    const uint32_t row_bytes = (uint32_t)(Nx * 8);
    const uint32_t tx_bytes = row_bytes + (PERIODIC ? 128u : 0u) + XREC_BYTES;   // row + wrap + record
    const int s_base = 1044 + em.Ef;
    const double grid = ldexp(1.0, em.Ef - 31);
    bool bad = false;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    if constexpr (!PERIODIC) {
        for (int s = 0; s < S; ++s) {
            double* b = bufs + (size_t)s * stride;
            for (int e = tid; e < PAD; e += nthreads) {
                b[e] = 0.0;
                b[PAD + Nx + e] = 0.0;
            }
        }
    }
    __syncthreads();

    auto issue = [&](int s, int r) {
        double* dst = bufs + (size_t)s * stride + PAD;
        const double* src = fin + (size_t)r * Nx;
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

    long long colacc[XE_MAXCH][XE_V];
#pragma unroll
    for (int c = 0; c < XE_MAXCH; ++c)
#pragma unroll
        for (int v = 0; v < XE_V; ++v) colacc[c][v] = 0;
    double kin = 0.0;

    int it = 0;
    int r = blockIdx.x;
    bool failed = false;
    for (; r < Np; r += G, ++it) {
        const int s = it % S;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((it / S) & 1), WAIT_LIMIT_NS);
        double* rowbuf = bufs + (size_t)s * stride + PAD;
        if (ok) convert_range(rowbuf, Nx + (PERIODIC ? 16 : 0), s_base, bad);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const XRec* rc = reinterpret_cast<const XRec*>(recs + (size_t)s * XREC_BYTES);
        const int n0 = rc->n0;
        EmulW w;
#pragma unroll
        for (int t = 0; t < NTAP; ++t) {
            w.Wh[t] = rc->Wh[t];
            w.wl[t] = rc->wl[t];
            w.wf[t] = rc->wf[t];
        }
        double g = 0.0, d = 0.0;
        if constexpr (!PERIODIC) {
            g = rc->g64;
            d = rc->d64;
        }
        const int A = (n0 - 4) & 1;
        int base;
        if constexpr (PERIODIC) {
            base = (n0 - 4 - A) % Nx;
            if (base < 0) base += Nx;
        } else {
            base = n0 - 4 - A;
        }
        const int2* src = reinterpret_cast<const int2*>(rowbuf);
        double* orow = fout + (size_t)r * Nx;
        long long rowsum = 0;
#pragma unroll
        for (int c = 0; c < XE_MAXCH; ++c) {
            const int i = XE_V * (tid + c * nthreads);
            if (i < Nx) {
                int e = i + base;
                if constexpr (PERIODIC) {
                    if (e >= Nx) e -= Nx;
                }
                long long Tv[XE_V];
                if (A == 0) emul_chunk<0>(src + e, w, Tv);
                else emul_chunk<1>(src + e, w, Tv);
                double out[XE_V];
#pragma unroll
                for (int v = 0; v < XE_V; ++v) out[v] = emul_to_f64(Tv[v], em.Ef);
                if constexpr (!PERIODIC) {
                    const int k = i + n0;
                    if (k < 0 || k + XE_V - 1 >= Nx - 1) {
                        // rare boundary chunk (f'' = 0 outside the row): outputs whose foot cell is
                        // outside are 0, the two touching the end take the row's edge filters, in
                        // the same integer/FP32 arithmetic as the interior
                        for (int v = 0; v < XE_V; ++v) {
                            const int kv = k + v;
                            if (kv >= 0 && kv < Nx - 1) continue;
                            if (kv < -1 || kv >= Nx) {
                                Tv[v] = 0;
                                out[v] = 0.0;
                                continue;
                            }
                            const int q = kv < 0 ? 0 : 1;
                            long long M = EMUL_M0;
                            float sa = 0.f, sb = 0.f;
                            for (int t = 0; t < NTAP; ++t) {
                                const int2 p = src[e + A + v + t];
                                M = mad_wide(rc->Whe[q][t], p.x, M);
                                sa = fmaf(rc->wle[q][t], __int2float_rn(p.x), sa);
                                sb = fmaf(rc->wfe[q][t], __int_as_float(p.y), sb);
                            }
                            Tv[v] = emul_finish(M, sa + sb);
                            out[v] = emul_to_f64(Tv[v], em.Ef);
                        }
                    }
                }
#pragma unroll
                for (int v = 0; v < XE_V; ++v) {
                    const long long Tc = Tv[v] >> 10;   // units 2^(Ef-51), rounded down
                    colacc[c][v] += Tc;
                    rowsum += Tc;
                }
                st_global_v4_f64(orow + i, out[0], out[1], out[2], out[3]);   // one full 32-byte sector
            }
        }
        if constexpr (KIN) {
            const double pj = a.pmin + (double)r * a.dp;
            kin = fma(0.5 * pj * pj, fx128_to_f64((i128)rowsum, 51 - em.Ef), kin);
        }
        __syncthreads();   // every thread done with stage s
        if (tid == 0) {
            const int rn = r + S * G;
            if (rn < Np) {
                fence_proxy_async_smem();
                issue(s, rn);
            }
        }
    }
    if (bad) atomicCAS(a.err, 0, DEV_ERR_RANGE);

    if (failed) {
        if (tid == 0) {
            atomicCAS(a.err, 0, DEV_ERR_XSHIFT_WAIT);
            for (int k = 0; k < S; ++k) {
                const int rr = r + k * G;
                if (rr >= Np) break;
                const int itk = it + k;
                mbar_wait_bounded(&bars[itk % S], (uint32_t)((itk / S) & 1), WAIT_LIMIT_NS);
            }
        }
        __syncthreads();
        return;
    }

    if (a.colacc) {
        // exact fixed-point column sums, added across CTAs: units 2^(Ef-51) -> 2^-k_col
        const int sh = a.k_col + em.Ef - 51;
#pragma unroll
        for (int c = 0; c < XE_MAXCH; ++c) {
            const int i = XE_V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < XE_V; ++v) {
                    const long long x = colacc[c][v];
                    const long long q = sh >= 0 ? (long long)((unsigned long long)x << sh) : ((x + (1ll << (-sh - 1))) >> (-sh));
                    atomicAdd(a.colacc + i + v, (unsigned long long)q);
                }
            }
        }
    } else if (a.colpart64) {
        // exact per-CTA column sums, one partial row per CTA (plain 32-byte stores, no atomics)
        const int sh = a.k_col + em.Ef - 51;
        long long* cp = a.colpart64 + (size_t)blockIdx.x * Nx;
#pragma unroll
        for (int c = 0; c < XE_MAXCH; ++c) {
            const int i = XE_V * (tid + c * nthreads);
            if (i < Nx) {
                long long q[XE_V];
#pragma unroll
                for (int v = 0; v < XE_V; ++v) {
                    const long long x = colacc[c][v];
                    q[v] = sh >= 0 ? (long long)((unsigned long long)x << sh) : ((x + (1ll << (-sh - 1))) >> (-sh));
                }
#pragma unroll
                for (int v = 0; v < XE_V; v += 4) st_global_v4_b64(cp + i + v, q[v], q[v + 1], q[v + 2], q[v + 3]);
            }
        }
    } else if (a.colpart) {
        double* cp = a.colpart + (size_t)blockIdx.x * Nx;
#pragma unroll
        for (int c = 0; c < XE_MAXCH; ++c) {
            const int i = XE_V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < XE_V; ++v) cp[i + v] = fx128_to_f64((i128)colacc[c][v], 51 - em.Ef);
            }
        }
    }
    if constexpr (KIN) {
        double v = kin;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < (nthreads + 31) / 32; ++q) s += red[q];
            a.kinpart[blockIdx.x] = s;
        }
    }
}

// ============================================================================ p-shift (emulated FP64)
template <bool PPER>
__global__ void __launch_bounds__(PS_TW * PS_RG, 2) pshift_e_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                    PShiftArgs a, EmulArgs em)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    double* bufs = reinterpret_cast<double*>(smem_raw + 128);
    constexpr int BUF = PSE_RB * PS_TW;

    const double* __restrict__ fin = static_cast<const double*>(a.fin);
    double* __restrict__ fout = static_cast<double*>(a.fout);
    const int Nx = a.Nx, Np = a.Np;
    const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 5;
    const int ntx = (Nx + PS_TW - 1) / PS_TW, nty = (Np + PS_TH - 1) / PS_TH;
    const int ntiles = ntx * nty;
    const int G = gridDim.x;
    const int s_base = 1044 + em.Ef;
    const double grid = ldexp(1.0, em.Ef - 31);
    bool bad = false;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        prefetch_tensormap(&tmap);
    }
    __syncthreads();

    auto issue = [&](int b, const TileWin& t) {
        if (t.smem_ok) {
            mbar_arrive_expect_tx(&bars[b], (uint32_t)(t.nb * PS_BH * PS_TW * 8));
            for (int q = 0; q < t.nb; ++q)
                tma_load_2d(bufs + (size_t)b * BUF + (size_t)q * PS_BH * PS_TW, &tmap, t.i0, t.r0 + q * PS_BH, &bars[b]);
        } else {
            mbar_arrive_expect_tx(&bars[b], 0u);
        }
    };

    int tile = blockIdx.x;
    if (grp == 0 && tile < ntiles) {
        int n0l;
        bool cv;
        TileWin t = tile_window<PPER, PSE_RB>(tile, ntx, em.n0, Nx, lane, n0l, cv);
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
            TileWin tn = tile_window<PPER, PSE_RB>(nt, ntx, em.n0, Nx, lane, n0l, cv);
            if (lane == 0) {
                fence_proxy_async_smem();
                issue(b ^ 1, tn);
            }
        }
        int n0_i;
        bool colvalid;
        const TileWin t = tile_window<PPER, PSE_RB>(tile, ntx, em.n0, Nx, lane, n0_i, colvalid);
        const int i = t.i0 + lane;
        EmulW w;
#pragma unroll
        for (int k = 0; k < NTAP; ++k) {
            w.Wh[k] = colvalid ? em.Wh[(size_t)k * Nx + i] : 0;
            w.wl[k] = colvalid ? em.wl[(size_t)k * Nx + i] : 0.f;
            w.wf[k] = colvalid ? em.wf[(size_t)k * Nx + i] : 0.f;
        }
        double g = 0.0, d = 0.0;
        if constexpr (!PPER) {
            if (colvalid) {
                g = em.gd[i];
                d = em.gd[Nx + i];
            }
        }
        const bool ok = mbar_wait_bounded(&bars[b], (uint32_t)((q >> 1) & 1), WAIT_LIMIT_NS);
        double* buf = bufs + (size_t)b * BUF;
        if (ok && t.smem_ok) convert_range(buf, t.nb * PS_BH * PS_TW, s_base, bad);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const int jb = t.j0 + grp * PS_RPT;
        // Input-stationary filter: walk the 25 window elements once; element u feeds outputs
        // rw = u-9 .. u (tap u - rw).  Keeps 16 int64 + 16 float accumulators live instead of the
        // whole converted window.
        long long M[PS_RPT];
        float Sacc[PS_RPT];
#pragma unroll
        for (int rw = 0; rw < PS_RPT; ++rw) {
            M[rw] = EMUL_M0;
            Sacc[rw] = 0.f;
        }
        const int2* sb = reinterpret_cast<const int2*>(buf);
        const int base = jb + n0_i - 4 - t.r0;
        auto feed = [&](int u, int kx, float rr) {
            const float kf = __int2float_rn(kx);
#pragma unroll
            for (int tap = 0; tap < NTAP; ++tap) {
                const int rw = u - tap;
                if (rw >= 0 && rw < PS_RPT) {
                    M[rw] = mad_wide(w.Wh[tap], kx, M[rw]);
                    Sacc[rw] = fmaf(w.wl[tap], kf, Sacc[rw]);
                    Sacc[rw] = fmaf(w.wf[tap], rr, Sacc[rw]);
                }
            }
        };
        if (t.smem_ok) {
#pragma unroll
            for (int u = 0; u < PS_RPT + 9; ++u) {
                const int2 v = sb[(base + u) * PS_TW + lane];
                feed(u, v.x, __int_as_float(v.y));
            }
        } else {
#pragma unroll
            for (int u = 0; u < PS_RPT + 9; ++u) {
                const double x = colvalid ? gload_p<double, PPER>(fin, jb + n0_i - 4 + u, i, Nx, Np) : 0.0;
                const EmulElem v = emul_split(x, s_base, bad);
                feed(u, v.kx, v.r);
            }
        }
        // a tile wholly inside the grid, every foot cell inside too (the common case): no per-row
        // edge or bounds checks
        const bool interior = t.i0 + PS_TW <= Nx && t.j0 + PS_TH <= Np &&
                              (PPER || (t.j0 + t.kmin >= 0 && t.j0 + PS_TH - 1 + t.kmax < Np - 1));
        if (interior) {
            double* __restrict__ op = fout + (size_t)jb * Nx + i;
#pragma unroll
            for (int rw = 0; rw < PS_RPT; ++rw) {
                *op = emul_to_f64(emul_finish(M[rw], Sacc[rw]), em.Ef);
                op += Nx;
            }
        } else {
            bool any_edge = false;
#pragma unroll
            for (int rw = 0; rw < PS_RPT; ++rw) {
                const int j = jb + rw;
                const double out = emul_to_f64(emul_finish(M[rw], Sacc[rw]), em.Ef);
                bool edge = false;
                if constexpr (!PPER) {
                    const int kk = j + n0_i;
                    edge = kk < 0 || kk >= Np - 1;
                }
                any_edge |= edge;
                if (colvalid && j < Np && !edge) fout[(size_t)j * Nx + i] = out;
            }
            if constexpr (!PPER) {
                if (any_edge && colvalid && em.Whe) {
                    // rare boundary rows (f'' = 0 outside the grid): 0 where the foot cell is outside,
                    // the column's edge filters where it touches the end, in the interior arithmetic
                    for (int rw = 0; rw < PS_RPT; ++rw) {
                        const int j = jb + rw, kk = j + n0_i;
                        if (j >= Np || !(kk < 0 || kk >= Np - 1)) continue;
                        if (kk < -1 || kk >= Np) {
                            fout[(size_t)j * Nx + i] = 0.0;
                            continue;
                        }
                        const int q = kk < 0 ? 0 : 1;
                        long long M = EMUL_M0;
                        float sa = 0.f, sbb = 0.f;
                        for (int u = 0; u < NTAP; ++u) {
                            int kx;
                            float rr;
                            if (t.smem_ok) {
                                const int2 v = sb[(base + rw + u) * PS_TW + lane];
                                kx = v.x;
                                rr = __int_as_float(v.y);
                            } else {
                                const double x = gload_p<double, PPER>(fin, j + n0_i - 4 + u, i, Nx, Np);
                                const EmulElem ev = emul_split(x, s_base, bad);
                                kx = ev.kx;
                                rr = ev.r;
                            }
                            const size_t idx = ((size_t)q * NTAP + u) * Nx + i;
                            M = mad_wide(em.Whe[idx], kx, M);
                            sa = fmaf(em.wle[idx], __int2float_rn(kx), sa);
                            sbb = fmaf(em.wfe[idx], rr, sbb);
                        }
                        fout[(size_t)j * Nx + i] = emul_to_f64(emul_finish(M, sa + sbb), em.Ef);
                    }
                } else if (any_edge && colvalid) {
                    // no edge filters (not given): recompute in FP64
                    for (int rw = 0; rw < PS_RPT; ++rw) {
                        const int j = jb + rw, kk = j + n0_i;
                        if (j >= Np || !(kk < 0 || kk >= Np - 1)) continue;
                        double xv[NTAP];
                        double acc = 0.0;
                        for (int u = 0; u < NTAP; ++u) {
                            double x;
                            if (t.smem_ok) {
                                const int2 v = sb[(base + rw + u) * PS_TW + lane];
                                x = ((double)v.x + (double)__int_as_float(v.y)) * grid;
                            } else {
                                x = gload_p<double, PPER>(fin, j + n0_i - 4 + u, i, Nx, Np);
                            }
                            xv[u] = x;
                            acc = fma(em.w64[(size_t)u * Nx + i], x, acc);
                        }
                        fout[(size_t)j * Nx + i] = emul_edge(acc, xv, kk, Np, g, d);
                    }
                }
            }
        }
        __syncthreads();   // every thread done with buffer b before it is refilled
    }
    if (bad) atomicCAS(a.err, 0, DEV_ERR_RANGE);
    if (failed && tid == 0) {
        atomicCAS(a.err, 0, DEV_ERR_PSHIFT_WAIT);
        if (tile + G < ntiles) mbar_wait_bounded(&bars[(q + 1) & 1], (uint32_t)(((q + 1) >> 1) & 1), WAIT_LIMIT_NS);
        mbar_wait_bounded(&bars[q & 1], (uint32_t)((q >> 1) & 1), WAIT_LIMIT_NS);
    }
}

int xshift_e_max_cols(int threads) { return XE_V * threads * XE_MAXCH; }

size_t pshift_e_smem_bytes() { return 256 + 2 * (size_t)PSE_RB * PS_TW * 8; }

cudaError_t xshift_e_occupancy(bool periodic, int threads, size_t smem, int* blocks)
{
    return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_e_kernel<true, true>, threads, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_e_kernel<false, true>, threads, smem);
}

cudaError_t pshift_e_occupancy(int* blocks)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pshift_e_kernel<false>, PS_TW * PS_RG, pshift_e_smem_bytes());
}

cudaError_t launch_xshift_e(bool periodic, bool kin, int grid, int threads, const XShiftArgs& a, const EmulArgs& em,
                            cudaStream_t st)
{
    if (a.rec == nullptr) return cudaErrorInvalidValue;   // the per-row record is staged with each row
    const size_t smem = xshift_smem_bytes(a.Nx, a.pad, a.stages, 8);
    if (periodic) {
        if (kin) xshift_e_kernel<true, true><<<grid, threads, smem, st>>>(a, em);
        else xshift_e_kernel<true, false><<<grid, threads, smem, st>>>(a, em);
    } else {
        if (kin) xshift_e_kernel<false, true><<<grid, threads, smem, st>>>(a, em);
        else xshift_e_kernel<false, false><<<grid, threads, smem, st>>>(a, em);
    }
    return cudaGetLastError();
}

cudaError_t launch_pshift_e(bool p_periodic, int grid, const CUtensorMap* tmap, const PShiftArgs& a, const EmulArgs& em,
                            cudaStream_t st)
{
    const size_t smem = pshift_e_smem_bytes();
    if (p_periodic) pshift_e_kernel<true><<<grid, PS_TW * PS_RG, smem, st>>>(*tmap, a, em);
    else pshift_e_kernel<false><<<grid, PS_TW * PS_RG, smem, st>>>(*tmap, a, em);
    return cudaGetLastError();
}

cudaError_t set_kernel_attributes_e(int max_smem)
{
    cudaError_t e = cudaSuccess;
#define VL_ATTR(fn) \
    if (e == cudaSuccess) e = allow_dynamic_smem(fn, max_smem)
    VL_ATTR((xshift_e_kernel<true, true>));
    VL_ATTR((xshift_e_kernel<true, false>));
    VL_ATTR((xshift_e_kernel<false, true>));
    VL_ATTR((xshift_e_kernel<false, false>));
    VL_ATTR((pshift_e_kernel<true>));
    VL_ATTR((pshift_e_kernel<false>));
#undef VL_ATTR
    return e;
}

// ============================================================================ filter split (emulated)
__global__ void emul_params_kernel(int n, const double* __restrict__ w, int* Wh, float* wl, float* wf)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * NTAP) return;
    int h;
    float l, f;
    emul_weight(w[idx], h, l, f);
    Wh[idx] = h;
    wl[idx] = l;
    wf[idx] = f;
}

cudaError_t launch_emul_params(int n, const double* w, int* Wh, float* wl, float* wf, cudaStream_t st)
{
    const int tot = n * NTAP;
    emul_params_kernel<<<(tot + 255) / 256, 256, 0, st>>>(n, w, Wh, wl, wf);
    return cudaGetLastError();
}

}  // namespace vl
