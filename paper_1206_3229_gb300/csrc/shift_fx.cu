// shift_fx.cu -- the two sweeps for 64-bit fixed-point storage (VLASOV_FX64).
//
// f is stored as X = round(f * 2^(61-Ef)) in int64 (|f| < 2^Ef, Ef = a bound four times the largest
// uploaded |f|): the same 8 bytes per cell as FP64, an absolute resolution of 2^-59 of max|f|, and no
// IEEE decoding.  Each staged element splits with two integer instructions into
//   X = kx * 2^30 + rem,  kx = X >> 30 (int32), rem in [0, 2^30)
// and the filter runs as in the emulated-FP64 sweeps (emul.cuh): 10 IMAD.WIDE on kx and 20 FP32
// FMAs on (float)kx and (float)rem; the int64 result T is already in storage units.  Data
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
static_assert(PSF_RB % PS_BH == 0, "a staged window is whole TMA boxes: the slot must hold nb * PS_BH rows");
// p-shift: PSF_RG compute warps and one producer warp (16 warps per SM at two CTAs, so
// that the compute warps keep 128 registers), tiles of PS_TW columns x PSF_TH rows, PSF_NB in flight
constexpr int PSF_RG = 7;
constexpr int PSF_TH = PSF_RG * PS_RPT;
constexpr int PSF_THREADS = PS_TW * (PSF_RG + 1);
constexpr int PSF_NB = 2;

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

// A chunk with an output whose foot cell touches or leaves a zero-outside row end (rare; kept out
// of line so that its registers do not weigh on the filter loop).  Outputs with the foot cell
// wholly outside are 0; the two touching the end take the row's edge filters (line_edge_weights) in
// the same fixed-point arithmetic as the interior; the others keep the interior results o.v.
// Window element m (m = 0 at f_{k-4} of the chunk's first output) is row[b0 + m] of a plain row,
// or of a padded row (PADDED: 8-element lines 10 elements apart).  Returned by value (no caller
// array needs an address), with the range bits of the recomputed outputs.
struct FxOut {
    long long v[XF_V];
    uint32_t rng;
};
__device__ __noinline__ FxOut fx_edge_chunk(FxOut o, const long long* row, int b0, bool padded, const XRec* rc,
                                            int k, int Nx)
{
    o.rng = 0;
    for (int v = 0; v < XF_V; ++v) {
        const int kv = k + v;
        if (kv >= 0 && kv < Nx - 1) continue;
        if (kv < -1 || kv >= Nx) {
            o.v[v] = 0;
            continue;
        }
        const int q = kv < 0 ? 0 : 1;
        long long M = EMUL_M0;
        float sl = 0.f, sr = 0.f;
        for (int t = 0; t < NTAP; ++t) {
            const int ee = b0 + v + t;
            int kx;
            float kf, rf;
            fx_split(padded ? row[(ee >> 3) * 10 + (ee & 7)] : row[ee], kx, kf, rf);
            M += (long long)rc->Whe[q][t] * (long long)kx;
            sl = fmaf(rc->wle[q][t], kf, sl);
            sr = fmaf(rc->wfe[q][t] * 9.313225746154785e-10f, rf, sr);   // * 2^-30
        }
        o.v[v] = fx_store(emul_finish(M, sl + sr), o.rng);
    }
    return o;
}

// One boundary output of a zero-outside column (window X = f_{kk-4} .., foot cell kk): 0 when the
// cell lies wholly outside, else the column's edge filter (em.Whe: [2][NTAP][Nx]) in the fixed-point
// arithmetic of the interior.  (Inline: an out-of-line call here cost the p-shift a stack frame
// and spills in its filter loop.)
struct FxOne {
    long long v;
    uint32_t rng;
};
__device__ __forceinline__ FxOne fx_edge_one(const long long* X, const EmulArgs& em, int i, int Nx, int kk, int Np)
{
    FxOne o{0, 0};
    if (kk < -1 || kk >= Np) return o;
    const int q = kk < 0 ? 0 : 1;
    long long M = EMUL_M0;
    float sl = 0.f, sr = 0.f;
    for (int t = 0; t < NTAP; ++t) {
        const size_t idx = ((size_t)q * NTAP + t) * Nx + i;
        int kx;
        float kf, rf;
        fx_split(X[t], kx, kf, rf);
        M += (long long)em.Whe[idx] * (long long)kx;
        sl = fmaf(em.wle[idx], kf, sl);
        sr = fmaf(em.wfe[idx] * 9.313225746154785e-10f, rf, sr);   // * 2^-30
    }
    o.v = fx_store(emul_finish(M, sl + sr), o.rng);
    return o;
}

// XF_V consecutive outputs of one x row from the staged fixed-point values f_{k-4-A} .. , read as
// pairs: pair h at q[h] in a plain row, or (PADDED) at q[h + (Q + h) / 4] in a padded row whose
// window starts at pair 4 m + Q (pair p at 16-byte slot p + p / 4, q = slot of the first pair).
// Input-stationary: each element is split once and fed to the outputs it touches.  The two FP32
// residual products of a tap are two scalar FMAs.
template <int A, bool PADDED = false>
__device__ __forceinline__ void fx_chunk(const longlong2* q, const FxW& w, long long (&out)[XF_V], uint32_t& rng,
                                         int Q = 0)
{
    long long M[XF_V];
    float2 S[XF_V];
#pragma unroll
    for (int v = 0; v < XF_V; ++v) {
        M[v] = EMUL_M0;
        S[v] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int h = 0; h < XF_W / 2; ++h) {
        const longlong2 pr = q[PADDED ? h + ((Q + h) >> 2) : h];
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
            // two scalar FMAs rather than one paired FFMA2: measured 11 % faster in the fused
            // x-shift, whose heavy FMA pipe (shared with the IMAD.WIDE products) was the busiest unit
            if (v0) {
                S[v].x = fmaf(w.wlr[t0].x, xa.x, S[v].x);
                S[v].y = fmaf(w.wlr[t0].y, xa.y, S[v].y);
            }
            if (v1) {
                S[v].x = fmaf(w.wlr[t1].x, xb.x, S[v].x);
                S[v].y = fmaf(w.wlr[t1].y, xb.y, S[v].y);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < XF_V; ++v) out[v] = fx_store(emul_finish(M[v], S[v].x + S[v].y), rng);
}

// End of an x-shift sweep: hand over this CTA's exact column sums acc[c][v] (column
// XF_V (tid + c blockDim) + v, units 2^(Ef-51)) in the form the arguments ask for.  Every thread
// of the block calls it (block reductions inside).
template <int CH>
__device__ __forceinline__ void fx_colsum_epilogue(const XShiftArgs& a, const long long (&acc)[CH][XF_V], int Ef,
                                                   i128* scratch)
{
    const int Nx = a.Nx, tid = threadIdx.x, nthreads = blockDim.x;
    if (a.colacc) {
        // exact fixed-point column sums, added across CTAs: units 2^(Ef-51) -> 2^-k_col
        const int sh = a.k_col + Ef - 51;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = XF_V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < XF_V; ++v) {
                    const long long x = acc[c][v];
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
        for (int c = 0; c < CH; ++c) {
            const int i = XF_V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < XF_V; ++v) {
                    const long long t = acc[c][v];
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
        const int sh = a.k_col + Ef - 51;
        long long* cp = a.colpart64 + (size_t)blockIdx.x * Nx;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = XF_V * (tid + c * nthreads);
            if (i < Nx) {
                long long q[XF_V];
#pragma unroll
                for (int v = 0; v < XF_V; ++v) {
                    const long long x = acc[c][v];
                    q[v] = sh >= 0 ? (long long)((unsigned long long)x << sh) : ((x + (1ll << (-sh - 1))) >> (-sh));
                }
#pragma unroll
                for (int v = 0; v < XF_V; v += 4) st_global_v4_b64(cp + i + v, q[v], q[v + 1], q[v + 2], q[v + 3]);
            }
        }
    } else if (a.colpart) {
        double* cp = a.colpart + (size_t)blockIdx.x * Nx;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = XF_V * (tid + c * nthreads);
            if (i < Nx) {
#pragma unroll
                for (int v = 0; v < XF_V; ++v) cp[i + v] = fx128_to_f64((i128)acc[c][v], 51 - Ef);
            }
        }
    }
}

// The CTA's kinetic sum (per-thread kin, units 2^(Ef-51-KIN_Q)): exact int128 when the
// arguments ask for it (the total is then independent of how rows were split over CTAs),
// else rounded to FP64.
__device__ __forceinline__ void fx_kin_epilogue(const XShiftArgs& a, i128 kin, int Ef, i128* scratch)
{
    const i128 t = block_sum_i128(kin, scratch);
    if (threadIdx.x == 0) {
        if (a.kin128) static_cast<i128*>(a.kin128)[blockIdx.x] = t;
        else a.kinpart[blockIdx.x] = fx128_to_f64(t, 51 + KIN_Q - Ef);
    }
}

// End of the fused x-shifts, HMF (blockDim >= 224): both passes' per-CTA sums (mass, cos- and
// sin-weighted column sums) and the exact kinetic sum in one pass over shared memory `sm`
// (7 blockDim int128): each thread stores its seven partials slot-major; warp w < 7 adds slot w with
// a lane-strided loop and one warp reduction (seven short reductions instead of three block-wide
// shuffle trees).  Weighted sums by exact split 32-bit products (Mac26).
__device__ __forceinline__ void xxf_hmf_epilogue(const XShiftArgs& a, const XShiftArgs& b,
                                                 const long long (&acc1)[1][XF_V], const long long (&acc2)[1][XF_V],
                                                 i128 kin, int Ef, i128* sm)
{
    const int Nx = a.Nx, tid = threadIdx.x, n = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int i = XF_V * tid;
    auto part = [&](const long long (&acc)[1][XF_V], int q) {
        long long m = 0;
        Mac26 x, y;
        if (i < Nx) {
#pragma unroll
            for (int v = 0; v < XF_V; ++v) {
                const long long t = acc[0][v];
                m += t;
                x.add(__ldg(a.cos50 + i + v), t);
                y.add(__ldg(a.sin50 + i + v), t);
            }
        }
        sm[(3 * q + 0) * n + tid] = (i128)m;
        sm[(3 * q + 1) * n + tid] = x.fold();
        sm[(3 * q + 2) * n + tid] = y.fold();
    };
    part(acc1, 0);
    part(acc2, 1);
    sm[6 * n + tid] = kin;
    __syncthreads();
    if (wid < 7) {
        i128 t = 0;
#pragma unroll 4
        for (int k = lane; k < n; k += 32) t += sm[wid * n + k];
        t = warp_sum_i128(t);
        if (lane == 0) {
            if (wid < 6) {
                const XShiftArgs& o = wid < 3 ? a : b;
                static_cast<i128*>(o.ctapart)[(size_t)blockIdx.x * 3 + wid % 3] = t;
            } else if (a.kin128) {
                static_cast<i128*>(a.kin128)[blockIdx.x] = t;
            } else {
                a.kinpart[blockIdx.x] = fx128_to_f64(t, 51 + KIN_Q - Ef);
            }
        }
    }
}

// Padded rows (fused x-shifts): 8-element lines 80 bytes apart, so that pair p (elements 2p, 2p+1)
// sits at 16-byte slot p + p / 4.  A warp's 16-byte window reads, 64 bytes apart per thread in a
// plain row (four-way bank conflicts), then hit distinct banks.  A TMA box of 10 x H elements over
// a tensor of 8-element lines writes this layout directly (the two columns past the line are out
// of bounds and arrive as zeros).
__host__ __device__ __forceinline__ int xxf_front(int pad, bool periodic) { return periodic ? 0 : (pad + 63) / 64 * 64; }
__host__ __device__ __forceinline__ int xxf_row_bytes(int Nx, int pad, bool periodic)
{
    const int lines = (2 * xxf_front(pad, periodic) + Nx + (periodic ? 16 : 0)) / 8;
    return (lines * 80 + 127) / 128 * 128;   // rows stay 128-byte aligned (TMA destinations)
}

// The chunk whose window starts at pair p0 of a padded row.
template <int A>
__device__ __forceinline__ void fx_chunk_padded(const longlong2* slots, int p0, const FxW& w, long long (&out)[XF_V],
                                                uint32_t& rng)
{
    // Q at run time: one instantiation (a compile-time Q, four copies of the unrolled chunk in
    // each pass, measured slower: instruction-cache misses)
    fx_chunk<A, true>(slots + 5 * (p0 >> 2) + (p0 & 3), w, out, rng, p0 & 3);
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
            const int base = PERIODIC ? rc->m4 - A : n0 - 4 - A;   // m4 has the parity of n0 - 4
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
                    const longlong2* q2 = reinterpret_cast<const longlong2*>(rowbuf + e);
                    if (A == 0) fx_chunk<0>(q2, w, out, rng);
                    else fx_chunk<1>(q2, w, out, rng);
                    if constexpr (!PERIODIC) {
                        const int k = i + n0;
                        if (k < 0 || k + XF_V - 1 >= Nx - 1) {
                            FxOut o;
#pragma unroll
                            for (int v = 0; v < XF_V; ++v) o.v[v] = out[v];
                            o = fx_edge_chunk(o, rowbuf, e + A, false, rc, k, Nx);
#pragma unroll
                            for (int v = 0; v < XF_V; ++v) out[v] = o.v[v];
                            rng |= o.rng;
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

    fx_colsum_epilogue<XF_MAXCH>(a, colacc, em.Ef, scratch);
    if constexpr (KIN) fx_kin_epilogue(a, kin, em.Ef, scratch);
}

template <bool PERIODIC, bool KIN>
__global__ void __launch_bounds__(XS_THREADS_MAX, 1) xshift_fx_kernel(XShiftArgs a, EmulArgs em)
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

// ============================================================================ fused x-shifts (FX64)
// The second x half-shift of step n and the first of step n+1 (Sec. 3, steps four and one of the
// Strang cycle) move row j by the same p_j dt/2 with the same filter, and neither needs anything
// from other rows.  So one launch stages each row once, filters it into a shared-memory row (the
// state f(t_n + dt) at the end of step n: its column sums and kinetic sum are step n's moments),
// filters that row again and writes only the result (f^(I) of step n+1, whose column sums give the
// next force).  The arithmetic of each pass is that of xshift_fx_body, so the result is the same
// bits as two launches; the HBM traffic is that of one.  One output chunk of XF_V columns per
// thread (Nx <= XF_V * blockDim.x); rows stride by the CTA count; S stages of whole rows in flight
// (TMA boxes of H lines into padded rows), two padded intermediate rows alternate so that one
// barrier per row suffices.
//   a: input, records, shape, and the outputs of the first pass (step n's moment sums, kinetic);
//   b: output row buffer (b.fout) and the column sums of the second pass.
template <bool PERIODIC>
__device__ __forceinline__ void xxshift_fx_body(const CUtensorMap* tmap, const XShiftArgs& a, const XShiftArgs& b,
                                                const EmulArgs& em)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    __shared__ unsigned int issued[8];     // copies issued into each stage

    const long long* __restrict__ fin = static_cast<const long long*>(a.fin);
    long long* __restrict__ fout = static_cast<long long*>(b.fout);
    const int Nx = a.Nx, Np = a.Np, PAD = a.pad, S = a.stages;
    const int PADR = xxf_front(PAD, PERIODIC);   // zero elements before the row (whole 640-byte line groups)
    const int sbytes = xxf_row_bytes(Nx, PAD, PERIODIC);
    const int H = a.box_h;                 // TMA box height in lines (a multiple of 8 dividing Nx / 8)
    unsigned char* stg = smem_raw + 128;
    long long* ibufs = reinterpret_cast<long long*>(stg + (size_t)S * sbytes);   // two padded rows
    const int istride = sbytes / 8;
    unsigned char* recs = reinterpret_cast<unsigned char*>(ibufs + 2 * (size_t)istride);
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int G = a.ctas > 0 ? a.ctas : (int)gridDim.x;
    const uint32_t tx_bytes = (uint32_t)(Nx / 8 * 80) + (PERIODIC ? 128u : 0u) + XREC_BYTES;   // boxes count whole
    const double unit = ldexp(1.0, em.Ef - FX_FRAC);
    const int i = XF_V * tid;              // this thread's output columns i .. i + XF_V - 1
    const bool act = i < Nx;
    uint32_t rng = 0;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&bars[s], 1);
            issued[s] = 0;
        }
        fence_barrier_init();
    }
    for (int e = tid; e < 2 * istride; e += nthreads) ibufs[e] = 0;
    if constexpr (!PERIODIC) {
        for (int s = 0; s < S; ++s) {   // zero halo lines of the stages
            long long* q = reinterpret_cast<long long*>(stg + (size_t)s * sbytes);
            for (int e = tid; e < PADR / 8 * 10; e += nthreads) q[e] = 0;
            for (int e = (PADR + Nx) / 8 * 10 + tid; e < istride; e += nthreads) q[e] = 0;
        }
    }
    __syncthreads();

    auto issue = [&](int s, int r) {
        unsigned char* dst = stg + (size_t)s * sbytes + PADR / 8 * 80;
        const long long* src = fin + (size_t)r * Nx;
        issued[s] += 1;
        mbar_arrive_expect_tx(&bars[s], tx_bytes);
        for (int l = 0; l < Nx / 8; l += H)   // boxes of 10 x H: 8 elements + 2 zero-filled per line
            tma_load_2d(dst + l * 80, tmap, 0, r * (Nx / 8) + l, &bars[s]);
        if constexpr (PERIODIC) {   // wrap lines
            bulk_g2s(dst + (Nx / 8) * 80, src, 64u, &bars[s]);
            bulk_g2s(dst + (Nx / 8 + 1) * 80, src + 8, 64u, &bars[s]);
        }
        bulk_g2s(recs + (size_t)s * XREC_BYTES, static_cast<const unsigned char*>(a.rec) + (size_t)r * XREC_BYTES,
                 XREC_BYTES, &bars[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            const int r = blockIdx.x + s * G;
            if (r < Np) issue(s, r);
        }
    }

    long long acc1[1][XF_V], acc2[1][XF_V];   // column sums of the two passes, units 2^(Ef-51)
#pragma unroll
    for (int v = 0; v < XF_V; ++v) {
        acc1[0][v] = 0;
        acc2[0][v] = 0;
    }
    i128 kin = 0;   // units 2^(Ef-51-KIN_Q), rows after the first pass

    int it = 0;
    bool failed = false;
    for (int r = blockIdx.x; r < Np; r += G, ++it) {
        const int s = it % S;
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[s], (uint32_t)((it / S) & 1), WAIT_LIMIT_NS));
        long long* ib = ibufs + (size_t)(it & 1) * istride;
        longlong2* ib2 = reinterpret_cast<longlong2*>(ib);
        FxW w;
        int n0 = 0, A = 0, e = 0;   // the row's shift; this thread's window start (both passes)
        long long p2q = 0, rowsum = 0;
        if (ok) {
            const unsigned char* sb = stg + (size_t)s * sbytes;
            const XRec* rc = reinterpret_cast<const XRec*>(recs + (size_t)s * XREC_BYTES);
            n0 = rc->n0;
            p2q = rc->p2q;
            A = (n0 - 4) & 1;
            e = i + (PERIODIC ? rc->m4 - A : n0 - 4 - A);   // m4 has the parity of n0 - 4
            if (PERIODIC && e >= Nx) e -= Nx;
#pragma unroll
            for (int t = 0; t < NTAP; ++t) {
                w.Wh[t] = rc->Wh[t];
                w.wlr[t] = make_float2(rc->wl[t], rc->wf[t] * 9.313225746154785e-10f);   // * 2^-30
            }
            if (act) {
                long long out[XF_V];
                const int p1 = (PADR + e) >> 1;
                const longlong2* sb2 = reinterpret_cast<const longlong2*>(sb);
                if (A == 0) fx_chunk_padded<0>(sb2, p1, w, out, rng);
                else fx_chunk_padded<1>(sb2, p1, w, out, rng);
                if constexpr (!PERIODIC) {
                    const int k = i + n0;
                    if (k < 0 || k + XF_V - 1 >= Nx - 1) {
                        FxOut o;
#pragma unroll
                        for (int v = 0; v < XF_V; ++v) o.v[v] = out[v];
                        o = fx_edge_chunk(o, reinterpret_cast<const long long*>(sb), PADR + e + A, true, rc, k, Nx);
#pragma unroll
                        for (int v = 0; v < XF_V; ++v) out[v] = o.v[v];
                        rng |= o.rng;
                    }
                }
#pragma unroll
                for (int v = 0; v < XF_V; ++v) {
                    const long long Tc = out[v] >> 10;
                    acc1[0][v] += Tc;
                    rowsum += Tc;
                }
                {
                    const int pb = (PADR + i) >> 1;
#pragma unroll
                    for (int k = 0; k < XF_V / 2; ++k) ib2[pb + k + ((pb + k) >> 2)] = make_longlong2(out[2 * k], out[2 * k + 1]);
                }
                if constexpr (PERIODIC) {
                    if (i < 16) {   // the wrap copy read by the second pass's last windows
                        const int pb = (PADR + Nx + i) >> 1;
#pragma unroll
                        for (int k = 0; k < XF_V / 2; ++k) ib2[pb + k + ((pb + k) >> 2)] = make_longlong2(out[2 * k], out[2 * k + 1]);
                    }
                }
            }
        }
        // every warp's first pass is done: the intermediate row is complete and stage s is free
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 32 * (it % (nthreads >> 5))) {   // the refill's issuer rotates over the warps
            const int rn = r + S * G;
            if (rn < Np) {
                fence_proxy_async_smem();
                issue(s, rn);
            }
        }
        kin += (i128)rowsum * (i128)p2q;
        if (act) {
            long long out[XF_V];
            const int p0 = (e + PADR) >> 1;
            if (A == 0) fx_chunk_padded<0>(ib2, p0, w, out, rng);
            else fx_chunk_padded<1>(ib2, p0, w, out, rng);
            if constexpr (!PERIODIC) {
                const int k = i + n0;
                if (k < 0 || k + XF_V - 1 >= Nx - 1) {
                    // the staged record may already be overwritten: read this row's from global memory
                    const XRec* rg = reinterpret_cast<const XRec*>(static_cast<const unsigned char*>(a.rec) +
                                                                   (size_t)r * XREC_BYTES);
                    FxOut o;
#pragma unroll
                    for (int v = 0; v < XF_V; ++v) o.v[v] = out[v];
                    o = fx_edge_chunk(o, ib, PADR + e + A, true, rg, k, Nx);
#pragma unroll
                    for (int v = 0; v < XF_V; ++v) out[v] = o.v[v];
                    rng |= o.rng;
                }
            }
#pragma unroll
            for (int v = 0; v < XF_V; ++v) acc2[0][v] += out[v] >> 10;
            long long* orow = fout + (size_t)r * Nx;
#pragma unroll
            for (int v = 0; v < XF_V; v += 4) st_global_v4_b64(orow + i + v, out[v], out[v + 1], out[v + 2], out[v + 3]);
        }
    }
    __syncthreads();   // every warp is done with the stage buffers
    if (rng >= (1u << 30)) atomicCAS(a.err, 0, DEV_ERR_RANGE);
    i128* scratch = reinterpret_cast<i128*>(stg);

    if (failed) {
        if (tid == 0) {
            atomicCAS(a.err, 0, DEV_ERR_XSHIFT_WAIT);
            for (int k = 0; k < S; ++k)   // the last copy issued into each stage must land before exit
                if (issued[k] > 0) mbar_wait_bounded(&bars[k], (uint32_t)((issued[k] - 1) & 1), WAIT_LIMIT_NS);
        }
        __syncthreads();
        return;
    }
    if (a.ctapart && b.ctapart && blockDim.x >= 7 * 32) {
        xxf_hmf_epilogue(a, b, acc1, acc2, kin, em.Ef, scratch);
        return;
    }
    fx_colsum_epilogue<1>(a, acc1, em.Ef, scratch);
    fx_kin_epilogue(a, kin, em.Ef, scratch);
    fx_colsum_epilogue<1>(b, acc2, em.Ef, scratch);
}

template <bool PERIODIC>
__global__ void __launch_bounds__(XXF_THREADS_MAX, 1) xxshift_fx_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                          XShiftArgs a, XShiftArgs b, EmulArgs em)
{
    xxshift_fx_body<PERIODIC>(&tmap, a, b, em);
}

// ============================================================================ p-shift (FX64)
// STAGED: warp 0 prepares each tile in shared memory one iteration ahead (single grids, measured
// faster there); otherwise every warp works out its tile's window and loads its filters, prefetched
// into L1 one tile ahead (the batched form, whose slots are small grids of few tiles per CTA: the
// staged form measured slower there).
// Input-stationary accumulation for the p-shift: elements u and u + 1 of a column's window (X0, X1;
// X1 absent when !second) fed to the PS_RPT outputs they touch.  Their two products for an output
// enter its int64 sum in one three-input add (two IMAD.WIDE + IADD3 + IADD3.X) instead of two 64-bit
// multiply-adds (three instructions each on this GPU).
__device__ __forceinline__ void psfx_feed2(int u, long long X0, long long X1, bool second, const FxW& w,
                                           long long (&M)[PS_RPT], float2 (&S)[PS_RPT])
{
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
        if (v0) {
            S[rw].x = fmaf(w.wlr[t0].x, xa.x, S[rw].x);
            S[rw].y = fmaf(w.wlr[t0].y, xa.y, S[rw].y);
        }
        if (v1) {
            S[rw].x = fmaf(w.wlr[t1].x, xb.x, S[rw].x);
            S[rw].y = fmaf(w.wlr[t1].y, xb.y, S[rw].y);
        }
    }
}

// The PS_RPT outputs of one column (rows jb ..) from the window: staged (buf, window element u at
// buf[(base + u) * PS_TW + lane]) or, for a tile whose window does not fit, loaded from f.
template <bool PPER>
__device__ __forceinline__ void psfx_accumulate(const TileWin& t, const long long* buf, int base, const long long* fin,
                                                int jb, int n0_i, int i, bool colvalid, int Nx, int Np, const FxW& w,
                                                long long (&M)[PS_RPT], float2 (&S)[PS_RPT])
{
#pragma unroll
    for (int rw = 0; rw < PS_RPT; ++rw) {
        M[rw] = EMUL_M0;
        S[rw] = make_float2(0.f, 0.f);
    }
    constexpr int NU = PS_RPT + 9;
    const int lane = threadIdx.x & 31;
    if (t.smem_ok) {
#pragma unroll
        for (int u = 0; u < NU; u += 2)
            psfx_feed2(u, buf[(base + u) * PS_TW + lane], u + 1 < NU ? buf[(base + u + 1) * PS_TW + lane] : 0ll,
                       u + 1 < NU, w, M, S);
    } else {
#pragma unroll
        for (int u = 0; u < NU; u += 2) {
            const long long X0 = colvalid ? gload_p<long long, PPER>(fin, jb + n0_i - 4 + u, i, Nx, Np) : 0ll;
            const long long X1 = (colvalid && u + 1 < NU) ? gload_p<long long, PPER>(fin, jb + n0_i - 3 + u, i, Nx, Np) : 0ll;
            psfx_feed2(u, X0, X1, u + 1 < NU, w, M, S);
        }
    }
}

// A tile wholly inside the grid, every foot cell inside too (the common case): its rows are stored
// without per-row edge or bounds checks.
template <bool PPER, int TH = PS_TH>
__device__ __forceinline__ bool psfx_interior(const TileWin& t, int Nx, int Np)
{
    return t.i0 + PS_TW <= Nx && t.j0 + TH <= Np &&
           (PPER || (t.j0 + t.kmin >= 0 && t.j0 + TH - 1 + t.kmax < Np - 1));
}

// Store the column's outputs.  Interior tiles: plain stores.  Otherwise rows past the grid are
// skipped and outputs whose foot cell touches or leaves a zero-outside column end are recomputed
// from the window (buf or f, as in psfx_accumulate) with the column's edge filters.
template <bool PPER>
__device__ __forceinline__ void psfx_store(bool interior, const TileWin& t, const long long* buf, int base,
                                           const long long* fin, long long* fout, int jb, int n0_i, int i,
                                           bool colvalid, int Nx, int Np, const EmulArgs& em,
                                           const long long (&M)[PS_RPT], const float2 (&S)[PS_RPT], uint32_t& rng)
{
    if (interior) {
        long long* __restrict__ op = fout + (size_t)jb * Nx + i;
#pragma unroll
        for (int rw = 0; rw < PS_RPT; ++rw) {
            *op = fx_store(emul_finish(M[rw], S[rw].x + S[rw].y), rng);
            op += Nx;
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    bool any_edge = false;
#pragma unroll
    for (int rw = 0; rw < PS_RPT; ++rw) {
        const int j = jb + rw;
        const long long out = fx_store(emul_finish(M[rw], S[rw].x + S[rw].y), rng);
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
            const double unit = ldexp(1.0, em.Ef - FX_FRAC);
            const double g = em.gd[i], d = em.gd[Nx + i];
            for (int rw = 0; rw < PS_RPT; ++rw) {
                const int j = jb + rw, kk = j + n0_i;
                if (j >= Np || !(kk < 0 || kk >= Np - 1)) continue;
                long long X[NTAP];
                for (int u = 0; u < NTAP; ++u)
                    X[u] = t.smem_ok ? buf[(base + rw + u) * PS_TW + lane]
                                     : gload_p<long long, PPER>(fin, j + n0_i - 4 + u, i, Nx, Np);
                if (em.Whe) {   // fixed point, with the column's edge filters
                    const FxOne o = fx_edge_one(X, em, i, Nx, kk, Np);
                    rng |= o.rng;
                    fout[(size_t)j * Nx + i] = o.v;
                } else {
                    fout[(size_t)j * Nx + i] = fx_edge(X, em.w64 + i, Nx, kk, Np, g, d, unit, em.Ef);
                }
            }
        }
    }
}

// p-shift, warp-specialised (single grids and the batched form): warp PSF_RG (the producer) prepares each tile of this CTA
// into one of PSF_NB slots -- its window of input rows by 2-D TMA boxes (zero fill), its columns'
// foot offsets and split filters -- and the PSF_RG compute warps take the slots in turn on full /
// empty mbarriers, with no CTA-wide barrier per tile.  Thread (warp g, lane c) computes the PS_RPT
// outputs of column c in rows j0 + g PS_RPT .., input-stationary over the PS_RPT + 9 staged rows.
template <bool PPER>
__device__ __forceinline__ void pshift_fx_ws_body(const CUtensorMap* tmap, const PShiftArgs& a, const EmulArgs& em)
{
    constexpr int NB = PSF_NB;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = align128(smem_dyn);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + NB;
    long long* bufs = reinterpret_cast<long long*>(smem_raw + 128);
    constexpr int BUF = PSF_RB * PS_TW;
    static_assert(2 * NB * 8 <= 128, "barriers fit in front of the buffers");

    const long long* __restrict__ fin = static_cast<const long long*>(a.fin);
    long long* __restrict__ fout = static_cast<long long*>(a.fout);
    const int Nx = a.Nx, Np = a.Np;
    const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 5;
    const int ntx = (Nx + PS_TW - 1) / PS_TW, nty = (Np + PSF_TH - 1) / PSF_TH;
    const int ntiles = ntx * nty;
    const int G = gridDim.x;

    struct TileInfo {
        int n0[PS_TW];
        int Wh[NTAP][PS_TW];
        float wl[NTAP][PS_TW], wr[NTAP][PS_TW];
        TileWin t;
    };
    __shared__ TileInfo info[NB];

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], PSF_RG);
        }
        fence_barrier_init();
        prefetch_tensormap(tmap);
    }
    __syncthreads();   // the last CTA-wide barrier: the roles part here

    if (grp == PSF_RG) {
        // ---- producer
        int k = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles; tile += G, ++k) {
            const int b = k % NB;
            // the tile's window, offsets and filters first: their global loads overlap the wait for
            // the slot
            int n0l;
            bool cv;
            const TileWin t = tile_window<PPER, PSF_RB, PSF_TH>(tile, ntx, em.n0, Nx, lane, n0l, cv);
            const size_t ic = (size_t)t.i0 + lane;
            int Whr[NTAP];
            float wlr[NTAP], wrr[NTAP];
#pragma unroll
            for (int q = 0; q < NTAP; ++q) {
                Whr[q] = cv ? em.Wh[(size_t)q * Nx + ic] : 0;
                wlr[q] = cv ? em.wl[(size_t)q * Nx + ic] : 0.f;
                wrr[q] = cv ? em.wf[(size_t)q * Nx + ic] * 9.313225746154785e-10f : 0.f;   // * 2^-30
            }
            if (k >= NB) ok = mbar_wait_bounded(&empty[b], (uint32_t)(((k / NB) - 1) & 1), WAIT_LIMIT_NS);
            if (!__all_sync(0xffffffffu, ok)) break;
#pragma unroll
            for (int q = 0; q < NTAP; ++q) {
                info[b].Wh[q][lane] = Whr[q];
                info[b].wl[q][lane] = wlr[q];
                info[b].wr[q][lane] = wrr[q];
            }
            info[b].n0[lane] = n0l;
            __syncwarp();
            if (lane == 0) {
                info[b].t = t;
                fence_proxy_async_smem();   // the compute warps' reads of buffer b before its refill
                mbar_arrive_expect_tx(&full[b], t.smem_ok ? (uint32_t)(t.nb * PS_BH * PS_TW * 8) : 0u);   // releases info[b]
                if (t.smem_ok)
                    for (int q = 0; q < t.nb; ++q)
                        tma_load_2d(bufs + (size_t)b * BUF + (size_t)q * PS_BH * PS_TW, tmap, t.i0, t.r0 + q * PS_BH, &full[b]);
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
    uint32_t rng = 0;   // OR of (high word + 2^29) of every stored result
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, ++k) {
        const int b = k % NB;
        if (!mbar_wait_bounded(&full[b], (uint32_t)((k / NB) & 1), WAIT_LIMIT_NS)) {
            if (lane == 0) atomicCAS(a.err, 0, DEV_ERR_PSHIFT_WAIT);
            break;
        }
        const TileWin t = info[b].t;
        const int n0_i = info[b].n0[lane];
        FxW w;
#pragma unroll
        for (int q = 0; q < NTAP; ++q) {
            w.Wh[q] = info[b].Wh[q][lane];
            w.wlr[q] = make_float2(info[b].wl[q][lane], info[b].wr[q][lane]);
        }
        const int i = t.i0 + lane;
        const bool colvalid = i < Nx;
        const int jb = t.j0 + grp * PS_RPT;   // first output row of this thread
        const int base = jb + n0_i - 4 - t.r0;
        const long long* buf = bufs + (size_t)b * BUF;
        long long M[PS_RPT];
        float2 S[PS_RPT];
        psfx_accumulate<PPER>(t, buf, base, fin, jb, n0_i, i, colvalid, Nx, Np, w, M, S);
        const bool interior = psfx_interior<PPER, PSF_TH>(t, Nx, Np);
        if (interior) {   // the window and slot are read: hand buffer b back before the stores
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
        }
        psfx_store<PPER>(interior, t, buf, base, fin, fout, jb, n0_i, i, colvalid, Nx, Np, em, M, S, rng);
        if (!interior) {   // edge outputs read the window again
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[b]);
        }
    }
    if (rng >= (1u << 30)) atomicCAS(a.err, 0, DEV_ERR_RANGE);
}

template <bool PPER>
__global__ void __launch_bounds__(PSF_THREADS, 2) pshift_fx_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                     PShiftArgs a, EmulArgs em)
{
    pshift_fx_ws_body<PPER>(&tmap, a, em);
}

// Batched form (the same warp-specialised body): the slot's tensor map sits in global memory next to
// its arguments.
template <bool PPER>
__global__ void __launch_bounds__(PSF_THREADS, 2) pshift_fx_batch_kernel(const CUtensorMap* __restrict__ tmaps,
                                                                           const PShiftArgs* __restrict__ args,
                                                                           const EmulArgs* __restrict__ ems,
                                                                           const int* __restrict__ ver)
{
    const int slot = blockIdx.y;
    const int k = slot * 2 + ver[slot];
    const PShiftArgs a = args[k];
    if (a.Nx <= 0) return;
    const EmulArgs em = ems[slot];
    pshift_fx_ws_body<PPER>(tmaps + k, a, em);
}

int xshift_fx_max_cols(int threads) { return XF_V * threads * XF_MAXCH; }

int pshift_fx_tile_rows() { return PSF_TH; }

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

int xxshift_fx_row_bytes(int Nx, int pad, bool periodic) { return xxf_row_bytes(Nx, pad, periodic); }

size_t xxshift_fx_smem_bytes(int Nx, int pad, int stages)
{
    const size_t sb = (size_t)std::max(xxf_row_bytes(Nx, pad, true), xxf_row_bytes(Nx, pad, false));
    return 256 + (size_t)stages * (sb + XREC_BYTES) + 2 * sb;
}

int xxshift_fx_threads(int Nx) { return std::max(32, (Nx / XF_V + 31) / 32 * 32); }

cudaError_t launch_xxshift_fx(bool periodic, int grid, const CUtensorMap* tmap, const XShiftArgs& a, const XShiftArgs& b,
                              const EmulArgs& em, cudaStream_t st)
{
    if (a.rec == nullptr || a.Nx > XF_V * XXF_THREADS_MAX || a.stages < 1 || a.stages > 8) return cudaErrorInvalidValue;
    const size_t smem = xxshift_fx_smem_bytes(a.Nx, a.pad, a.stages);
    const int threads = xxshift_fx_threads(a.Nx);
    if (periodic) xxshift_fx_kernel<true><<<grid, threads, smem, st>>>(*tmap, a, b, em);
    else xxshift_fx_kernel<false><<<grid, threads, smem, st>>>(*tmap, a, b, em);
    return cudaGetLastError();
}

cudaError_t xxshift_fx_occupancy(bool periodic, int Nx, size_t smem, int* blocks)
{
    const int threads = xxshift_fx_threads(Nx);
    return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xxshift_fx_kernel<true>, threads, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xxshift_fx_kernel<false>, threads, smem);
}

cudaError_t launch_pshift_fx(bool p_periodic, int grid, const CUtensorMap* tmap, const PShiftArgs& a,
                             const EmulArgs& em, cudaStream_t st)
{
    const size_t smem = pshift_fx_smem_bytes();
    if (p_periodic) pshift_fx_kernel<true><<<grid, PSF_THREADS, smem, st>>>(*tmap, a, em);
    else pshift_fx_kernel<false><<<grid, PSF_THREADS, smem, st>>>(*tmap, a, em);
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
    pshift_fx_batch_kernel<false><<<grid, PSF_THREADS, pshift_fx_smem_bytes(), st>>>(tmaps, args, ems, ver);
    return cudaGetLastError();
}

cudaError_t set_kernel_attributes_fx(int max_smem)
{
    cudaError_t e = cudaSuccess;
#define VL_ATTR(fn) \
    if (e == cudaSuccess) e = allow_dynamic_smem(fn, max_smem)
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
    VL_ATTR((xxshift_fx_kernel<true>));
    VL_ATTR((xxshift_fx_kernel<false>));
#undef VL_ATTR
    return e;
}

cudaError_t xshift_fx_occupancy(bool periodic, int threads, size_t smem, int* blocks)
{
    return periodic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_fx_kernel<true, true>, threads, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, xshift_fx_kernel<false, true>, threads, smem);
}

cudaError_t pshift_fx_occupancy(int* blocks)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pshift_fx_kernel<false>, PSF_THREADS,
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
