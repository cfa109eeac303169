// vlasov_api.cu -- host runtime behind the C ABI of include/vlasov.h.
//
// A handle owns two ping-pong copies of f, the per-row x-shift filters (fixed for the run: they
// depend only on p_j, dt and dx), the per-column p-shift filters (rewritten every step by the
// force), reduction scratch, a ring of per-step moment records, and two CUDA graphs holding one
// Strang step each (one per starting buffer).  vlasov_step(n) launches those graphs n times.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vlasov.h"
#include "emul.cuh"
#include "fixed_point.cuh"
#include "vlasov_internal.cuh"

using namespace vl;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU_TRY(expr)                                                                                 \
    do {                                                                                             \
        cudaError_t e_ = (expr);                                                                     \
        if (e_ != cudaSuccess) return fail(VLASOV_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));   \
    } while (0)

PFN_cuTensorMapEncodeTiled_v12000 get_encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

constexpr int ALIGN_N = 8;

}  // namespace

// Graph runs: whole steps (or middle pieces of fused steps) are launched in graphs of 2^L of them,
// L < RUN_LEVELS.
constexpr int RUN_LEVELS = 6;

struct vlasov_sim {
    int model = 0, Nx = 0, Np = 0, prec = 0, esz = 8;
    int msz = 8;                // bytes of the filter/parameter type: 8 (FP64 modes) or 4 (FP32, BF16 storage)
    bool xper = true, pper = false;
    double xmin = 0, xmax = 0, pmin = 0, pmax = 0, dx = 0, dp = 0, dt = 0, eps = 0, G = 1;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int dev = 0, nsm = 0, max_smem = 0;   // max_smem: opt-in shared memory per block

    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    bool has_f = false;

    bool emul = false;          // FP64 storage, integer/FP32 filter arithmetic (emul.cuh)
    bool fx = false;            // 64-bit fixed-point storage, same filter arithmetic (shift_fx.cu)
    LineParamsDev xp, pp, sp;   // x rows (fixed), p columns (per step), scratch for substeps
    EmulParamsDev xe, pe, se;   // their emulated-FP64 splits
    void* xrec = nullptr;       // [Np] XRec of the fixed x rows
    void* srec = nullptr;       // [max(Nx, Np)] XRec scratch for x substeps
    int xthreads = 256, xstages = 1, xpad = 16, xgrid = 1, pgrid = 1, crgrid = 1;
    bool gs = false;            // global-spline sweeps (vlasov_set_spline)
    double* gs_h = nullptr;     // [GS_HTAPS] their filter h
    int gspgrid = 0;

    double* colpart = nullptr;  // [xgrid][Nx]
    unsigned long long* colacc = nullptr;  // [Nx] exact column sums added by the x-shift
    double* kinpart = nullptr;  // [xgrid]
    double* rho = nullptr;
    long long* colfx = nullptr; // [Nx] fixed-point column sums
    double* Qd = nullptr;       // [Nx] sheet prefix combination
    double* F = nullptr;
    double* Fout = nullptr;
    void* blockpart = nullptr;  // int128 [crgrid][3]
    void* ringpart = nullptr;   // int128 [(Nx+7)/8]
    unsigned int* tickets = nullptr;  // [0] colreduce, [1] ring, [2] colreduce of the end state (fused ring)
    unsigned long long* maxbits = nullptr;
    Scalars* sc = nullptr;
    double* costab = nullptr;
    double* sintab = nullptr;
    long long* cosfx = nullptr;
    long long* sinfx = nullptr;
    long long* cos50 = nullptr;   // round(cos x_i 2^50), round(sin x_i 2^50)
    long long* sin50 = nullptr;
    void* ctapart = nullptr;      // [xgrid][3] int128 per-CTA HMF partials
    bool hmf_cta = false;         // HMF: reductions from per-CTA partials (no per-column pass)
    bool hmf_cta_fd = false;      //   its value with the spline of Eq. findif (the global-spline
                                  //   sweeps hand over column partials)
    void* ringdV = nullptr;     // in the storage type
    void* ringV = nullptr;
    // ring force methods (ring.cu): exact fixed-point tables and scratch, FFT spectra and twiddles
    int ring_method = RING_M_FIXED;
    long long* ringKq = nullptr;
    long long* ringVq = nullptr;
    int ring_sK = 0, ring_sV = 0, ring_ksplit = 1;
    void* ring_gpart = nullptr;
    unsigned int* ring_gticket = nullptr;
    void* ring_upart = nullptr;
    void* ring_fft64 = nullptr;   // [khat N | vhat N | twiddles N/2] double2
    void* ring_fft32 = nullptr;   // same as float2
    void* ring_tcK = nullptr;     // tensor-core method: Toeplitz block images of V' and V
    void* ring_tcV = nullptr;
    // fused ring steps: the moments of the end of a step and the force of the next step's f^(I) are
    // reduced and convolved side by side, so the end state has its own copies of these
    double* rho_m = nullptr;
    long long* colfx_m = nullptr;
    Scalars* sc_m = nullptr;
    void* blockpart_m = nullptr;
    void* ring_gpart_m = nullptr;
    unsigned int* ring_gticket_m = nullptr;
    long long* ring_tcacc = nullptr;   // [N] fixed-point sums of the blocks' partial results
    unsigned int* ring_tcticket = nullptr;
    double ring_tcmax[2] = {0, 0};     // max |V'|, max |V| (scale of those sums)
    // fixed-point scales of the reductions (from a bound 2^Ef >= 4 max|f|)
    int Ef = 0, k_col = 0, k_kin = 0, k_pot = 0;
    bool scales_set = false;
    MomentRec* hist = nullptr;
    long long* dstep = nullptr;
    long long read_step = 0;
    int* err = nullptr;

    // Fused x-shifts (FX64, Nx <= 4096): the second x half-shift of a step and the first of the
    // next run as one launch (xxshift_fx), so vlasov_step(n) runs head (x-shift, force, p-shift),
    // n-1 times mid (fused x-shifts, moments, force, p-shift) and tail (x-shift, moments).
    bool fuse_ok = false, fuse = false;
    int xxgrid = 0, xxstages = 0;
    int nctas = 0;                    // max(xgrid, xxgrid): entries of the per-CTA partial buffers
    void* ctapart_m = nullptr;        // [nctas][3] int128 HMF partials of the fused launch's first pass
    long long* colpart_m = nullptr;   // [nctas][Nx] its per-CTA column sums (other models)
    void* kin128 = nullptr;           // [nctas] int128 per-CTA kinetic sums (FX64)

    CUtensorMap tmap[2];
    CUtensorMap xtmap[2];             // fused x-shifts: f[b] as 8-element lines, boxes of 10 x xbox_h
    int xbox_h = 0;
    // per starting buffer: runs of 2^L whole steps, head and tail pieces, runs of 2^L middle pieces
    cudaGraphExec_t grun[2][RUN_LEVELS] = {};
    cudaGraphExec_t ghead[2] = {nullptr, nullptr}, gtail[2] = {nullptr, nullptr};
    cudaGraphExec_t gmid[2][RUN_LEVELS] = {};
};

namespace {

void free_params(LineParamsDev& p)
{
    cudaFree(p.n0);
    cudaFree(p.w);
    cudaFree(p.gd);
    cudaFree(p.beta);
    p = LineParamsDev{};
}

int alloc_params(LineParamsDev& p, int n, int esz)
{
    CU_TRY(cudaMalloc(&p.n0, sizeof(int) * (size_t)n));
    CU_TRY(cudaMalloc(&p.w, (size_t)esz * NTAP * (size_t)n));
    CU_TRY(cudaMalloc(&p.gd, (size_t)esz * 2 * (size_t)n));
    CU_TRY(cudaMalloc(&p.beta, sizeof(double) * (size_t)n));
    return VLASOV_OK;
}

void free_emul(EmulParamsDev& e)
{
    cudaFree(e.Wh);
    cudaFree(e.wl);
    cudaFree(e.wf);
    cudaFree(e.Whe);
    cudaFree(e.wle);
    cudaFree(e.wfe);
    e = EmulParamsDev{};
}

int alloc_emul(EmulParamsDev& e, int n)
{
    CU_TRY(cudaMalloc(&e.Wh, sizeof(int) * NTAP * (size_t)n));
    CU_TRY(cudaMalloc(&e.wl, sizeof(float) * NTAP * (size_t)n));
    CU_TRY(cudaMalloc(&e.wf, sizeof(float) * NTAP * (size_t)n));
    CU_TRY(cudaMalloc(&e.Whe, sizeof(int) * 2 * NTAP * (size_t)n));
    CU_TRY(cudaMalloc(&e.wle, sizeof(float) * 2 * NTAP * (size_t)n));
    CU_TRY(cudaMalloc(&e.wfe, sizeof(float) * 2 * NTAP * (size_t)n));
    return VLASOV_OK;
}

// Host-side filters for n lines with displacements disp[] (cells), uploaded to p (and, for the
// emulated FP64 sweeps, their integer/FP32 split to e; and as staged x-shift records to rec).
int upload_params(vlasov_sim* s, LineParamsDev& p, const double* disp, int n, int* max_abs_n0,
                  EmulParamsDev* e = nullptr, void* rec = nullptr, bool rows_are_p = false)
{
    if (rec) {
        std::vector<unsigned char> buf((size_t)n * XREC_BYTES, 0);
        for (int l = 0; l < n; ++l) {
            LineSplit L;
            line_split(disp[l], L);
            XRec r;
            std::memset(&r, 0, sizeof r);
            r.n0 = L.n0;
            r.m4 = (int)((((long long)L.n0 - 4) % s->Nx + s->Nx) % s->Nx);
            r.g64 = L.g;
            r.d64 = L.d;
            r.g32 = (float)L.g;
            r.d32 = (float)L.d;
            for (int t = 0; t < NTAP; ++t) {
                r.w64[t] = L.w[t];
                r.w32[t] = (float)L.w[t];
                emul_weight(L.w[t], r.Wh[t], r.wl[t], r.wf[t]);
            }
            double we[2][NTAP];
            line_edge_weights(L, we);
            for (int q = 0; q < 2; ++q)
                for (int t = 0; t < NTAP; ++t) emul_weight(we[q][t], r.Whe[q][t], r.wle[q][t], r.wfe[q][t]);
            if (rows_are_p) {
                const double pj = s->pmin + (double)l * s->dp;   // as the kernels' p_j
                r.p2q = std::llround(std::ldexp(0.5 * pj * pj, KIN_Q));
                r.p2h = (float)(0.5 * pj * pj);
            }
            std::memcpy(&buf[(size_t)l * XREC_BYTES], &r, sizeof r);
        }
        CU_TRY(cudaMemcpyAsync(rec, buf.data(), buf.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
    }
    std::vector<int> n0(n);
    std::vector<double> w((size_t)NTAP * n), gd(2 * (size_t)n), we((size_t)2 * NTAP * n), beta(n);
    int mx = 0;
    for (int l = 0; l < n; ++l) {
        LineSplit L;
        line_split(disp[l], L);
        n0[l] = L.n0;
        beta[l] = L.beta;
        mx = std::max(mx, std::abs(L.n0));
        for (int t = 0; t < NTAP; ++t) w[(size_t)t * n + l] = L.w[t];
        gd[l] = L.g;
        gd[(size_t)n + l] = L.d;
        double e2[2][NTAP];
        line_edge_weights(L, e2);
        for (int q = 0; q < 2; ++q)
            for (int t = 0; t < NTAP; ++t) we[((size_t)q * NTAP + t) * n + l] = e2[q][t];
    }
    if (max_abs_n0) *max_abs_n0 = mx;
    CU_TRY(cudaMemcpyAsync(p.n0, n0.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s->st));
    CU_TRY(cudaMemcpyAsync(p.beta, beta.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s->st));
    if ((s->emul || s->fx) && e) {
        std::vector<int> Wh(w.size());
        std::vector<float> wl(w.size()), wf(w.size());
        for (size_t q = 0; q < w.size(); ++q) emul_weight(w[q], Wh[q], wl[q], wf[q]);
        CU_TRY(cudaMemcpyAsync(e->Wh, Wh.data(), sizeof(int) * Wh.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaMemcpyAsync(e->wl, wl.data(), sizeof(float) * wl.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaMemcpyAsync(e->wf, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice, s->st));
        std::vector<int> Whe(we.size());
        std::vector<float> wle(we.size()), wfe(we.size());
        for (size_t q = 0; q < we.size(); ++q) emul_weight(we[q], Whe[q], wle[q], wfe[q]);
        CU_TRY(cudaMemcpyAsync(e->Whe, Whe.data(), sizeof(int) * Whe.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaMemcpyAsync(e->wle, wle.data(), sizeof(float) * wle.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaMemcpyAsync(e->wfe, wfe.data(), sizeof(float) * wfe.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
    }
    if (s->msz == 8) {
        CU_TRY(cudaMemcpyAsync(p.w, w.data(), 8 * w.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaMemcpyAsync(p.gd, gd.data(), 8 * gd.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
    } else {
        std::vector<float> wf(w.begin(), w.end()), gf(gd.begin(), gd.end());
        CU_TRY(cudaMemcpyAsync(p.w, wf.data(), 4 * wf.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaMemcpyAsync(p.gd, gf.data(), 4 * gf.size(), cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
    }
    return VLASOV_OK;
}

int make_tmap(vlasov_sim* s, int b)
{
    auto enc = get_encode_tiled();
    if (!enc) return fail(VLASOV_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)s->Nx, (cuuint64_t)s->Np};
    cuuint64_t strides[1] = {(cuuint64_t)s->Nx * (cuuint64_t)s->esz};
    cuuint32_t box[2] = {(cuuint32_t)PS_TW, (cuuint32_t)PS_BH};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = s->fx ? CU_TENSOR_MAP_DATA_TYPE_INT64
                                   : s->esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : s->esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(&s->tmap[b], dt, 2,
                     s->f[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(VLASOV_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    if (s->fuse_ok && s->fx) {
        // rows of f as 8-element lines; a box of 10 x xbox_h lands as padded lines (2 zero columns)
        cuuint64_t ldims[2] = {8, (cuuint64_t)s->Nx * (cuuint64_t)s->Np / 8};
        cuuint64_t lstrides[1] = {64};
        cuuint32_t lbox[2] = {10, (cuuint32_t)s->xbox_h};
        r = enc(&s->xtmap[b], CU_TENSOR_MAP_DATA_TYPE_INT64, 2, s->f[b], ldims, lstrides, lbox, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(VLASOV_ECUDA, "cuTensorMapEncodeTiled (row lines) failed (%d)", (int)r);
    }
    return VLASOV_OK;
}

XShiftArgs xargs(vlasov_sim* s, const void* in, void* out, const LineParamsDev& p, bool reduce, bool kin,
                 const void* rec = nullptr)
{
    XShiftArgs a;
    a.rec = rec;
    a.fin = in;
    a.fout = out;
    a.Nx = s->Nx;
    a.Np = s->Np;
    a.pad = s->xpad;
    a.stages = s->xstages;
    a.n0 = p.n0;
    a.w = p.w;
    a.gd = p.gd;
    // Column sums of the output: every sweep but the hardware-FP64 one writes exact int64 partial
    // rows (one per CTA; 4096 atomics per CTA at the end of a sweep cost more than these 10 MB of
    // stores, and FP64 partial rows would be added by slow dependent FP64 additions); hardware FP64
    // adds exact sums atomically.
    const bool part64 = s->fx || s->emul || s->esz <= 4;
    const bool atomics = s->esz == 8 && !part64;
    a.colpart = nullptr;
    a.colacc = (reduce && atomics) ? s->colacc : nullptr;
    a.colpart64 = (reduce && part64 && !s->hmf_cta) ? reinterpret_cast<long long*>(s->colpart) : nullptr;
    a.ctapart = (reduce && s->hmf_cta) ? s->ctapart : nullptr;
    a.cos50 = s->cos50;
    a.sin50 = s->sin50;
    a.Ef = s->Ef;
    a.k_col = s->k_col;
    a.kinpart = kin ? s->kinpart : nullptr;
    a.kin128 = (kin && s->fx) ? s->kin128 : nullptr;
    a.pmin = s->pmin;
    a.dp = s->dp;
    a.err = s->err;
    a.beta = p.beta;
    a.gs_h = s->gs_h;
    return a;
}

PShiftArgs pargs(vlasov_sim* s, const void* in, void* out, const LineParamsDev& p)
{
    PShiftArgs a;
    a.fin = in;
    a.fout = out;
    a.Nx = s->Nx;
    a.Np = s->Np;
    a.n0 = p.n0;
    a.w = p.w;
    a.gd = p.gd;
    a.err = s->err;
    a.beta = p.beta;
    a.gs_h = s->gs_h;
    return a;
}

// Cells a chunk's window reaches past |n0| on a zero-outside row: 4 taps + (V - 1) alignment slack,
// V = 16 bytes / cell, at least the 8 the 8-byte and FP32 kernels always had.
int xhalo_extra(int esz) { return esz == 2 ? 12 : 8; }

// bf16 of a double, rounded to nearest even in one step (as the device's double-to-bf16
// conversion): the value is rounded to 8 significant bits (or to the 2^-133 grid of the smallest
// bf16), which an FP32 holds exactly, and the bf16 is that FP32's high half.
uint16_t bf16_bits(double x)
{
    float r = (float)x;   // zero, non-finite, or overflow: the FP32 value decides
    if (x != 0.0 && std::isfinite(x) && std::fabs(x) < 3.0e38) {
        int e = 0;
        std::frexp(x, &e);                                  // |x| in [2^(e-1), 2^e)
        const int ue = std::max(e - 8, -133);               // exponent of the last kept bit
        const double q = std::nearbyint(std::ldexp(x, -ue));   // default rounding: to nearest even
        r = (float)std::ldexp(q, ue);
    }
    uint32_t u;
    std::memcpy(&u, &r, 4);
    return (uint16_t)(u >> 16);
}

int ceil_log2(double v)
{
    int e = 0;
    const double m = std::frexp(v, &e);   // v = m 2^e, m in [0.5, 1)
    return m == 0.5 ? e - 1 : e;
}

void drop_graphs(vlasov_sim* s)
{
    auto drop = [](cudaGraphExec_t* g) {
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    };
    for (int b = 0; b < 2; ++b) {
        drop(&s->ghead[b]);
        drop(&s->gtail[b]);
        for (int L = 0; L < RUN_LEVELS; ++L) {
            drop(&s->grun[b][L]);
            drop(&s->gmid[b][L]);
        }
    }
}

// Fixed-point shifts of the reductions from the largest |f| (bound 2^Ef >= 4 max|f|).  Kernel
// arguments are captured in the step graphs, so a change of scale drops the graphs.
void update_scales(vlasov_sim* s, double maxabs)
{
    int e = 0;
    if (maxabs > 0 && std::isfinite(maxabs)) std::frexp(maxabs, &e);   // maxabs < 2^e
    const int Ef = e + 2;
    const int Lp = ceil_log2((double)s->Np), Lx = ceil_log2((double)s->Nx);
    const double pm = std::max(std::fabs(s->pmin), std::fabs(s->pmax));
    const int k_col = 61 - Ef - Lp;
    const int k_kin = 124 - ceil_log2(0.5 * pm * pm * (double)s->Np * (double)s->Nx) - Ef;
    int k_pot = 0;
    if (s->model == VLASOV_SHEET) k_pot = 124 - (3 * Lx + 2 * (Lp + Ef));
    if (s->model == VLASOV_RING) {
        const double vmax = 1.0 / std::sqrt(2.0 * s->eps);
        const double rmax = s->dp * (double)s->Np * std::ldexp(1.0, Ef);
        k_pot = 124 - ceil_log2((double)s->Nx * (double)s->Nx * s->dx * vmax * rmax * rmax);
    }
    if (!s->scales_set || Ef != s->Ef || k_col != s->k_col || k_kin != s->k_kin || k_pot != s->k_pot) drop_graphs(s);
    s->Ef = Ef;
    s->k_col = k_col;
    s->k_kin = k_kin;
    s->k_pot = k_pot;
    s->scales_set = true;
}

EmulArgs emargs(vlasov_sim* s, const LineParamsDev& p, const EmulParamsDev& e)
{
    EmulArgs a;
    a.Ef = s->Ef;
    a.n0 = p.n0;
    a.Wh = e.Wh;
    a.wl = e.wl;
    a.wf = e.wf;
    a.gd = static_cast<const double*>(p.gd);
    a.w64 = static_cast<const double*>(p.w);
    a.Whe = e.Whe;
    a.wle = e.wle;
    a.wfe = e.wfe;
    return a;
}

cudaError_t run_xshift(vlasov_sim* s, const XShiftArgs& a, const LineParamsDev& p, const EmulParamsDev& e, bool kin)
{
    if (s->gs) return launch_gs_xshift(s->esz, s->xper, kin, s->xgrid, a, s->st);   // partials: xgrid rows
    if (s->fx) return launch_xshift_fx(s->xper, kin, s->xgrid, s->xthreads, a, emargs(s, p, e), s->st);
    if (s->emul) return launch_xshift_e(s->xper, kin, s->xgrid, s->xthreads, a, emargs(s, p, e), s->st);
    return launch_xshift(s->esz, s->xper, kin, s->xgrid, s->xthreads, a, s->st);
}

// HMF with FP32-class storage: the p-shift forms its filters itself from the x-shift's per-CTA
// numbers (no filter launch).
bool hmf_filters_in_pshift(const vlasov_sim* s) { return s->hmf_cta && !s->fx && s->esz <= 4; }

cudaError_t run_pshift(vlasov_sim* s, const CUtensorMap* tmap, const PShiftArgs& a, const LineParamsDev& p,
                       const EmulParamsDev& e, const HmfFiltArgs* hf = nullptr)
{
    if (s->gs) return launch_gs_pshift(s->esz, s->pper, s->gspgrid, a, s->st);
    if (s->fx) return launch_pshift_fx(s->pper, s->pgrid, tmap, a, emargs(s, p, e), s->st);
    if (s->emul) return launch_pshift_e(s->pper, s->pgrid, tmap, a, emargs(s, p, e), s->st);
    return launch_pshift(s->esz, s->pper, s->pgrid, tmap, a, hf, s->st);
}

ColReduceArgs crargs(vlasov_sim* s, int B, bool kin, bool final_moments, bool from_acc = true, bool fused_m = false)
{
    ColReduceArgs a;
    const bool part64 = from_acc && (s->fx || s->emul || s->esz <= 4);
    a.colacc = (from_acc && s->esz == 8 && !part64) ? s->colacc : nullptr;
    a.colpart64 = part64 ? (fused_m ? s->colpart_m : reinterpret_cast<const long long*>(s->colpart)) : nullptr;
    a.colpart = s->colpart;
    a.B = B;
    a.kinpart = (kin && !s->fx) ? s->kinpart : nullptr;
    a.kin128 = (kin && s->fx) ? s->kin128 : nullptr;
    a.kin_frac = 51 + KIN_Q - s->Ef;
    a.Nx = s->Nx;
    a.k_col = s->k_col;
    a.k_kin = s->k_kin;
    a.k_pot = s->k_pot;
    a.dp = s->dp;
    a.dxdp = s->dx * s->dp;
    a.pot_scale = 2.0 * 3.14159265358979323846 * s->G * s->dx * s->dx * s->dx * s->dp * s->dp;
    a.cosfx = s->cosfx;
    a.sinfx = s->sinfx;
    a.rho = s->rho;
    a.colfx = s->colfx;
    a.Qd = s->Qd;
    a.blockpart = s->blockpart;
    a.ticket = &s->tickets[0];
    a.sc = s->sc;
    a.model = s->model;
    a.final_moments = final_moments ? 1 : 0;
    a.hist = s->hist;
    a.step = s->dstep;
    a.dt = s->dt;
    return a;
}

RingArgs ringargs(vlasov_sim* s, bool final_moments)
{
    RingArgs a;
    a.N = s->Nx;
    a.dx = s->dx;
    a.rho = s->rho;
    a.dV = s->ringdV;
    a.V = s->ringV;
    a.F = s->F;
    a.blockpart = s->ringpart;
    a.k_pot = s->k_pot;
    a.pot_scale = 0.5 * s->dx;
    a.ticket = &s->tickets[1];
    a.sc = s->sc;
    a.final_moments = final_moments ? 1 : 0;
    a.hist = s->hist;
    a.step = s->dstep;
    a.dt = s->dt;
    a.colfx = s->colfx;
    a.Kq = s->ringKq;
    a.Vq = s->ringVq;
    a.k_col = s->k_col;
    a.sK = s->ring_sK;
    a.sV = s->ring_sV;
    a.dp = s->dp;
    a.ksplit = s->ring_ksplit;
    a.gpart = s->ring_gpart;
    a.gticket = s->ring_gticket;
    a.upart = s->ring_upart;
    const bool f64 = s->ring_method != RING_M_FFT32;
    const size_t e2 = f64 ? 16 : 8;
    unsigned char* t = static_cast<unsigned char*>(f64 ? s->ring_fft64 : s->ring_fft32);
    a.khat = t;
    a.vhat = t ? t + e2 * (size_t)s->Nx : nullptr;
    a.twid = t ? t + 2 * e2 * (size_t)s->Nx : nullptr;
    a.tcK = s->ring_tcK;
    a.tcV = s->ring_tcV;
    a.tcacc = s->ring_tcacc;
    a.tcticket = s->ring_tcticket;
    // |partial result| <= N max|table| max rho, max rho <= dp Np 2^Ef: N/128 such sums stay below 2^62
    {
        const double bound = (double)s->Nx * s->ring_tcmax[final_moments ? 1 : 0] * s->dp * (double)s->Np *
                             std::ldexp(1.0, s->Ef);
        a.tcq = bound > 0 ? 57 - ceil_log2(bound) : 0;
        a.tcq = std::max(-100, std::min(100, a.tcq));
    }
    a.err = s->err;
    return a;
}

PParamsArgs pparams_args(const vlasov_sim* s, double* Fout);

// Ring force with the fixed-point sums: its launch also writes the p-shift filters of the columns
// (one launch fewer per step).
bool ring_filters_in_force(const vlasov_sim* s) { return s->model == VLASOV_RING && s->ring_method == RING_M_FIXED; }

// The ring force (final_moments = false) or potential and moment record (true) by the handle's
// method; one launch either way (with_filters: the force launch of the fixed-point method also
// writes the p-shift filters).
cudaError_t run_ring(vlasov_sim* s, bool final_moments, bool with_filters = false)
{
    RingArgs a = ringargs(s, final_moments);
    if (with_filters && !final_moments && ring_filters_in_force(s)) {
        a.pp = pparams_args(s, nullptr);
        a.pp_on = 1;
        a.pp_fixed = s->msz == 8 ? 1 : 0;
    }
    switch (s->ring_method) {
    case RING_M_FIXED: return launch_ring_fixed(a, s->st);
    case RING_M_FFT64: return launch_ring_fft(true, a, s->st);
    case RING_M_FFT32: return launch_ring_fft(false, a, s->st);
    case RING_M_TENSOR: return launch_ring_tc(a, s->st);
    default: return launch_ring(s->msz, a, s->st);
    }
}

PParamsArgs pparams_args(const vlasov_sim* s, double* Fout)
{
    PParamsArgs a;
    a.Nx = s->Nx;
    a.model = s->model;
    a.sc = s->sc;
    a.costab = s->costab;
    a.sintab = s->sintab;
    a.Fin = s->model == VLASOV_SHEET ? s->Qd : s->F;
    a.Fscale = -2.0 * 3.14159265358979323846 * s->G * s->dx * s->dp;
    a.cp = s->dt / s->dp;
    a.n0 = s->pp.n0;
    a.w = s->pp.w;
    a.gd = s->pp.gd;
    a.Fout = Fout;
    a.Wh = (s->emul || s->fx) ? s->pe.Wh : nullptr;
    a.wl = (s->emul || s->fx) ? s->pe.wl : nullptr;
    a.wf = (s->emul || s->fx) ? s->pe.wf : nullptr;
    a.Whe = (s->emul || s->fx) ? s->pe.Whe : nullptr;
    a.wle = (s->emul || s->fx) ? s->pe.wle : nullptr;
    a.wfe = (s->emul || s->fx) ? s->pe.wfe : nullptr;
    a.beta = s->gs ? s->pp.beta : nullptr;
    return a;
}

int launch_pparams_only(vlasov_sim* s, double* Fout, bool from_cta = false, int ctas = 0)
{
    PParamsArgs a = pparams_args(s, Fout);
    if (from_cta) {
        a.ctapart = s->ctapart;
        a.ctas = ctas > 0 ? ctas : s->xgrid;
        a.Ef = s->Ef;
        a.dxdp = s->dx * s->dp;
        CU_TRY(launch_pparams_hmf_cta(s->msz, a, s->st));
        return VLASOV_OK;
    }
    CU_TRY(launch_pparams(s->msz, a, s->st));
    return VLASOV_OK;
}

int launch_force_params(vlasov_sim* s, double* Fout)
{
    if (s->model == VLASOV_RING) CU_TRY(run_ring(s, false));
    return launch_pparams_only(s, Fout);
}

// Optional per-launch event marks (vlasov_step_timed): ev[k] is recorded before launch k and
// ev[k+1] after it.
struct Marks {
    cudaEvent_t* ev = nullptr;
    int k = 0;
};

int mark(vlasov_sim* s, Marks* m)
{
    if (m && m->ev) CU_TRY(cudaEventRecord(m->ev[m->k++], s->st));
    return VLASOV_OK;
}

#define MARK()                    \
    do {                          \
        int rc_ = mark(s, marks); \
        if (rc_) return rc_;      \
    } while (0)

// Step 1 from buffer c into c^1: f^(I) = f(x - p dt/2, p), with the density partials of f^(I).
int enq_x1(vlasov_sim* s, int c, Marks* marks)
{
    CU_TRY(run_xshift(s, xargs(s, s->f[c], s->f[c ^ 1], s->xp, true, false, s->xrec), s->xp, s->xe, false));
    MARK();
    return VLASOV_OK;
}

// Steps 2-3: rho, F^(I) and the p-shift filters from the density partials of `ctas` CTAs, then the
// p-shift f^(II) = f^(I)(x, p - F dt) from buffer c^1 into c.
int enq_force_p(vlasov_sim* s, int c, int ctas, Marks* marks)
{
    const int o = c ^ 1;
    HmfFiltArgs hf{};
    if (hmf_filters_in_pshift(s)) {   // Mx, My from the per-CTA partials, inside the p-shift
        hf.ctapart = s->ctapart;
        hf.ctas = ctas > 0 ? ctas : s->xgrid;
        hf.Ef = s->Ef;
        hf.on = 1;
        hf.dxdp = s->dx * s->dp;
        hf.cp = s->dt / s->dp;
        hf.costab = s->costab;
        hf.sintab = s->sintab;
    } else if (s->hmf_cta) {
        int rc = launch_pparams_only(s, nullptr, true, ctas);   // Mx, My from the per-CTA partials
        if (rc) return rc;
        MARK();
    } else {
        CU_TRY(launch_colreduce(crargs(s, ctas, false, false), s->crgrid, s->st));
        MARK();
        if (s->model == VLASOV_RING) {
            CU_TRY(run_ring(s, false, true));
            MARK();
        }
        if (!ring_filters_in_force(s)) {
            int rc = launch_pparams_only(s, nullptr);
            if (rc) return rc;
            MARK();
        }
    }
    CU_TRY(run_pshift(s, &s->tmap[o], pargs(s, s->f[o], s->f[c], s->pp), s->pp, s->pe, hf.on ? &hf : nullptr));
    MARK();
    return VLASOV_OK;
}

// The moment record of the state just written, from the partials of `ctas` CTAs (those of the
// fused launch's first pass when fused_m).
int enq_moments(vlasov_sim* s, int ctas, bool fused_m, Marks* marks)
{
    if (s->hmf_cta) {
        ColReduceArgs c = crargs(s, ctas, true, true);
        c.ctapart = fused_m ? s->ctapart_m : s->ctapart;
        c.Ef = s->Ef;
        CU_TRY(launch_colreduce_cta(c, s->st));
    } else {
        CU_TRY(launch_colreduce(crargs(s, ctas, true, true, true, fused_m), s->crgrid, s->st));
    }
    MARK();
    if (s->model == VLASOV_RING) {
        CU_TRY(run_ring(s, true));
        MARK();
    }
    return VLASOV_OK;
}

// Step 4 from buffer c into c^1: f(t+dt) = f^(II)(x - p dt/2, p), then the moments.
int enq_x2(vlasov_sim* s, int c, Marks* marks)
{
    CU_TRY(run_xshift(s, xargs(s, s->f[c], s->f[c ^ 1], s->xp, true, true, s->xrec), s->xp, s->xe, true));
    MARK();
    return enq_moments(s, s->xgrid, false, marks);
}

// Step 4 of this step and step 1 of the next in one launch, buffer c into c^1; then the moments of
// the state between them (the end of this step).
int enq_xx(vlasov_sim* s, int c, Marks* marks)
{
    XShiftArgs a = xargs(s, s->f[c], nullptr, s->xp, true, true, s->xrec);
    a.stages = s->xxstages;
    a.box_h = s->xbox_h;
    a.ctapart = s->hmf_cta ? s->ctapart_m : nullptr;
    a.colpart64 = s->hmf_cta ? nullptr : s->colpart_m;
    XShiftArgs b = xargs(s, nullptr, s->f[c ^ 1], s->xp, true, false, s->xrec);
    if (s->fx) CU_TRY(launch_xxshift_fx(s->xper, s->xxgrid, &s->xtmap[c], a, b, emargs(s, s->xp, s->xe), s->st));
    else CU_TRY(launch_xxshift(s->esz, s->xper, s->xxgrid, a, b, s->st));
    MARK();
    return enq_moments(s, s->xxgrid, true, marks);
}

// Fused ring steps with the exact fixed-point convolutions: the two column reductions (end of this
// step, f^(I) of the next) in one launch and the two convolutions (the end state's potential and
// record, the next step's force) in one launch.
bool ring_merged(const vlasov_sim* s)
{
    return s->model == VLASOV_RING && s->fuse && s->ring_method == RING_M_FIXED && s->ring_gpart_m != nullptr &&
           s->colpart_m != nullptr;
}

int enq_mid_ring_merged(vlasov_sim* s, int c, Marks* marks)
{
    XShiftArgs a = xargs(s, s->f[c], nullptr, s->xp, true, true, s->xrec);
    a.stages = s->xxstages;
    a.box_h = s->xbox_h;
    a.ctapart = nullptr;
    a.colpart64 = s->colpart_m;
    XShiftArgs b = xargs(s, nullptr, s->f[c ^ 1], s->xp, true, false, s->xrec);
    if (s->fx) CU_TRY(launch_xxshift_fx(s->xper, s->xxgrid, &s->xtmap[c], a, b, emargs(s, s->xp, s->xe), s->st));
    else CU_TRY(launch_xxshift(s->esz, s->xper, s->xxgrid, a, b, s->st));
    MARK();
    ColReduceArgs cm = crargs(s, s->xxgrid, true, true, true, true);   // end of this step: moments
    cm.rho = s->rho_m;
    cm.colfx = s->colfx_m;
    cm.sc = s->sc_m;
    cm.blockpart = s->blockpart_m;
    cm.ticket = &s->tickets[2];
    ColReduceArgs cd = crargs(s, s->xxgrid, false, false);             // f^(I) of the next step: density
    if (!cm.colpart64 || !cd.colpart64 || cm.colacc || cd.colacc) return fail(VLASOV_ECUDA, "merged reduction needs partial rows");
    CU_TRY(launch_colreduce_p64_dual(cm, cd, s->st));
    MARK();
    RingArgs rf = ringargs(s, false);   // with the p-shift filters of its columns
    rf.pp = pparams_args(s, nullptr);
    rf.pp_on = 1;
    rf.pp_fixed = s->msz == 8 ? 1 : 0;
    RingArgs rp = ringargs(s, true);
    rp.colfx = s->colfx_m;
    rp.rho = s->rho_m;
    rp.sc = s->sc_m;
    rp.gpart = s->ring_gpart_m;
    rp.gticket = s->ring_gticket_m;
    CU_TRY(launch_ring_fixed_dual(rf, rp, s->st));
    MARK();
    const int o = c ^ 1;
    CU_TRY(run_pshift(s, &s->tmap[o], pargs(s, s->f[o], s->f[c], s->pp), s->pp, s->pe));
    MARK();
    return VLASOV_OK;
}

// One whole Strang step from buffer c (result in c^1).
int enqueue_step(vlasov_sim* s, int c, Marks* marks = nullptr)
{
    MARK();
    int rc = enq_x1(s, c, marks);
    if (!rc) rc = enq_force_p(s, c, s->xgrid, marks);
    if (!rc) rc = enq_x2(s, c, marks);
    return rc;
}

// Pieces of a run of fused steps from buffer c (result in c^1): head, mid between steps, tail.
enum Piece { P_HEAD, P_MID, P_TAIL };
int enqueue_piece(vlasov_sim* s, int c, Piece k, Marks* marks = nullptr)
{
    MARK();
    if (k == P_HEAD) {
        int rc = enq_x1(s, c, marks);
        return rc ? rc : enq_force_p(s, c, s->xgrid, marks);
    }
    if (k == P_MID) {
        if (ring_merged(s)) return enq_mid_ring_merged(s, c, marks);
        int rc = enq_xx(s, c, marks);
        return rc ? rc : enq_force_p(s, c, s->xxgrid, marks);
    }
    return enq_x2(s, c, marks);
}
#undef MARK

template <typename F>
int capture(vlasov_sim* s, cudaGraphExec_t* out, F&& enqueue)
{
    if (*out) return VLASOV_OK;
    cudaGraph_t g = nullptr;
    CU_TRY(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue();
    const cudaError_t e = cudaStreamEndCapture(s->st, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(VLASOV_ECUDA, "stream capture: %s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return fail(VLASOV_ECUDA, "graph instantiate: %s", cudaGetErrorString(e2));
    return VLASOV_OK;
}

// Graphs of 2^L whole steps from buffer c (L = 0: one step, ending on c^1; L > 0 ends on c).  All
// levels are captured at the first call (for both starting buffers), so that no capture falls
// between two launches of a later call.
int build_graphs(vlasov_sim* s, int c)
{
    int rc = VLASOV_OK;
    for (int L = 0; L < RUN_LEVELS && !rc; ++L)
        rc = capture(s, &s->grun[c][L], [&] {
            int r = VLASOV_OK;
            for (int k = 0; k < (1 << L) && !r; ++k) r = enqueue_step(s, c ^ (k & 1));
            return r;
        });
    return rc;
}

// Head, tail, and runs of 2^L middle pieces (each from buffer c back into c).
int build_fused_graphs(vlasov_sim* s, int c)
{
    int rc = capture(s, &s->ghead[c], [&] { return enqueue_piece(s, c, P_HEAD); });
    if (!rc) rc = capture(s, &s->gtail[c], [&] { return enqueue_piece(s, c, P_TAIL); });
    for (int L = 0; L < RUN_LEVELS && !rc; ++L)
        rc = capture(s, &s->gmid[c][L], [&] {
            int r = VLASOV_OK;
            for (int k = 0; k < (1 << L) && !r; ++k) r = enqueue_piece(s, c, P_MID);
            return r;
        });
    return rc;
}

// Launches per piece: x-shift 1; force (reductions, filters); p-shift; x-shift 4 or the fused
// x-shifts; moments.
int force_launches(const vlasov_sim* s)
{
    if (hmf_filters_in_pshift(s)) return 0;
    if (s->hmf_cta) return 1;
    if (s->model == VLASOV_RING) return ring_filters_in_force(s) ? 2 : 3;
    return 2;
}
int moment_launches(const vlasov_sim* s) { return s->model == VLASOV_RING ? 2 : 1; }

int check_dev_err(vlasov_sim* s)
{
    int h = 0;
    CU_TRY(cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    CU_TRY(cudaStreamSynchronize(s->st));
    if (h != DEV_ERR_NONE) {
        cudaMemsetAsync(s->err, 0, sizeof(int), s->st);
        if (h == DEV_ERR_RANGE)
            return fail(VLASOV_ERANGE, "|f| outgrew the fixed-point range (4x the largest uploaded |f|); "
                                       "results since the last check are void");
        return fail(VLASOV_ETIMEOUT, "a bounded device wait expired (code %d); results since the last check are void", h);
    }
    return VLASOV_OK;
}

}  // namespace

namespace vl {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace vl

extern "C" {

const char* vlasov_last_error(void) { return g_err.c_str(); }

void vlasov_destroy(vlasov_sim* s)
{
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    drop_graphs(s);
    for (int b = 0; b < 2; ++b) cudaFree(s->f[b]);
    free_params(s->xp);
    free_params(s->pp);
    free_params(s->sp);
    free_emul(s->xe);
    free_emul(s->pe);
    free_emul(s->se);
    void* bufs[] = {s->colpart, s->colacc, s->kinpart, s->rho, s->colfx, s->Qd, s->F, s->Fout, s->blockpart, s->ringpart,
                    s->tickets, s->maxbits, s->sc, s->costab, s->sintab, s->cosfx, s->sinfx, s->ringdV, s->ringV,
                    s->hist, s->dstep, s->err, s->xrec, s->srec, s->cos50, s->sin50, s->ctapart,
                    s->ctapart_m, s->colpart_m, s->kin128, s->gs_h, s->ringKq, s->ringVq, s->ring_gpart,
                    s->ring_gticket, s->ring_upart, s->ring_fft64, s->ring_fft32, s->ring_tcK, s->ring_tcV,
                    s->ring_tcacc, s->ring_tcticket, s->rho_m, s->colfx_m, s->sc_m, s->blockpart_m, s->ring_gpart_m,
                    s->ring_gticket_m};
    for (void* p : bufs) cudaFree(p);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    delete s;
}

int vlasov_create(int model, int Nx, int Np, const vlasov_domain* d, double dt, vlasov_sim** out)
{
    if (!out) return fail(VLASOV_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d) return fail(VLASOV_EINVAL, "domain is NULL");
    if (model < VLASOV_HMF || model > VLASOV_FREE) return fail(VLASOV_EINVAL, "unknown model %d", model);
    if (d->precision != VLASOV_F64 && d->precision != VLASOV_F32 && d->precision != VLASOV_F64_NATIVE &&
        d->precision != VLASOV_FX64 && d->precision != VLASOV_BF16)
        return fail(VLASOV_EINVAL, "unknown precision %d", d->precision);
    const int esz = d->precision == VLASOV_F32 ? 4 : d->precision == VLASOV_BF16 ? 2 : 8;
    if (Nx < 16 || Np < 16 || Nx % ALIGN_N || Np % ALIGN_N)
        return fail(VLASOV_EINVAL, "Nx=%d, Np=%d: both must be multiples of %d and >= 16", Nx, Np, ALIGN_N);
    // x rows are staged whole: 256-thread CTAs cover 8192 FP32 or BF16 cells and 4096 8-byte cells;
    // longer 8-byte rows (up to 8192) run on 512-thread CTAs
    const int xs_threads = (esz == 8 && Nx > xshift_max_cols(esz, XS_THREADS_MIN)) ? XS_THREADS_MAX : XS_THREADS_MIN;
    if (Nx > xshift_max_cols(esz, xs_threads))
        return fail(VLASOV_EINVAL, "Nx=%d exceeds %d for this precision", Nx, xshift_max_cols(esz, xs_threads));
    if (!(dt > 0) || !std::isfinite(dt)) return fail(VLASOV_EINVAL, "dt must be > 0");
    if (!(d->xmax > d->xmin) || !(d->pmax > d->pmin)) return fail(VLASOV_EINVAL, "empty domain");
    if (model == VLASOV_RING && !(d->eps > 0)) return fail(VLASOV_EINVAL, "ring model needs eps > 0");
    if (std::max(std::fabs(d->pmin), std::fabs(d->pmax)) >= 2896.0)
        return fail(VLASOV_EINVAL, "|p| must stay below 2896 (fixed-point kinetic weights)");

    vlasov_sim* s = new vlasov_sim();
    s->model = model;
    s->Nx = Nx;
    s->Np = Np;
    s->prec = d->precision;
    s->esz = esz;
    s->msz = esz == 8 ? 8 : 4;
    s->emul = d->precision == VLASOV_F64;
    s->fx = d->precision == VLASOV_FX64;
    s->xper = d->x_periodic != 0;
    s->pper = d->p_periodic != 0;
    s->xmin = d->xmin;
    s->xmax = d->xmax;
    s->pmin = d->pmin;
    s->pmax = d->pmax;
    s->dx = (d->xmax - d->xmin) / (double)Nx;
    s->dp = (d->pmax - d->pmin) / (double)Np;
    s->dt = dt;
    s->eps = d->eps;
    s->G = d->G;

    auto bail = [&](int rc) {
        vlasov_destroy(s);
        return rc;
    };
#define TRY(expr)                 \
    do {                          \
        int rc_ = (expr);         \
        if (rc_) return bail(rc_); \
    } while (0)
#define CTRY(expr)                                                                                       \
    do {                                                                                                 \
        cudaError_t e_ = (expr);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? VLASOV_ENOMEM : VLASOV_ECUDA, "%s: %s", #expr, \
                             cudaGetErrorString(e_)));                                                   \
    } while (0)

    CTRY(cudaGetDevice(&s->dev));
    CTRY(cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->dev));
    int max_optin = 0;
    CTRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->dev));
    s->max_smem = max_optin;
    if (d->stream) {
        s->st = static_cast<cudaStream_t>(d->stream);
    } else {
        CTRY(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
        s->own_stream = true;
    }
    CTRY(set_kernel_attributes(max_optin - 1024));
    CTRY(set_kernel_attributes_e(max_optin - 1024));
    CTRY(set_kernel_attributes_fx(max_optin - 1024));
    CTRY(set_ring_attributes(max_optin - 1024));
    CTRY(set_ringfx_attributes(max_optin - 1024));

    const size_t cells = (size_t)Nx * (size_t)Np;
    for (int b = 0; b < 2; ++b) {
        CTRY(cudaMalloc(&s->f[b], cells * esz));
        CTRY(cudaMemsetAsync(s->f[b], 0, cells * esz, s->st));
    }

    // x-shift filters: row j moves by s_j = p_j * ((dt/2)/dx) cells.
    std::vector<double> srow(Np);
    {
        const double cx = (0.5 * dt) / s->dx;
        for (int j = 0; j < Np; ++j) {
            const double p = s->pmin + (double)j * s->dp;
            srow[j] = p * cx;
        }
    }
    TRY(alloc_params(s->xp, Np, s->msz));
    TRY(alloc_params(s->pp, Nx, s->msz));
    TRY(alloc_params(s->sp, std::max(Nx, Np), s->msz));
    if (s->emul || s->fx) {
        TRY(alloc_emul(s->xe, Np));
        TRY(alloc_emul(s->pe, Nx));
        TRY(alloc_emul(s->se, std::max(Nx, Np)));
    }
    int max_n0 = 0;
    CTRY(cudaMalloc(&s->xrec, (size_t)XREC_BYTES * Np));
    CTRY(cudaMalloc(&s->srec, (size_t)XREC_BYTES * std::max(Nx, Np)));
    TRY(upload_params(s, s->xp, srow.data(), Np, &max_n0, &s->xe, s->xrec, true));

    // x-shift launch shape: whole rows staged per CTA.
    s->xthreads = xs_threads;
    // zero halo of non-periodic rows: the window of a chunk reaches |n0| + 4 + (V - 1) cells past the
    // row, V = 16 bytes / cell (8 for BF16 storage)
    s->xpad = s->xper ? 16 : ((max_n0 + xhalo_extra(esz) + 15) / 16) * 16;
    const size_t row_bytes = (size_t)(Nx + 2 * s->xpad) * esz + XREC_BYTES;
    const size_t smem_budget = (size_t)max_optin - 2048;
    s->xstages = (int)std::min<size_t>(4, (smem_budget - 256) / row_bytes);
    if (s->emul || s->fx) {
        // two CTAs per SM: up to three rows in flight each
        const size_t half = (size_t)max_optin / 2 - 2048;
        const int st2 = (int)std::min<size_t>(3, (half - 256) / row_bytes);
        if (st2 >= 2) s->xstages = st2;
    }
    if (s->xstages < 1) return bail(fail(VLASOV_EINVAL, "a row of Nx=%d (+%d halo) does not fit shared memory", Nx, s->xpad));
    int occ = 0;
    if (s->fx) CTRY(xshift_fx_occupancy(s->xper, s->xthreads, xshift_smem_bytes(Nx, s->xpad, s->xstages, esz), &occ));
    else if (s->emul) CTRY(xshift_e_occupancy(s->xper, s->xthreads, xshift_smem_bytes(Nx, s->xpad, s->xstages, esz), &occ));
    else CTRY(xshift_occupancy(esz, s->xper, s->xthreads, xshift_smem_bytes(Nx, s->xpad, s->xstages, esz), &occ));
    occ = std::max(occ, 1);
    s->xgrid = std::min(Np, s->nsm * occ);

    int pocc = 0;
    if (s->fx) CTRY(pshift_fx_occupancy(&pocc));
    else if (s->emul) CTRY(pshift_e_occupancy(&pocc));
    else CTRY(pshift_occupancy(esz, &pocc));
    pocc = std::max(pocc, 1);
    const int pth = s->fx ? pshift_fx_tile_rows() : PS_TH;
    const int ptiles = ((Nx + PS_TW - 1) / PS_TW) * ((Np + pth - 1) / pth);
    s->pgrid = std::min(ptiles, s->nsm * pocc);
    s->crgrid = (Nx + 31) / 32;

    // Fused x-shifts: S stages of whole rows and two intermediate rows in one CTA's shared memory;
    // rows arrive in TMA boxes of xbox_h 8-element lines (a multiple of 8 lines dividing Nx / 8,
    // so that every box lands 128-byte aligned)
    for (int d = 32; d >= 1 && Nx % 64 == 0; --d)
        if ((Nx / 64) % d == 0) {
            s->xbox_h = 8 * d;
            break;
        }
    if (s->fx && Nx <= XF_FUSED_MAX_NX && s->xbox_h > 0) {
        const size_t row = (size_t)std::max(xxshift_fx_row_bytes(Nx, s->xpad, true), xxshift_fx_row_bytes(Nx, s->xpad, false));
        const size_t budget = (size_t)max_optin - 2048;
        const int st = budget > 256 + 2 * row ? (int)std::min<size_t>(3, (budget - 256 - 2 * row) / (row + XREC_BYTES)) : 0;
        if (st >= 2) {
            int xocc = 0;
            CTRY(xxshift_fx_occupancy(s->xper, Nx, xxshift_fx_smem_bytes(Nx, s->xpad, st), &xocc));
            if (xocc >= 1) {
                s->xxstages = st;
                s->xxgrid = std::min(Np, s->nsm * xocc);
                s->fuse_ok = true;
                // on by default for periodic rows; on zero-outside rows (sheet) the separate
                // x-shifts measured faster (each fused row barrier waits for the rows' edge outputs)
                s->fuse = s->xper;
            }
        }
    } else if (!s->fx && !s->emul && esz <= 4 && Nx <= XXS_MAX_NX) {
        // FP32-class storage: whole padded rows by bulk copies, as the separate x-shift stages them;
        // two CTAs per SM (a CTA waits at a barrier every row) with up to three rows in flight each
        const size_t row = (size_t)(Nx + 2 * s->xpad) * esz;
        auto stages_in = [&](size_t budget) {
            return budget > 256 + 2 * row ? (int)std::min<size_t>(3, (budget - 256 - 2 * row) / (row + XREC_BYTES)) : 0;
        };
        int st = stages_in((size_t)max_optin / XXS_CTAS_PER_SM - 2048);
        if (st < 2) st = stages_in((size_t)max_optin - 2048);
        if (st >= 2) {
            int xocc = 0;
            CTRY(xxshift_occupancy(esz, s->xper, xxshift_smem_bytes(Nx, s->xpad, st, esz), &xocc));
            if (xocc >= 1) {
                s->xxstages = st;
                s->xxgrid = std::min(Np, s->nsm * xocc);
                s->fuse_ok = true;
                // on by default for FP32 and BF16 storage (measured faster: HMF 4096^2 BF16
                // 0.0950 -> 0.0875 ms per step once the row loop does no FP64 arithmetic)
                s->fuse = true;
            }
        }
    }
    s->nctas = std::max(s->xgrid, s->xxgrid);

    // per-CTA column partial rows; also the scratch of vlasov_casimirs (2 * CAS_BLOCKS + 2 doubles)
    CTRY(cudaMalloc(&s->colpart, sizeof(double) * std::max((size_t)s->nctas * Nx, (size_t)2 * CAS_BLOCKS + 2)));
    CTRY(cudaMalloc(&s->ctapart, 48 * (size_t)s->nctas));
    CTRY(cudaMalloc(&s->kin128, 16 * (size_t)s->nctas));
    if (s->fuse_ok) {
        CTRY(cudaMalloc(&s->ctapart_m, 48 * (size_t)s->nctas));
        CTRY(cudaMalloc(&s->colpart_m, sizeof(long long) * (size_t)s->nctas * Nx));
    }
    // HMF needs no per-column density: the x-shifts hand over three exact numbers per CTA (bounded
    // in int128 while Nx * Np <= 2^24).
    s->hmf_cta = (s->fx || esz <= 4) && model == VLASOV_HMF && (double)Nx * (double)Np <= 16777216.0;
    s->hmf_cta_fd = s->hmf_cta;
    CTRY(cudaMalloc(&s->colacc, sizeof(unsigned long long) * (size_t)Nx));
    CTRY(cudaMemsetAsync(s->colacc, 0, sizeof(unsigned long long) * (size_t)Nx, s->st));
    CTRY(cudaMalloc(&s->kinpart, sizeof(double) * (size_t)s->nctas));
    CTRY(cudaMalloc(&s->rho, sizeof(double) * Nx));
    CTRY(cudaMalloc(&s->colfx, sizeof(long long) * Nx));
    CTRY(cudaMalloc(&s->Qd, sizeof(double) * Nx));
    CTRY(cudaMemsetAsync(s->Qd, 0, sizeof(double) * Nx, s->st));
    CTRY(cudaMalloc(&s->F, sizeof(double) * Nx));
    CTRY(cudaMemsetAsync(s->F, 0, sizeof(double) * Nx, s->st));
    CTRY(cudaMalloc(&s->Fout, sizeof(double) * Nx));
    CTRY(cudaMalloc(&s->blockpart, 16 * 3 * (size_t)s->crgrid));
    CTRY(cudaMalloc(&s->ringpart, 16 * (size_t)ring_blocks(Nx)));
    CTRY(cudaMalloc(&s->maxbits, sizeof(unsigned long long)));
    CTRY(cudaMalloc(&s->tickets, sizeof(unsigned int) * 4));
    CTRY(cudaMemsetAsync(s->tickets, 0, sizeof(unsigned int) * 4, s->st));
    CTRY(cudaMalloc(&s->sc, sizeof(Scalars)));
    CTRY(cudaMemsetAsync(s->sc, 0, sizeof(Scalars), s->st));
    CTRY(cudaMalloc(&s->hist, sizeof(MomentRec) * HIST_CAP));
    CTRY(cudaMalloc(&s->dstep, sizeof(long long)));
    CTRY(cudaMemsetAsync(s->dstep, 0, sizeof(long long), s->st));
    CTRY(cudaMalloc(&s->err, sizeof(int)));
    CTRY(cudaMemsetAsync(s->err, 0, sizeof(int), s->st));

    // Tables on the x nodes: cos/sin for HMF (Eq. hmfmeanforce, mxmydef); ring kernel V, V'.
    {
        std::vector<double> c(Nx), sn(Nx), dV(Nx), V(Nx);
        std::vector<long long> cfx(Nx), sfx(Nx), c50(Nx), s50(Nx);
        for (int i = 0; i < Nx; ++i) {
            const double th = s->xmin + (double)i * s->dx;
            c[i] = std::cos(th);
            sn[i] = std::sin(th);
            cfx[i] = std::llround(std::ldexp(c[i], 62));
            sfx[i] = std::llround(std::ldexp(sn[i], 62));
            c50[i] = std::llround(std::ldexp(c[i], 50));
            s50[i] = std::llround(std::ldexp(sn[i], 50));
            const double u = (double)i * s->dx;
            if (model == VLASOV_RING) {
                const double q = 1.0 - std::cos(u) + s->eps;
                dV[i] = std::sin(u) / (2.0 * std::sqrt(2.0) * q * std::sqrt(q));   // V'(u), Eq. (ringpot)
                V[i] = -1.0 / (std::sqrt(2.0) * std::sqrt(q));                      // V(u)
            } else {
                dV[i] = V[i] = 0.0;
            }
        }
        double h[GS_HTAPS];
        gs_filter_h(h);
        CTRY(cudaMalloc(&s->gs_h, sizeof h));
        CTRY(cudaMemcpy(s->gs_h, h, sizeof h, cudaMemcpyHostToDevice));
        CTRY(cudaMalloc(&s->costab, sizeof(double) * Nx));
        CTRY(cudaMalloc(&s->sintab, sizeof(double) * Nx));
        CTRY(cudaMalloc(&s->cosfx, sizeof(long long) * Nx));
        CTRY(cudaMalloc(&s->sinfx, sizeof(long long) * Nx));
        CTRY(cudaMalloc(&s->cos50, sizeof(long long) * Nx));
        CTRY(cudaMalloc(&s->sin50, sizeof(long long) * Nx));
        CTRY(cudaMalloc(&s->ringdV, (size_t)s->msz * Nx));
        CTRY(cudaMalloc(&s->ringV, (size_t)s->msz * Nx));
        CTRY(cudaMemcpyAsync(s->costab, c.data(), sizeof(double) * Nx, cudaMemcpyHostToDevice, s->st));
        CTRY(cudaMemcpyAsync(s->sintab, sn.data(), sizeof(double) * Nx, cudaMemcpyHostToDevice, s->st));
        CTRY(cudaMemcpyAsync(s->cosfx, cfx.data(), sizeof(long long) * Nx, cudaMemcpyHostToDevice, s->st));
        CTRY(cudaMemcpyAsync(s->sinfx, sfx.data(), sizeof(long long) * Nx, cudaMemcpyHostToDevice, s->st));
        CTRY(cudaMemcpyAsync(s->cos50, c50.data(), sizeof(long long) * Nx, cudaMemcpyHostToDevice, s->st));
        CTRY(cudaMemcpyAsync(s->sin50, s50.data(), sizeof(long long) * Nx, cudaMemcpyHostToDevice, s->st));
        if (s->msz == 8) {
            CTRY(cudaMemcpyAsync(s->ringdV, dV.data(), sizeof(double) * Nx, cudaMemcpyHostToDevice, s->st));
            CTRY(cudaMemcpyAsync(s->ringV, V.data(), sizeof(double) * Nx, cudaMemcpyHostToDevice, s->st));
            CTRY(cudaStreamSynchronize(s->st));
        } else {
            std::vector<float> dVf(dV.begin(), dV.end()), Vf(V.begin(), V.end());
            CTRY(cudaMemcpyAsync(s->ringdV, dVf.data(), sizeof(float) * Nx, cudaMemcpyHostToDevice, s->st));
            CTRY(cudaMemcpyAsync(s->ringV, Vf.data(), sizeof(float) * Nx, cudaMemcpyHostToDevice, s->st));
            CTRY(cudaStreamSynchronize(s->st));
        }
        if (model == VLASOV_RING) {
            // tables and scratch of the exact fixed-point method
            std::vector<long long> Kq(Nx), Vq(Nx);
            ring_fixed_tables(Nx, s->dx, s->eps, Kq.data(), Vq.data(), &s->ring_sK, &s->ring_sV);
            s->ring_ksplit = ringfx_ksplit(Nx, s->nsm);
            const int ngrp = (Nx + 31) / 32;
            CTRY(cudaMalloc(&s->ringKq, sizeof(long long) * Nx));
            CTRY(cudaMalloc(&s->ringVq, sizeof(long long) * Nx));
            CTRY(cudaMalloc(&s->ring_gpart, 16 * (size_t)s->ring_ksplit * Nx));
            CTRY(cudaMalloc(&s->ring_gticket, sizeof(unsigned int) * ngrp));
            CTRY(cudaMemsetAsync(s->ring_gticket, 0, sizeof(unsigned int) * ngrp, s->st));
            CTRY(cudaMalloc(&s->ring_gpart_m, 16 * (size_t)s->ring_ksplit * Nx));
            CTRY(cudaMalloc(&s->ring_gticket_m, sizeof(unsigned int) * ngrp));
            CTRY(cudaMemsetAsync(s->ring_gticket_m, 0, sizeof(unsigned int) * ngrp, s->st));
            CTRY(cudaMalloc(&s->rho_m, sizeof(double) * Nx));
            CTRY(cudaMalloc(&s->colfx_m, sizeof(long long) * Nx));
            CTRY(cudaMalloc(&s->sc_m, sizeof(Scalars)));
            CTRY(cudaMemsetAsync(s->sc_m, 0, sizeof(Scalars), s->st));
            CTRY(cudaMalloc(&s->blockpart_m, 16 * 3 * (size_t)s->crgrid));
            CTRY(cudaMalloc(&s->ring_upart, 16 * (size_t)ngrp));
            CTRY(cudaMemcpyAsync(s->ringKq, Kq.data(), sizeof(long long) * Nx, cudaMemcpyHostToDevice, s->st));
            CTRY(cudaMemcpyAsync(s->ringVq, Vq.data(), sizeof(long long) * Nx, cudaMemcpyHostToDevice, s->st));
            CTRY(cudaStreamSynchronize(s->st));
            if (ringfx_smem_bytes(Nx, s->ring_ksplit) + 8192 > (size_t)max_optin) s->ring_method = RING_M_DIRECT;
        }
    }
    TRY(make_tmap(s, 0));
    TRY(make_tmap(s, 1));
#undef TRY
#undef CTRY
    *out = s;
    return VLASOV_OK;
}

int vlasov_set_f(vlasov_sim* s, const double* host_f)
{
    if (!s || !host_f) return fail(VLASOV_EINVAL, "NULL argument");
    const size_t cells = (size_t)s->Nx * s->Np;
    if (s->esz == 8) {
        // 8-byte storage: the FP64 upload lands in the state buffer (FP64 modes) or in the other one
        // (FX64, converted from there); the bound on |f| and the conversion run on the device
        void* dst = s->f[s->fx ? s->cur ^ 1 : s->cur];
        CU_TRY(cudaMemcpyAsync(dst, host_f, cells * 8, cudaMemcpyHostToDevice, s->st));
        return vlasov_set_f_device(s, static_cast<const double*>(dst));
    }
    double mx = 0.0;
    for (size_t k = 0; k < cells; ++k) mx = std::max(mx, std::fabs(host_f[k]));
    if (!std::isfinite(mx)) return fail(VLASOV_EINVAL, "f holds a non-finite value");
    update_scales(s, mx);
    if (s->esz == 2) {
        std::vector<uint16_t> tmp(cells);
        for (size_t k = 0; k < cells; ++k) tmp[k] = bf16_bits(host_f[k]);
        CU_TRY(cudaMemcpyAsync(s->f[s->cur], tmp.data(), cells * 2, cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));   // tmp is released on return
    } else {
        std::vector<float> tmp(cells);
        for (size_t k = 0; k < cells; ++k) tmp[k] = (float)host_f[k];
        CU_TRY(cudaMemcpyAsync(s->f[s->cur], tmp.data(), cells * 4, cudaMemcpyHostToDevice, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
    }
    CU_TRY(cudaMemsetAsync(s->dstep, 0, sizeof(long long), s->st));
    CU_TRY(cudaStreamSynchronize(s->st));
    s->read_step = 0;
    s->has_f = true;
    return VLASOV_OK;
}

int vlasov_set_f_device(vlasov_sim* s, const double* dev_f)
{
    if (!s || !dev_f) return fail(VLASOV_EINVAL, "NULL argument");
    const size_t cells = (size_t)s->Nx * s->Np;
    CU_TRY(cudaMemsetAsync(s->dstep, 0, sizeof(long long), s->st));
    unsigned long long bits = 0;
    CU_TRY(launch_maxabs(8, dev_f, cells, s->maxbits, s->st));
    CU_TRY(cudaMemcpyAsync(&bits, s->maxbits, sizeof bits, cudaMemcpyDeviceToHost, s->st));
    CU_TRY(cudaStreamSynchronize(s->st));
    double mx;
    std::memcpy(&mx, &bits, sizeof mx);
    if (!std::isfinite(mx)) return fail(VLASOV_EINVAL, "f holds a non-finite value");
    update_scales(s, mx);
    if (s->fx) CU_TRY(launch_f64_to_fx(dev_f, static_cast<long long*>(s->f[s->cur]), cells, s->Ef, s->st));
    else if (dev_f != s->f[s->cur]) CU_TRY(launch_convert(dev_f, 8, s->f[s->cur], s->esz, cells, s->st));
    s->read_step = 0;
    s->has_f = true;
    return VLASOV_OK;
}

int vlasov_init_waterbag(vlasov_sim* s, double x0, double p0, double noise, unsigned long long seed, int mode,
                         double mode_amp)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    if (!(x0 > 0) || !(p0 > 0) || !std::isfinite(x0) || !std::isfinite(p0))
        return fail(VLASOV_EINVAL, "waterbag half-widths must be finite and > 0");
    if (mode != 0 && mode != 1) return fail(VLASOV_EINVAL, "mode must be 0 (box) or 1 (homogeneous + cos mode)");
    if (!(noise >= 0 && noise < 1) || !(std::fabs(mode_amp) < 1))
        return fail(VLASOV_EINVAL, "noise must be in [0, 1) and |mode_amp| < 1");
    const int Nx = s->Nx, Np = s->Np;
    const size_t cells = (size_t)Nx * Np;
    // profile tables of Sec. 4's waterbags on the nodes x_i = xmin + i dx, p_j = pmin + j dp
    std::vector<double> tab((size_t)Nx + Np);
    double* rowv = tab.data();
    double* colv = rowv + Np;
    double rows = 0, cmax = 0;
    for (int j = 0; j < Np; ++j) {
        const double p = s->pmin + (double)j * s->dp;
        rowv[j] = std::fabs(p) < p0 ? 1.0 : 0.0;
        rows += rowv[j];
    }
    const double L = s->xmax - s->xmin, half_x = 0.5 * L;
    for (int i = 0; i < Nx; ++i) {
        const double x = s->xmin + (double)i * s->dx;
        if (mode == 0) colv[i] = (x0 >= half_x || std::fabs(x) < x0) ? 1.0 / (4.0 * x0 * p0) : 0.0;
        else colv[i] = (1.0 / (2.0 * p0 * L)) * (1.0 + mode_amp * std::cos(x));
        cmax = std::max(cmax, std::fabs(colv[i]));
    }
    if (!(rows > 0) || !(cmax > 0)) return fail(VLASOV_EINVAL, "initial state is empty on this grid");

    // one temporary block: tables, int128 block partials, ticket, mass
    const size_t off_part = ((tab.size() * 8 + 15) / 16) * 16;
    const size_t off_tail = off_part + 16 * (size_t)WB_BLOCKS;
    char* tmp = nullptr;
    CU_TRY(cudaMalloc(&tmp, off_tail + 16));
    WaterbagArgs a;
    a.rowv = reinterpret_cast<const double*>(tmp);
    a.colv = a.rowv + Np;
    a.Nx = Nx;
    a.Np = Np;
    a.noise = mode == 0 ? noise : 0.0;
    a.seed = seed;
    a.k_m = 120 - ceil_log2((double)cells * cmax * (1.0 + a.noise) * 2.0 + 1.0);
    a.dxdp = s->dx * s->dp;
    a.part = tmp + off_part;
    a.ticket = reinterpret_cast<unsigned int*>(tmp + off_tail);
    a.mass = reinterpret_cast<double*>(tmp + off_tail + 8);
    a.maxbits = s->maxbits;
    // 8-byte storage: the FP64 state goes through vlasov_set_f_device (FX64 from the other buffer)
    void* dst = s->f[(s->esz == 8 && s->fx) ? s->cur ^ 1 : s->cur];
    cudaError_t e = cudaMemcpyAsync(tmp, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = launch_waterbag(a, s->esz, dst, s->st);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, s->maxbits, sizeof bits, cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(VLASOV_ECUDA, "vlasov_init_waterbag: %s", cudaGetErrorString(e));
    if (s->esz == 8) return vlasov_set_f_device(s, static_cast<const double*>(dst));
    double mx;
    std::memcpy(&mx, &bits, sizeof mx);
    if (!std::isfinite(mx)) return fail(VLASOV_EINVAL, "initial state holds a non-finite value");
    update_scales(s, mx);
    CU_TRY(cudaMemsetAsync(s->dstep, 0, sizeof(long long), s->st));
    CU_TRY(cudaStreamSynchronize(s->st));
    s->read_step = 0;
    s->has_f = true;
    return VLASOV_OK;
}

int vlasov_get_f(vlasov_sim* s, double* host_f)
{
    if (!s || !host_f) return fail(VLASOV_EINVAL, "NULL argument");
    const size_t cells = (size_t)s->Nx * s->Np;
    if (s->fx) {
        // decoded on the device into the other state buffer (free between steps), then one copy
        double* tmp = static_cast<double*>(s->f[s->cur ^ 1]);
        CU_TRY(launch_fx_to_f64(static_cast<const long long*>(s->f[s->cur]), tmp, cells, s->Ef, s->st));
        CU_TRY(cudaMemcpyAsync(host_f, tmp, cells * 8, cudaMemcpyDeviceToHost, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
    } else if (s->esz == 8) {
        CU_TRY(cudaMemcpyAsync(host_f, s->f[s->cur], cells * 8, cudaMemcpyDeviceToHost, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
    } else if (s->esz == 2) {
        std::vector<uint16_t> tmp(cells);
        CU_TRY(cudaMemcpyAsync(tmp.data(), s->f[s->cur], cells * 2, cudaMemcpyDeviceToHost, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
        for (size_t k = 0; k < cells; ++k) {
            const uint32_t u = (uint32_t)tmp[k] << 16;   // a bf16 is the high half of an FP32
            float v;
            std::memcpy(&v, &u, 4);
            host_f[k] = (double)v;
        }
    } else {
        std::vector<float> tmp(cells);
        CU_TRY(cudaMemcpyAsync(tmp.data(), s->f[s->cur], cells * 4, cudaMemcpyDeviceToHost, s->st));
        CU_TRY(cudaStreamSynchronize(s->st));
        for (size_t k = 0; k < cells; ++k) host_f[k] = (double)tmp[k];
    }
    return check_dev_err(s);
}

int vlasov_get_f_device(vlasov_sim* s, double* dev_f)
{
    if (!s || !dev_f) return fail(VLASOV_EINVAL, "NULL argument");
    const size_t cells = (size_t)s->Nx * s->Np;
    if (s->fx) CU_TRY(launch_fx_to_f64(static_cast<const long long*>(s->f[s->cur]), dev_f, cells, s->Ef, s->st));
    else CU_TRY(launch_convert(s->f[s->cur], s->esz, dev_f, 8, cells, s->st));
    return VLASOV_OK;
}

int vlasov_step(vlasov_sim* s, int n)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    if (n < 0) return fail(VLASOV_EINVAL, "n < 0");
    if (!s->has_f) return fail(VLASOV_ESTATE, "vlasov_step before vlasov_set_f");
    if (s->fuse && n >= 2) {
        const int c = s->cur;
        // both starting buffers' graphs at the first call, so that no later call captures
        int rc = build_fused_graphs(s, c);
        if (!rc) rc = build_fused_graphs(s, c ^ 1);
        if (rc) return rc;
        // one graph launch per run of 2^L middle pieces, largest runs first (a graph launch costs
        // the stream a few microseconds more than a kernel boundary inside a graph)
        CU_TRY(cudaGraphLaunch(s->ghead[c], s->st));
        int m = n - 1;
        for (int L = RUN_LEVELS - 1; L >= 0; --L)
            for (; m >= (1 << L); m -= 1 << L) CU_TRY(cudaGraphLaunch(s->gmid[c][L], s->st));
        CU_TRY(cudaGraphLaunch(s->gtail[c], s->st));
        s->cur ^= 1;
        return VLASOV_OK;
    }
    int m = n;
    for (int L = RUN_LEVELS - 1; L >= 0; --L)
        for (; m >= (1 << L); m -= 1 << L) {
            int rc = build_graphs(s, s->cur);
            if (!rc) rc = build_graphs(s, s->cur ^ 1);
            if (rc) return rc;
            CU_TRY(cudaGraphLaunch(s->grun[s->cur][L], s->st));
            if (L == 0) s->cur ^= 1;
        }
    return VLASOV_OK;
}

int vlasov_moments(vlasov_sim* s, vlasov_moments_t* out, int max, int* count)
{
    if (!s || (!out && max > 0)) return fail(VLASOV_EINVAL, "NULL argument");
    long long h = 0;
    CU_TRY(cudaMemcpyAsync(&h, s->dstep, sizeof h, cudaMemcpyDeviceToHost, s->st));
    CU_TRY(cudaStreamSynchronize(s->st));
    long long first = std::max(s->read_step, h - (long long)HIST_CAP);
    long long n = std::min<long long>(h - first, (long long)std::max(max, 0));
    std::vector<MomentRec> tmp((size_t)std::max<long long>(n, 0));
    // the records are contiguous in the ring except across its wrap: at most two copies
    for (long long k = 0; k < n;) {
        const long long idx = (first + k) % HIST_CAP;
        const long long len = std::min<long long>(n - k, (long long)HIST_CAP - idx);
        CU_TRY(cudaMemcpyAsync(&tmp[(size_t)k], s->hist + idx, sizeof(MomentRec) * (size_t)len,
                               cudaMemcpyDeviceToHost, s->st));
        k += len;
    }
    CU_TRY(cudaStreamSynchronize(s->st));
    for (long long k = 0; k < n; ++k) {
        const MomentRec& r = tmp[(size_t)k];
        out[k].t = r.t;
        out[k].mass = r.mass;
        out[k].Mx = r.Mx;
        out[k].My = r.My;
        out[k].kinetic = r.kinetic;
        out[k].potential = r.potential;
        out[k].energy = r.energy;
        out[k].step = r.step;
    }
    s->read_step = first + n;
    if (count) *count = (int)n;
    return check_dev_err(s);
}

int vlasov_substep(vlasov_sim* s, int axis, const double* host_disp)
{
    if (!s || !host_disp) return fail(VLASOV_EINVAL, "NULL argument");
    if (axis != 0 && axis != 1) return fail(VLASOV_EINVAL, "axis must be 0 (x) or 1 (p)");
    if (!s->has_f) return fail(VLASOV_ESTATE, "substep before vlasov_set_f");
    const int c = s->cur, o = c ^ 1;
    if (axis == 0) {
        int mx = 0;
        int rc = upload_params(s, s->sp, host_disp, s->Np, &mx, &s->se, s->srec);
        if (rc) return rc;
        XShiftArgs a = xargs(s, s->f[c], s->f[o], s->sp, false, false, s->srec);
        if (!s->xper && mx + xhalo_extra(s->esz) > s->xpad) {
            // wider zero halo for this call: the staged row grows, fewer rows in flight
            a.pad = ((mx + xhalo_extra(s->esz) + 15) / 16) * 16;
            int max_optin = 0;
            CU_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->dev));
            const size_t row_bytes = (size_t)(s->Nx + 2 * a.pad) * s->esz + XREC_BYTES;
            const size_t budget = (size_t)max_optin - 2048 - 256;
            a.stages = (int)std::min<size_t>(4, budget / row_bytes);
            if (a.stages < 1) return fail(VLASOV_EINVAL, "x displacement of %d cells does not fit shared memory", mx);
        }
        CU_TRY(run_xshift(s, a, s->sp, s->se, false));
    } else {
        int rc = upload_params(s, s->sp, host_disp, s->Nx, nullptr, &s->se);
        if (rc) return rc;
        CU_TRY(run_pshift(s, &s->tmap[c], pargs(s, s->f[c], s->f[o], s->sp), s->sp, s->se));
    }
    s->cur = o;
    CU_TRY(cudaStreamSynchronize(s->st));
    return check_dev_err(s);
}

int vlasov_density_force(vlasov_sim* s, double* host_rho, double* host_F)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    if (!s->has_f) return fail(VLASOV_ESTATE, "density before vlasov_set_f");
    if (s->fx) CU_TRY(launch_colsum_fx(static_cast<const long long*>(s->f[s->cur]), s->Nx, s->Np, s->Ef, s->colpart, s->st));
    else CU_TRY(launch_colsum(s->esz, s->f[s->cur], s->Nx, s->Np, s->colpart, 1, s->st));
    CU_TRY(launch_colreduce(crargs(s, 1, false, false, false), s->crgrid, s->st));
    int rc = launch_force_params(s, s->Fout);
    if (rc) return rc;
    if (host_rho) CU_TRY(cudaMemcpyAsync(host_rho, s->rho, sizeof(double) * s->Nx, cudaMemcpyDeviceToHost, s->st));
    if (host_F) CU_TRY(cudaMemcpyAsync(host_F, s->Fout, sizeof(double) * s->Nx, cudaMemcpyDeviceToHost, s->st));
    CU_TRY(cudaStreamSynchronize(s->st));
    return check_dev_err(s);
}

int vlasov_casimirs(vlasov_sim* s, double* entropy, double* l2)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    if (!s->has_f) return fail(VLASOV_ESTATE, "vlasov_casimirs before vlasov_set_f");
    const size_t cells = (size_t)s->Nx * s->Np;
    const int kind = s->fx ? 0 : (s->esz == 8 ? 1 : s->esz == 4 ? 2 : 3);
    const double unit = s->fx ? std::ldexp(1.0, s->Ef - FX_FRAC) : 1.0;
    // scratch: the column partial rows (at least 2 * CAS_BLOCKS + 2 doubles)
    double* part = s->colpart;
    double* out = s->colpart + 2 * CAS_BLOCKS;
    CU_TRY(launch_casimirs(kind, s->f[s->cur], cells, unit, s->dx * s->dp, part, out, s->st));
    double h[2] = {0.0, 0.0};
    CU_TRY(cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, s->st));
    CU_TRY(cudaStreamSynchronize(s->st));
    if (entropy) *entropy = h[0];
    if (l2) *l2 = h[1];
    return check_dev_err(s);
}

// Spectra and twiddles of the FFT ring method, computed once per handle and arithmetic type.
// Toeplitz block images of the tensor-core ring method, built once per handle.
static int ring_tc_setup(vlasov_sim* s)
{
    if (s->ring_tcK) return VLASOV_OK;
    const int N = s->Nx, N1 = N / RING_TC_M;
    std::vector<double> dV(N), V(N);
    for (int i = 0; i < N; ++i) {
        const double u = (double)i * s->dx;
        const double q = 1.0 - std::cos(u) + s->eps;
        dV[i] = std::sin(u) / (2.0 * std::sqrt(2.0) * q * std::sqrt(q));
        V[i] = -1.0 / (std::sqrt(2.0) * std::sqrt(q));
    }
    const size_t bytes = (size_t)N1 * 2 * RING_TC_IMG;
    std::vector<float> img(bytes / 4);
    CU_TRY(cudaMalloc(&s->ring_tcK, bytes));
    CU_TRY(cudaMalloc(&s->ring_tcV, bytes));
    CU_TRY(cudaMalloc(&s->ring_tcacc, sizeof(long long) * (size_t)N));
    CU_TRY(cudaMemset(s->ring_tcacc, 0, sizeof(long long) * (size_t)N));
    CU_TRY(cudaMalloc(&s->ring_tcticket, sizeof(unsigned int)));
    CU_TRY(cudaMemset(s->ring_tcticket, 0, sizeof(unsigned int)));
    for (int i = 0; i < N; ++i) {
        s->ring_tcmax[0] = std::max(s->ring_tcmax[0], std::fabs(dV[i]));
        s->ring_tcmax[1] = std::max(s->ring_tcmax[1], std::fabs(V[i]));
    }
    ring_tc_tables(dV.data(), N, img.data());
    CU_TRY(cudaMemcpy(s->ring_tcK, img.data(), bytes, cudaMemcpyHostToDevice));
    ring_tc_tables(V.data(), N, img.data());
    CU_TRY(cudaMemcpy(s->ring_tcV, img.data(), bytes, cudaMemcpyHostToDevice));
    return VLASOV_OK;
}

static int ring_fft_tables(vlasov_sim* s, bool f64)
{
    void** slot = f64 ? &s->ring_fft64 : &s->ring_fft32;
    if (*slot) return VLASOV_OK;
    const int N = s->Nx;
    std::vector<double> dV(N), V(N), kh(2 * (size_t)N), vh(2 * (size_t)N);
    for (int i = 0; i < N; ++i) {
        const double u = (double)i * s->dx;
        const double q = 1.0 - std::cos(u) + s->eps;
        dV[i] = std::sin(u) / (2.0 * std::sqrt(2.0) * q * std::sqrt(q));
        V[i] = -1.0 / (std::sqrt(2.0) * std::sqrt(q));
    }
    ring_dft_host(dV.data(), N, kh.data());
    ring_dft_host(V.data(), N, vh.data());
    std::vector<double> all(2 * (size_t)N * 2 + (size_t)N);   // khat, vhat (N complex each), twiddles (N/2)
    std::copy(kh.begin(), kh.end(), all.begin());
    std::copy(vh.begin(), vh.end(), all.begin() + 2 * (size_t)N);
    for (int m = 0; m < N / 2; ++m) {
        const double ang = 2.0 * 3.14159265358979323846 * (double)m / (double)N;
        all[4 * (size_t)N + 2 * m] = std::cos(ang);
        all[4 * (size_t)N + 2 * m + 1] = -std::sin(ang);
    }
    const size_t n = all.size();
    if (f64) {
        CU_TRY(cudaMalloc(slot, n * sizeof(double)));
        CU_TRY(cudaMemcpy(*slot, all.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> af(all.begin(), all.end());
        CU_TRY(cudaMalloc(slot, n * sizeof(float)));
        CU_TRY(cudaMemcpy(*slot, af.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    }
    return VLASOV_OK;
}

int vlasov_set_ring_method(vlasov_sim* s, int method)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    if (s->model != VLASOV_RING) return fail(VLASOV_EINVAL, "not a ring-model handle");
    if (method == VLASOV_RING_FIXED) {
        if (ringfx_smem_bytes(s->Nx, s->ring_ksplit) + 8192 > (size_t)s->max_smem)
            return fail(VLASOV_EINVAL, "fixed-point ring method: Nx too large for shared memory");
    } else if (method == VLASOV_RING_FFT || method == VLASOV_RING_FFT_F32) {
        if (!ring_fft_ok(s->Nx)) return fail(VLASOV_EINVAL, "FFT ring method needs Nx a power of two <= 4096");
        const bool f64 = method == VLASOV_RING_FFT;
        if (ring_fft_smem_bytes(s->Nx, f64) + 8192 > (size_t)s->max_smem)
            return fail(VLASOV_EINVAL, "FFT ring method: Nx too large for shared memory");
        int rc = ring_fft_tables(s, f64);
        if (rc) return rc;
    } else if (method == VLASOV_RING_TENSOR) {
        if (!ring_tc_ok(s->Nx)) return fail(VLASOV_EINVAL, "tensor-core ring method needs Nx = 128 k, 256 <= Nx <= 4096");
        if (ring_tc_smem_bytes() + 2048 > (size_t)s->max_smem)
            return fail(VLASOV_EINVAL, "tensor-core ring method: not enough shared memory");
        int rc = ring_tc_setup(s);
        if (rc) return rc;
    } else if (method != VLASOV_RING_DIRECT) {
        return fail(VLASOV_EINVAL, "unknown ring method %d", method);
    }
    CU_TRY(cudaStreamSynchronize(s->st));
    if (s->ring_method != method) drop_graphs(s);
    s->ring_method = method;
    return VLASOV_OK;
}

int vlasov_ring_method(const vlasov_sim* s) { return (s && s->model == VLASOV_RING) ? s->ring_method : 0; }

int vlasov_ring_timings(vlasov_sim* s, int reps, double* us)
{
    if (!s || !us) return fail(VLASOV_EINVAL, "NULL argument");
    if (s->model != VLASOV_RING) return fail(VLASOV_EINVAL, "not a ring-model handle");
    if (!s->has_f) return fail(VLASOV_ESTATE, "vlasov_ring_timings before vlasov_set_f");
    if (reps < 1 || reps > 100000) return fail(VLASOV_EINVAL, "reps must be in [1, 1e5]");
    for (int m = 0; m < VLASOV_RING_METHODS; ++m) us[m] = 0.0;
    // density of the current f (as vlasov_density_force), then each method's force launch
    if (s->fx) CU_TRY(launch_colsum_fx(static_cast<const long long*>(s->f[s->cur]), s->Nx, s->Np, s->Ef, s->colpart, s->st));
    else CU_TRY(launch_colsum(s->esz, s->f[s->cur], s->Nx, s->Np, s->colpart, 1, s->st));
    CU_TRY(launch_colreduce(crargs(s, 1, false, false, false), s->crgrid, s->st));
    const int keep = s->ring_method;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU_TRY(cudaEventCreate(&e0));
    CU_TRY(cudaEventCreate(&e1));
    int rc = VLASOV_OK;
    for (int m = VLASOV_RING_DIRECT; m < VLASOV_RING_METHODS && !rc; ++m) {
        if (m == VLASOV_RING_TENSOR) {
            if (!ring_tc_ok(s->Nx) || ring_tc_smem_bytes() + 2048 > (size_t)s->max_smem) continue;
            if ((rc = ring_tc_setup(s)) != VLASOV_OK) break;
        }
        const bool fft = m == VLASOV_RING_FFT || m == VLASOV_RING_FFT_F32;
        if (fft && !ring_fft_ok(s->Nx)) continue;
        if (fft && ring_fft_smem_bytes(s->Nx, m == VLASOV_RING_FFT) + 8192 > (size_t)s->max_smem) continue;
        if (fft && (rc = ring_fft_tables(s, m == VLASOV_RING_FFT)) != VLASOV_OK) break;
        if (m == VLASOV_RING_FIXED && ringfx_smem_bytes(s->Nx, s->ring_ksplit) + 8192 > (size_t)s->max_smem) continue;
        s->ring_method = m;
        cudaError_t e = run_ring(s, false);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s->st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = run_ring(s, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = fail(VLASOV_ECUDA, "ring timing: %s", cudaGetErrorString(e));
        else us[m] = 1e3 * (double)ms / reps;
    }
    s->ring_method = keep;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return check_dev_err(s);
}

int vlasov_test_expire_wait(vlasov_sim* s, long long limit_ns)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    if (limit_ns < 1000 || limit_ns > 2000000000ll)
        return fail(VLASOV_EINVAL, "limit_ns must be in [1e3, 2e9]");
    CU_TRY(launch_expire_wait(s->err, (unsigned long long)limit_ns, s->st));
    return VLASOV_OK;
}

int vlasov_sync(vlasov_sim* s)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    CU_TRY(cudaStreamSynchronize(s->st));
    return check_dev_err(s);
}

int vlasov_step_timed(vlasov_sim* s, int n, double* ms_per_launch, int max_launches, int* nlaunch)
{
    if (!s || n < 1 || !ms_per_launch) return fail(VLASOV_EINVAL, "bad argument");
    if (!s->has_f) return fail(VLASOV_ESTATE, "vlasov_step_timed before vlasov_set_f");
    const bool fused = s->fuse && n >= 2;
    const int L = vlasov_kernels_per_step(s);
    if (max_launches < L) return fail(VLASOV_EINVAL, "max_launches < %d", L);
    // fused: head, n-1 timed mids, tail (the slots are those of a mid piece); else n whole steps
    const int reps = fused ? n - 1 : n;
    std::vector<cudaEvent_t> ev((size_t)(L + 1) * reps, nullptr);
    for (auto& e : ev) CU_TRY(cudaEventCreate(&e));
    int rc = VLASOV_OK;
    const int c = s->cur;
    if (fused) {
        rc = enqueue_piece(s, c, P_HEAD);
        for (int k = 0; k < reps && !rc; ++k) {
            Marks m;
            m.ev = ev.data() + (size_t)k * (L + 1);
            rc = enqueue_piece(s, c, P_MID, &m);
        }
        if (!rc) rc = enqueue_piece(s, c, P_TAIL);
        s->cur ^= 1;
    } else {
        for (int k = 0; k < reps && !rc; ++k) {
            Marks m;
            m.ev = ev.data() + (size_t)k * (L + 1);
            rc = enqueue_step(s, s->cur, &m);
            s->cur ^= 1;
        }
    }
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess) rc = fail(VLASOV_ECUDA, "sync: %s", cudaGetErrorString(e));
    }
    if (!rc) {
        for (int q = 0; q < L; ++q) {
            double acc = 0.0;
            for (int k = 0; k < reps; ++k) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[(size_t)k * (L + 1) + q], ev[(size_t)k * (L + 1) + q + 1]);
                acc += ms;
            }
            ms_per_launch[q] = acc / reps;
        }
        if (nlaunch) *nlaunch = L;
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (rc) return rc;
    return check_dev_err(s);
}

int vlasov_kernels_per_step(const vlasov_sim* s)
{
    if (!s) return 0;
    if (ring_merged(s)) return 4;   // fused x-shifts, both reductions, both convolutions (+ filters), p-shift
    return (s->fuse ? 2 : 3) + force_launches(s) + moment_launches(s);
}

long long vlasov_launches(const vlasov_sim* s, int n)
{
    if (!s || n < 1) return 0;
    if (!(s->fuse && n >= 2)) return (long long)n * (3 + force_launches(s) + moment_launches(s));
    // head (x-shift, force, p-shift), n-1 mids, tail (x-shift, moments)
    return (2 + force_launches(s)) + (long long)(n - 1) * vlasov_kernels_per_step(s) + (1 + moment_launches(s));
}

int vlasov_set_fused_x(vlasov_sim* s, int on)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    if (on && s->gs) return fail(VLASOV_EINVAL, "fused x-shifts run the spline of Eq. findif only");
    if (on && !s->fuse_ok)
        return fail(VLASOV_EINVAL, "fused x-shifts need VLASOV_FX64 (Nx <= %d), VLASOV_F32 or VLASOV_BF16 (Nx <= %d) storage",
                    XF_FUSED_MAX_NX, XXS_MAX_NX);
    s->fuse = on != 0;
    return VLASOV_OK;
}

int vlasov_fused_x(const vlasov_sim* s) { return (s && s->fuse) ? 1 : 0; }

int vlasov_set_spline(vlasov_sim* s, int spline)
{
    if (!s) return fail(VLASOV_EINVAL, "NULL handle");
    if (spline != VLASOV_SPLINE_FD && spline != VLASOV_SPLINE_GS) return fail(VLASOV_EINVAL, "unknown spline %d", spline);
    const bool gs = spline == VLASOV_SPLINE_GS;
    if (gs == s->gs) return VLASOV_OK;
    if (gs) {
        if (s->fx || s->emul || s->esz == 2)
            return fail(VLASOV_EINVAL, "the global spline runs with VLASOV_F64_NATIVE or VLASOV_F32 storage");
        if (s->Nx < GS_MIN_N || s->Np < GS_MIN_N || s->Nx > GS_XTHREADS * GS_XCH)
            return fail(VLASOV_EINVAL, "the global spline needs %d <= Nx <= %d and Np >= %d", GS_MIN_N,
                        GS_XTHREADS * GS_XCH, GS_MIN_N);
        if (s->gspgrid == 0) {
            int occ = 0;
            CU_TRY(gs_occupancy(s->esz, false, gs_pshift_smem_bytes(s->esz), &occ));
            const int tiles = ((s->Nx + 31) / 32) * ((s->Np + GS_PTH - 1) / GS_PTH);
            s->gspgrid = std::max(1, std::min(tiles, s->nsm * std::max(occ, 1)));
        }
        s->fuse = false;
    }
    CU_TRY(cudaStreamSynchronize(s->st));
    drop_graphs(s);
    s->gs = gs;
    s->hmf_cta = gs ? false : s->hmf_cta_fd;
    return VLASOV_OK;
}

int vlasov_spline(const vlasov_sim* s) { return (s && s->gs) ? VLASOV_SPLINE_GS : VLASOV_SPLINE_FD; }

}  // extern "C"
