// vlasov_internal.cuh -- shared declarations of the CUDA library (kernels + host runtime).
//
// Layout (Sec. 3 of arXiv:1206.3229): f[j*Nx + i], x contiguous, p rows.  Two ping-pong buffers
// hold f; a Strang step is x-shift (A->B), p-shift (B->A), x-shift (A->B).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace vl {

// ---------------------------------------------------------------------------------------------
// Eq. (findif): f''(u_k) du^2 = sum_{m=-4..4} c_|m| f(u_{k+m}), c = -205/72, 8/5, -1/5, 8/315, -1/560.
#define VL_FD_C0 (-205.0 / 72.0)
#define VL_FD_C1 (8.0 / 5.0)
#define VL_FD_C2 (-1.0 / 5.0)
#define VL_FD_C3 (8.0 / 315.0)
#define VL_FD_C4 (-1.0 / 560.0)

constexpr int NTAP = 10;          // the spline + FD stencil spans f_{k-4} .. f_{k+5}
constexpr int FX_FRAC = 61;       // 64-bit fixed-point storage: X = round(f * 2^(FX_FRAC - Ef))
constexpr int HIST_CAP = 4096;    // moment records kept on the device

// Spline weights of one line for a displacement s (cells).  Eqs. (splinegen, splinecoeffs) with
// f''_k = D_k/du^2 and D_k = sum_m c_|m| f_{k+m}: the du^2 of gamma/delta cancels, so
//   f_new(i) = alpha f_k + beta f_{k+1} + g D_k + d D_{k+1},  k = i + n0,
//   g = (alpha^3 - alpha)/6, d = (beta^3 - beta)/6,
// which is the 10-tap filter  f_new(i) = sum_{t=0..9} w_t f_{k-4+t}.
struct LineSplit {
    int n0;
    double alpha, beta, g, d;
    double w[NTAP];
};

__host__ __device__ inline void line_split(double s, LineSplit& L)
{
    const double ms = -s;
    const double fl = floor(ms);
    L.n0 = (int)fl;
    L.beta = ms - fl;
    L.alpha = 1.0 - L.beta;
    const double a = L.alpha, b = L.beta;
    L.g = (a * a * a - a) / 6.0;
    L.d = (b * b * b - b) / 6.0;
    const double g = L.g, d = L.d;
    L.w[0] = g * VL_FD_C4;
    L.w[1] = g * VL_FD_C3 + d * VL_FD_C4;
    L.w[2] = g * VL_FD_C2 + d * VL_FD_C3;
    L.w[3] = g * VL_FD_C1 + d * VL_FD_C2;
    L.w[4] = a + g * VL_FD_C0 + d * VL_FD_C1;
    L.w[5] = b + g * VL_FD_C1 + d * VL_FD_C0;
    L.w[6] = g * VL_FD_C2 + d * VL_FD_C1;
    L.w[7] = g * VL_FD_C3 + d * VL_FD_C2;
    L.w[8] = g * VL_FD_C4 + d * VL_FD_C3;
    L.w[9] = d * VL_FD_C4;
}

// Zero-outside lines take f'' = 0 at nodes outside the grid.  Outputs whose foot cell lies wholly
// outside are 0; the two whose cell touches the end need the filter without one f'' term:
//   we[0]: k = -1, without g D_k   (D_k spans taps 0..8 with c_|t-4|),
//   we[1]: k = n - 1, without d D_{k+1}  (taps 1..9 with c_|t-5|).
__host__ __device__ inline void line_edge_weights(const LineSplit& L, double we[2][NTAP])
{
    const double c[5] = {VL_FD_C0, VL_FD_C1, VL_FD_C2, VL_FD_C3, VL_FD_C4};
    for (int t = 0; t < NTAP; ++t) {
        const int m0 = t - 4, m1 = t - 5;
        we[0][t] = L.w[t] - (m0 >= -4 && m0 <= 4 ? L.g * c[m0 < 0 ? -m0 : m0] : 0.0);
        we[1][t] = L.w[t] - (m1 >= -4 && m1 <= 4 ? L.d * c[m1 < 0 ? -m1 : m1] : 0.0);
    }
}

// Per-line parameters in device memory, structure-of-arrays over `n` lines:
//   n0[line], w[t*n + line] (t < 10), gd[line] = g, gd[n + line] = d  (in the storage type T).
struct LineParamsDev {
    int* n0 = nullptr;
    void* w = nullptr;
    void* gd = nullptr;
    double* beta = nullptr;   // foot fraction per line (global-spline sweeps)
};

// Global-spline variant (Eq. tridiagsys).  On a periodic line the cyclic system's inverse is the
// circulant g_m = r^|m| / (2 sqrt 3), r = sqrt 3 - 2 (|r|^31 < 2e-18: truncated at |m| <= GS_R it is
// exact to FP64 rounding for lines of >= 2 GS_R + 1 nodes).  On a zero-outside line (f = f'' = 0 at
// the nodes -1 and n) the same holds for the data extended oddly about -1 and n.  So the spline
// value at a foot k + beta is a filter of GS_TAPS taps over the extended line, starting at node
// k - GS_R - 1: W_u = alpha [u = 0] + beta [u = 1] + gamma h_u + delta h_(u-1), u = -GS_R-1 .. GS_R+2,
// with h = 6 g * (1, -2, 1) (GS_HTAPS taps, u = -GS_R-1 .. GS_R+1) and gamma, delta of Eq.
// splinecoeffs in cell units.
constexpr int GS_R = 30;
constexpr int GS_HTAPS = 2 * GS_R + 3;
constexpr int GS_TAPS = 2 * GS_R + 4;
constexpr int GS_HALO = GS_R + 2;          // extended nodes each side of a staged line
constexpr int GS_MIN_N = 2 * GS_R + 4;     // lines this short or longer
constexpr int GS_XTHREADS = 512;
constexpr int GS_XCH = 16;                 // columns per x-shift thread: Nx <= GS_XTHREADS * GS_XCH
constexpr int GS_PROWS = 256;              // staged rows of a p-shift tile (32 columns)
constexpr int GS_PTH = 64;                 // output rows of a p-shift tile (8 warps x 8)

inline void gs_filter_h(double h[GS_HTAPS])
{
    const double r = std::sqrt(3.0) - 2.0;
    double g[2 * GS_R + 1];
    double rm = 1.0;
    for (int m = 0; m <= GS_R; ++m) {
        g[GS_R + m] = g[GS_R - m] = rm / (2.0 * std::sqrt(3.0));
        rm *= r;
    }
    auto gm = [&](int m) { return (m >= -GS_R && m <= GS_R) ? g[GS_R + m] : 0.0; };
    for (int u = -GS_R - 1; u <= GS_R + 1; ++u) h[u + GS_R + 1] = 6.0 * (gm(u - 1) - 2.0 * gm(u) + gm(u + 1));
}

// Device-side error codes written to the handle's flag by a bounded wait that gave up.
enum : int { DEV_ERR_NONE = 0, DEV_ERR_XSHIFT_WAIT = 1, DEV_ERR_PSHIFT_WAIT = 2, DEV_ERR_RANGE = 3,
             DEV_ERR_TEST_WAIT = 4, DEV_ERR_RING_WAIT = 5 };

// Scalars produced by the reductions of one sweep (device struct).
struct Scalars {
    double mass, Mx, My, kinetic, potential;
};

// One moment record (mirrors vlasov_moments_t).
struct MomentRec {
    double t, mass, Mx, My, kinetic, potential, energy;
    long long step;
};

// ---------------------------------------------------------------------------------------------
// Launch arguments.
// Per-row filter record of the x-shift, staged into shared memory next to its row by the same bulk
// copy transaction (all precisions' forms of the ten weights; filled on the host).
struct XRec {
    int n0;
    int m4;               // (n0 - 4) mod Nx in [0, Nx): where a periodic row's window for output 0 starts
    double w64[NTAP];
    double g64, d64;
    int Wh[NTAP];
    float wl[NTAP];
    float wf[NTAP];
    float w32[NTAP];
    float g32, d32;
    long long p2q;        // round(p_j^2 / 2 * 2^KIN_Q) of the row: exact kinetic-energy weight
    // zero-outside rows: line_edge_weights split as Wh/wl/wf (the fixed-point sweeps' edge outputs)
    int Whe[2][NTAP];
    float wle[2][NTAP];
    float wfe[2][NTAP];
    float p2h;            // p_j^2 / 2 of the row in FP32 (kinetic weight of the FP32-class sweeps)
    float pad_;
};
constexpr int XREC_BYTES = 528;
constexpr int KIN_Q = 40;   // |p| < 2896 keeps p^2/2 * 2^KIN_Q below 2^62
static_assert(sizeof(XRec) <= XREC_BYTES, "XRec must fit its staged slot");

struct XShiftArgs {
    const void* rec = nullptr;   // [Np] records of XREC_BYTES, or null: read the arrays below
    const void* fin;
    void* fout;
    int Nx, Np;
    int pad;              // zero/halo elements each side of a staged row
    int stages;           // rows in flight per CTA
    const int* n0;        // per row
    const void* w;        // [10][Np] in T
    const void* gd;       // [2][Np] in T
    double* colpart;      // [gridDim.x][Nx] column sums of the output, or null
    unsigned long long* colacc = nullptr;   // or: [Nx] exact int64 column sums (round(x 2^k_col)), atomically added
    long long* colpart64 = nullptr;          // or: [ctas][Nx] exact int64 per-CTA column sums (units 2^-k_col)
    void* ctapart = nullptr;                 // or (HMF): [ctas][3] int128 per-CTA sum_i t_i, sum_i cos50_i t_i,
                                             // sum_i sin50_i t_i of the CTA's column sums t_i (units 2^(Ef-51))
    const long long* cos50 = nullptr;        //   round(cos x_i 2^50), round(sin x_i 2^50)
    int Ef = 0;                              //   (FP32-class storage: the bound 2^Ef of those units)
    const long long* sin50 = nullptr;
    int k_col = 0;
    double* kinpart;      // [gridDim.x] sum_j p_j^2/2 sum_i out, or null
    void* kin128 = nullptr;   // FX64: [ctas] int128 per-CTA kinetic sums instead (units 2^(Ef-51-KIN_Q))
    double pmin, dp;
    const double* beta = nullptr;   // global spline: foot fraction per row, and the filter h
    const double* gs_h = nullptr;
    int* err;
    int box_h = 0;        // fused x-shifts: lines of 8 elements per TMA box (divides Nx / 8, <= 256)
    int ctas = 0;         // CTAs that share the rows (row stride; the partials above have this many
                          // entries); 0: gridDim.x.  CTAs at or past it do nothing.
};

// Filters of the emulated-FP64 sweeps (emul.cuh), structure-of-arrays over n lines:
//   Wh[t*n + line] (int32), wl[t*n + line], wf[t*n + line] (float), plus n0 and gd (FP64) as above.
struct EmulArgs {
    int Ef;               // fixed-point bound: |f| < 2^Ef
    const int* n0;
    const int* Wh;
    const float* wl;
    const float* wf;
    const double* gd;
    const double* w64;    // the FP64 weights [10][n] (boundary rows are recomputed in FP64)
    const int* Whe = nullptr;     // or: the edge filters [2][10][n] of zero-outside lines, split as
    const float* wle = nullptr;   //   Wh/wl/wf (the boundary outputs in fixed-point arithmetic)
    const float* wfe = nullptr;
};

struct EmulParamsDev {
    int* Wh = nullptr;
    float* wl = nullptr;
    float* wf = nullptr;
    int* Whe = nullptr;     // [2][NTAP][n]: the edge filters of zero-outside lines (line_edge_weights)
    float* wle = nullptr;
    float* wfe = nullptr;
};

struct PShiftArgs {
    const void* fin;
    void* fout;
    int Nx, Np;
    const int* n0;        // per column
    const void* w;        // [10][Nx] in T
    const void* gd;       // [2][Nx] in T
    int* err;
    const double* beta = nullptr;   // global spline: foot fraction per column, and the filter h
    const double* gs_h = nullptr;
};

struct ColReduceArgs {
    unsigned long long* colacc;   // [Nx] int64 column sums added by the x-shift (read and cleared), or null
    const double* colpart;   // else [B][Nx] per-CTA column sums of f
    const long long* colpart64 = nullptr;   // or [B][Nx] exact per-CTA column sums (units 2^-k_col)
    const void* ctapart = nullptr;          // or (HMF) [B][3] int128 per-CTA partials of the x-shift
    int Ef = 0;                             //   (their units: 2^(Ef-51), 2^(Ef-101))
    int B;
    const double* kinpart;   // [B] per-CTA sum_j p_j^2/2 sum_i f, or null
    const void* kin128 = nullptr;   // or [B] int128 per-CTA kinetic sums in units 2^-kin_frac (exact total)
    int kin_frac = 0;
    int Nx;
    int k_col;               // fixed-point shift of column sums: X = round(x * 2^k_col) (int64)
    int k_kin;               // shift of the kinetic partials (int128)
    int k_pot;               // shift of the sheet potential terms (int128)
    double dp;
    double dxdp;             // dx * dp
    double pot_scale;        // sheet: 2 pi G dx^3 dp^2
    const long long* cosfx;  // round(cos(x_i) * 2^62), round(sin(x_i) * 2^62)
    const long long* sinfx;
    double* rho;             // [Nx] out: dp * column sum
    long long* colfx;        // [Nx] out: fixed-point column sums
    double* Qd;              // [Nx] out (sheet): (2 C_i + s_i - S) * 2^-k_col, C_i = sum_{k<i} s_k
    void* blockpart;         // [gridDim.x][3] int128 scratch
    unsigned int* ticket;    // zero on entry; reset by the last block
    Scalars* sc;             // out
    int model;
    int final_moments;       // 1: write the moment record (all models but ring)
    MomentRec* hist;
    long long* step;
    double dt;
};

// HMF p-shift filters formed inside the p-shift (FP32-class storage): the x-shift's per-CTA numbers
// give Mx, My (one warp per CTA sums them exactly), and the producer warp forms each tile's filters.
struct HmfFiltArgs {
    const void* ctapart = nullptr;   // [ctas][3] int128
    int ctas = 0, Ef = 0, on = 0;
    double dxdp = 0, cp = 0;         // dx dp; dt / dp
    const double* costab = nullptr;
    const double* sintab = nullptr;
};

struct PParamsArgs {
    // HMF from the x-shift's per-CTA partials: every block adds the same [ctas][3] int128 partials
    // (exactly) to get Mx, My.
    const void* ctapart = nullptr;
    int ctas = 0, Ef = 0;
    double dxdp = 0;
    int Nx, model;
    const Scalars* sc;
    const double* costab;
    const double* sintab;
    const double* Fin;       // ring: force [Nx]; sheet: Qd [Nx]
    double Fscale;           // sheet: F_i = Fscale * Qd_i
    double cp;               // dt / dp
    int* n0;
    void* w;
    void* gd;
    double* Fout;            // optional copy of F [Nx]
    int* Wh;                 // emulated-FP64 split of the weights, or null
    float* wl;
    float* wf;
    int* Whe = nullptr;      // and of the edge filters [2][NTAP][Nx], or null
    float* wle = nullptr;
    float* wfe = nullptr;
    double* beta = nullptr;  // foot fraction per column (global-spline sweeps), or null
};

struct RingArgs {
    int N;
    double dx;
    const double* rho;
    const void* dV;          // V'(m dx), m = 0..N-1 (double, or float for FP32 storage)
    const void* V;           // V(m dx)
    double* F;               // out
    void* blockpart;         // [gridDim.x] int128
    int k_pot;               // shift of the potential terms rho_i * Phi_i
    double pot_scale;        // 0.5 * dx
    unsigned int* ticket;
    Scalars* sc;
    int final_moments;
    MomentRec* hist;
    long long* step;
    double dt;
    // exact fixed-point form (ring.cu): t_k = exact column sums (rho_k = dp t_k 2^-k_col), kernel
    // tables round(V'(m dx) 2^sK) and round(V(m dx) 2^sV)
    const long long* colfx;
    const long long* Kq;
    const long long* Vq;
    int k_col, sK, sV;
    double dp;
    int ksplit;              // blocks per group of 32 outputs
    // the force launch of the fixed-point form can also write the p-shift filters of its columns
    // (the filter launch's work, same values): pp_on, with pp_fixed for 8-byte storage
    PParamsArgs pp{};
    int pp_on = 0, pp_fixed = 0;
    void* gpart;             // int128 [ksplit][N] partial sums
    unsigned int* gticket;   // [ceil(N/32)] per-group tickets
    void* upart;             // int128 [ceil(N/32)] potential partials per group
    // FFT form (ring.cu): spectra of the kernel tables and the twiddles exp(-2 pi i m / N), m < N/2,
    // in the FFT's arithmetic type (double2 or float2)
    const void* khat;
    const void* vhat;
    const void* twid;
    // tensor-core form (ring.cu): per column block e of 128, the 128 x 128 Toeplitz block of V' (tcK)
    // or V (tcV) as shared-memory images (TF32 high part, then low part)
    const void* tcK;
    const void* tcV;
    long long* tcacc;        // [N] exact fixed-point sums of the blocks' partial results (scale 2^tcq)
    int tcq;
    unsigned int* tcticket;
    int* err;                // device error flag of the handle (bounded waits that gave up)
};

// Ring force and potential by method (ring.cu): VLASOV_RING_DIRECT runs ring_kernel (FMA in the
// arithmetic type); FIXED the exact fixed-point sum; FFT_F64 / FFT_F32 the shared-memory FFT.
enum : int { RING_M_DIRECT = 1, RING_M_FIXED = 2, RING_M_FFT64 = 3, RING_M_FFT32 = 4, RING_M_TENSOR = 5 };
constexpr int RINGFX_THREADS = 256;
constexpr int RING_FFT_THREADS = 1024;
int ringfx_ksplit(int N, int nsm);
size_t ringfx_smem_bytes(int N, int ksplit);
cudaError_t set_ringfx_attributes(int max_smem);
cudaError_t launch_ring_fixed(const RingArgs& a, cudaStream_t st);
// Fixed-point force of one state and potential (and moment record) of another in one launch.
cudaError_t launch_ring_fixed_dual(const RingArgs& f, const RingArgs& p, cudaStream_t st);
// Batched fixed-point form: grid.y = slot; each slot's split follows its own N (as a single grid),
// the launch covers the split of max_n.
cudaError_t launch_ring_fixed_batch(bool pot, int slots, int max_n, int nsm, const RingArgs* args, cudaStream_t st);
// Host: the fixed-point kernel tables of a ring grid of N nodes (Kq, Vq: N entries; shifts sK, sV).
void ring_fixed_tables(int N, double dx, double eps, long long* Kq, long long* Vq, int* sK, int* sV);
// Tensor-core form: N = 128 N1 (256 <= N <= 4096), one CTA per column block, tcgen05 MMAs in
// 3xTF32 split precision.  Table images: N1 blocks x (hi, lo) x RING_TC_IMG bytes.
constexpr int RING_TC_M = 128;
constexpr int RING_TC_N = 32;                            // MMA N: N1 padded to a multiple of 16 (<= 32)
constexpr size_t RING_TC_IMG = (size_t)RING_TC_M * RING_TC_M * 4;   // one 128 x 128 TF32 block
bool ring_tc_ok(int N);
size_t ring_tc_smem_bytes();
cudaError_t launch_ring_tc(const RingArgs& a, cudaStream_t st);
void ring_tc_tables(const double* table, int N, float* images);   // images: N/128 x 2 x 128 x 128 floats
bool ring_fft_ok(int N);
size_t ring_fft_smem_bytes(int N, bool f64);
cudaError_t launch_ring_fft(bool f64, const RingArgs& a, cudaStream_t st);
// Host: exact DFT of a real table (FP64 accumulation over an FP64 twiddle table), out[2k] = Re, out[2k+1] = Im.
void ring_dft_host(const double* v, int N, double* out);

// ---------------------------------------------------------------------------------------------
// Launchers (return cudaError_t of the launch).
constexpr int XS_THREADS_MIN = 256;
constexpr int XS_THREADS_MAX = 512;   // 8-byte rows longer than 256 threads cover (Nx <= 8192)
int xshift_max_cols(int elem_bytes, int threads);
size_t xshift_smem_bytes(int Nx, int pad, int stages, int elem_bytes);
cudaError_t launch_xshift(int elem_bytes, bool periodic, bool kin, int grid, int threads,
                          const XShiftArgs& a, cudaStream_t st);

constexpr int PS_TW = 32;        // columns per tile (one warp lane per column)
constexpr int PS_RG = 8;         // row groups (warps) per CTA
constexpr int PS_RPT = 16;       // output rows per thread
constexpr int PS_TH = PS_RG * PS_RPT;  // output rows per tile
constexpr int PS_BH = 32;        // rows per TMA box
constexpr int PS_RB = 256;       // staged rows per buffer
static_assert(PS_RB % PS_BH == 0, "a staged window is whole TMA boxes: the slot must hold nb * PS_BH rows");
// FP32-class p-shift: PS_RG compute warps and one producer warp per CTA, PS_NB staged tiles in flight
constexpr int PS_THREADS = PS_TW * (PS_RG + 1);
constexpr int PS_NB = 2;
constexpr int PS_MINB = 3;       // CTAs per SM the register budget is set for, 4-byte storage (faster than 2)
size_t pshift_smem_bytes(int elem_bytes);
// hf (may be NULL): form the HMF filters inside the launch (4-byte and 2-byte storage)
cudaError_t launch_pshift(int elem_bytes, bool p_periodic, int grid, const CUtensorMap* tmap,
                          const PShiftArgs& a, const HmfFiltArgs* hf, cudaStream_t st);

// Opt a kernel into the dynamic shared memory it may use: the per-block limit max_smem less its own
// static shared memory.
template <typename K>
inline cudaError_t allow_dynamic_smem(K kernel, int max_smem)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
}
cudaError_t set_kernel_attributes(int max_smem);
cudaError_t set_kernel_attributes_e(int max_smem);
int xshift_e_max_cols(int threads);
int xshift_fx_max_cols(int threads);
size_t pshift_e_smem_bytes();
cudaError_t xshift_e_occupancy(bool periodic, int threads, size_t smem, int* blocks);
cudaError_t pshift_e_occupancy(int* blocks);
cudaError_t launch_xshift_e(bool periodic, bool kin, int grid, int threads, const XShiftArgs& a, const EmulArgs& em,
                            cudaStream_t st);
cudaError_t launch_pshift_e(bool p_periodic, int grid, const CUtensorMap* tmap, const PShiftArgs& a, const EmulArgs& em,
                            cudaStream_t st);
cudaError_t xshift_occupancy(int elem_bytes, bool periodic, int threads, size_t smem, int* blocks);
cudaError_t pshift_occupancy(int elem_bytes, int* blocks);

cudaError_t set_kernel_attributes_fx(int max_smem);
size_t pshift_fx_smem_bytes();
cudaError_t xshift_fx_occupancy(bool periodic, int threads, size_t smem, int* blocks);
cudaError_t pshift_fx_occupancy(int* blocks);
int pshift_fx_tile_rows();   // output rows per tile of the single-grid FX64 p-shift
cudaError_t launch_xshift_fx(bool periodic, bool kin, int grid, int threads, const XShiftArgs& a, const EmulArgs& em,
                             cudaStream_t st);
// Global-spline sweeps (IEEE FP64 or FP32 storage and arithmetic).
size_t gs_xshift_smem_bytes(int Nx, int elem_bytes);
size_t gs_pshift_smem_bytes(int elem_bytes);
cudaError_t launch_gs_xshift(int elem_bytes, bool periodic, bool kin, int grid, const XShiftArgs& a, cudaStream_t st);
cudaError_t launch_gs_pshift(int elem_bytes, bool p_periodic, int grid, const PShiftArgs& a, cudaStream_t st);
cudaError_t gs_occupancy(int elem_bytes, bool xdir, size_t smem, int* blocks);

// Fused x-shifts with FP32-class storage (elem_bytes 4: FP32, 2: BF16): XXS_THREADS threads share
// rows of up to XXS_MAX_NX columns; XXS_CTAS_PER_SM CTAs per SM.
constexpr int XXS_THREADS = 512;
constexpr int XXS_CTAS_PER_SM = 2;
constexpr int XXS_MAX_NX = 4096;
size_t xxshift_smem_bytes(int Nx, int pad, int stages, int elem_bytes);
cudaError_t launch_xxshift(int elem_bytes, bool periodic, int grid, const XShiftArgs& a, const XShiftArgs& b,
                           cudaStream_t st);
cudaError_t xxshift_occupancy(int elem_bytes, bool periodic, size_t smem, int* blocks);

// Fused x-shifts (second half of step n, first half of step n+1) with FX64 storage.
constexpr int XXF_THREADS_MAX = 512;   // one chunk of 8 columns per thread: Nx <= 4096
constexpr int XF_FUSED_MAX_NX = 8 * XXF_THREADS_MAX;
int xxshift_fx_row_bytes(int Nx, int pad, bool periodic);   // one padded row in shared memory
size_t xxshift_fx_smem_bytes(int Nx, int pad, int stages);
int xxshift_fx_threads(int Nx);
cudaError_t xxshift_fx_occupancy(bool periodic, int Nx, size_t smem, int* blocks);
// tmap: f as a 2-D tensor of 8-element lines ({8, Nx * Np / 8}, 64-byte stride) with a box of
// {10, a.box_h} (the two extra columns read as zeros: padded rows in shared memory).
cudaError_t launch_xxshift_fx(bool periodic, int grid, const CUtensorMap* tmap, const XShiftArgs& a, const XShiftArgs& b,
                              const EmulArgs& em, cudaStream_t st);
cudaError_t launch_pshift_fx(bool p_periodic, int grid, const CUtensorMap* tmap, const PShiftArgs& a,
                             const EmulArgs& em, cudaStream_t st);
// Casimirs (entropy, integral of f^2) of a stored f: kind 0 FX64 (unit = 2^(Ef-61)), 1 double, 2 float.
constexpr int CAS_BLOCKS = 8 * 152;
cudaError_t launch_casimirs(int kind, const void* f, size_t n, double unit, double dxdp, double* part, double* out,
                            cudaStream_t st);
cudaError_t launch_f64_to_fx(const double* s, long long* d, size_t n, int Ef, cudaStream_t st);
// Failure-path check: one CTA waits on an mbarrier that nothing arrives on, with the bounded wait
// of the sweep kernels and the given limit, then records DEV_ERR_TEST_WAIT in *err and returns.
cudaError_t launch_expire_wait(int* err, unsigned long long limit_ns, cudaStream_t st);
// Waterbag initial states (Sec. 4) written on the device; see aux_kernels.cu.
constexpr int WB_BLOCKS = 4 * 152;
constexpr int WB_THREADS = 256;
struct WaterbagArgs {
    const double* rowv;          // [Np] momentum profile (device)
    const double* colv;          // [Nx] position profile (device)
    int Nx, Np;
    double noise;                // 0: no noise
    unsigned long long seed;
    int k_m;                     // fixed-point shift of the exact mass sum
    double dxdp;
    void* part;                  // int128 [WB_BLOCKS]
    unsigned int* ticket;
    double* mass;                // out: dx dp sum of the unnormalised f
    unsigned long long* maxbits; // out: bits of the largest |f| after normalisation
};
// f (elem_bytes 8: double, 4: float, 2: bf16) = the normalised state; two launches, no sync.
cudaError_t launch_waterbag(const WaterbagArgs& a, int elem_bytes, void* f, cudaStream_t st);
cudaError_t launch_fx_to_f64(const long long* s, double* d, size_t n, int Ef, cudaStream_t st);
cudaError_t launch_colsum_fx(const long long* f, int Nx, int Np, int Ef, double* colpart, cudaStream_t st);

cudaError_t launch_colreduce(const ColReduceArgs& a, int grid, cudaStream_t st);
// Two reductions of exact per-CTA partial rows (colpart64) in one launch.
cudaError_t launch_colreduce_p64_dual(const ColReduceArgs& a, const ColReduceArgs& b, cudaStream_t st);

// Batched forms (FP32 or FX64 storage): grid.y = slot; per-slot arguments (two buffer parities
// for the sweeps) live in device arrays, so one captured graph serves any set of occupied slots.
cudaError_t launch_xshift_batch(bool periodic, bool kin, int slots, int ctas_per_slot, size_t smem,
                                const XShiftArgs* args, const int* ver, cudaStream_t st);
cudaError_t launch_pshift_batch(int slots, int ctas_per_slot, const CUtensorMap* tmaps, const PShiftArgs* args,
                                const int* ver, cudaStream_t st);
cudaError_t launch_xshift_fx_batch(bool periodic, bool kin, int slots, int ctas_per_slot, size_t smem,
                                   const XShiftArgs* args, const EmulArgs* ems, const int* ver, cudaStream_t st);
cudaError_t launch_pshift_fx_batch(int slots, int ctas_per_slot, const CUtensorMap* tmaps, const PShiftArgs* args,
                                   const EmulArgs* ems, const int* ver, cudaStream_t st);
cudaError_t launch_colreduce_batch(int slots, int blocks_per_slot, const ColReduceArgs* args, cudaStream_t st);
cudaError_t launch_pparams_batch(int elem_bytes, int slots, int max_n, const PParamsArgs* args, cudaStream_t st);
cudaError_t launch_pparams(int elem_bytes, const PParamsArgs& a, cudaStream_t st);
// HMF, 8-byte storage, from the x-shift's per-CTA partials: force and p-shift parameters
// (pparams_hmf_cta), and the moments after the second x-shift (colreduce_cta, one block).
cudaError_t launch_pparams_hmf_cta(int elem_bytes, const PParamsArgs& a, cudaStream_t st);
cudaError_t set_ring_attributes(int max_smem);
cudaError_t launch_colreduce_cta(const ColReduceArgs& a, cudaStream_t st);
cudaError_t launch_ring(int elem_bytes, const RingArgs& a, cudaStream_t st);
int ring_blocks(int N);
cudaError_t launch_colsum(int elem_bytes, const void* f, int Nx, int Np, double* colpart, int B,
                          cudaStream_t st);
void set_last_error(const char* msg);   // text returned by vlasov_last_error() on this thread

cudaError_t launch_convert(const void* src, int src_bytes, void* dst, int dst_bytes, size_t n,
                           cudaStream_t st);
cudaError_t launch_maxabs(int elem_bytes, const void* f, size_t n, unsigned long long* out, cudaStream_t st);

}  // namespace vl
