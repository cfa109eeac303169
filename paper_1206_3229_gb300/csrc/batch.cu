// batch.cu -- many grids of uneven size and different models advanced together (FP32 storage, or
// FX64: the FP64-accurate 64-bit fixed point of shift_fx.cu), and a continuous-batching serving
// loop on top.
//
// A batch has a fixed number of slots.  Every slot owns its buffers inside one device arena (a
// first-fit allocator over a single allocation, so admission is limited by HBM footprint, not by a
// fixed per-slot size).  The kernels of a Strang step are the single-grid kernels launched once per
// sub-step with gridDim.y = slots: each CTA reads its slot's arguments from device arrays (two
// copies per sweep, one per buffer parity, selected by a per-slot parity word that a one-block
// kernel flips at the end of the step).  Free slots carry zero sizes and exit at once.  Because the
// launch parameters never change, one captured CUDA graph runs every batched step, whatever the
// occupancy; admission and retirement only rewrite a slot's argument entries in stream order.
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <thread>
#include <vector>

#include "../../include/vlasov.h"
#include "emul.cuh"
#include "fixed_point.cuh"
#include "vlasov_internal.cuh"

using namespace vl;

namespace {

constexpr int B_CTAS_X_MAX = 512;   // most x-shift CTAs per slot (sizes the kinetic partials)
constexpr int B_ROWS_PER_CTA = 16;  // default x-shift rows per CTA (the CTA count of a slot depends on its Np only)
constexpr int B_TILES_PER_CTA = 8;  // default p-shift tiles per CTA of the largest grid of a batch
constexpr int B_PAD_ZERO = 64;   // zero halo of non-periodic rows (|x displacement| <= 55 cells)
constexpr int B_STAGES = 3;
constexpr int B_INIT_BLOCKS = 128;

int slot_ctas_x(int Np, int rows_per_cta)
{
    return std::min(B_CTAS_X_MAX, std::max(16, (Np + rows_per_cta - 1) / rows_per_cta));
}

int bfail(int code, const char* msg)
{
    set_last_error(msg);
    return code;
}

#define B_TRY(expr)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            char b_[256];                                                                      \
            snprintf(b_, sizeof b_, "%s: %s", #expr, cudaGetErrorString(e_));                  \
            return bfail(e_ == cudaErrorMemoryAllocation ? VLASOV_ENOMEM : VLASOV_ECUDA, b_);  \
        }                                                                                      \
    } while (0)

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

int clog2(double v)
{
    int e = 0;
    const double m = std::frexp(v, &e);
    return m == 0.5 ? e - 1 : e;
}

// ------------------------------------------------------------------------------------------- arena
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes, coalesced

    bool alloc(size_t bytes, size_t* off)
    {
        bytes = al256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = al256(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// ------------------------------------------------------------------------------------------- device init
// f_ij = rowv[j] * colv[i] * (1 + noise * xi_ij) in FP32, xi from the (j*Nx+i+1)-th SplitMix64 output
// of `seed` (top 24 bits); the int128 fixed-point sum of f gives the mass, the last block stores
// 1/mass; a second kernel scales f to unit mass.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long k)
{
    unsigned long long z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct InitArgs {
    float* f;
    int Nx, Np;
    const float* rowv;
    const float* colv;
    float noise;
    unsigned long long seed;
    int k_m;                 // fixed-point shift of the mass sum
    double dxdp;
    void* part;              // int128 [B_INIT_BLOCKS]
    unsigned int* ticket;
    double* inv_mass;
};

__global__ void __launch_bounds__(256) init_fill_kernel(InitArgs a)
{
    __shared__ i128 red[33];
    __shared__ bool is_last;
    const size_t n = (size_t)a.Nx * a.Np;
    i128 acc = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / a.Nx), i = (int)(k - (size_t)j * a.Nx);
        float v = a.rowv[j] * a.colv[i];
        if (v != 0.f && a.noise != 0.f) {
            const unsigned long long z = splitmix64_at(a.seed, (unsigned long long)k + 1ull);
            const float xi = __uint2float_rn((unsigned int)(z >> 40)) * 1.1920928955078125e-07f - 1.0f;   // 2u - 1
            v = v * (1.0f + a.noise * xi);
        }
        a.f[k] = v;
        acc += fx128_from_f32(v, a.k_m);
    }
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
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += vp[b];
    t = block_sum_i128(t, red);
    if (threadIdx.x == 0) {
        const double mass = a.dxdp * fx128_to_f64(t, a.k_m);
        *a.inv_mass = mass > 0 ? 1.0 / mass : 0.0;
        *a.ticket = 0u;
    }
}

__global__ void init_scale_kernel(float* f, size_t n, const double* inv_mass)
{
    const float s = (float)*inv_mass;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) f[k] *= s;
}

__global__ void flip_kernel(int* ver, int slots)
{
    for (int s = threadIdx.x; s < slots; s += blockDim.x) ver[s] ^= 1;
}

// FX64 slots: the same initial state in FP64 (xi from the top 53 bits of the SplitMix64 output, as
// the shared input generator draws it), its exact fixed-point mass, then scaling to unit mass and
// conversion to the fixed-point storage.
struct InitArgs64 {
    double* f;               // FP64 staging (the slot's second f buffer)
    int Nx, Np;
    const double* rowv;
    const double* colv;
    double noise;
    unsigned long long seed;
    int k_m;
    double dxdp;
    void* part;
    unsigned int* ticket;
    double* inv_mass;
};

__global__ void __launch_bounds__(256) init_fill64_kernel(InitArgs64 a)
{
    __shared__ i128 red[33];
    __shared__ bool is_last;
    const size_t n = (size_t)a.Nx * a.Np;
    i128 acc = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / a.Nx), i = (int)(k - (size_t)j * a.Nx);
        double v = a.rowv[j] * a.colv[i];
        if (v != 0.0 && a.noise != 0.0) {
            const unsigned long long z = splitmix64_at(a.seed, (unsigned long long)k + 1ull);
            const double xi = 2.0 * ((double)(z >> 11) * 1.1102230246251565e-16) - 1.0;   // 2u - 1, u = top 53 bits
            v = v * (1.0 + a.noise * xi);
        }
        a.f[k] = v;
        acc += fx128_from_f64(v, a.k_m);
    }
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
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += vp[b];
    t = block_sum_i128(t, red);
    if (threadIdx.x == 0) {
        const double mass = a.dxdp * fx128_to_f64(t, a.k_m);
        *a.inv_mass = mass > 0 ? 1.0 / mass : 0.0;
        *a.ticket = 0u;
    }
}

__global__ void init_scale_fx_kernel(const double* src, long long* dst, size_t n, const double* inv_mass, int k)
{
    const double s = *inv_mass;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        dst[q] = (long long)fx128_from_f64(src[q] * s, k);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// ------------------------------------------------------------------------------------------- slot layout
struct SlotLayout {
    size_t f[2], xrec, pn0, pw, pgd, pWh, pwl, pwf, pWhe, pwle, pwfe, colpart, colacc, kinpart, rho, F, Qd, colfx, blockpart,
        tickets, sc, hist, dstep, err, costab, sintab, cosfx, sinfx, rowv, colv, initpart, inv_mass,
        ringKq, ringVq, ringgpart, ringgticket, ringupart, total;
};

// esz: bytes per cell (4: FP32 storage, 8: FX64 storage)
// Largest split of the ring's fixed-point sums for Nx nodes (the split itself follows the device).
int ring_split_of(int Nx) { return std::max(1, Nx / 256); }

SlotLayout layout(int Nx, int Np, int esz)
{
    SlotLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o += al256(bytes);
        return r;
    };
    const size_t cells = (size_t)Nx * Np;
    L.f[0] = take(cells * esz);
    L.f[1] = take(cells * esz);
    L.xrec = take((size_t)Np * XREC_BYTES);
    L.pn0 = take((size_t)Nx * 4);
    L.pw = take((size_t)NTAP * Nx * esz);
    L.pgd = take((size_t)2 * Nx * esz);
    L.pWh = esz == 8 ? take((size_t)NTAP * Nx * 4) : 0;
    L.pwl = esz == 8 ? take((size_t)NTAP * Nx * 4) : 0;
    L.pwf = esz == 8 ? take((size_t)NTAP * Nx * 4) : 0;
    L.pWhe = esz == 8 ? take((size_t)2 * NTAP * Nx * 4) : 0;   // edge filters of the zero-outside p columns
    L.pwle = esz == 8 ? take((size_t)2 * NTAP * Nx * 4) : 0;
    L.pwfe = esz == 8 ? take((size_t)2 * NTAP * Nx * 4) : 0;
    L.colacc = take((size_t)Nx * 8);
    L.kinpart = take((size_t)B_CTAS_X_MAX * 16);   // FP64 (F32 storage) or int128 (FX64) per CTA
    L.rho = take((size_t)Nx * 8);
    L.F = take((size_t)Nx * 8);
    L.Qd = take((size_t)Nx * 8);
    L.colfx = take((size_t)Nx * 8);
    L.blockpart = take((size_t)((Nx + 31) / 32) * 48);
    L.tickets = take(16);
    L.sc = take(sizeof(Scalars));
    L.hist = take(sizeof(MomentRec) * HIST_CAP);
    L.dstep = take(8);
    L.err = take(8);
    L.costab = take((size_t)Nx * 8);
    L.sintab = take((size_t)Nx * 8);
    L.cosfx = take((size_t)Nx * 8);
    L.sinfx = take((size_t)Nx * 8);
    L.rowv = take((size_t)Np * esz);
    L.colv = take((size_t)Nx * esz);
    L.initpart = take((size_t)B_INIT_BLOCKS * 16);
    L.inv_mass = take(8);
    // ring: exact fixed-point force and potential (ring.cu); a slot's split follows its own Nx
    L.ringKq = take((size_t)Nx * 8);
    L.ringVq = take((size_t)Nx * 8);
    L.ringgpart = take((size_t)16 * ring_split_of(Nx) * Nx);
    L.ringgticket = take((size_t)((Nx + 31) / 32) * 4);
    L.ringupart = take((size_t)((Nx + 31) / 32) * 16);
    L.total = o;
    return L;
}

struct Slot {
    bool used = false;       // buffers allocated (admitted, possibly finished and draining)
    bool active = false;     // advanced by batched steps
    vlasov_request req;
    size_t off = 0, bytes = 0;
    SlotLayout L;
    int steps_done = 0;
    int Ef = 0, k_col = 0, k_kin = 0, k_pot = 0;
    int ring_sK = 0, ring_sV = 0;   // shifts of the ring's fixed-point kernel tables
    double admit_s = 0;
    int done_event = -1;     // index into the step-event ring of the step that finished it
    long long result_index = -1;
};

}  // namespace

// ------------------------------------------------------------------------------------------- the batch
struct vlasov_batch {
    int S = 0, max_n = 0;
    int prec = VLASOV_F32;           // VLASOV_F32 or VLASOV_FX64, for every slot
    int esz = 4;
    int ctas_x = 16, ctas_p = 32;    // CTAs per slot of the batched sweeps (fixed at capture)
    int nsm = 0;                     // SMs of the device (the ring sums' split follows it)
    vlasov_batch_shape shape = {B_ROWS_PER_CTA, B_TILES_PER_CTA};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    Arena arena;
    std::vector<Slot> slots;
    // device argument arrays and their host mirrors
    XShiftArgs* d_xa = nullptr;      // [4][S][2]: periodic/zero x (step 1), periodic/zero x (step 4)
    PShiftArgs* d_pa = nullptr;      // [S][2]
    CUtensorMap* d_tm = nullptr;     // [S][2]
    ColReduceArgs* d_cr = nullptr;   // [2][S]: after step 1, after step 4
    RingArgs* d_rg = nullptr;        // [2][S]
    PParamsArgs* d_pp = nullptr;     // [S]
    EmulArgs* d_em = nullptr;        // [S] (FX64)
    int* d_ver = nullptr;            // [S]
    std::vector<XShiftArgs> xa;
    std::vector<PShiftArgs> pa;
    std::vector<CUtensorMap> tm;
    std::vector<ColReduceArgs> cr;
    std::vector<RingArgs> rg;
    std::vector<PParamsArgs> pp;
    std::vector<EmulArgs> em;
    size_t xsmem = 0;
    cudaGraphExec_t graph = nullptr;
    long long steps_launched = 0;
};

namespace {

char* P(vlasov_batch* b, const Slot& s, size_t off) { return b->arena.base + s.off + off; }

void clear_slot_args(vlasov_batch* b, int k)
{
    for (int kind = 0; kind < 4; ++kind)
        for (int v = 0; v < 2; ++v) {
            XShiftArgs& a = b->xa[((size_t)kind * b->S + k) * 2 + v];
            a = XShiftArgs{};
            a.Np = 0;
            a.Nx = 0;
        }
    for (int v = 0; v < 2; ++v) {
        PShiftArgs& a = b->pa[(size_t)k * 2 + v];
        std::memset(&a, 0, sizeof a);
    }
    for (int q = 0; q < 2; ++q) {
        std::memset(&b->cr[(size_t)q * b->S + k], 0, sizeof(ColReduceArgs));
        std::memset(&b->rg[(size_t)q * b->S + k], 0, sizeof(RingArgs));
    }
    std::memset(&b->pp[k], 0, sizeof(PParamsArgs));
    std::memset(&b->em[k], 0, sizeof(EmulArgs));
}

int upload_slot_args(vlasov_batch* b, int k)
{
    const size_t S = b->S;
    for (int kind = 0; kind < 4; ++kind)
        B_TRY(cudaMemcpyAsync(b->d_xa + (kind * S + k) * 2, &b->xa[(kind * S + k) * 2], 2 * sizeof(XShiftArgs),
                              cudaMemcpyHostToDevice, b->st));
    B_TRY(cudaMemcpyAsync(b->d_pa + (size_t)k * 2, &b->pa[(size_t)k * 2], 2 * sizeof(PShiftArgs), cudaMemcpyHostToDevice, b->st));
    B_TRY(cudaMemcpyAsync(b->d_tm + (size_t)k * 2, &b->tm[(size_t)k * 2], 2 * sizeof(CUtensorMap), cudaMemcpyHostToDevice, b->st));
    for (int q = 0; q < 2; ++q) {
        B_TRY(cudaMemcpyAsync(b->d_cr + q * S + k, &b->cr[q * S + k], sizeof(ColReduceArgs), cudaMemcpyHostToDevice, b->st));
        B_TRY(cudaMemcpyAsync(b->d_rg + q * S + k, &b->rg[q * S + k], sizeof(RingArgs), cudaMemcpyHostToDevice, b->st));
    }
    B_TRY(cudaMemcpyAsync(b->d_pp + k, &b->pp[k], sizeof(PParamsArgs), cudaMemcpyHostToDevice, b->st));
    B_TRY(cudaMemcpyAsync(b->d_em + k, &b->em[k], sizeof(EmulArgs), cudaMemcpyHostToDevice, b->st));
    return VLASOV_OK;
}

// Fill the argument entries of an occupied slot (both buffer parities) from its layout.
int fill_slot_args(vlasov_batch* b, int k)
{
    Slot& s = b->slots[k];
    const vlasov_request& r = s.req;
    const int Nx = r.Nx, Np = r.Np;
    const double dx = (r.xmax - r.xmin) / Nx, dp = (r.pmax - r.pmin) / Np;
    const bool per = r.x_periodic != 0;
    void* fbuf[2] = {P(b, s, s.L.f[0]), P(b, s, s.L.f[1])};
    for (int v = 0; v < 2; ++v) {          // v = buffer holding f at the start of the step
        for (int step4 = 0; step4 < 2; ++step4) {
            for (int kind_per = 0; kind_per < 2; ++kind_per) {
                const int kind = step4 * 2 + (kind_per ? 0 : 1);   // 0 per/step1, 1 zero/step1, 2 per/step4, 3 zero/step4
                XShiftArgs& a = b->xa[((size_t)kind * b->S + k) * 2 + v];
                a = XShiftArgs{};
                if ((kind_per == 1) != per) {
                    a.Nx = a.Np = 0;
                    continue;
                }
                a.rec = P(b, s, s.L.xrec);
                a.fin = fbuf[v];          // both x half-shifts of the step read buffer v
                a.fout = fbuf[v ^ 1];
                a.Nx = Nx;
                a.Np = Np;
                a.pad = per ? 16 : B_PAD_ZERO;
                a.stages = B_STAGES;
                a.n0 = nullptr;
                a.w = nullptr;
                a.gd = nullptr;
                a.colpart = nullptr;
                a.colacc = reinterpret_cast<unsigned long long*>(P(b, s, s.L.colacc));
                a.k_col = s.k_col;
                a.kinpart = step4 ? reinterpret_cast<double*>(P(b, s, s.L.kinpart)) : nullptr;
                a.kin128 = (step4 && b->esz == 8) ? P(b, s, s.L.kinpart) : nullptr;   // FX64: exact
                a.pmin = r.pmin;
                a.dp = dp;
                a.err = reinterpret_cast<int*>(P(b, s, s.L.err));
                a.ctas = slot_ctas_x(Np, b->shape.rows_per_cta);
            }
        }
        // p-shift: reads the other buffer, writes back into v
        PShiftArgs& pa = b->pa[(size_t)k * 2 + v];
        pa.fin = fbuf[v ^ 1];
        pa.fout = fbuf[v];
        pa.Nx = Nx;
        pa.Np = Np;
        pa.n0 = reinterpret_cast<const int*>(P(b, s, s.L.pn0));
        pa.w = P(b, s, s.L.pw);
        pa.gd = P(b, s, s.L.pgd);
        pa.err = reinterpret_cast<int*>(P(b, s, s.L.err));
        auto enc = encode_tiled();
        if (!enc) return bfail(VLASOV_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
        cuuint64_t dims[2] = {(cuuint64_t)Nx, (cuuint64_t)Np};
        cuuint64_t strides[1] = {(cuuint64_t)Nx * b->esz};
        cuuint32_t box[2] = {(cuuint32_t)PS_TW, (cuuint32_t)PS_BH};
        cuuint32_t estr[2] = {1, 1};
        const CUtensorMapDataType dt = b->esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_INT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        if (enc(&b->tm[(size_t)k * 2 + v], dt, 2, fbuf[v ^ 1], dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return bfail(VLASOV_ECUDA, "cuTensorMapEncodeTiled failed for a batch slot");
    }
    const int B = std::min(slot_ctas_x(Np, b->shape.rows_per_cta), Np);
    for (int q = 0; q < 2; ++q) {
        ColReduceArgs& c = b->cr[(size_t)q * b->S + k];
        c.colacc = reinterpret_cast<unsigned long long*>(P(b, s, s.L.colacc));
        c.colpart = nullptr;   // the x-shifts add exact column sums into colacc
        c.B = B;
        c.kinpart = (q && b->esz == 4) ? reinterpret_cast<const double*>(P(b, s, s.L.kinpart)) : nullptr;
        c.kin128 = (q && b->esz == 8) ? P(b, s, s.L.kinpart) : nullptr;   // exact sum of int128 partials
        c.kin_frac = 51 + KIN_Q - s.Ef;
        c.Nx = Nx;
        c.k_col = s.k_col;
        c.k_kin = s.k_kin;
        c.k_pot = s.k_pot;
        c.dp = dp;
        c.dxdp = dx * dp;
        c.pot_scale = 2.0 * 3.14159265358979323846 * r.G * dx * dx * dx * dp * dp;
        c.cosfx = reinterpret_cast<const long long*>(P(b, s, s.L.cosfx));
        c.sinfx = reinterpret_cast<const long long*>(P(b, s, s.L.sinfx));
        c.rho = reinterpret_cast<double*>(P(b, s, s.L.rho));
        c.colfx = reinterpret_cast<long long*>(P(b, s, s.L.colfx));
        c.Qd = reinterpret_cast<double*>(P(b, s, s.L.Qd));
        c.blockpart = P(b, s, s.L.blockpart);
        c.ticket = reinterpret_cast<unsigned int*>(P(b, s, s.L.tickets));
        c.sc = reinterpret_cast<Scalars*>(P(b, s, s.L.sc));
        c.model = r.model;
        c.final_moments = q;
        c.hist = reinterpret_cast<MomentRec*>(P(b, s, s.L.hist));
        c.step = reinterpret_cast<long long*>(P(b, s, s.L.dstep));
        c.dt = r.dt;
        RingArgs& g = b->rg[(size_t)q * b->S + k];
        std::memset(&g, 0, sizeof g);
        if (r.model == VLASOV_RING) {
            g.N = Nx;
            g.dx = dx;
            g.rho = c.rho;
            g.F = reinterpret_cast<double*>(P(b, s, s.L.F));
            g.k_pot = s.k_pot;
            g.pot_scale = 0.5 * dx;
            g.ticket = reinterpret_cast<unsigned int*>(P(b, s, s.L.tickets)) + 1;
            g.sc = c.sc;
            g.final_moments = q;
            g.hist = c.hist;
            g.step = c.step;
            g.dt = r.dt;
            g.colfx = c.colfx;
            g.Kq = reinterpret_cast<const long long*>(P(b, s, s.L.ringKq));
            g.Vq = reinterpret_cast<const long long*>(P(b, s, s.L.ringVq));
            g.k_col = s.k_col;
            g.sK = s.ring_sK;
            g.sV = s.ring_sV;
            g.dp = dp;
            g.ksplit = ringfx_ksplit(Nx, b->nsm);
            g.gpart = P(b, s, s.L.ringgpart);
            g.gticket = reinterpret_cast<unsigned int*>(P(b, s, s.L.ringgticket));
            g.upart = P(b, s, s.L.ringupart);
        }
    }
    PParamsArgs& p = b->pp[k];
    p.Nx = Nx;
    p.model = r.model;
    p.sc = reinterpret_cast<const Scalars*>(P(b, s, s.L.sc));
    p.costab = reinterpret_cast<const double*>(P(b, s, s.L.costab));
    p.sintab = reinterpret_cast<const double*>(P(b, s, s.L.sintab));
    p.Fin = reinterpret_cast<const double*>(P(b, s, r.model == VLASOV_SHEET ? s.L.Qd : s.L.F));
    p.Fscale = -2.0 * 3.14159265358979323846 * r.G * dx * dp;
    p.cp = r.dt / dp;
    p.n0 = reinterpret_cast<int*>(P(b, s, s.L.pn0));
    p.w = P(b, s, s.L.pw);
    p.gd = P(b, s, s.L.pgd);
    p.Fout = nullptr;
    const bool fx = b->esz == 8;
    p.Wh = fx ? reinterpret_cast<int*>(P(b, s, s.L.pWh)) : nullptr;
    p.wl = fx ? reinterpret_cast<float*>(P(b, s, s.L.pwl)) : nullptr;
    p.wf = fx ? reinterpret_cast<float*>(P(b, s, s.L.pwf)) : nullptr;
    p.Whe = fx ? reinterpret_cast<int*>(P(b, s, s.L.pWhe)) : nullptr;
    p.wle = fx ? reinterpret_cast<float*>(P(b, s, s.L.pwle)) : nullptr;
    p.wfe = fx ? reinterpret_cast<float*>(P(b, s, s.L.pwfe)) : nullptr;
    EmulArgs& e = b->em[k];
    std::memset(&e, 0, sizeof e);
    if (fx) {
        e.Ef = s.Ef;
        e.n0 = p.n0;
        e.Wh = p.Wh;
        e.wl = p.wl;
        e.wf = p.wf;
        e.gd = reinterpret_cast<const double*>(p.gd);
        e.w64 = reinterpret_cast<const double*>(p.w);
        e.Whe = p.Whe;
        e.wle = p.wle;
        e.wfe = p.wfe;
    }
    return VLASOV_OK;
}

int validate_request(const vlasov_request* r, int max_n)
{
    if (!r) return bfail(VLASOV_EINVAL, "NULL request");
    if (r->model < VLASOV_HMF || r->model > VLASOV_FREE) return bfail(VLASOV_EINVAL, "unknown model");
    if (r->Nx < 16 || r->Np < 16 || r->Nx % 8 || r->Np % 8) return bfail(VLASOV_EINVAL, "Nx, Np: multiples of 8, >= 16");
    if (r->Nx > max_n || r->Np > max_n) return bfail(VLASOV_EINVAL, "grid larger than the batch maximum");
    if (!(r->dt > 0) || !(r->xmax > r->xmin) || !(r->pmax > r->pmin)) return bfail(VLASOV_EINVAL, "bad domain or dt");
    if (r->model == VLASOV_RING && !(r->eps > 0)) return bfail(VLASOV_EINVAL, "ring needs eps > 0");
    if (std::max(std::fabs(r->pmin), std::fabs(r->pmax)) >= 2896.0)
        return bfail(VLASOV_EINVAL, "|p| must stay below 2896 (fixed-point kinetic weights)");
    if (r->steps < 0) return bfail(VLASOV_EINVAL, "steps < 0");
    return VLASOV_OK;
}

// Launch shapes picked by vlasov_batch_autotune, per (device, max_n, precision), for this process.
std::mutex g_shape_mu;
std::map<std::tuple<int, int, int>, vlasov_batch_shape> g_shapes;

void tuned_shape(int max_n, int precision, vlasov_batch_shape* out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_shapes.find(std::make_tuple(dev, max_n, precision));
    *out = it != g_shapes.end() ? it->second : vlasov_batch_shape{B_ROWS_PER_CTA, B_TILES_PER_CTA};
}

}  // namespace

// ================================================================================== C ABI
extern "C" {

void vlasov_batch_destroy(vlasov_batch* b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->arena.base);
    void* bufs[] = {b->d_xa, b->d_pa, b->d_tm, b->d_cr, b->d_rg, b->d_pp, b->d_em, b->d_ver};
    for (void* p : bufs) cudaFree(p);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
}

int vlasov_batch_create(int slots, int max_n, long long mem_budget_bytes, int precision, void* stream,
                        vlasov_batch** out)
{
    return vlasov_batch_create_shaped(slots, max_n, mem_budget_bytes, precision, stream, nullptr, out);
}

int vlasov_batch_shape_of(const vlasov_batch* b, vlasov_batch_shape* out)
{
    if (!b || !out) return bfail(VLASOV_EINVAL, "NULL argument");
    *out = b->shape;
    return VLASOV_OK;
}

int vlasov_batch_autotune(int max_n, int precision, void* stream, vlasov_batch_shape* best, double* ms_per_step)
{
    if (!best) return bfail(VLASOV_EINVAL, "best is NULL");
    static const int R[4] = {8, 16, 32, 64}, T[4] = {2, 4, 8, 16};
    // eight synthetic HMF waterbags: two each of max_n, max_n/2, max_n/4, max_n/8 (>= 16)
    std::vector<vlasov_request> reqs;
    long long budget = 1 << 20;
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 2; ++c) {
            vlasov_request r;
            std::memset(&r, 0, sizeof r);
            const int n = std::max(16, (max_n >> k) / 8 * 8);
            r.model = VLASOV_HMF;
            r.Nx = r.Np = n;
            r.xmin = -3.14159265358979323846;
            r.xmax = 3.14159265358979323846;
            r.pmin = -2.0;
            r.pmax = 2.0;
            r.x_periodic = 1;
            r.dt = 0.05;
            r.init = 0;
            r.x0 = 1.5;
            r.p0 = 0.8;
            r.noise = 1e-4;
            r.seed = (unsigned long long)(2 * k + c + 1);
            r.steps = 1000;
            const long long fp = vlasov_batch_footprint(&r, precision);
            if (fp < 0) return bfail(VLASOV_EINVAL, "autotune: precision must be VLASOV_F32 or VLASOV_FX64");
            budget += fp + 4096;
            reqs.push_back(r);
        }
    double best_ms = 0.0;
    int last_rc = VLASOV_OK;
    for (int q = 0; q < 16; ++q) {
        const vlasov_batch_shape sh = {R[q / 4], T[q % 4]};
        if (ms_per_step) ms_per_step[q] = 0.0;
        vlasov_batch* b = nullptr;
        int rc = vlasov_batch_create_shaped(8, max_n, budget, precision, stream, &sh, &b);
        for (size_t k = 0; k < reqs.size() && !rc; ++k) {
            int slot = -1;
            rc = vlasov_batch_admit(b, &reqs[k], nullptr, &slot);
        }
        float ms = 0.f;
        if (!rc) rc = vlasov_batch_step(b, 2);
        if (!rc) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            cudaError_t e = cudaEventCreate(&e0);
            if (e == cudaSuccess) e = cudaEventCreate(&e1);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->st);
            if (e == cudaSuccess) rc = vlasov_batch_step(b, 8);
            if (e == cudaSuccess && !rc) e = cudaEventRecord(e1, b->st);
            if (e == cudaSuccess && !rc) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess && !rc) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (e != cudaSuccess && !rc) {
                char m[256];
                snprintf(m, sizeof m, "autotune timing: %s", cudaGetErrorString(e));
                rc = bfail(VLASOV_ECUDA, m);
            }
        }
        vlasov_batch_destroy(b);
        if (rc) {
            last_rc = rc;
            continue;
        }
        const double per = ms / 8.0;
        if (ms_per_step) ms_per_step[q] = per;
        if (best_ms == 0.0 || per < best_ms) {
            best_ms = per;
            *best = sh;
        }
    }
    if (best_ms == 0.0) return last_rc ? last_rc : bfail(VLASOV_ECUDA, "autotune: no candidate ran");
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shapes[std::make_tuple(dev, max_n, precision)] = *best;
    return VLASOV_OK;
}

int vlasov_batch_create_shaped(int slots, int max_n, long long mem_budget_bytes, int precision, void* stream,
                               const vlasov_batch_shape* shape, vlasov_batch** out)
{
    if (!out) return bfail(VLASOV_EINVAL, "out is NULL");
    *out = nullptr;
    if (slots < 1 || slots > 4096) return bfail(VLASOV_EINVAL, "slots must be in 1..4096");
    if (max_n < 16 || max_n % 8 || max_n > 8192) return bfail(VLASOV_EINVAL, "max_n must be a multiple of 8 in 16..8192");
    if (mem_budget_bytes <= 0) return bfail(VLASOV_EINVAL, "memory budget must be positive");
    if (precision != VLASOV_F32 && precision != VLASOV_FX64)
        return bfail(VLASOV_EINVAL, "batch precision must be VLASOV_F32 or VLASOV_FX64");
    if (precision == VLASOV_FX64 && max_n > xshift_fx_max_cols(XS_THREADS_MIN))
        return bfail(VLASOV_EINVAL, "FX64 batch: max_n above the x-shift row limit");
    if (shape && (shape->rows_per_cta < 1 || shape->rows_per_cta > 4096 || shape->tiles_per_cta < 1 ||
                  shape->tiles_per_cta > 1024))
        return bfail(VLASOV_EINVAL, "batch shape: rows_per_cta in 1..4096, tiles_per_cta in 1..1024");
    vlasov_batch* b = new vlasov_batch();
    if (shape) b->shape = *shape;
    else tuned_shape(max_n, precision, &b->shape);
    b->S = slots;
    b->max_n = max_n;
    b->prec = precision;
    b->esz = precision == VLASOV_FX64 ? 8 : 4;
    // Work per slot grows with its grid while the launch shape is fixed for every slot: the launch
    // has the CTAs the largest grid needs (B_ROWS_PER_CTA rows, B_TILES_PER_CTA tiles each); a slot
    // uses as many x-shift CTAs as its own Np calls for, independent of the batch (so its column and
    // kinetic partial sums, and its results, do not depend on what else is in the batch), and the
    // surplus CTAs exit at once.
    b->ctas_x = slot_ctas_x(max_n, b->shape.rows_per_cta);
    {
        const int th = precision == VLASOV_FX64 ? pshift_fx_tile_rows() : PS_TH;
        const int tiles = ((max_n + PS_TW - 1) / PS_TW) * ((max_n + th - 1) / th);
        b->ctas_p = std::min(1024, std::max(32, tiles / b->shape.tiles_per_cta));
    }
    auto bail = [&](int rc) {
        vlasov_batch_destroy(b);
        return rc;
    };
#define BC(expr)                                  \
    do {                                          \
        int rc_ = [&]() -> int {                  \
            B_TRY(expr);                          \
            return VLASOV_OK;                     \
        }();                                      \
        if (rc_) return bail(rc_);                \
    } while (0)
    if (stream) {
        b->st = static_cast<cudaStream_t>(stream);
    } else {
        BC(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    int dev = 0, optin = 0;
    BC(cudaGetDevice(&dev));
    BC(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    BC(set_kernel_attributes(optin - 1024));
    BC(set_kernel_attributes_fx(optin - 1024));
    BC(set_ringfx_attributes(optin - 1024));
    BC(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
    BC(cudaMalloc(&b->arena.base, (size_t)mem_budget_bytes));
    b->arena.size = (size_t)mem_budget_bytes;
    b->arena.free_[0] = (size_t)mem_budget_bytes;
    b->slots.resize(slots);
    const size_t S = slots;
    b->xa.assign(4 * S * 2, XShiftArgs{});
    b->pa.assign(S * 2, PShiftArgs{});
    b->tm.assign(S * 2, CUtensorMap{});
    b->cr.assign(2 * S, ColReduceArgs{});
    b->rg.assign(2 * S, RingArgs{});
    b->pp.assign(S, PParamsArgs{});
    b->em.assign(S, EmulArgs{});
    for (int k = 0; k < slots; ++k) clear_slot_args(b, k);
    BC(cudaMalloc(&b->d_xa, sizeof(XShiftArgs) * b->xa.size()));
    BC(cudaMalloc(&b->d_pa, sizeof(PShiftArgs) * b->pa.size()));
    BC(cudaMalloc(&b->d_tm, sizeof(CUtensorMap) * b->tm.size()));
    BC(cudaMalloc(&b->d_cr, sizeof(ColReduceArgs) * b->cr.size()));
    BC(cudaMalloc(&b->d_rg, sizeof(RingArgs) * b->rg.size()));
    BC(cudaMalloc(&b->d_pp, sizeof(PParamsArgs) * b->pp.size()));
    BC(cudaMalloc(&b->d_em, sizeof(EmulArgs) * b->em.size()));
    BC(cudaMalloc(&b->d_ver, sizeof(int) * S));
    BC(cudaMemsetAsync(b->d_ver, 0, sizeof(int) * S, b->st));
    BC(cudaMemcpyAsync(b->d_xa, b->xa.data(), sizeof(XShiftArgs) * b->xa.size(), cudaMemcpyHostToDevice, b->st));
    BC(cudaMemcpyAsync(b->d_pa, b->pa.data(), sizeof(PShiftArgs) * b->pa.size(), cudaMemcpyHostToDevice, b->st));
    BC(cudaMemsetAsync(b->d_tm, 0, sizeof(CUtensorMap) * b->tm.size(), b->st));
    BC(cudaMemcpyAsync(b->d_cr, b->cr.data(), sizeof(ColReduceArgs) * b->cr.size(), cudaMemcpyHostToDevice, b->st));
    BC(cudaMemcpyAsync(b->d_rg, b->rg.data(), sizeof(RingArgs) * b->rg.size(), cudaMemcpyHostToDevice, b->st));
    BC(cudaMemcpyAsync(b->d_pp, b->pp.data(), sizeof(PParamsArgs) * b->pp.size(), cudaMemcpyHostToDevice, b->st));
    BC(cudaMemcpyAsync(b->d_em, b->em.data(), sizeof(EmulArgs) * b->em.size(), cudaMemcpyHostToDevice, b->st));
    BC(cudaStreamSynchronize(b->st));
    b->xsmem = xshift_smem_bytes(max_n, B_PAD_ZERO, B_STAGES, b->esz);

    // capture one batched Strang step
    cudaGraph_t g = nullptr;
    BC(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    int rc = VLASOV_OK;
    auto L = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == VLASOV_OK) {
            char m[256];
            snprintf(m, sizeof m, "batched launch: %s", cudaGetErrorString(e));
            rc = bfail(VLASOV_ECUDA, m);
        }
    };
    const int crb = (max_n + 31) / 32;
    const bool fx = b->esz == 8;
    auto xs = [&](bool per, bool kin, const XShiftArgs* a) {
        return fx ? launch_xshift_fx_batch(per, kin, slots, b->ctas_x, b->xsmem, a, b->d_em, b->d_ver, b->st)
                  : launch_xshift_batch(per, kin, slots, b->ctas_x, b->xsmem, a, b->d_ver, b->st);
    };
    L(xs(true, false, b->d_xa + 0 * S * 2));
    L(xs(false, false, b->d_xa + 1 * S * 2));
    L(launch_colreduce_batch(slots, crb, b->d_cr, b->st));
    L(launch_ring_fixed_batch(false, slots, max_n, b->nsm, b->d_rg, b->st));
    L(launch_pparams_batch(b->esz, slots, max_n, b->d_pp, b->st));
    L(fx ? launch_pshift_fx_batch(slots, b->ctas_p, b->d_tm, b->d_pa, b->d_em, b->d_ver, b->st)
         : launch_pshift_batch(slots, b->ctas_p, b->d_tm, b->d_pa, b->d_ver, b->st));
    L(xs(true, true, b->d_xa + 2 * S * 2));
    L(xs(false, true, b->d_xa + 3 * S * 2));
    L(launch_colreduce_batch(slots, crb, b->d_cr + S, b->st));
    L(launch_ring_fixed_batch(true, slots, max_n, b->nsm, b->d_rg + S, b->st));
    flip_kernel<<<1, 256, 0, b->st>>>(b->d_ver, slots);
    L(cudaGetLastError());
    cudaError_t ec = cudaStreamEndCapture(b->st, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return bail(rc);
    }
    if (ec != cudaSuccess) return bail(bfail(VLASOV_ECUDA, "batch graph capture failed"));
    ec = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ec != cudaSuccess) return bail(bfail(VLASOV_ECUDA, "batch graph instantiate failed"));
#undef BC
    *out = b;
    return VLASOV_OK;
}

// Bytes of device memory a request occupies in a batch arena.
long long vlasov_batch_footprint(const vlasov_request* r, int precision)
{
    if (!r || r->Nx <= 0 || r->Np <= 0) return -1;
    if (precision != VLASOV_F32 && precision != VLASOV_FX64) return -1;
    return (long long)layout(r->Nx, r->Np, precision == VLASOV_FX64 ? 8 : 4).total;
}

int vlasov_batch_admit(vlasov_batch* b, const vlasov_request* r, const double* host_f0, int* slot_out)
{
    if (!b || !slot_out) return bfail(VLASOV_EINVAL, "NULL argument");
    *slot_out = -1;
    int rc = validate_request(r, b->max_n);
    if (rc) return rc;
    int k = -1;
    for (int q = 0; q < b->S; ++q)
        if (!b->slots[q].used) {
            k = q;
            break;
        }
    if (k < 0) return bfail(VLASOV_ESTATE, "no free slot");
    const SlotLayout L = layout(r->Nx, r->Np, b->esz);
    const bool fx = b->esz == 8;
    size_t off = 0;
    if (!b->arena.alloc(L.total, &off)) return bfail(VLASOV_ENOMEM, "request does not fit the batch memory budget now");
    Slot& s = b->slots[k];
    s = Slot{};
    s.used = true;
    s.req = *r;
    s.off = off;
    s.bytes = L.total;
    s.L = L;
    const int Nx = r->Nx, Np = r->Np;
    const double dx = (r->xmax - r->xmin) / Nx, dp = (r->pmax - r->pmin) / Np;
    const bool per = r->x_periodic != 0;

    // host-side tables: node coordinates, initial profile factors, trig and ring tables, row filters
    std::vector<double> rowv(Np), colv(Nx);
    double colsum = 0, rowsum = 0;
    for (int j = 0; j < Np; ++j) {
        const double p = r->pmin + (double)j * dp;
        const double v = std::fabs(p) < r->p0 ? 1.0 : 0.0;
        rowv[j] = v;
        rowsum += v;
    }
    const double half_x = 0.5 * (r->xmax - r->xmin);
    for (int i = 0; i < Nx; ++i) {
        const double x = r->xmin + (double)i * dx;
        double v;
        if (r->init == 0) v = (r->x0 >= half_x || std::fabs(x) < r->x0) ? 1.0 / (4.0 * r->x0 * r->p0) : 0.0;
        else v = (1.0 / (2.0 * r->p0 * (r->xmax - r->xmin))) * (1.0 + r->amp * std::cos(x));
        colv[i] = fx ? v : (double)(float)v;   // FP32 slots build f from the FP32 profile
        colsum += v;
    }
    const double mass_est = dx * dp * colsum * rowsum;
    if (!(mass_est > 0)) {
        b->arena.release(off, L.total);
        s = Slot{};
        return bfail(VLASOV_EINVAL, "initial state is empty on this grid");
    }
    double fmax = 0;
    for (int i = 0; i < Nx; ++i) fmax = std::max(fmax, (double)colv[i]);
    fmax = fmax * (1.0 + std::fabs(r->noise)) / mass_est;   // after normalisation
    const size_t cells = (size_t)Nx * Np;
    double fscale = fmax;   // bound 2^Ef >= 4 max|f|: from the given f0 (as the single-grid path), else the estimate
    if (host_f0 && fx) {
        fscale = 0;
        for (size_t q = 0; q < cells; ++q) fscale = std::max(fscale, std::fabs(host_f0[q]));
    }
    {
        int e = 0;
        std::frexp(fscale, &e);
        s.Ef = e + 2;
        const int Lp = clog2((double)Np), Lx = clog2((double)Nx);
        const double pm = std::max(std::fabs(r->pmin), std::fabs(r->pmax));
        s.k_col = 61 - s.Ef - Lp;
        s.k_kin = 124 - clog2(0.5 * pm * pm * (double)Np * (double)Nx) - s.Ef;
        s.k_pot = 0;
        if (r->model == VLASOV_SHEET) s.k_pot = 124 - (3 * Lx + 2 * (Lp + s.Ef));
        if (r->model == VLASOV_RING) {
            const double vmax = 1.0 / std::sqrt(2.0 * r->eps);
            const double rmax = dp * (double)Np * std::ldexp(1.0, s.Ef);
            s.k_pot = 124 - clog2((double)Nx * (double)Nx * dx * vmax * rmax * rmax);
        }
    }
    std::vector<double> c(Nx), sn(Nx);
    std::vector<long long> cfx(Nx), sfx(Nx);
    for (int i = 0; i < Nx; ++i) {
        const double th = r->xmin + (double)i * dx;
        c[i] = std::cos(th);
        sn[i] = std::sin(th);
        cfx[i] = std::llround(std::ldexp(c[i], 62));
        sfx[i] = std::llround(std::ldexp(sn[i], 62));
    }
    std::vector<unsigned char> recs((size_t)Np * XREC_BYTES, 0);
    const double cx = (0.5 * r->dt) / dx;
    int max_n0 = 0;
    for (int j = 0; j < Np; ++j) {
        const double p = r->pmin + (double)j * dp;
        LineSplit Ls;
        line_split(p * cx, Ls);
        XRec rc_;
        std::memset(&rc_, 0, sizeof rc_);
        rc_.n0 = Ls.n0;
        rc_.m4 = (int)((((long long)Ls.n0 - 4) % Nx + Nx) % Nx);
        rc_.p2q = std::llround(std::ldexp(0.5 * p * p, KIN_Q));
        rc_.p2h = (float)(0.5 * p * p);
        max_n0 = std::max(max_n0, std::abs(Ls.n0));
        rc_.g64 = Ls.g;
        rc_.d64 = Ls.d;
        rc_.g32 = (float)Ls.g;
        rc_.d32 = (float)Ls.d;
        for (int t = 0; t < NTAP; ++t) {
            rc_.w64[t] = Ls.w[t];
            rc_.w32[t] = (float)Ls.w[t];
            emul_weight(Ls.w[t], rc_.Wh[t], rc_.wl[t], rc_.wf[t]);
        }
        double we[2][NTAP];
        line_edge_weights(Ls, we);
        for (int q = 0; q < 2; ++q)
            for (int t = 0; t < NTAP; ++t) emul_weight(we[q][t], rc_.Whe[q][t], rc_.wle[q][t], rc_.wfe[q][t]);
        std::memcpy(&recs[(size_t)j * XREC_BYTES], &rc_, sizeof rc_);
    }
    if (!per && max_n0 + 8 > B_PAD_ZERO) {
        b->arena.release(off, L.total);
        s = Slot{};
        return bfail(VLASOV_EINVAL, "x displacement too large for the batched zero halo (55 cells)");
    }
    auto H2D = [&](size_t o, const void* src, size_t bytes) {
        return cudaMemcpyAsync(P(b, s, o), src, bytes, cudaMemcpyHostToDevice, b->st);
    };
    B_TRY(cudaMemsetAsync(P(b, s, 0), 0, L.total, b->st));
    B_TRY(H2D(L.costab, c.data(), 8 * (size_t)Nx));
    B_TRY(H2D(L.sintab, sn.data(), 8 * (size_t)Nx));
    B_TRY(H2D(L.cosfx, cfx.data(), 8 * (size_t)Nx));
    B_TRY(H2D(L.sinfx, sfx.data(), 8 * (size_t)Nx));
    std::vector<long long> Kq(Nx), Vq(Nx);
    if (r->model == VLASOV_RING) {
        ring_fixed_tables(Nx, dx, r->eps, Kq.data(), Vq.data(), &s.ring_sK, &s.ring_sV);
        B_TRY(H2D(L.ringKq, Kq.data(), 8 * (size_t)Nx));
        B_TRY(H2D(L.ringVq, Vq.data(), 8 * (size_t)Nx));
    }
    B_TRY(H2D(L.xrec, recs.data(), recs.size()));
    if (host_f0 && fx) {
        std::vector<long long> tmp(cells);
        for (size_t q = 0; q < cells; ++q) tmp[q] = (long long)fx128_from_f64(host_f0[q], FX_FRAC - s.Ef);
        B_TRY(H2D(L.f[0], tmp.data(), cells * 8));
        B_TRY(cudaStreamSynchronize(b->st));
    } else if (host_f0) {
        std::vector<float> tmp(cells);
        for (size_t q = 0; q < cells; ++q) tmp[q] = (float)host_f0[q];
        B_TRY(H2D(L.f[0], tmp.data(), cells * 4));
        B_TRY(cudaStreamSynchronize(b->st));
    } else if (fx) {
        B_TRY(H2D(L.rowv, rowv.data(), 8 * (size_t)Np));
        B_TRY(H2D(L.colv, colv.data(), 8 * (size_t)Nx));
        InitArgs64 ia;
        ia.f = reinterpret_cast<double*>(P(b, s, L.f[1]));
        ia.Nx = Nx;
        ia.Np = Np;
        ia.rowv = reinterpret_cast<const double*>(P(b, s, L.rowv));
        ia.colv = reinterpret_cast<const double*>(P(b, s, L.colv));
        ia.noise = r->init == 0 ? r->noise : 0.0;
        ia.seed = r->seed;
        ia.k_m = 120 - clog2((double)cells * fmax * mass_est * 2.0 + 1.0);
        ia.dxdp = dx * dp;
        ia.part = P(b, s, L.initpart);
        ia.ticket = reinterpret_cast<unsigned int*>(P(b, s, L.tickets));
        ia.inv_mass = reinterpret_cast<double*>(P(b, s, L.inv_mass));
        init_fill64_kernel<<<B_INIT_BLOCKS, 256, 0, b->st>>>(ia);
        B_TRY(cudaGetLastError());
        init_scale_fx_kernel<<<256, 256, 0, b->st>>>(ia.f, reinterpret_cast<long long*>(P(b, s, L.f[0])), cells,
                                                     ia.inv_mass, FX_FRAC - s.Ef);
        B_TRY(cudaGetLastError());
    } else {
        std::vector<float> rowf(rowv.begin(), rowv.end()), colf(colv.begin(), colv.end());
        B_TRY(H2D(L.rowv, rowf.data(), 4 * (size_t)Np));
        B_TRY(H2D(L.colv, colf.data(), 4 * (size_t)Nx));
        InitArgs ia;
        ia.f = reinterpret_cast<float*>(P(b, s, L.f[0]));
        ia.Nx = Nx;
        ia.Np = Np;
        ia.rowv = reinterpret_cast<const float*>(P(b, s, L.rowv));
        ia.colv = reinterpret_cast<const float*>(P(b, s, L.colv));
        ia.noise = (float)(r->init == 0 ? r->noise : 0.0);
        ia.seed = r->seed;
        ia.k_m = 120 - clog2((double)cells * fmax * mass_est * 2.0 + 1.0);
        ia.dxdp = dx * dp;
        ia.part = P(b, s, L.initpart);
        ia.ticket = reinterpret_cast<unsigned int*>(P(b, s, L.tickets));
        ia.inv_mass = reinterpret_cast<double*>(P(b, s, L.inv_mass));
        init_fill_kernel<<<B_INIT_BLOCKS, 256, 0, b->st>>>(ia);
        B_TRY(cudaGetLastError());
        init_scale_kernel<<<256, 256, 0, b->st>>>(ia.f, cells, ia.inv_mass);
        B_TRY(cudaGetLastError());
    }
    // this slot starts at buffer 0: its parity word must read 0 at its first step
    const int zero = 0;
    B_TRY(cudaMemcpyAsync(b->d_ver + k, &zero, sizeof(int), cudaMemcpyHostToDevice, b->st));
    rc = fill_slot_args(b, k);
    if (rc) {
        b->arena.release(off, L.total);
        s = Slot{};
        return rc;
    }
    if (r->steps == 0) clear_slot_args(b, k);
    rc = upload_slot_args(b, k);
    if (rc) return rc;
    // the small host tables above are staged by the runtime when copied from pageable memory, so
    // they may go out of scope without waiting for the stream (admission overlaps running steps)
    s.active = r->steps > 0;
    *slot_out = k;
    return VLASOV_OK;
}

int vlasov_batch_step(vlasov_batch* b, int n)
{
    if (!b || n < 0) return bfail(VLASOV_EINVAL, "bad argument");
    for (int it = 0; it < n; ++it) {
        bool any = false;
        for (auto& s : b->slots) any |= s.active;
        if (!any) break;
        B_TRY(cudaGraphLaunch(b->graph, b->st));
        ++b->steps_launched;
        for (int k = 0; k < b->S; ++k) {
            Slot& s = b->slots[k];
            if (!s.active) continue;
            if (++s.steps_done >= s.req.steps) {
                // finished: no further batched step may touch it
                s.active = false;
                clear_slot_args(b, k);
                int rc = upload_slot_args(b, k);
                if (rc) return rc;
            }
        }
    }
    return VLASOV_OK;
}

int vlasov_batch_slot_steps(vlasov_batch* b, int slot, int* steps_done)
{
    if (!b || slot < 0 || slot >= b->S || !steps_done) return bfail(VLASOV_EINVAL, "bad argument");
    *steps_done = b->slots[slot].steps_done;
    return VLASOV_OK;
}

int vlasov_batch_get(vlasov_batch* b, int slot, double* host_f, vlasov_moments_t* out, int max, int* count)
{
    if (!b || slot < 0 || slot >= b->S) return bfail(VLASOV_EINVAL, "bad argument");
    Slot& s = b->slots[slot];
    if (!s.used) return bfail(VLASOV_ESTATE, "slot is free");
    B_TRY(cudaStreamSynchronize(b->st));
    const size_t cells = (size_t)s.req.Nx * s.req.Np;
    if (host_f) {
        const int cur = s.steps_done & 1;
        if (b->esz == 8) {
            std::vector<long long> tmp(cells);
            B_TRY(cudaMemcpy(tmp.data(), P(b, s, s.L.f[cur]), cells * 8, cudaMemcpyDeviceToHost));
            for (size_t q = 0; q < cells; ++q) host_f[q] = fx128_to_f64((i128)tmp[q], FX_FRAC - s.Ef);
        } else {
            std::vector<float> tmp(cells);
            B_TRY(cudaMemcpy(tmp.data(), P(b, s, s.L.f[cur]), cells * 4, cudaMemcpyDeviceToHost));
            for (size_t q = 0; q < cells; ++q) host_f[q] = (double)tmp[q];
        }
    }
    if (count) *count = 0;
    if (out && max > 0) {
        const int n = std::min(std::min(max, s.steps_done), HIST_CAP);
        std::vector<MomentRec> rec(HIST_CAP);
        B_TRY(cudaMemcpy(rec.data(), P(b, s, s.L.hist), sizeof(MomentRec) * HIST_CAP, cudaMemcpyDeviceToHost));
        const int first = s.steps_done - n;
        for (int q = 0; q < n; ++q) {
            const MomentRec& m = rec[(size_t)(first + q) % HIST_CAP];
            out[q].t = m.t;
            out[q].mass = m.mass;
            out[q].Mx = m.Mx;
            out[q].My = m.My;
            out[q].kinetic = m.kinetic;
            out[q].potential = m.potential;
            out[q].energy = m.energy;
            out[q].step = m.step;
        }
        if (count) *count = n;
    }
    int h = 0;
    B_TRY(cudaMemcpy(&h, P(b, s, s.L.err), sizeof(int), cudaMemcpyDeviceToHost));
    if (h) return bfail(h == DEV_ERR_RANGE ? VLASOV_ERANGE : VLASOV_ETIMEOUT, "device error flag set for this slot");
    return VLASOV_OK;
}

int vlasov_batch_release(vlasov_batch* b, int slot)
{
    if (!b || slot < 0 || slot >= b->S) return bfail(VLASOV_EINVAL, "bad argument");
    Slot& s = b->slots[slot];
    if (!s.used) return VLASOV_OK;
    if (s.active) {
        s.active = false;
        clear_slot_args(b, slot);
        int rc = upload_slot_args(b, slot);
        if (rc) return rc;
    }
    B_TRY(cudaStreamSynchronize(b->st));   // nothing in flight may still use its memory
    b->arena.release(s.off, s.bytes);
    s = Slot{};
    return VLASOV_OK;
}

// ------------------------------------------------------------------------------------------- serving loop
}  // extern "C"

namespace {

// The batch of the serving loop with its queue of requests, the events that mark its launched
// steps, and the slots whose last step is still in flight.
struct ServeLane {
    vlasov_batch* b = nullptr;
    std::vector<int> queue;        // request indices, in arrival order
    size_t next = 0;               // first queue entry not yet admitted
    std::vector<cudaEvent_t> ev;   // one per launched batched step (ring of NE)
    std::vector<long long> ev_step;
    cudaEvent_t ev0 = nullptr;     // recorded at the start of the run
    struct Draining {
        int slot, req;
        long long step_index;
    };
    std::vector<Draining> draining;
    std::vector<int> slot_req;
    std::vector<MomentRec> hostrec;
    long long launched = 0;
};
constexpr int SERVE_NE = 256;

void lane_free(ServeLane& L)
{
    for (auto& e : L.ev)
        if (e) cudaEventDestroy(e);
    if (L.ev0) cudaEventDestroy(L.ev0);
    vlasov_batch_destroy(L.b);
    L = ServeLane{};
}

int lane_init(ServeLane& L, int slots, int max_n, long long budget, int prec, void* stream)
{
    int rc = vlasov_batch_create(std::max(1, slots), max_n, budget, prec, stream, &L.b);
    if (rc) return rc;
    L.ev.assign(SERVE_NE, nullptr);
    L.ev_step.assign(SERVE_NE, -1);
    for (auto& e : L.ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bfail(VLASOV_ECUDA, "event create");
    if (cudaEventCreate(&L.ev0) != cudaSuccess) return bfail(VLASOV_ECUDA, "event create");
    L.slot_req.assign(L.b->S, -1);
    L.hostrec.resize(2 * (size_t)L.b->S);
    return VLASOV_OK;
}

// Admit this lane's arrived requests in arrival order while a slot and memory are free.
template <typename Now>
void lane_admit(ServeLane& L, const vlasov_request* reqs, vlasov_result* results, int* finished, Now now_s)
{
    vlasov_batch* b = L.b;
    while (L.next < L.queue.size() && reqs[L.queue[L.next]].arrival_s <= now_s()) {
        const int q = L.queue[L.next];
        int slot = -1;
        const int r2 = vlasov_batch_admit(b, &reqs[q], nullptr, &slot);
        if (r2 == VLASOV_ESTATE || r2 == VLASOV_ENOMEM) {
            // full now: admit later, unless nothing is running (then it can never fit)
            bool busy = false;
            for (auto& sl : b->slots) busy |= sl.used;
            if (busy) break;
            results[q].status = r2;
            ++*finished;
            ++L.next;
            continue;
        }
        if (r2) {
            results[q].status = r2;
            ++*finished;
            ++L.next;
            continue;
        }
        results[q].admit_s = now_s();
        L.slot_req[slot] = q;
        ++L.next;
        if (reqs[q].steps == 0) {
            results[q].status = 0;
            results[q].done_s = results[q].admit_s;
            vlasov_batch_release(b, slot);
            L.slot_req[slot] = -1;
            ++*finished;
        }
    }
}

// Launch one batched step if any slot is active (at most `depth` steps in flight).  Returns 1 if a
// step was launched, 0 if none was active, or a negative error.
int lane_step(ServeLane& L, int depth)
{
    vlasov_batch* b = L.b;
    bool any_active = false;
    for (auto& sl : b->slots) any_active |= sl.active;
    if (!any_active) return 0;
    if (L.launched >= depth) cudaEventSynchronize(L.ev[(size_t)((L.launched - depth) % SERVE_NE)]);
    std::vector<int> was_active(b->S, 0);
    for (int k = 0; k < b->S; ++k) was_active[k] = b->slots[k].active;
    const int rc = vlasov_batch_step(b, 1);
    if (rc) return rc;
    const int e = (int)(L.launched % SERVE_NE);
    cudaEventRecord(L.ev[e], b->st);
    L.ev_step[e] = L.launched;
    for (int k = 0; k < b->S; ++k) {
        if (was_active[k] && !b->slots[k].active) {
            // copy its last and first moment records (stream-ordered after the step) and drain
            Slot& sl = b->slots[k];
            const int last = (sl.steps_done - 1) % HIST_CAP;
            cudaMemcpyAsync(&L.hostrec[2 * k], P(b, sl, sl.L.hist) + sizeof(MomentRec) * last, sizeof(MomentRec),
                            cudaMemcpyDeviceToHost, b->st);
            cudaMemcpyAsync(&L.hostrec[2 * k + 1], P(b, sl, sl.L.hist), sizeof(MomentRec), cudaMemcpyDeviceToHost, b->st);
            L.draining.push_back({k, L.slot_req[k], L.launched});
        }
    }
    ++L.launched;
    return 1;
}

// Retire drained slots whose last step has completed on the GPU.
template <typename Now>
void lane_retire(ServeLane& L, vlasov_result* results, int* finished, Now now_s)
{
    vlasov_batch* b = L.b;
    for (size_t d = 0; d < L.draining.size();) {
        const ServeLane::Draining dr = L.draining[d];
        const int e = (int)(dr.step_index % SERVE_NE);
        const bool recycled = L.ev_step[e] != dr.step_index;
        if (!recycled && cudaEventQuery(L.ev[e]) != cudaSuccess) {
            ++d;
            continue;
        }
        if (recycled) cudaStreamSynchronize(b->st);
        else cudaEventSynchronize(L.ev[e]);
        cudaStreamSynchronize(b->st);   // the record copies were enqueued after the event
        vlasov_result& out = results[dr.req];
        float ms = 0.f;
        if (!recycled) cudaEventElapsedTime(&ms, L.ev0, L.ev[e]);
        else ms = (float)(now_s() * 1e3);
        out.done_s = ms * 1e-3;
        out.status = 0;
        out.steps = b->slots[dr.slot].steps_done;
        const MomentRec* m2[2] = {&L.hostrec[2 * dr.slot], &L.hostrec[2 * dr.slot + 1]};
        vlasov_moments_t* dst[2] = {&out.last, &out.first};
        for (int z = 0; z < 2; ++z) {
            dst[z]->t = m2[z]->t;
            dst[z]->mass = m2[z]->mass;
            dst[z]->Mx = m2[z]->Mx;
            dst[z]->My = m2[z]->My;
            dst[z]->kinetic = m2[z]->kinetic;
            dst[z]->potential = m2[z]->potential;
            dst[z]->energy = m2[z]->energy;
            dst[z]->step = m2[z]->step;
        }
        vlasov_batch_release(b, dr.slot);
        L.slot_req[dr.slot] = -1;
        ++*finished;
        L.draining.erase(L.draining.begin() + (long)d);
    }
}

}  // namespace

extern "C" {

int vlasov_serve(const vlasov_request* reqs, int n, const vlasov_serve_options* opt, vlasov_result* results,
                 double* makespan_s)
{
    if (!reqs || n < 0 || !opt || !results) return bfail(VLASOV_EINVAL, "NULL argument");
    int max_n = opt->max_n;
    if (max_n <= 0)
        for (int q = 0; q < n; ++q) max_n = std::max(max_n, std::max(reqs[q].Nx, reqs[q].Np));
    max_n = std::max(16, max_n);
    const int prec = opt->precision ? opt->precision : VLASOV_F32;
    if (prec != VLASOV_F32 && prec != VLASOV_FX64)
        return bfail(VLASOV_EINVAL, "serving precision must be VLASOV_F32 or VLASOV_FX64");
    if (opt->autotune) {
        vlasov_batch_shape sh;
        const int rc0 = vlasov_batch_autotune(max_n, prec, opt->stream, &sh, nullptr);
        if (rc0) return rc0;
    }
    ServeLane L;
    {
        const int rc0 = lane_init(L, opt->slots, max_n, opt->mem_budget_bytes, prec, opt->stream);
        if (rc0) {
            lane_free(L);
            return rc0;
        }
    }
    std::vector<int> order(n);
    for (int q = 0; q < n; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return reqs[a].arrival_s < reqs[c].arrival_s; });
    L.queue = order;
    for (int q = 0; q < n; ++q) {
        std::memset(&results[q], 0, sizeof(vlasov_result));
        results[q].status = 1;   // pending
        results[q].arrival_s = reqs[q].arrival_s;
    }
    cudaStreamSynchronize(L.b->st);
    const auto t0 = std::chrono::steady_clock::now();
    cudaEventRecord(L.ev0, L.b->st);
    auto now_s = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    const int depth = std::max(1, opt->max_inflight);
    int finished = 0, rc = VLASOV_OK;
    while (finished < n && rc == VLASOV_OK) {
        lane_admit(L, reqs, results, &finished, now_s);
        const int r = lane_step(L, depth);
        if (r < 0) {
            rc = r;
            break;
        }
        if (r == 0 && L.next < L.queue.size()) {
            // nothing running: sleep until the next arrival
            const double wait = reqs[L.queue[L.next]].arrival_s - now_s();
            if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
        }
        lane_retire(L, results, &finished, now_s);
    }
    cudaStreamSynchronize(L.b->st);
    if (makespan_s) *makespan_s = now_s();
    lane_free(L);
    return rc;
}

}  // extern "C"
