// noalloc.cu -- an x-shift sweep with its density epilogue that allocates no memory.
//
// Who this is for: code that runs where it may not call cudaMalloc -- for example inside a host
// callback or a custom allocator hook, under a framework that owns every device allocation and
// forbids others, or in a plug-in that must not grow the process' device footprint after start-up.
// Such a caller hands in device buffers for the input, the output and the density, and this entry
// point does its work in a fixed scratch area that is part of the library image itself.
//
// The scratch is a file-scope __device__ array: every GPU on which the library is loaded holds
// it (NOALLOC_SCRATCH_BYTES) until the process exits, whether or not this entry point is called.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "../../include/vlasov.h"
#include "vlasov_internal.cuh"

using namespace vl;

namespace {

constexpr int NA_MAX_NX = 4096;     // longest row (FP64)
constexpr int NA_MAX_NP = 4096;     // most rows
constexpr int NA_MAX_CTAS = 152;    // CTAs of the sweep = rows of column partials
constexpr int NA_PAD_ZERO = 64;     // zero halo each side of a staged row (non-periodic x)
constexpr int NA_PAD_PERIODIC = 16;

// Scratch layout (bytes): [error flag | row filters | column partials]
constexpr size_t NA_OFF_N0 = 256;
constexpr size_t NA_N0_BYTES = sizeof(int) * NA_MAX_NP;
constexpr size_t NA_W_BYTES = sizeof(double) * NTAP * NA_MAX_NP;
constexpr size_t NA_GD_BYTES = sizeof(double) * 2 * NA_MAX_NP;
constexpr size_t NA_PART_BYTES = sizeof(double) * (size_t)NA_MAX_CTAS * NA_MAX_NX;
constexpr size_t NA_OFF_W = NA_OFF_N0 + 256 * ((NA_N0_BYTES + 255) / 256);
constexpr size_t NA_OFF_GD = NA_OFF_W + NA_W_BYTES;
constexpr size_t NA_OFF_PART = 256 * ((NA_OFF_GD + NA_GD_BYTES + 255) / 256);
constexpr size_t NOALLOC_SCRATCH_BYTES = NA_OFF_PART + NA_PART_BYTES;   // ~5.1 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};   // device address of the scratch, per device
int g_na_smem[NA_MAX_DEVICES] = {};

int na_fail(int code, const char* msg, cudaError_t e = cudaSuccess)
{
    char buf[256];
    if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
    else snprintf(buf, sizeof buf, "%s", msg);
    set_last_error(buf);
    return code;
}

// Filters of each row from its displacement (cells): the same split as every other x-shift.  A
// displacement beyond the staged halo (|n0| > max_n0) is clamped, so the sweep stays inside its
// shared-memory window, and the error flag is raised (the density then comes out as NaN).
__global__ void na_row_filters(const double* __restrict__ disp, int Np, int max_n0, int* n0, double* w, double* gd,
                               int* flag)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Np) return;
    const double s = disp[j];
    LineSplit L;
    line_split(fabs(s) < 1.0e9 ? s : 0.0, L);   // NaN or huge: a harmless split, flagged below
    if (!(fabs(s) < 1.0e9) || L.n0 < -max_n0 || L.n0 > max_n0) {
        atomicExch(flag, 1);
        L.n0 = max(-max_n0, min(max_n0, L.n0));
    }
    n0[j] = L.n0;
#pragma unroll
    for (int t = 0; t < NTAP; ++t) w[(size_t)t * Np + j] = L.w[t];
    gd[j] = L.g;
    gd[Np + j] = L.d;
}

// rho_i = dp * sum_b part[b][i], partial rows summed in a fixed order; NaN if the flag is up
// (a displacement was out of range, or a bounded wait in the sweep gave up).
__global__ void na_density(const double* __restrict__ part, int B, int Nx, double dp, const int* flag,
                           double* __restrict__ rho)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nx) return;
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += part[(size_t)b * Nx + i];
    rho[i] = *flag ? __longlong_as_double(0x7ff8000000000000ll) : dp * s;
}

// Once per device, with that device current: look up the scratch's device address (in host code
// the array's name is only a host-side stand-in) and opt the sweep kernels into their shared memory.
int na_setup(int dev, unsigned char** ptr, int* smem)
{
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(VLASOV_EINVAL, "device ordinal out of range");
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return na_fail(VLASOV_ECUDA, "cudaGetSymbolAddress(scratch)", e);
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return na_fail(VLASOV_ECUDA, "cudaDeviceGetAttribute", e);
        e = set_kernel_attributes(optin - 1024);
        if (e != cudaSuccess) return na_fail(VLASOV_ECUDA, "cudaFuncSetAttribute", e);
        g_na_smem[dev] = optin;
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *ptr = g_na_ptr[dev];
    *smem = g_na_smem[dev];
    return VLASOV_OK;
}

}  // namespace

extern "C" int vlasov_xshift_density_noalloc(const double* dev_fin, double* dev_fout, double* dev_rho, int Nx, int Np,
                                             double pmin, double pmax, int x_periodic, const double* dev_disp,
                                             void* stream)
{
    if (!dev_fin || !dev_fout || !dev_rho || !dev_disp) return na_fail(VLASOV_EINVAL, "NULL buffer");
    if (Nx < 16 || Np < 16 || Nx % 8 || Np % 8) return na_fail(VLASOV_EINVAL, "Nx, Np must be multiples of 8 and >= 16");
    if (Nx > NA_MAX_NX || Np > NA_MAX_NP) return na_fail(VLASOV_EINVAL, "Nx or Np above the scratch maximum of 4096");
    if (!(pmax > pmin)) return na_fail(VLASOV_EINVAL, "empty p domain");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(VLASOV_ECUDA, "cudaGetDevice", e);
    unsigned char* scratch = nullptr;
    int optin = 0;
    int rc = na_setup(dev, &scratch, &optin);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    int* flag = reinterpret_cast<int*>(scratch);
    int* n0 = reinterpret_cast<int*>(scratch + NA_OFF_N0);
    double* w = reinterpret_cast<double*>(scratch + NA_OFF_W);
    double* gd = reinterpret_cast<double*>(scratch + NA_OFF_GD);
    double* part = reinterpret_cast<double*>(scratch + NA_OFF_PART);
    const int pad = x_periodic ? NA_PAD_PERIODIC : NA_PAD_ZERO;
    // periodic rows wrap, so any displacement is in range; zero-extended rows need |n0| + 8 <= pad
    const int max_n0 = x_periodic ? 0x3fffffff : pad - 8;

    // staged rows in flight: as many as fit the opted-in shared memory, at most 4, at least 1
    const long long row_bytes = (long long)(Nx + 2 * pad) * (long long)sizeof(double) + XREC_BYTES;
    const long long room = (long long)optin - 2048 - 256;
    const int stages = room > 0 ? (int)std::min<long long>(4, room / row_bytes) : 0;
    if (stages < 1) return na_fail(VLASOV_EINVAL, "a staged row does not fit in this device's shared memory");

    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess) return na_fail(VLASOV_ECUDA, "clear flag", e);
    na_row_filters<<<(Np + 127) / 128, 128, 0, st>>>(dev_disp, Np, max_n0, n0, w, gd, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(VLASOV_ECUDA, "row filters launch", e);

    XShiftArgs a;
    a.fin = dev_fin;
    a.fout = dev_fout;
    a.Nx = Nx;
    a.Np = Np;
    a.pad = pad;
    a.stages = stages;
    a.n0 = n0;
    a.w = w;
    a.gd = gd;
    a.colpart = part;
    a.kinpart = nullptr;
    a.pmin = pmin;
    a.dp = (pmax - pmin) / (double)Np;
    a.err = flag;
    const int B = std::min(Np, NA_MAX_CTAS);
    if ((e = launch_xshift(8, x_periodic != 0, false, B, XS_THREADS_MIN, a, st)) != cudaSuccess)
        return na_fail(VLASOV_ECUDA, "x-shift launch", e);
    na_density<<<(Nx + 255) / 256, 256, 0, st>>>(part, B, Nx, a.dp, flag, dev_rho);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(VLASOV_ECUDA, "density launch", e);
    return VLASOV_OK;
}
