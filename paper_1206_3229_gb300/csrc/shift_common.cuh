// shift_common.cuh -- pieces shared by the FP32/FP64 and the emulated-FP64 sweep kernels.
#pragma once
#include "ptx.cuh"
#include "vlasov_internal.cuh"

namespace vl {

// Dynamic shared memory rounded up to a 128-byte boundary (TMA destinations); every launch
// reserves 128 extra bytes for this.
__device__ __forceinline__ unsigned char* align128(unsigned char* p)
{
    const uint32_t a = smem_u32(p);
    return p + ((128u - (a & 127u)) & 127u);
}


// D_k of Eq. (findif) (undivided) for a window starting at f_{k-4}.
template <typename T>
__device__ __forceinline__ T fd_undivided(const T* x)
{
    const T c0 = T(VL_FD_C0), c1 = T(VL_FD_C1), c2 = T(VL_FD_C2), c3 = T(VL_FD_C3), c4 = T(VL_FD_C4);
    return c4 * (x[0] + x[8]) + c3 * (x[1] + x[7]) + c2 * (x[2] + x[6]) + c1 * (x[3] + x[5]) + c0 * x[4];
}

// Non-periodic axes take f'' = 0 at nodes outside the grid.  The 10-tap filter evaluates D at
// k and k+1 from the zero-extended f, so remove those terms when k or k+1 lies outside [0, n).
// `x` starts at f_{k-4}.
template <typename T>
__device__ __forceinline__ T edge_fix(T out, const T* x, int k, int n, T g, T d)
{
    if (k < 0 || k >= n) out -= g * fd_undivided(x);
    if (k + 1 < 0 || k + 1 >= n) out -= d * fd_undivided(x + 1);
    return out;
}

struct TileWin {
    int i0, j0, r0, nb;
    int kmin, kmax;   // least and greatest foot offset n0 over the tile's columns
    bool smem_ok;
};

// Window of input rows a tile of TH rows needs: [j0 + kmin - 4, j0 + TH - 1 + kmax + 5].  Called by whole
// warps (all lanes hold one column); identical in every warp.  tile_window_of takes this lane's foot
// offset n0_lane (any value where !colvalid, replaced there by the tile's least offset); tile_window
// loads it from n0.
template <bool PPER, int RB = PS_RB, int TH = PS_TH>
__device__ __forceinline__ TileWin tile_window_of(int tile, int ntx, bool colvalid, int& n0_lane)
{
    TileWin t;
    const int tx = tile % ntx, ty = tile / ntx;
    t.i0 = tx * PS_TW;
    t.j0 = ty * TH;
    int kmin = colvalid ? n0_lane : 0x7fffffff;
    int kmax = colvalid ? n0_lane : (int)0x80000000;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (!colvalid) n0_lane = kmin;   // columns past Nx read (and discard) the tile's own window
    t.kmin = kmin;
    t.kmax = kmax;
    t.r0 = t.j0 + kmin - 4;
    const long long R = (long long)TH + 9 + ((long long)kmax - (long long)kmin);
    t.smem_ok = !PPER && R <= RB;
    t.nb = t.smem_ok ? (int)((R + PS_BH - 1) / PS_BH) : 0;
    return t;
}

template <bool PPER, int RB = PS_RB, int TH = PS_TH>
__device__ __forceinline__ TileWin tile_window(int tile, int ntx, const int* __restrict__ n0, int Nx, int lane,
                                               int& n0_lane, bool& colvalid)
{
    const int i = (tile % ntx) * PS_TW + lane;
    colvalid = i < Nx;
    n0_lane = colvalid ? n0[i] : 0;
    return tile_window_of<PPER, RB, TH>(tile, ntx, colvalid, n0_lane);
}

template <typename T, bool PPER>
__device__ __forceinline__ T gload_p(const T* __restrict__ f, int row, int col, int Nx, int Np)
{
    if constexpr (PPER) {
        int rr = row % Np;
        if (rr < 0) rr += Np;
        return f[(size_t)rr * Nx + col];
    } else {
        return (row >= 0 && row < Np) ? f[(size_t)row * Nx + col] : T(0);
    }
}

}  // namespace vl
