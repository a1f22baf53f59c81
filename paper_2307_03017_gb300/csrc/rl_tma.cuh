// rl_tma.cuh -- shared-memory plane staging for the warp kernels (sm_103a).
//
// A block handles a TX x TY tile of view pixels.  For plane d every pixel samples the MPI
// at p = q + a(q) + rho_d b(q); over the tile these positions lie in a small window of
// the reference image.  The window's top-left corner follows from per-block bounds of
// q + a(q) and b(q) (rho_d > 0), so it is known before any sample is taken.  One thread
// fetches the window -- a fixed BW x BH box of RGBA voxels of plane d -- with a TMA tensor
// copy (cp.async.bulk.tensor), whose out-of-image part the copy engine fills with zeros:
// exactly the zero padding of the bilinear sampler.  Two stages alternate so that the
// copy of the next plane overlaps the arithmetic on the current one.  Samples whose taps
// leave the window (extreme warps) fall back to direct global loads; results never
// depend on the window being large enough.
//
// Every wait on an mbarrier is bounded in time; a wait that gives up records
// RL_DEVFLAG_TIMEOUT in the device status word and the block stops.
#pragma once
#include <cuda.h>

#include "rl_common.cuh"

#define RL_DEVFLAG_TIMEOUT 1u

namespace rltma {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int BW = 48, BH = 16;  // staged window in voxels
constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it did not complete in ~1 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Per-block bounds of q + a(q) and b(q) over the tile's pixels (x and y).
struct TileBounds {
    float axl, axh, bxl, bxh, ayl, ayh, byl, byh;
};

// Block-wide min/max reduction of the warp coefficients; `scratch` holds 8 floats per warp.
__device__ __forceinline__ TileBounds tile_bounds(float ux, float uy, float bx, float by, bool ok, float* scratch) {
    float v[8] = {ok ? ux : INFINITY, ok ? -ux : INFINITY, ok ? bx : INFINITY, ok ? -bx : INFINITY,
                  ok ? uy : INFINITY, ok ? -uy : INFINITY, ok ? by : INFINITY, ok ? -by : INFINITY};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = fminf(v[i], __shfl_xor_sync(0xffffffffu, v[i], o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 8; ++i) scratch[warp * 8 + i] = v[i];
    __syncthreads();
    float r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = INFINITY;
    for (int w = 0; w < NT / 32; ++w)
#pragma unroll
        for (int i = 0; i < 8; ++i) r[i] = fminf(r[i], scratch[w * 8 + i]);
    __syncthreads();
    TileBounds b;
    b.axl = r[0]; b.axh = -r[1]; b.bxl = r[2]; b.bxh = -r[3];
    b.ayl = r[4]; b.ayh = -r[5]; b.byl = r[6]; b.byh = -r[7];
    return b;
}

// Window of plane rho: top-left corner (xlo, ylo) of the staged box and the extent
// (nx, ny) <= (BW, BH) that can hold taps.  xlo is even so that the TMA start
// coordinate is 16-byte aligned for 2-byte storage as well.
struct Window {
    int xlo, ylo, nx, ny;
};

__device__ __forceinline__ int clamp_coord(float v) { return (int)fminf(fmaxf(v, -1048576.f), 1048576.f); }

__device__ __forceinline__ Window window_for(const TileBounds& tb, float rho) {
    Window w;
    if (!(tb.axl <= tb.axh)) {  // no pixel of the tile has a usable ray
        w.xlo = 0; w.ylo = 0; w.nx = 0; w.ny = 0;
        return w;
    }
    w.xlo = (clamp_coord(floorf(fmaf(rho, tb.bxl, tb.axl))) - 1) & ~1;
    w.ylo = clamp_coord(floorf(fmaf(rho, tb.byl, tb.ayl))) - 1;
    const int xhi = clamp_coord(floorf(fmaf(rho, tb.bxh, tb.axh))) + 2;
    const int yhi = clamp_coord(floorf(fmaf(rho, tb.byh, tb.ayh))) + 2;
    w.nx = min(max(xhi - w.xlo + 1, 0), BW);
    w.ny = min(max(yhi - w.ylo + 1, 0), BH);
    return w;
}

// Bilinear sample from a staged window (all four taps inside it; zero-padded by TMA).
template <typename Tm>
__device__ __forceinline__ float4 window_sample(const Tm* st, int lx, int ly, float fx, float fy) {
    const Tm* p = st + (ly * BW + lx) * 4;
    const float4 v00 = RLStore<Tm>::load4_nc(p), v10 = RLStore<Tm>::load4_nc(p + 4);
    const float4 v01 = RLStore<Tm>::load4_nc(p + BW * 4), v11 = RLStore<Tm>::load4_nc(p + BW * 4 + 4);
    const float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy), w01 = (1.f - fx) * fy, w11 = fx * fy;
    float4 a;
    a.x = fmaf(w11, v11.x, fmaf(w01, v01.x, fmaf(w10, v10.x, w00 * v00.x)));
    a.y = fmaf(w11, v11.y, fmaf(w01, v01.y, fmaf(w10, v10.y, w00 * v00.y)));
    a.z = fmaf(w11, v11.z, fmaf(w01, v01.z, fmaf(w10, v10.z, w00 * v00.z)));
    a.w = fmaf(w11, v11.w, fmaf(w01, v01.w, fmaf(w10, v10.w, w00 * v00.w)));
    return a;
}

}  // namespace rltma
