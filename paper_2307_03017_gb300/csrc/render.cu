// render.cu -- novel-view rendering (Eq. eq_render, Eq. eq_over) and warp diagnostics.
//
// One thread per target pixel: for d = D-1 .. 0 (nearest first) sample plane d at
// p = q + a(q) + rho_d b(q) (bilinear, zero padding per tap) and accumulate
// C += T alpha c, T *= (1 - alpha).  The loop stops once T is exactly zero, after which
// every further term is exactly zero.
#include "rl_internal.h"

namespace {

constexpr int kRenderBX = 32, kRenderBY = 4;
#ifndef RL_RENDER_MIN_BLOCKS
#define RL_RENDER_MIN_BLOCKS 1  // no register cap: measured fastest
#endif

// Blocks are ordered view-fastest (grid x = view) so that the views of a tile, whose plane
// footprints overlap, run together and share the MPI through L2.
template <typename Tm>
__global__ void __launch_bounds__(kRenderBX* kRenderBY, RL_RENDER_MIN_BLOCKS)
k_render(const Tm* __restrict__ M, int D, int H, int W, const __grid_constant__ RLViews views, int tiles_x,
         float* __restrict__ out) {
    const int view = blockIdx.x;  // grid (views, tiles_x, tiles_y): views of a tile run together
    const int qx = blockIdx.y * kRenderBX + threadIdx.x;
    const int qy = blockIdx.z * kRenderBY + threadIdx.y;
    if (qx >= W || qy >= H) return;
    const RLWarp w = rl_warp_coeffs(views.v[view], (float)qx, (float)qy);
    const size_t plane = (size_t)H * W * 4;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll 2
    for (int d = D - 1; d >= 0; --d) {
        const RLTaps t = rl_taps(w, views.rho[d], qx, qy);
        const float4 m = rl_sample_fast(M + d * plane, H, W, t);
        const float a = T * m.w;
        c0 = fmaf(a, m.x, c0);
        c1 = fmaf(a, m.y, c1);
        c2 = fmaf(a, m.z, c2);
        T = T * (1.f - m.w);
        if (T == 0.f) break;
    }
    float* o = out + (((size_t)view * H + qy) * W + qx) * 3;
    o[0] = c0;
    o[1] = c1;
    o[2] = c2;
}

__global__ void k_warp_offsets(int D, int H, int W, const __grid_constant__ RLViews views, float* __restrict__ out) {
    const int qx = blockIdx.x * blockDim.x + threadIdx.x;
    const int qy = blockIdx.y;
    if (qx >= W) return;
    const RLWarp w = rl_warp_coeffs(views.v[0], (float)qx, (float)qy);
    for (int d = 0; d < D; ++d) {
        const float rho = views.rho[d];
        const bool ok = w.dir_ok && (fmaf(-rho, w.cz, 1.0f) > 0.0f);
        float* o = out + (((size_t)d * H + qy) * W + qx) * 2;
        o[0] = ok ? fmaf(rho, w.bx, w.ax) : __int_as_float(0x7fc00000);
        o[1] = ok ? fmaf(rho, w.by, w.ay) : __int_as_float(0x7fc00000);
    }
}

}  // namespace

rl_status rl_launch_render(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, float* out,
                           cudaStream_t s) {
    const int path = rl_kernel_path(H, W, views.n);
    if (path == 1) {
        CUtensorMap map;
        if (rl_encode_mpi_tmap(&map, M, dt, D, H, W)) return rl_launch_render_tma(map, M, dt, D, H, W, views, out, s);
    }
    if (path != 2) return rl_launch_render_pp(M, dt, D, H, W, views, out, s);
    dim3 block(kRenderBX, kRenderBY);
    const int tiles_x = (W + kRenderBX - 1) / kRenderBX, tiles_y = (H + kRenderBY - 1) / kRenderBY;
    const dim3 grid((unsigned)views.n, (unsigned)tiles_x, (unsigned)tiles_y);
    if (dt == RL_F32) {
        RLTraceScope ts("render_f32", s);
        k_render<float><<<grid, block, 0, s>>>((const float*)M, D, H, W, views, tiles_x, out);
    } else {
        RLTraceScope ts("render_bf16", s);
        k_render<__nv_bfloat16><<<grid, block, 0, s>>>((const __nv_bfloat16*)M, D, H, W, views, tiles_x, out);
    }
    return rl_check_launch("render");
}

rl_status rl_launch_warp_offsets(int D, int H, int W, const RLViews& views, float* out, cudaStream_t s) {
    RLTraceScope ts("warp_offsets", s);
    k_warp_offsets<<<dim3((W + 127) / 128, H), 128, 0, s>>>(D, H, W, views, out);
    return rl_check_launch("warp_offsets");
}
