// render.cu -- novel-view rendering (Eq. eq_render, Eq. eq_over) and warp diagnostics.
//
// One thread per target pixel: for d = D-1 .. 0 (nearest first) sample plane d at
// p = q + a(q) + rho_d b(q) (bilinear, zero padding per tap; coordinates anchored per block in
// FP64, rl_common.cuh) and accumulate
// C += T alpha c, T *= (1 - alpha).  The loop stops once T is exactly zero, after which
// every further term is exactly zero.  Views that are pure shifts of the reference (no
// rotation, no depth offset, same focal lengths) take a kernel that computes each plane's
// shift and weights once per block and renders four pixels of a column per thread, loading
// each tap row once.
#include "rl_internal.h"

namespace {

constexpr int kRenderBX = 32, kRenderBY = 4;
#ifndef RL_RENDER_MIN_BLOCKS
#define RL_RENDER_MIN_BLOCKS 1  // no register cap: measured fastest
#endif

// Blocks are ordered view-fastest (grid x = view) so that the views of a tile, whose plane
// footprints overlap, run together and share the MPI through L2.
template <typename Tm, bool ANCH>
__global__ void __launch_bounds__(kRenderBX* kRenderBY, RL_RENDER_MIN_BLOCKS)
k_render(const Tm* __restrict__ M, int D, int H, int W, const __grid_constant__ RLViews views, int tiles_x,
         float* __restrict__ out) {
    __shared__ RLAnchor sA;
    const int view = blockIdx.x;  // grid (views, tiles_x, tiles_y): views of a tile run together
    if (ANCH)
        rl_anchor_build(&sA, views, view, blockIdx.y * kRenderBX + kRenderBX / 2,
                        blockIdx.z * kRenderBY + kRenderBY / 2, D, threadIdx.y * kRenderBX + threadIdx.x,
                        kRenderBX * kRenderBY);
    const int qx = blockIdx.y * kRenderBX + threadIdx.x;
    const int qy = blockIdx.z * kRenderBY + threadIdx.y;
    if (qx >= W || qy >= H) return;
    const RLPixWarp<ANCH> w = rl_pix_warp<ANCH>(sA, views.v[view], qx, qy);
    const size_t plane = (size_t)H * W * 4;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll 1
    for (int d = D - 1; d >= 0; --d) {
        const RLTaps t = w.taps(sA, d, views.rho[d], qx, qy);
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

// Views with no rotation relative to the reference, no depth offset and the reference's
// focal lengths: the warp offset p - q = a + rho_d b is the same for every pixel of a plane,
// so the taps' integer shift and the bilinear weights are computed once per plane from the
// block's FP64 anchor table (rl_common.cuh) and read from shared memory.  Same samples, same
// results as k_render.
struct RLPlaneShift {
    int ix, iy, ok;
    float fx, fy;
    float w00, w10, w01, w11;
};

// One thread renders kShiftRows vertically adjacent pixels of a column: for each plane their
// taps span kShiftRows + 1 rows of two columns, loaded once (kShiftRows + 1 rows x 2 loads
// instead of kShiftRows x 4).
constexpr int kShiftRows = 4;

template <typename Tm>
__global__ void __launch_bounds__(kRenderBX* kRenderBY, 8)
k_render_shift(const Tm* __restrict__ M, int D, int H, int W, const __grid_constant__ RLViews views,
               float* __restrict__ out) {
    __shared__ RLPlaneShift sp[RL_DEV_MAX_PLANES];
    const int view = blockIdx.x;  // grid (views, tiles_x, tiles_y of kRenderBY * kShiftRows rows)
    const int tid = threadIdx.y * kRenderBX + threadIdx.x;
    if (tid < D) {
        // a pure shift: p - q = (c_r - c_v) + rho_d f_r C_xy for every pixel, formed in FP64 and
        // split into an integer and an FP32 fraction (the anchors of rl_common.cuh, exactly)
        const RLViewParam64& P = views.v64[view];
        const double rho = views.rho64[tid];
        const double kx = P.dcx + rho * (P.fxr * P.C[0]), ky = P.dcy + rho * (P.fyr * P.C[1]);
        const double flx = floor(kx), fly = floor(ky);
        RLPlaneShift p;
        p.ok = fabs(kx) < 1e9 && fabs(ky) < 1e9;
        p.ix = p.ok ? (int)flx : 0;
        p.iy = p.ok ? (int)fly : 0;
        p.fx = (float)(kx - flx);
        p.fy = (float)(ky - fly);
        p.w00 = (1.f - p.fx) * (1.f - p.fy);
        p.w10 = p.fx * (1.f - p.fy);
        p.w01 = (1.f - p.fx) * p.fy;
        p.w11 = p.fx * p.fy;
        sp[tid] = p;
    }
    __syncthreads();
    const int qx = blockIdx.y * kRenderBX + threadIdx.x;
    const int qy0 = (blockIdx.z * kRenderBY + threadIdx.y) * kShiftRows;
    if (qx >= W || qy0 >= H) return;
    const size_t plane = (size_t)H * W * 4;
    float T[kShiftRows], c0[kShiftRows], c1[kShiftRows], c2[kShiftRows];
#pragma unroll
    for (int r = 0; r < kShiftRows; ++r) { T[r] = 1.f; c0[r] = c1[r] = c2[r] = 0.f; }
    for (int d = D - 1; d >= 0; --d) {
        const RLPlaneShift p = sp[d];
        const int x0 = qx + p.ix, y0 = qy0 + p.iy;
        float4 m[kShiftRows];
        if (p.ok && (unsigned)x0 < (unsigned)(W - 1) && y0 >= 0 && y0 + kShiftRows < H) {
            // all kShiftRows + 1 tap rows inside: load each once
            const Tm* q = M + d * plane + (unsigned)(y0 * W + x0) * 4u;
            float4 a0 = RLStore<Tm>::load4(q), a1 = RLStore<Tm>::load4(q + 4);
#pragma unroll
            for (int r = 0; r < kShiftRows; ++r) {
                const Tm* qr = q + (r + 1) * 4 * W;
                const float4 b0 = RLStore<Tm>::load4(qr), b1 = RLStore<Tm>::load4(qr + 4);
                float2 lo = __fmul2_rn(make_float2(p.w00, p.w00), make_float2(a0.x, a0.y));
                float2 hi = __fmul2_rn(make_float2(p.w00, p.w00), make_float2(a0.z, a0.w));
                lo = __ffma2_rn(make_float2(p.w10, p.w10), make_float2(a1.x, a1.y), lo);
                hi = __ffma2_rn(make_float2(p.w10, p.w10), make_float2(a1.z, a1.w), hi);
                lo = __ffma2_rn(make_float2(p.w01, p.w01), make_float2(b0.x, b0.y), lo);
                hi = __ffma2_rn(make_float2(p.w01, p.w01), make_float2(b0.z, b0.w), hi);
                lo = __ffma2_rn(make_float2(p.w11, p.w11), make_float2(b1.x, b1.y), lo);
                hi = __ffma2_rn(make_float2(p.w11, p.w11), make_float2(b1.z, b1.w), hi);
                m[r] = make_float4(lo.x, lo.y, hi.x, hi.y);
                a0 = b0;
                a1 = b1;
            }
        } else {
#pragma unroll
            for (int r = 0; r < kShiftRows; ++r) {
                RLTaps t;
                t.x0 = x0;
                t.y0 = y0 + r;
                t.fx = p.fx;
                t.fy = p.fy;
                t.ok = p.ok != 0;
                m[r] = rl_sample(M + d * plane, H, W, t);
            }
        }
        bool any = false;
#pragma unroll
        for (int r = 0; r < kShiftRows; ++r) {
            const float a = T[r] * m[r].w;
            c0[r] = fmaf(a, m[r].x, c0[r]);
            c1[r] = fmaf(a, m[r].y, c1[r]);
            c2[r] = fmaf(a, m[r].z, c2[r]);
            T[r] = T[r] * (1.f - m[r].w);
            any |= T[r] != 0.f;
        }
        if (!any) break;  // every further term of every pixel is exactly zero
    }
#pragma unroll
    for (int r = 0; r < kShiftRows; ++r) {
        if (qy0 + r >= H) break;
        float* o = out + (((size_t)view * H + qy0 + r) * W + qx) * 3;
        o[0] = c0[r];
        o[1] = c1[r];
        o[2] = c2[r];
    }
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
    if (path != 2) return rl_launch_render_pp(M, dt, D, H, W, views, out, s);
    dim3 block(kRenderBX, kRenderBY);
    const int tiles_x = (W + kRenderBX - 1) / kRenderBX, tiles_y = (H + kRenderBY - 1) / kRenderBY;
    const dim3 grid((unsigned)views.n, (unsigned)tiles_x, (unsigned)tiles_y);
    if (rl_views_are_shifts(views)) {
        const dim3 sgrid((unsigned)views.n, (unsigned)tiles_x,
                         (unsigned)((H + kRenderBY * kShiftRows - 1) / (kRenderBY * kShiftRows)));
        if (dt == RL_F32) {
            RLTraceScope ts("render_shift_f32", s);
            k_render_shift<float><<<sgrid, block, 0, s>>>((const float*)M, D, H, W, views, out);
        } else {
            RLTraceScope ts("render_shift_bf16", s);
            k_render_shift<__nv_bfloat16><<<sgrid, block, 0, s>>>((const __nv_bfloat16*)M, D, H, W, views, out);
        }
        return rl_check_launch("render");
    }
    if (dt == RL_F32) {
        RLTraceScope ts("render_f32", s);
        if (views.anchored) k_render<float, true><<<grid, block, 0, s>>>((const float*)M, D, H, W, views, tiles_x, out);
        else k_render<float, false><<<grid, block, 0, s>>>((const float*)M, D, H, W, views, tiles_x, out);
    } else {
        RLTraceScope ts("render_bf16", s);
        if (views.anchored)
            k_render<__nv_bfloat16, true><<<grid, block, 0, s>>>((const __nv_bfloat16*)M, D, H, W, views, tiles_x, out);
        else
            k_render<__nv_bfloat16, false><<<grid, block, 0, s>>>((const __nv_bfloat16*)M, D, H, W, views, tiles_x, out);
    }
    return rl_check_launch("render");
}

rl_status rl_launch_warp_offsets(int D, int H, int W, const RLViews& views, float* out, cudaStream_t s) {
    RLTraceScope ts("warp_offsets", s);
    k_warp_offsets<<<dim3((W + 127) / 128, H), 128, 0, s>>>(D, H, W, views, out);
    return rl_check_launch("warp_offsets");
}

RL_DEBUG_READER(render)
