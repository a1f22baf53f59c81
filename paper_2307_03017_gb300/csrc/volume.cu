// volume.cu -- the sparsified gradient volume V_s of Sec. 3.3 (Eq. eq_simplifiedGradients and
// eq_V): for every kept voxel (slot j of level pixel p, plane d = S[j][p]) the C = 4N + 4
// channels [P (3N, view-major), A^{w^-1}_1..N (N), M_l (4)], stored [C][k][h][w] FP32.
//
// k_view_alpha (one thread per view pixel q, all views in one launch, view-fastest blocks):
//   the alpha weights of the level MPI warped into view i (Eq. eq_gradient on M_i),
//   A_{i,d}(q) = alpha_d(q) prod_{j>d}(1 - alpha_j(q)), nearest plane first, stored
//   [N][D][h][w] FP32.  The warp and the bilinear alpha sample are the render's.
// k_volume (one thread per kept voxel and view): the level pixel carried into view i by the
//   inverse warp (reference -> view) at plane d; a bilinear sample (zero padding) of A_{i,d}
//   there; the PSV channels as the mean of the full-resolution PSV samples of the 2^l x 2^l
//   child pixels (Sec. 3.2 downsamples the full-resolution volume); and M_l[d][p].
// k_volume_packed: the same channels, written as the learned network's BF16 channels-last
//   input instead of the FP32 [C][k][h][w] volume.
#include "rl_internal.h"

namespace {

constexpr int kAlphaBX = 32, kAlphaBY = 4;

// Bilinear sample (zero padding per tap) of the alpha channel of one plane [H][W][4].
template <typename Tm>
__device__ __forceinline__ float sample_alpha(const Tm* __restrict__ plane, int H, int W, const RLTaps& t) {
    if (!t.ok) return 0.f;
    const float w00 = (1.f - t.fx) * (1.f - t.fy), w10 = t.fx * (1.f - t.fy);
    const float w01 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
    const size_t r0 = (size_t)t.y0 * W, r1 = r0 + W;
    if ((unsigned)t.x0 < (unsigned)(W - 1) && (unsigned)t.y0 < (unsigned)(H - 1)) {
        // all four taps inside: the same products in the same order, without the per-tap tests
        float a = fmaf(w00, RLStore<Tm>::load1(plane + (r0 + t.x0) * 4 + 3), 0.f);
        a = fmaf(w10, RLStore<Tm>::load1(plane + (r0 + t.x0 + 1) * 4 + 3), a);
        a = fmaf(w01, RLStore<Tm>::load1(plane + (r1 + t.x0) * 4 + 3), a);
        return fmaf(w11, RLStore<Tm>::load1(plane + (r1 + t.x0 + 1) * 4 + 3), a);
    }
    const bool x0in = (unsigned)t.x0 < (unsigned)W, x1in = (unsigned)(t.x0 + 1) < (unsigned)W;
    const bool y0in = (unsigned)t.y0 < (unsigned)H, y1in = (unsigned)(t.y0 + 1) < (unsigned)H;
    float a = 0.f;
    if (y0in && x0in) a = fmaf(w00, RLStore<Tm>::load1(plane + (r0 + t.x0) * 4 + 3), a);
    if (y0in && x1in) a = fmaf(w10, RLStore<Tm>::load1(plane + (r0 + t.x0 + 1) * 4 + 3), a);
    if (y1in && x0in) a = fmaf(w01, RLStore<Tm>::load1(plane + (r1 + t.x0) * 4 + 3), a);
    if (y1in && x1in) a = fmaf(w11, RLStore<Tm>::load1(plane + (r1 + t.x0 + 1) * 4 + 3), a);
    return a;
}

// Bilinear sample (zero padding per tap) of a [H][W][C] FP32 map; C = 1 or 3.
template <int C>
__device__ __forceinline__ void sample_map(const float* __restrict__ img, int H, int W, const RLTaps& t, float* out) {
#pragma unroll
    for (int c = 0; c < C; ++c) out[c] = 0.f;
    if (!t.ok) return;
    const float wt[4] = {(1.f - t.fx) * (1.f - t.fy), t.fx * (1.f - t.fy), (1.f - t.fx) * t.fy, t.fx * t.fy};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = t.x0 + (k & 1), y = t.y0 + (k >> 1);
        if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) continue;
        const float* v = img + ((size_t)y * W + x) * C;
#pragma unroll
        for (int c = 0; c < C; ++c) out[c] = fmaf(wt[k], __ldg(v + c), out[c]);
    }
}

template <typename Tm, bool ANCH>
__global__ void __launch_bounds__(kAlphaBX * kAlphaBY)
k_view_alpha(const Tm* __restrict__ M, int D, int H, int W, const __grid_constant__ RLViews views,
             float* __restrict__ A) {
    __shared__ RLAnchor sA;
    const int view = blockIdx.x;  // grid (views, tiles_x, tiles_y)
    if (ANCH)
        rl_anchor_build(&sA, views, view, blockIdx.y * kAlphaBX + kAlphaBX / 2, blockIdx.z * kAlphaBY + kAlphaBY / 2,
                        D, threadIdx.y * kAlphaBX + threadIdx.x, kAlphaBX * kAlphaBY);
    const int qx = blockIdx.y * kAlphaBX + threadIdx.x;
    const int qy = blockIdx.z * kAlphaBY + threadIdx.y;
    if (qx >= W || qy >= H) return;
    const RLPixWarp<ANCH> w = rl_pix_warp<ANCH>(sA, views.v[view], qx, qy);
    const size_t plane = (size_t)H * W * 4, hw = (size_t)H * W;
    float* out = A + (size_t)view * D * hw + (size_t)qy * W + qx;
    float T = 1.f;
    for (int d = D - 1; d >= 0; --d) {
        const RLTaps t = w.taps(sA, d, views.rho[d], qx, qy);
        const float a = sample_alpha(M + d * plane, H, W, t);
        out[(size_t)d * hw] = a * T;
        T = T * (1.f - a);
    }
}

// Channels of kept voxel (p = (x, y), plane d) from view i: the inverse-warped alpha weight a
// and the PSV colour psv[3] (the mean of the full-resolution samples of p's children).
__device__ __forceinline__ void voxel_view(const float* __restrict__ A, const float* __restrict__ images,
                                           const RLInvViews& iv, int D, int h, int w, int level, int x, int y,
                                           int d, int i, float& a, float (&psv)[3]) {
    const long long hw = (long long)h * w;
    const float rho = iv.rho[d];
    const int s = 1 << level, H = h << level, W = w << level;
    const float inv_area = 1.f / (float)(s * s);
    // inverse-warped alpha weight of view i, at level l
    const RLInvWarp c = rl_inv_coeffs(iv.lv[i], (float)x, (float)y);
    sample_map<1>(A + ((size_t)i * D + d) * hw, h, w, rl_inv_taps(c, iv.lv[i], rho, x, y), &a);
    // PSV of view i: mean over the full-resolution children of p
    float acc[3] = {0.f, 0.f, 0.f};
    const float* img = images + (size_t)i * H * W * 3;
    for (int yy = 0; yy < s; ++yy)
        for (int xx = 0; xx < s; ++xx) {
            const int X = x * s + xx, Y = y * s + yy;
            const RLInvWarp cf = rl_inv_coeffs(iv.full[i], (float)X, (float)Y);
            float v[3];
            sample_map<3>(img, H, W, rl_inv_taps(cf, iv.full[i], rho, X, Y), v);
            acc[0] += v[0];
            acc[1] += v[1];
            acc[2] += v[2];
        }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) psv[ch] = acc[ch] * inv_area;
}

template <typename Tm>
__global__ void __launch_bounds__(128)
k_volume(const Tm* __restrict__ Ml, int D, int h, int w, int level, const uint8_t* __restrict__ S, int k,
         const float* __restrict__ A, const float* __restrict__ images, const __grid_constant__ RLInvViews iv,
         float* __restrict__ V) {
    // grid (pixel blocks, k, N): one thread per (kept voxel, view); view 0 also writes M_l
    const long long hw = (long long)h * w;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, i = blockIdx.z;
    if (p >= hw) return;
    const int y = (int)(p / w), x = (int)(p % w);
    const int d = __ldg(S + (size_t)j * hw + p);
    const int N = iv.n;
    const size_t cstride = (size_t)k * hw;  // channel stride of V
    float* out = V + (size_t)j * hw + p;
    if (d >= D) {  // not a plane: the voxel's channels are zero
        out[(size_t)(3 * i) * cstride] = 0.f;
        out[(size_t)(3 * i + 1) * cstride] = 0.f;
        out[(size_t)(3 * i + 2) * cstride] = 0.f;
        out[(size_t)(3 * N + i) * cstride] = 0.f;
        if (i == 0)
            for (int c = 0; c < 4; ++c) out[(size_t)(4 * N + c) * cstride] = 0.f;
        return;
    }
    if (!RL_IN(d, D)) return;
    float a, psv[3];
    voxel_view(A, images, iv, D, h, w, level, x, y, d, i, a, psv);
    out[(size_t)(3 * N + i) * cstride] = a;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) out[(size_t)(3 * i + ch) * cstride] = psv[ch];
    if (i == 0) {
        const float4 m = RLStore<Tm>::load4(Ml + ((size_t)d * hw + p) * 4);
        out[(size_t)(4 * N + 0) * cstride] = m.x;
        out[(size_t)(4 * N + 1) * cstride] = m.y;
        out[(size_t)(4 * N + 2) * cstride] = m.z;
        out[(size_t)(4 * N + 3) * cstride] = m.w;
    }
}

// The same volume as the network's input: act [k][h][w][32] BF16 channels-last (round to
// nearest even), channels >= 4N + 4 zero.  Block = N warps over 32 consecutive voxels of one
// slot, warp i computing view i (the gathers of a warp stay those of one view); the voxels'
// channels meet in shared memory and leave as one contiguous 64-byte record per voxel.
template <typename Tm>
__global__ void __launch_bounds__(32 * RL_DEV_MAX_VIEWS)
k_volume_packed(const Tm* __restrict__ Ml, int D, int h, int w, int level, const uint8_t* __restrict__ S,
                const float* __restrict__ A, const float* __restrict__ images, const __grid_constant__ RLInvViews iv,
                __nv_bfloat16* __restrict__ act) {
    __shared__ float rec[32][33];  // 32 voxels x 32 channels (+1: rows start on different banks)
    const long long hw = (long long)h * w;
    const int lane = threadIdx.x & 31, i = threadIdx.x >> 5;
    const long long p0 = (long long)blockIdx.x * 32;
    const long long p = p0 + lane;
    const int j = blockIdx.y;
    const int N = iv.n, C = 4 * N + 4;
    if (p < hw) {
        // each warp writes every channel it owns, zeros included, so no fill is needed
        float a = 0.f, psv[3] = {0.f, 0.f, 0.f};
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
        const int d = __ldg(S + (size_t)j * hw + p);
        if (d < D) {
            const int y = (int)(p / w), x = (int)(p % w);
            voxel_view(A, images, iv, D, h, w, level, x, y, d, i, a, psv);
            if (i == 0) m = RLStore<Tm>::load4(Ml + ((size_t)d * hw + p) * 4);
        }
        rec[lane][3 * i] = psv[0];
        rec[lane][3 * i + 1] = psv[1];
        rec[lane][3 * i + 2] = psv[2];
        rec[lane][3 * N + i] = a;
        if (i == 0) {
            rec[lane][4 * N + 0] = m.x;
            rec[lane][4 * N + 1] = m.y;
            rec[lane][4 * N + 2] = m.z;
            rec[lane][4 * N + 3] = m.w;
        }
    }
    __syncthreads();
    // 32 voxels x 4 chunks of 8 channels, 16 bytes each; channels >= C are zero
    for (int t = threadIdx.x; t < 128; t += blockDim.x) {
        const int v = t >> 2, chunk = t & 3;
        if (p0 + v >= hw) continue;
        float r[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) r[e] = chunk * 8 + e < C ? rec[v][chunk * 8 + e] : 0.f;
        uint4 pk;
        __nv_bfloat162 q0 = __floats2bfloat162_rn(r[0], r[1]), q1 = __floats2bfloat162_rn(r[2], r[3]);
        __nv_bfloat162 q2 = __floats2bfloat162_rn(r[4], r[5]), q3 = __floats2bfloat162_rn(r[6], r[7]);
        pk.x = *reinterpret_cast<uint32_t*>(&q0);
        pk.y = *reinterpret_cast<uint32_t*>(&q1);
        pk.z = *reinterpret_cast<uint32_t*>(&q2);
        pk.w = *reinterpret_cast<uint32_t*>(&q3);
        *reinterpret_cast<uint4*>(act + ((size_t)j * hw + p0 + v) * 32 + chunk * 8) = pk;
    }
}

}  // namespace

rl_status rl_launch_view_alpha(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, float* A,
                               cudaStream_t s) {
    const dim3 grid((unsigned)views.n, (unsigned)((W + kAlphaBX - 1) / kAlphaBX),
                    (unsigned)((H + kAlphaBY - 1) / kAlphaBY));
    const dim3 block(kAlphaBX, kAlphaBY);
    if (dt == RL_F32) {
        RLTraceScope ts("view_alpha_f32", s);
        if (views.anchored) k_view_alpha<float, true><<<grid, block, 0, s>>>((const float*)M, D, H, W, views, A);
        else k_view_alpha<float, false><<<grid, block, 0, s>>>((const float*)M, D, H, W, views, A);
    } else {
        RLTraceScope ts("view_alpha_bf16", s);
        if (views.anchored)
            k_view_alpha<__nv_bfloat16, true><<<grid, block, 0, s>>>((const __nv_bfloat16*)M, D, H, W, views, A);
        else
            k_view_alpha<__nv_bfloat16, false><<<grid, block, 0, s>>>((const __nv_bfloat16*)M, D, H, W, views, A);
    }
    return rl_check_launch("view_alpha");
}

rl_status rl_launch_volume(const void* Ml, rl_dtype dt, int D, int h, int w, int level, const uint8_t* S, int k,
                           const float* A, const float* images, const RLInvViews& iv, float* V, cudaStream_t s,
                           void* act) {
    const long long hw = (long long)h * w;
    if (act) {
        const dim3 grid((unsigned)((hw + 31) / 32), (unsigned)k);
        const unsigned block = 32u * (unsigned)iv.n;
        if (dt == RL_F32) {
            RLTraceScope ts("volume_packed_f32", s);
            k_volume_packed<float><<<grid, block, 0, s>>>((const float*)Ml, D, h, w, level, S, A, images, iv,
                                                          (__nv_bfloat16*)act);
        } else {
            RLTraceScope ts("volume_packed_bf16", s);
            k_volume_packed<__nv_bfloat16><<<grid, block, 0, s>>>((const __nv_bfloat16*)Ml, D, h, w, level, S, A,
                                                                  images, iv, (__nv_bfloat16*)act);
        }
        return rl_check_launch("volume");
    }
    const dim3 grid((unsigned)((hw + 127) / 128), (unsigned)k, (unsigned)iv.n);
    if (dt == RL_F32) {
        RLTraceScope ts("volume_f32", s);
        k_volume<float><<<grid, 128, 0, s>>>((const float*)Ml, D, h, w, level, S, k, A, images, iv, V);
    } else {
        RLTraceScope ts("volume_bf16", s);
        k_volume<__nv_bfloat16><<<grid, 128, 0, s>>>((const __nv_bfloat16*)Ml, D, h, w, level, S, k, A, images, iv,
                                                     V);
    }
    return rl_check_launch("volume");
}

RL_DEBUG_READER(volume)
