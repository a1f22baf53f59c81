// update.cu -- masked update M_{n+1} = M_n + R(-lambda G_s, S) (Sec. 3.3, "Sparse Gradient
// Update"), with the coarse-to-fine nearest-neighbour upsampling of a level-l step.
//
// One thread per full-resolution pixel (y, x): for each kept slot j of its level-l pixel
// p = (y >> l, x >> l), plane d = S[j][p] takes M[d][y][x] -= lambda G[j][p], clamped to
// [0, 1] when asked, then rounded to the storage type (round to nearest even for BF16).
// Only k of the D planes are read and written.  With lambda_s != 0 the sparsity prior of
// Sec. 3.4 joins the alpha step: lambda_s sign(0.5 - a) / ((1.5 - |0.5 - a|) h w D), with a
// the alpha of the level MPI Ml.
#include "rl_internal.h"

namespace {

template <typename Tm>
__global__ void __launch_bounds__(128)
k_update(Tm* __restrict__ M, int D, int H, int W, int level, const uint8_t* __restrict__ S,
         const float* __restrict__ G, int k, float lambda, int clamp01, const Tm* __restrict__ Ml, float prior_scale) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const int w = W >> level, h = H >> level;
    const size_t hw = (size_t)h * w;
    const size_t p = (size_t)(y >> level) * w + (x >> level);
    for (int j = 0; j < k; ++j) {
        const int d = __ldg(S + (size_t)j * hw + p);
        if (d >= D) continue;
        float4 g = __ldg(reinterpret_cast<const float4*>(G) + (size_t)j * hw + p);
        if (prior_scale != 0.f) {
            const float a = RLStore<Tm>::load1(Ml + ((size_t)d * hw + p) * 4 + 3);
            const float sg = a < 0.5f ? 1.f : (a > 0.5f ? -1.f : 0.f);
            g.w += prior_scale * sg / (1.5f - fabsf(0.5f - a));
        }
        Tm* ptr = M + (((size_t)d * H + y) * W + x) * 4;
        float4 v = RLStore<Tm>::load4_nc(ptr);
        v.x = fmaf(-lambda, g.x, v.x);
        v.y = fmaf(-lambda, g.y, v.y);
        v.z = fmaf(-lambda, g.z, v.z);
        v.w = fmaf(-lambda, g.w, v.w);
        if (clamp01) {
            v.x = fminf(fmaxf(v.x, 0.f), 1.f);
            v.y = fminf(fmaxf(v.y, 0.f), 1.f);
            v.z = fminf(fmaxf(v.z, 0.f), 1.f);
            v.w = fminf(fmaxf(v.w, 0.f), 1.f);
        }
        RLStore<Tm>::store4(ptr, v);
    }
}

}  // namespace

rl_status rl_launch_update(void* M, rl_dtype dt, int D, int H, int W, int level, const uint8_t* S, const float* G,
                           int k, float lambda, int clamp01, cudaStream_t s, const void* Ml, float lambda_s) {
    dim3 grid((W + 127) / 128, H);
    // lambda_s / (h w D): the mean in L_s is over the level MPI's voxels
    const float prior_scale =
        (Ml && lambda_s != 0.f) ? (float)((double)lambda_s / ((double)(H >> level) * (W >> level) * D)) : 0.f;
    if (dt == RL_F32) {
        RLTraceScope ts("update_f32", s);
        k_update<float><<<grid, 128, 0, s>>>((float*)M, D, H, W, level, S, G, k, lambda, clamp01, (const float*)Ml,
                                             prior_scale);
    } else {
        RLTraceScope ts("update_bf16", s);
        k_update<__nv_bfloat16><<<grid, 128, 0, s>>>((__nv_bfloat16*)M, D, H, W, level, S, G, k, lambda, clamp01,
                                                     (const __nv_bfloat16*)Ml, prior_scale);
    }
    return rl_check_launch("update");
}
