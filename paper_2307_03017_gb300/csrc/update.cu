// update.cu -- masked update M_{n+1} = M_n + R(-lambda G_s, S) (Sec. 3.3, "Sparse Gradient
// Update"), with the coarse-to-fine nearest-neighbour upsampling of a level-l step.
//
// One thread per full-resolution pixel (y, x): for each kept slot j of its level-l pixel
// p = (y >> l, x >> l), plane d = S[j][p] takes M[d][y][x] -= lambda G[j][p], clamped to
// [0, 1] when asked, then rounded to the storage type (round to nearest even for BF16).
// Only k of the D planes are read and written.  With lambda_s != 0 the sparsity prior of
// Sec. 3.4 joins the alpha step: lambda_s sign(0.5 - a) / ((1.5 - |0.5 - a|) h w D), with a
// the alpha of the level MPI Ml.
#include <type_traits>

#include "rl_internal.h"

namespace {

template <typename Tm>
__device__ __forceinline__ void update_pixel(Tm* __restrict__ M, int D, int H, int W, int level,
                                             const uint8_t* __restrict__ S, const float* __restrict__ G, int k,
                                             float lambda, int clamp01, const Tm* __restrict__ Ml, float prior_scale,
                                             int x, int y) {
    if (x >= W || y >= H) return;
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
        const size_t e = ((size_t)d * H + y) * W + x;
        if (!RL_IN(e, (size_t)D * H * W)) continue;
        Tm* ptr = M + e * 4;
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

template <typename Tm>
__global__ void __launch_bounds__(128)
k_update(Tm* __restrict__ M, int D, int H, int W, int level, const uint8_t* __restrict__ S,
         const float* __restrict__ G, int k, float lambda, int clamp01, const Tm* __restrict__ Ml, float prior_scale) {
    update_pixel<Tm>(M, D, H, W, level, S, G, k, lambda, clamp01, Ml, prior_scale, blockIdx.x * blockDim.x + threadIdx.x,
                     blockIdx.y);
}

// Batched update: one persistent launch walks the update units of every item of a batch table
// (a unit is 128 pixels of one full-resolution row of one item, as k_update's grid).
template <typename Tm>
__global__ void __launch_bounds__(128)
k_update_batch(const RLBatchHeader* __restrict__ hdr, const RLBatchItem* __restrict__ items) {
    const unsigned n = hdr->n, total = hdr->upd_units;
    if (hdr->dtype != (std::is_same<Tm, float>::value ? (unsigned)RL_F32 : (unsigned)RL_BF16)) return;
    __shared__ unsigned next_slot;
    for (unsigned u = rl_batch_next(hdr, 3, &next_slot); u < total; u = rl_batch_next(hdr, 3, &next_slot)) {
        const RLBatchItem& it = items[rl_batch_find(items, n, u, &RLBatchItem::upd_begin)];
        const unsigned local = u - it.upd_begin;
        const int x = (int)(local % it.upd_tiles_x) * 128 + threadIdx.x, y = (int)(local / it.upd_tiles_x);
        update_pixel<Tm>(static_cast<Tm*>(it.M), it.D, it.H, it.W, it.level, it.S, it.G, it.k, it.lambda, it.clamp01,
                         static_cast<const Tm*>(it.Ml), it.prior_scale, x, y);
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

rl_status rl_launch_update_batch(const void* table, rl_dtype dt, cudaStream_t s) {
    const RLBatchHeader* hdr = static_cast<const RLBatchHeader*>(table);
    const RLBatchItem* items = rl_batch_items(table);
    const int grid = dt == RL_F32 ? rl_persistent_grid<k_update_batch<float>>(128, 0)
                                  : rl_persistent_grid<k_update_batch<__nv_bfloat16>>(128, 0);
    if (dt == RL_F32) {
        RLTraceScope ts("update_batch_f32", s);
        k_update_batch<float><<<grid, 128, 0, s>>>(hdr, items);
    } else {
        RLTraceScope ts("update_batch_bf16", s);
        k_update_batch<__nv_bfloat16><<<grid, 128, 0, s>>>(hdr, items);
    }
    return rl_check_launch("update_batch");
}

RL_DEBUG_READER(update)
