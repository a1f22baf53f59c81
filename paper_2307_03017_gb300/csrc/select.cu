// select.cu -- level pyramid of the MPI, the content-aligned top-k selection (Sec. 3.3
// "Gradient Sparsification") and image/tensor box downsampling.
//
// Pyramid: one thread per level-l voxel, the mean of its 2^l x 2^l full-resolution voxels
// (Sec. 3.2, hierarchical downsampling), rounded to the storage type.
//
// Selection: one thread per pixel.  Walking the planes nearest first, it forms the
// reference-view alpha weight A_d = alpha_d T_d (Eq. eq_gradient / eq_overA) with
// T_d = prod_{j>d}(1 - alpha_j), and keeps the k largest keys under the order
// (key descending, d ascending).  The kept planes become a 64-bit mask and the compact
// index list S[j][p] in ascending depth order, and the slot map used by the adjoint
// (slot j of plane S[j][p], RL_SLOT_NONE for the planes not kept); the compact gradient
// slots of the pixel are zeroed for the adjoint that follows.
//   k <= 8: a register-resident sorted list, one compare-exchange pass per plane.
//   k  > 8: rank counting over the D keys (O(D^2) per pixel, kept in local memory).
// MVS-sampling mode keeps instead the k consecutive planes around the argmax of the keys
// (ties to the lower d), shifted to stay within [0, D).
#include "rl_internal.h"

namespace {

__device__ __forceinline__ bool beats(float a, int ia, float b, int ib) { return a > b || (a == b && ia < ib); }

template <typename Tm, bool FROM_KEYS, int KMAX>
__global__ void __launch_bounds__(128)
k_select(const Tm* __restrict__ M, const float* __restrict__ keys, int D, int h, int w, int k,
         uint8_t* __restrict__ S, uint64_t* __restrict__ mask_out, uint8_t* __restrict__ slots,
         float* __restrict__ Gzero, unsigned* __restrict__ counter_zero, int mode) {
    const long long hw = (long long)h * w;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && counter_zero) *counter_zero = 0u;  // block counter of the loss epilogue that follows
    if (p >= hw) return;

    constexpr bool SMALL = KMAX <= 8;
    float kv[SMALL ? KMAX : 1];
    int ki[SMALL ? KMAX : 1];
    float allk[SMALL ? 1 : RL_DEV_MAX_PLANES];
    if constexpr (SMALL) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j) { kv[j] = -INFINITY; ki[j] = 255; }
    }
    // keys are formed nearest plane first; the loads of 16 planes are issued together
    constexpr int kBatch = 16;
    float T = 1.f;
    float best_key = -INFINITY;
    int best = D - 1;
    for (int d0 = D - 1; d0 >= 0; d0 -= kBatch) {
        float raw[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int d = d0 - u;
            if constexpr (FROM_KEYS)
                raw[u] = d >= 0 ? __ldg(keys + (size_t)d * hw + p) : 0.f;
            else
                raw[u] = d >= 0 ? RLStore<Tm>::load1(M + ((size_t)d * hw + p) * 4 + 3) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int d = d0 - u;
            if (d < 0) break;
            float key;
            if constexpr (FROM_KEYS) {
                key = raw[u];
            } else {
                key = raw[u] * T;
                T = T * (1.f - raw[u]);
            }
            if (!(key == key)) key = -INFINITY;  // NaN keys rank last
            if (key >= best_key) {  // walking towards lower d: ties go to the lower plane
                best_key = key;
                best = d;
            }
            if (mode == 1) continue;
            if constexpr (SMALL) {
                float cv = key;
                int ci = d;
#pragma unroll
                for (int j = 0; j < KMAX; ++j) {
                    if (j < k && beats(cv, ci, kv[j], ki[j])) {
                        const float tv = kv[j]; const int ti = ki[j];
                        kv[j] = cv; ki[j] = ci;
                        cv = tv; ci = ti;
                    }
                }
            } else {
                allk[d] = key;
            }
        }
    }
    uint64_t mk = 0;
    if (mode == 1) {
        int start = best - (k - 1) / 2;
        start = max(0, min(start, D - k));
        mk = (k >= 64 ? ~0ull : ((1ull << k) - 1ull)) << start;
    } else if constexpr (SMALL) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j < k) mk |= 1ull << ki[j];
    } else {
        for (int d = 0; d < D; ++d) {
            int rank = 0;
            for (int e = 0; e < D; ++e) rank += beats(allk[e], e, allk[d], d) ? 1 : 0;
            if (rank < k) mk |= 1ull << d;
        }
    }
    if (mask_out) mask_out[p] = mk;
    if (slots) {
        int j = 0;
        for (int d = 0; d < D; ++d) {
            const bool kept = (mk >> d) & 1ull;
            slots[(size_t)d * hw + p] = kept ? (uint8_t)j : (uint8_t)RL_SLOT_NONE;
            j += kept;
        }
    }
    uint64_t rem = mk;
    for (int j = 0; j < k; ++j) {
        const int d = __ffsll((long long)rem) - 1;
        rem &= rem - 1ull;
        if (S) S[(size_t)j * hw + p] = (uint8_t)d;
        if (Gzero) *reinterpret_cast<float4*>(Gzero + ((size_t)j * hw + p) * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <typename Tm, bool FROM_KEYS>
void launch_select_t(const void* M, const float* keys, int D, int h, int w, int k, uint8_t* S, uint64_t* mask,
                     uint8_t* slots, float* Gzero, unsigned* counter_zero, int mode, cudaStream_t s) {
    const long long hw = (long long)h * w;
    const int blocks = (int)((hw + 127) / 128);
    if (k <= 8 || mode == 1)
        k_select<Tm, FROM_KEYS, 8><<<blocks, 128, 0, s>>>((const Tm*)M, keys, D, h, w, k, S, mask, slots, Gzero,
                                                          counter_zero, mode);
    else
        k_select<Tm, FROM_KEYS, 64><<<blocks, 128, 0, s>>>((const Tm*)M, keys, D, h, w, k, S, mask, slots, Gzero,
                                                           counter_zero, mode);
}

template <typename Tm>
__global__ void __launch_bounds__(256)
k_pyramid(const Tm* __restrict__ M, int D, int H, int W, int level, Tm* __restrict__ Ml) {
    const int h = H >> level, w = W >> level, s = 1 << level;
    const long long n = (long long)D * h * w;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % w);
    const long long r = i / w;
    const int y = (int)(r % h);
    const int d = (int)(r / h);
    const Tm* base = M + (((size_t)d * H + (size_t)y * s) * W + (size_t)x * s) * 4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int yy = 0; yy < s; ++yy)
#pragma unroll 4
        for (int xx = 0; xx < s; ++xx) {
            const float4 v = RLStore<Tm>::load4(base + ((size_t)yy * W + xx) * 4);
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
    const float inv = 1.f / (float)(s * s);
    acc.x *= inv; acc.y *= inv; acc.z *= inv; acc.w *= inv;
    RLStore<Tm>::store4(Ml + (size_t)i * 4, acc);
}

__global__ void k_mask_to_slots(const uint64_t* __restrict__ mask, int D, int hw, uint8_t* __restrict__ slots) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= hw) return;
    const uint64_t mk = mask[p];
    int j = 0;
    for (int d = 0; d < D; ++d) {
        const bool kept = (mk >> d) & 1ull;
        slots[(size_t)d * hw + p] = kept ? (uint8_t)j : (uint8_t)RL_SLOT_NONE;
        j += kept;
    }
}

__global__ void k_downsample_f32(const float* __restrict__ x, int P, int H, int W, int C, int level,
                                 float* __restrict__ y) {
    const int h = H >> level, w = W >> level, s = 1 << level;
    const long long n = (long long)P * h * w * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int xx = (int)(r % w); r /= w;
    const int yy = (int)(r % h);
    const long long pl = r / h;
    const float* b = x + ((pl * H + (long long)yy * s) * W + (long long)xx * s) * C + c;
    float acc = 0.f;
    for (int a = 0; a < s; ++a)
        for (int bb = 0; bb < s; ++bb) acc += b[((long long)a * W + bb) * C];
    y[i] = acc * (1.f / (float)(s * s));
}

}  // namespace

rl_status rl_launch_select(const void* M, rl_dtype dt, const float* keys, int D, int h, int w, int k, uint8_t* S,
                           uint64_t* mask, uint8_t* slots, float* Gzero, cudaStream_t s, unsigned* counter_zero,
                           int mode) {
    if (keys) {
        RLTraceScope ts("select_keys", s);
        launch_select_t<float, true>(nullptr, keys, D, h, w, k, S, mask, slots, Gzero, counter_zero, mode, s);
    } else if (dt == RL_F32) {
        RLTraceScope ts("select_f32", s);
        launch_select_t<float, false>(M, nullptr, D, h, w, k, S, mask, slots, Gzero, counter_zero, mode, s);
    } else {
        RLTraceScope ts("select_bf16", s);
        launch_select_t<__nv_bfloat16, false>(M, nullptr, D, h, w, k, S, mask, slots, Gzero, counter_zero, mode, s);
    }
    return rl_check_launch("select");
}

rl_status rl_launch_pyramid(const void* M, rl_dtype dt, int D, int H, int W, int level, void* Ml, cudaStream_t s) {
    const long long n = (long long)D * (H >> level) * (W >> level);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (dt == RL_F32) {
        RLTraceScope ts("pyramid_f32", s);
        k_pyramid<float><<<blocks, 256, 0, s>>>((const float*)M, D, H, W, level, (float*)Ml);
    } else {
        RLTraceScope ts("pyramid_bf16", s);
        k_pyramid<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)M, D, H, W, level,
                                                        (__nv_bfloat16*)Ml);
    }
    return rl_check_launch("pyramid");
}

rl_status rl_launch_mask_to_slots(const uint64_t* mask, int D, int hw, uint8_t* slots, cudaStream_t s) {
    RLTraceScope ts("mask_to_slots", s);
    k_mask_to_slots<<<(hw + 255) / 256, 256, 0, s>>>(mask, D, hw, slots);
    return rl_check_launch("mask_to_slots");
}

rl_status rl_launch_downsample_f32(const float* x, int P, int H, int W, int C, int level, float* y, cudaStream_t s) {
    const long long n = (long long)P * (H >> level) * (W >> level) * C;
    if (n == 0) return RL_OK;
    RLTraceScope ts("downsample_f32", s);
    k_downsample_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, P, H, W, C, level, y);
    return rl_check_launch("downsample");
}
