// select.cu -- level pyramid of the MPI fused with the content-aligned top-k selection
// (Sec. 3.3 "Gradient Sparsification"), image/tensor box downsampling.
//
// One thread per level-l pixel.  Walking the planes nearest first, it forms the level-l
// voxel (mean of the 2^l x 2^l full-resolution voxels, stored to the level MPI), the
// reference-view alpha weight A_d = alpha_d T_d (Eq. eq_gradient / eq_overA) with
// T_d = prod_{j>d}(1 - alpha_j), and keeps the k largest keys under the order
// (key descending, d ascending).  The kept planes become a 64-bit mask and the compact
// index list S[j][p] in ascending depth order; the compact gradient slots of the pixel
// are zeroed for the adjoint that follows.
//   k <= 8: a register-resident sorted list, one compare-exchange pass per plane.
//   k  > 8: rank counting over the D keys (O(D^2) per pixel, kept in local memory).
#include "rl_internal.h"

namespace {

__device__ __forceinline__ bool beats(float a, int ia, float b, int ib) { return a > b || (a == b && ia < ib); }

template <typename Tm, bool FROM_KEYS, int KMAX>
__global__ void __launch_bounds__(128)
k_select(const Tm* __restrict__ M, const float* __restrict__ keys, int D, int Hf, int Wf, int level,
         Tm* __restrict__ Ml, int k, uint8_t* __restrict__ S, uint64_t* __restrict__ mask_out,
         float* __restrict__ Gzero) {
    const int h = Hf >> level, w = Wf >> level;
    const long long hw = (long long)h * w;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= hw) return;
    const int py = (int)(p / w), px = (int)(p - (long long)py * w);
    const int s = 1 << level;
    const float inv_area = 1.f / (float)(s * s);

    constexpr bool SMALL = KMAX <= 8;
    float kv[SMALL ? KMAX : 1];
    int ki[SMALL ? KMAX : 1];
    float allk[SMALL ? 1 : RL_DEV_MAX_PLANES];
    if constexpr (SMALL) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j) { kv[j] = -INFINITY; ki[j] = 255; }
    }
    float T = 1.f;
    for (int d = D - 1; d >= 0; --d) {
        float key;
        if constexpr (FROM_KEYS) {
            key = __ldg(keys + (size_t)d * hw + p);
        } else {
            float alpha;
            if (level == 0) {
                alpha = RLStore<Tm>::load1(M + ((size_t)d * hw + p) * 4 + 3);
            } else {
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                const Tm* base = M + ((size_t)d * Hf + (size_t)py * s) * Wf * 4;
                for (int yy = 0; yy < s; ++yy)
                    for (int xx = 0; xx < s; ++xx) {
                        const float4 v = RLStore<Tm>::load4(base + ((size_t)yy * Wf + (size_t)px * s + xx) * 4);
                        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
                    }
                acc.x *= inv_area; acc.y *= inv_area; acc.z *= inv_area; acc.w *= inv_area;
                Tm* dst = Ml + ((size_t)d * hw + p) * 4;
                RLStore<Tm>::store4(dst, acc);
                alpha = RLStore<Tm>::round1(acc.w);  // the stored value, which the adjoint will see
            }
            key = alpha * T;
            T = T * (1.f - alpha);
        }
        if (!(key == key)) key = -INFINITY;  // NaN keys rank last
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
    uint64_t mk = 0;
    if constexpr (SMALL) {
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
    uint64_t rem = mk;
    for (int j = 0; j < k; ++j) {
        const int d = __ffsll((long long)rem) - 1;
        rem &= rem - 1ull;
        if (S) S[(size_t)j * hw + p] = (uint8_t)d;
        if (Gzero) *reinterpret_cast<float4*>(Gzero + ((size_t)j * hw + p) * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <typename Tm, bool FROM_KEYS>
void launch_select_t(const void* M, const float* keys, int D, int Hf, int Wf, int level, void* Ml, int k,
                     uint8_t* S, uint64_t* mask, float* Gzero, cudaStream_t s) {
    const long long hw = (long long)(Hf >> level) * (Wf >> level);
    const int blocks = (int)((hw + 127) / 128);
    if (k <= 8)
        k_select<Tm, FROM_KEYS, 8><<<blocks, 128, 0, s>>>((const Tm*)M, keys, D, Hf, Wf, level, (Tm*)Ml, k, S, mask, Gzero);
    else
        k_select<Tm, FROM_KEYS, 64><<<blocks, 128, 0, s>>>((const Tm*)M, keys, D, Hf, Wf, level, (Tm*)Ml, k, S, mask, Gzero);
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

rl_status rl_launch_select(const void* M, rl_dtype dt, const float* keys, int D, int Hf, int Wf, int level, void* Ml,
                           int k, uint8_t* S, uint64_t* mask, float* Gzero, cudaStream_t s) {
    if (keys) {
        RLTraceScope ts("select_keys", s);
        launch_select_t<float, true>(nullptr, keys, D, Hf, Wf, 0, nullptr, k, S, mask, Gzero, s);
    } else if (dt == RL_F32) {
        RLTraceScope ts(level ? "pyramid_select_f32" : "select_f32", s);
        launch_select_t<float, false>(M, nullptr, D, Hf, Wf, level, Ml, k, S, mask, Gzero, s);
    } else {
        RLTraceScope ts(level ? "pyramid_select_bf16" : "select_bf16", s);
        launch_select_t<__nv_bfloat16, false>(M, nullptr, D, Hf, Wf, level, Ml, k, S, mask, Gzero, s);
    }
    return rl_check_launch("select");
}

rl_status rl_launch_downsample_f32(const float* x, int P, int H, int W, int C, int level, float* y, cudaStream_t s) {
    const long long n = (long long)P * (H >> level) * (W >> level) * C;
    if (n == 0) return RL_OK;
    RLTraceScope ts("downsample_f32", s);
    k_downsample_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, P, H, W, C, level, y);
    return rl_check_launch("downsample");
}
