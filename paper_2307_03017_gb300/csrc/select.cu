// select.cu -- level pyramid of the MPI, the content-aligned top-k selection (Sec. 3.3
// "Gradient Sparsification") and image/tensor box downsampling.
//
// Pyramid: each level-l voxel is the mean of its 2^l x 2^l full-resolution voxels (Sec. 3.2,
// hierarchical downsampling), rounded to the storage type.
//
// Selection: one thread per pixel.  Walking the planes nearest first, it forms the
// reference-view alpha weight A_d = alpha_d T_d (Eq. eq_gradient / eq_overA) with
// T_d = prod_{j>d}(1 - alpha_j), and keeps the k largest keys under the order
// (key descending, d ascending).  The kept planes become a 64-bit mask and the compact
// index list S[j][p] in ascending depth order, and the slot map used by the adjoint
// (slot j of plane S[j][p], RL_SLOT_NONE for the planes not kept); the compact gradient
// slots of the pixel are zeroed for the adjoint that follows.
//   k <= 8: a register-resident sorted list (compiled for each k), entered only by planes
//           whose key reaches its last entry.
//   k  > 8: rank counting over the D keys (O(D^2) per pixel, kept in local memory).
// MVS-sampling mode keeps instead the k consecutive planes around the argmax of the keys
// (ties to the lower d), shifted to stay within [0, D).
// On the coarse levels of an HSGD step the pyramid and the selection run as one kernel: the
// level voxels of a tile of pixels go to Ml and, through shared memory, to the selection.
// The same pass writes the level source images (2^l x 2^l means of the full-resolution
// images) that the gradient of that level reads, one pixel a view.
#include <type_traits>

#include "rl_internal.h"

namespace {

__device__ __forceinline__ bool beats(float a, int ia, float b, int ib) { return a > b || (a == b && ia < ib); }

// Per-pixel selection.  raw_at(d) gives alpha_d (keys mode: the key of plane d).  Returns the
// 64-bit mask of the kept planes.
//   K <= 8: a register-resident list of the K best, sorted by (key descending, d ascending);
//   its first k <= K entries are kept.  The walk
//   visits the planes in descending d, so a new plane is below every listed one and wins
//   every tie: it enters iff key >= the last listed key, and the insertion is a chain of
//   `>=` compare-exchanges.  Planes that cannot enter cost one comparison.
//   K == 64: rank counting over the D keys (O(D^2), kept in local memory).
// mode 1 (MVS sampling) keeps the k consecutive planes around the argmax of the keys.
template <int K, bool FROM_KEYS, typename RawFn>
__device__ __forceinline__ uint64_t select_mask(const RawFn& raw_at, int D, int k, int mode) {
    constexpr bool SMALL = K <= 8;
    float kv[SMALL ? K : 1];
    int ki[SMALL ? K : 1];
    float allk[SMALL ? 1 : RL_DEV_MAX_PLANES];
    if constexpr (SMALL) {
#pragma unroll
        for (int j = 0; j < K; ++j) { kv[j] = -INFINITY; ki[j] = 255; }
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
            raw[u] = d >= 0 ? raw_at(d) : 0.f;
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
            if (mode == 1) {
                if (key >= best_key) {  // walking towards lower d: ties go to the lower plane
                    best_key = key;
                    best = d;
                }
                continue;
            }
            if constexpr (SMALL) {
                if (key >= kv[K - 1]) {
                    float cv = key;
                    int ci = d;
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        if (cv >= kv[j]) {
                            const float tv = kv[j]; const int ti = ki[j];
                            kv[j] = cv; ki[j] = ci;
                            cv = tv; ci = ti;
                        }
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
        // the list holds the top K in order; its first k entries are the top k (k <= K)
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (j < k) mk |= 1ull << ki[j];
    } else {
        for (int d = 0; d < D; ++d) {
            int rank = 0;
            for (int e = 0; e < D; ++e) rank += beats(allk[e], e, allk[d], d) ? 1 : 0;
            if (rank < k) mk |= 1ull << d;
        }
    }
    return mk;
}

// Writes the selection of pixel p: mask, slot map, compact list S (ascending depth) and
// zeroes the pixel's compact gradient slots.
__device__ __forceinline__ void write_selection(uint64_t mk, int D, int k, long long hw, long long p,
                                                uint8_t* __restrict__ S, uint64_t* __restrict__ mask_out,
                                                uint8_t* __restrict__ slots, float* __restrict__ Gzero) {
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
        if (S && RL_IN(d, D)) S[(size_t)j * hw + p] = (uint8_t)d;
        if (Gzero) *reinterpret_cast<float4*>(Gzero + ((size_t)j * hw + p) * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <typename Tm, bool FROM_KEYS, int K>
__global__ void __launch_bounds__(128)
k_select(const Tm* __restrict__ M, const float* __restrict__ keys, int D, int h, int w, int k,
         uint8_t* __restrict__ S, uint64_t* __restrict__ mask_out, uint8_t* __restrict__ slots,
         float* __restrict__ Gzero, unsigned* __restrict__ counter_zero, int mode) {
    const long long hw = (long long)h * w;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && counter_zero) *counter_zero = 0u;  // block counter of the loss epilogue that follows
    if (p >= hw) return;
    const uint64_t mk = select_mask<K, FROM_KEYS>(
        [&](int d) {
            if constexpr (FROM_KEYS) return __ldg(keys + (size_t)d * hw + p);
            else return RLStore<Tm>::load1(M + ((size_t)d * hw + p) * 4 + 3);
        },
        D, k, mode);
    write_selection(mk, D, k, hw, p, S, mask_out, slots, Gzero);
}

// Mean of the 2^l x 2^l full-resolution voxels of level voxel (d, y, x), summed row by row.
template <typename Tm, int LOG>
__device__ __forceinline__ float4 pyramid_mean(const Tm* __restrict__ M, int H, int W, int level, int d, int y,
                                               int x) {
    const int s = LOG >= 0 ? (1 << LOG) : (1 << level);
    const Tm* base = M + (((size_t)d * H + (size_t)y * s) * W + (size_t)x * s) * 4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (LOG >= 0) {
        constexpr int SS = 1 << LOG;
        float4 v[SS * SS];
#pragma unroll
        for (int yy = 0; yy < SS; ++yy)
#pragma unroll
            for (int xx = 0; xx < SS; ++xx) v[yy * SS + xx] = RLStore<Tm>::load4(base + ((size_t)yy * W + xx) * 4);
#pragma unroll
        for (int i = 0; i < SS * SS; ++i) {
            acc.x += v[i].x; acc.y += v[i].y; acc.z += v[i].z; acc.w += v[i].w;
        }
    } else {
        for (int yy = 0; yy < s; ++yy)
#pragma unroll 4
            for (int xx = 0; xx < s; ++xx) {
                const float4 v = RLStore<Tm>::load4(base + ((size_t)yy * W + xx) * 4);
                acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
            }
    }
    const float inv = 1.f / (float)(s * s);
    acc.x *= inv; acc.y *= inv; acc.z *= inv; acc.w *= inv;
    return acc;
}

// Pyramid level l and its selection in one pass.  A block takes kTile consecutive level
// pixels: its threads form the kTile x D level voxels (a warp per plane row of the tile),
// store them to Ml and keep their alphas, as stored, in shared memory; the first warp then
// selects for the tile's pixels from shared memory.  Same arithmetic as forming Ml and then
// running the selection kernel on it.
constexpr int kTile = 32;

template <typename Tm, int K, int LOG>
__device__ __forceinline__ void pyramid_select_tile(const Tm* __restrict__ M, int D, int H, int W, int level,
                                                    Tm* __restrict__ Ml, int k, uint8_t* __restrict__ S,
                                                    uint8_t* __restrict__ slots, float* __restrict__ Gzero,
                                                    unsigned* __restrict__ counter_zero, int mode, long long p0,
                                                    float (*alpha)[kTile]) {
    const int h = H >> level, w = W >> level;
    const long long hw = (long long)h * w;
    if (p0 == 0 && threadIdx.x == 0 && counter_zero) *counter_zero = 0u;
    // level 1: the loads of NB voxels (4 full-resolution voxels each) are issued together
    constexpr int NB = LOG == 1 ? 4 : 1;
    for (int i0 = threadIdx.x; i0 < D * kTile; i0 += NB * blockDim.x) {
        float4 v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = i0 + b * blockDim.x;
            const long long p = p0 + i % kTile;
            if (i < D * kTile && p < hw)
                v[b] = pyramid_mean<Tm, LOG>(M, H, W, level, i / kTile, (int)(p / w), (int)(p % w));
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = i0 + b * blockDim.x;
            const int d = i / kTile, j = i % kTile;
            const long long p = p0 + j;
            if (i >= D * kTile || p >= hw) continue;
            RLStore<Tm>::store4(Ml + ((size_t)d * hw + p) * 4, v[b]);
            alpha[d][j] = RLStore<Tm>::round1(v[b].w);
        }
    }
    __syncthreads();
    const int j = threadIdx.x;
    const long long p = p0 + j;
    if (j < kTile && p < hw) {
        const uint64_t mk = select_mask<K, false>([&](int d) { return alpha[d][j]; }, D, k, mode);
        write_selection(mk, D, k, hw, p, S, nullptr, slots, Gzero);
    }
}

// The level-l source images Il [N][h][w][3]: each value the mean of the 2^l x 2^l
// full-resolution pixels, summed row by row and scaled by 1 / 4^l -- exactly what the gradient
// kernels form on the fly from full-resolution images -- for the tile's kTile pixels.
template <int LOG>
__device__ __forceinline__ void level_image_means(const float* __restrict__ images, int N, int H, int W, int level,
                                                  float* __restrict__ Il, long long p0) {
    const int s = LOG >= 0 ? (1 << LOG) : (1 << level), h = H >> level, w = W >> level;
    const long long hw = (long long)h * w;
    const float inv_area = 1.f / (float)(s * s);
    for (int i = threadIdx.x; i < N * kTile; i += blockDim.x) {
        const int v = i / kTile;
        const long long p = p0 + i % kTile;
        if (p >= hw) continue;
        const int y = (int)(p / w), x = (int)(p % w);
        const float* img = images + (size_t)v * H * W * 3;
        float i0 = 0.f, i1 = 0.f, i2 = 0.f;
        if constexpr (LOG >= 0) {
            // every load of the 4^l children issued before the first add (same sums, same order)
            constexpr int SS = 1 << LOG;
            float c[SS * SS * 3];
#pragma unroll
            for (int yy = 0; yy < SS; ++yy)
#pragma unroll
                for (int xx = 0; xx < SS; ++xx) {
                    const float* px = img + ((size_t)(y * SS + yy) * W + (x * SS + xx)) * 3;
                    c[(yy * SS + xx) * 3] = __ldg(px);
                    c[(yy * SS + xx) * 3 + 1] = __ldg(px + 1);
                    c[(yy * SS + xx) * 3 + 2] = __ldg(px + 2);
                }
#pragma unroll
            for (int q = 0; q < SS * SS; ++q) {
                i0 += c[q * 3];
                i1 += c[q * 3 + 1];
                i2 += c[q * 3 + 2];
            }
        } else {
            for (int yy = 0; yy < s; ++yy)
                for (int xx = 0; xx < s; ++xx) {
                    const float* px = img + ((size_t)(y * s + yy) * W + (x * s + xx)) * 3;
                    i0 += __ldg(px);
                    i1 += __ldg(px + 1);
                    i2 += __ldg(px + 2);
                }
        }
        float* o = Il + ((size_t)v * hw + p) * 3;
        o[0] = __fmul_rn(i0, inv_area);
        o[1] = __fmul_rn(i1, inv_area);
        o[2] = __fmul_rn(i2, inv_area);
    }
}

// With Il != NULL the block also writes the tile's level images (level_image_means), so that
// the gradient that follows reads one pixel per view instead of 4^l.
template <typename Tm, int K, int LOG>
__global__ void __launch_bounds__(256)
k_pyramid_select(const Tm* __restrict__ M, int D, int H, int W, int level, Tm* __restrict__ Ml, int k,
                 uint8_t* __restrict__ S, uint8_t* __restrict__ slots, float* __restrict__ Gzero,
                 unsigned* __restrict__ counter_zero, int mode, const float* __restrict__ images, int N,
                 float* __restrict__ Il) {
    __shared__ float alpha[RL_DEV_MAX_PLANES][kTile];
    if (Il) level_image_means<LOG>(images, N, H, W, level, Il, (long long)blockIdx.x * kTile);
    pyramid_select_tile<Tm, K, LOG>(M, D, H, W, level, Ml, k, S, slots, Gzero, counter_zero, mode,
                                    (long long)blockIdx.x * kTile, alpha);
}

// ------------------------------------------------------------------ batched selection
//
// One persistent launch selects for every item of a batch table (the selection stage of one
// HSGD iteration of each request): a unit is 256 level-0 pixels (one a thread, as k_select)
// or one 32-pixel pyramid tile (as k_pyramid_select) of one item.  The list holds 8 keys for
// k <= 8 (its first k entries are kept), so one instantiation serves every k; the rank-count
// selection of k > 8 is kept out of line so that the common path keeps few registers.
template <typename Tm>
__device__ __noinline__ uint64_t select_l0_ranked(const Tm* __restrict__ M, long long hw, long long p, int D, int k,
                                                 int mode) {
    return select_mask<64, false>([&](int d) { return RLStore<Tm>::load1(M + ((size_t)d * hw + p) * 4 + 3); }, D, k,
                                  mode);
}

template <typename Tm, int LOG>
__device__ __noinline__ void pyramid_select_tile_ranked(const Tm* __restrict__ M, int D, int H, int W, int level,
                                                        Tm* __restrict__ Ml, int k, uint8_t* __restrict__ S,
                                                        uint8_t* __restrict__ slots, float* __restrict__ Gzero,
                                                        unsigned* __restrict__ counter_zero, int mode, long long p0,
                                                        float (*alpha)[kTile]) {
    pyramid_select_tile<Tm, 64, LOG>(M, D, H, W, level, Ml, k, S, slots, Gzero, counter_zero, mode, p0, alpha);
}

template <typename Tm>
__global__ void __launch_bounds__(256, 4)
k_select_batch(const RLBatchHeader* __restrict__ hdr, const RLBatchItem* __restrict__ items) {
    __shared__ float alpha[RL_DEV_MAX_PLANES][kTile];
    const unsigned n = hdr->n, total = hdr->sel_units;
    if (hdr->dtype != (std::is_same<Tm, float>::value ? (unsigned)RL_F32 : (unsigned)RL_BF16)) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && hdr->status) atomicOr(hdr->status, RL_DEVFLAG_BATCH);
        return;
    }
    __shared__ unsigned next_slot;
    for (unsigned u = rl_batch_next(hdr, 0, &next_slot); u < total; u = rl_batch_next(hdr, 0, &next_slot)) {
        const RLBatchItem& it = items[rl_batch_find(items, n, u, &RLBatchItem::sel_begin)];
        const long long local = (long long)(u - it.sel_begin);
        const bool ranked = it.mode != 1 && it.k > 8;
        const Tm* M = static_cast<const Tm*>(it.M);
        if (it.level == 0) {
            const long long hw = (long long)it.H * it.W;
            const long long p = local * 256 + threadIdx.x;
            if (p == 0) *it.counter = 0u;  // block counter of the loss epilogue that follows
            if (p < hw) {
                const uint64_t mk =
                    ranked ? select_l0_ranked<Tm>(M, hw, p, it.D, it.k, it.mode)
                           : select_mask<8, false>([&](int d) { return RLStore<Tm>::load1(M + ((size_t)d * hw + p) * 4 + 3); },
                                                   it.D, it.k, it.mode);
                write_selection(mk, it.D, it.k, hw, p, it.S, nullptr, it.slots, it.G);
            }
        } else {
            Tm* Ml = static_cast<Tm*>(it.Ml);
#define RL_PSB(LL)                                                                                                 \
    if (ranked)                                                                                                    \
        pyramid_select_tile_ranked<Tm, LL>(M, it.D, it.H, it.W, it.level, Ml, it.k, it.S, it.slots, it.G, it.counter, \
                                           it.mode, local * kTile, alpha);                                         \
    else                                                                                                           \
        pyramid_select_tile<Tm, 8, LL>(M, it.D, it.H, it.W, it.level, Ml, it.k, it.S, it.slots, it.G, it.counter,     \
                                       it.mode, local * kTile, alpha)
            if (it.level == 1) { level_image_means<1>(it.images, it.N, it.H, it.W, 1, it.Il, local * kTile); RL_PSB(1); }
            else if (it.level == 2) { level_image_means<2>(it.images, it.N, it.H, it.W, 2, it.Il, local * kTile); RL_PSB(2); }
            else { level_image_means<-1>(it.images, it.N, it.H, it.W, it.level, it.Il, local * kTile); RL_PSB(-1); }
#undef RL_PSB
        }
        __syncthreads();  // alpha is reused by the next unit
    }
}

template <typename Tm, bool FROM_KEYS>
void launch_select_t(const void* M, const float* keys, int D, int h, int w, int k, uint8_t* S, uint64_t* mask,
                     uint8_t* slots, float* Gzero, unsigned* counter_zero, int mode, cudaStream_t s) {
    const long long hw = (long long)h * w;
    const int blocks = (int)((hw + 127) / 128);
#define RL_SEL(KK)                                                                                          \
    k_select<Tm, FROM_KEYS, KK><<<blocks, 128, 0, s>>>((const Tm*)M, keys, D, h, w, k, S, mask, slots, Gzero, \
                                                       counter_zero, mode)
    switch (mode == 1 ? 1 : k) {
        case 1: RL_SEL(1); break;
        case 2: RL_SEL(2); break;
        case 3: RL_SEL(3); break;
        case 4: RL_SEL(4); break;
        case 5: RL_SEL(5); break;
        case 6: RL_SEL(6); break;
        case 7: RL_SEL(7); break;
        case 8: RL_SEL(8); break;
        default: RL_SEL(64); break;
    }
#undef RL_SEL
}

template <typename Tm, int LOG>
void launch_pyramid_select_l(const Tm* M, int D, int H, int W, int level, Tm* Ml, int k, uint8_t* S,
                             uint8_t* slots, float* Gzero, unsigned* counter_zero, int mode, cudaStream_t s,
                             const float* images, int N, float* Il) {
    const long long hw = (long long)(H >> level) * (W >> level);
    const unsigned blocks = (unsigned)((hw + kTile - 1) / kTile);
#define RL_PS(KK)                                                                                                 \
    k_pyramid_select<Tm, KK, LOG><<<blocks, 256, 0, s>>>(M, D, H, W, level, Ml, k, S, slots, Gzero, counter_zero, mode, \
                                                         images, N, Il)
    switch (mode == 1 ? 1 : k) {
        case 1: RL_PS(1); break;
        case 2: RL_PS(2); break;
        case 3: RL_PS(3); break;
        case 4: RL_PS(4); break;
        case 5: RL_PS(5); break;
        case 6: RL_PS(6); break;
        case 7: RL_PS(7); break;
        case 8: RL_PS(8); break;
        default: RL_PS(64); break;
    }
#undef RL_PS
}

template <typename Tm>
void launch_pyramid_select_t(const void* M, int D, int H, int W, int level, void* Ml, int k, uint8_t* S,
                             uint8_t* slots, float* Gzero, unsigned* counter_zero, int mode, cudaStream_t s,
                             const float* images, int N, float* Il) {
    if (level == 1)
        launch_pyramid_select_l<Tm, 1>((const Tm*)M, D, H, W, level, (Tm*)Ml, k, S, slots, Gzero, counter_zero,
                                       mode, s, images, N, Il);
    else if (level == 2)
        launch_pyramid_select_l<Tm, 2>((const Tm*)M, D, H, W, level, (Tm*)Ml, k, S, slots, Gzero, counter_zero,
                                       mode, s, images, N, Il);
    else
        launch_pyramid_select_l<Tm, -1>((const Tm*)M, D, H, W, level, (Tm*)Ml, k, S, slots, Gzero, counter_zero,
                                        mode, s, images, N, Il);
}

__global__ void k_mask_to_slots(const uint64_t* __restrict__ mask, int D, int k, int hw,
                                uint8_t* __restrict__ slots) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= hw) return;
    const uint64_t mk = mask[p];
    int j = 0;
    for (int d = 0; d < D; ++d) {
        const bool kept = ((mk >> d) & 1ull) && j < k;  // the compact gradient holds k slots
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

rl_status rl_launch_pyramid_select(const void* M, rl_dtype dt, int D, int H, int W, int level, void* Ml, int k,
                                   uint8_t* S, uint8_t* slots, float* Gzero, unsigned* counter_zero, int mode,
                                   cudaStream_t s, const float* images, int N, float* Il) {
    if (!images) Il = nullptr;
    if (dt == RL_F32) {
        RLTraceScope ts("pyramid_select_f32", s);
        launch_pyramid_select_t<float>(M, D, H, W, level, Ml, k, S, slots, Gzero, counter_zero, mode, s, images, N,
                                       Il);
    } else {
        RLTraceScope ts("pyramid_select_bf16", s);
        launch_pyramid_select_t<__nv_bfloat16>(M, D, H, W, level, Ml, k, S, slots, Gzero, counter_zero, mode, s,
                                               images, N, Il);
    }
    return rl_check_launch("pyramid_select");
}

rl_status rl_launch_select_batch(const void* table, rl_dtype dt, cudaStream_t s) {
    const RLBatchHeader* hdr = static_cast<const RLBatchHeader*>(table);
    const RLBatchItem* items = rl_batch_items(table);
    const int grid = dt == RL_F32 ? rl_persistent_grid<k_select_batch<float>>(256, 0)
                                  : rl_persistent_grid<k_select_batch<__nv_bfloat16>>(256, 0);
    if (dt == RL_F32) {
        RLTraceScope ts("select_batch_f32", s);
        k_select_batch<float><<<grid, 256, 0, s>>>(hdr, items);
    } else {
        RLTraceScope ts("select_batch_bf16", s);
        k_select_batch<__nv_bfloat16><<<grid, 256, 0, s>>>(hdr, items);
    }
    return rl_check_launch("select_batch");
}

rl_status rl_launch_mask_to_slots(const uint64_t* mask, int D, int k, int hw, uint8_t* slots, cudaStream_t s) {
    RLTraceScope ts("mask_to_slots", s);
    k_mask_to_slots<<<(hw + 255) / 256, 256, 0, s>>>(mask, D, k, hw, slots);
    return rl_check_launch("mask_to_slots");
}

rl_status rl_launch_downsample_f32(const float* x, int P, int H, int W, int C, int level, float* y, cudaStream_t s) {
    const long long n = (long long)P * (H >> level) * (W >> level) * C;
    if (n == 0) return RL_OK;
    RLTraceScope ts("downsample_f32", s);
    k_downsample_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, P, H, W, C, level, y);
    return rl_check_launch("downsample");
}

RL_DEBUG_READER(select)
