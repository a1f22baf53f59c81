// grad.cu -- fused warp + composite + photometric residual + exact adjoint (one launch for
// all source views), the render backward used by autograd, and the loss reduction.
//
// Per view pixel q (one thread), with T_d = prod_{j>d}(1 - alpha_j) (Eq. eq_over):
//   pass 1, d = D-1 .. 0:  m_d = bilinear(M[d], p_d(q)); T_d -> shared memory;
//                           C += T_d alpha_d c_d; T *= (1 - alpha_d)
//   residual:               r = (C - I(q)) / N  (loss mode; L = 1/(2N) sum |C - I|^2; I the
//                           level image: given at the level's resolution, img_level 0, or formed
//                           on the fly from its 2^l x 2^l full-resolution pixels)
//                           or r = dL/dC given by the caller (backward mode)
//   pass 2, d = 0 .. D-1:  dL/dc_d = T_d alpha_d r;  dL/dalpha_d = T_d <c_d - B_d, r>,
//                           B_d the composite of the planes below d (B_0 = 0,
//                           B_{d+1} = c_d alpha_d + (1 - alpha_d) B_d);
//                           the bilinear transpose adds w_tap * dL/dm_d to the 4 taps.
// Sparse mode adds only into voxels kept by the selection (Sec. 3.3): the slot map
// slots[d][y][x] gives the compact slot of a kept voxel (its rank among the kept planes of
// the pixel) or RL_SLOT_NONE.  No division by (1 - alpha).
#include <type_traits>

#include "rl_internal.h"

namespace {

constexpr int kGradBX = 32, kGradBY = 4, kGradThreads = kGradBX * kGradBY;
#ifndef RL_GRAD_MIN_BLOCKS
#define RL_GRAD_MIN_BLOCKS 10  // resident blocks per SM the register budget must allow (measured best)
#endif

template <bool SPARSE>
__device__ __forceinline__ void scatter_tap(float* __restrict__ G, const uint8_t* __restrict__ slots_d, int d,
                                            unsigned hw, int H, int W, int x, int y, float wt, float4 g, unsigned ng) {
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return;
    const unsigned pix = (unsigned)(y * W + x);
    const unsigned slot = SPARSE ? (unsigned)__ldg(slots_d + pix) : (unsigned)d;
    if ((SPARSE && slot == RL_SLOT_NONE) || !RL_IN(slot, ng)) return;
    atomicAdd(reinterpret_cast<float4*>(G) + (slot * hw + pix), make_float4(wt * g.x, wt * g.y, wt * g.z, wt * g.w));
}

// Bilinear transpose of one sample's gradient g onto its four taps.
template <bool SPARSE>
__device__ __forceinline__ void scatter4(float* __restrict__ G, const uint8_t* __restrict__ slots_d, int d,
                                         unsigned hw, int H, int W, const RLTaps& t, float4 g, unsigned ng) {
    const float w00 = (1.f - t.fx) * (1.f - t.fy), w10 = t.fx * (1.f - t.fy);
    const float w01 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
    if ((unsigned)t.x0 < (unsigned)(W - 1) && (unsigned)t.y0 < (unsigned)(H - 1)) {
        const unsigned p = (unsigned)(t.y0 * W + t.x0);
        unsigned s00 = d, s10 = d, s01 = d, s11 = d;
        if (SPARSE) {
            s00 = __ldg(slots_d + p);
            s10 = __ldg(slots_d + p + 1);
            s01 = __ldg(slots_d + p + W);
            s11 = __ldg(slots_d + p + W + 1);
        }
        float4* G4 = reinterpret_cast<float4*>(G);
        if ((!SPARSE || s00 != RL_SLOT_NONE) && RL_IN(s00, ng))
            atomicAdd(G4 + (s00 * hw + p), make_float4(w00 * g.x, w00 * g.y, w00 * g.z, w00 * g.w));
        if ((!SPARSE || s10 != RL_SLOT_NONE) && RL_IN(s10, ng))
            atomicAdd(G4 + (s10 * hw + p + 1), make_float4(w10 * g.x, w10 * g.y, w10 * g.z, w10 * g.w));
        if ((!SPARSE || s01 != RL_SLOT_NONE) && RL_IN(s01, ng))
            atomicAdd(G4 + (s01 * hw + p + W), make_float4(w01 * g.x, w01 * g.y, w01 * g.z, w01 * g.w));
        if ((!SPARSE || s11 != RL_SLOT_NONE) && RL_IN(s11, ng))
            atomicAdd(G4 + (s11 * hw + p + W + 1), make_float4(w11 * g.x, w11 * g.y, w11 * g.z, w11 * g.w));
        return;
    }
    scatter_tap<SPARSE>(G, slots_d, d, hw, H, W, t.x0, t.y0, w00, g, ng);
    scatter_tap<SPARSE>(G, slots_d, d, hw, H, W, t.x0 + 1, t.y0, w10, g, ng);
    scatter_tap<SPARSE>(G, slots_d, d, hw, H, W, t.x0, t.y0 + 1, w01, g, ng);
    scatter_tap<SPARSE>(G, slots_d, d, hw, H, W, t.x0 + 1, t.y0 + 1, w11, g, ng);
}

// One block's tile of 32 x 4 view pixels of one view.  bid / nblocks index the block among
// the launch's (or the batch item's) blocks for the loss epilogue.
template <typename Tm, bool SPARSE, bool LOSS, bool ANCH>
__device__ __forceinline__ void grad_tile(const Tm* __restrict__ M, int D, int H, int W, const RLViews& views, int view,
                                          int qx, int qy, int tid, float* __restrict__ sT,
                                          const float* __restrict__ images, int img_level,
                                          const float* __restrict__ grad_out, const uint8_t* __restrict__ slots,
                                          float* __restrict__ G, float inv_n, float* __restrict__ partials,
                                          unsigned bid, unsigned nblocks, float* __restrict__ loss_out,
                                          unsigned* __restrict__ counter, float loss_scale) {
    float lsum = 0.f;
    __shared__ RLAnchor sA;  // the tile's anchor: its centre pixel
    if (ANCH)
        rl_anchor_build(&sA, views, view, (qx & ~(kGradBX - 1)) + kGradBX / 2, qy - qy % kGradBY + kGradBY / 2, D,
                        tid, kGradThreads);
    if (qx < W && qy < H) {
        const RLPixWarp<ANCH> w = rl_pix_warp<ANCH>(sA, views.v[view], qx, qy);
        const size_t plane = (size_t)H * W * 4;
        float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll 1
        for (int d = D - 1; d >= 0; --d) {
            const RLTaps t = w.taps(sA, d, views.rho[d], qx, qy);
            const float4 m = rl_sample_fast(M + d * plane, H, W, t);
            sT[d * kGradThreads + tid] = T;
            const float a = T * m.w;
            c0 = fmaf(a, m.x, c0);
            c1 = fmaf(a, m.y, c1);
            c2 = fmaf(a, m.z, c2);
            T = T * (1.f - m.w);
        }
        float r0, r1, r2;
        if (LOSS) {
            // source image at this level: mean of the 2^l x 2^l full-resolution block
            const int s = 1 << img_level;
            const int Wf = W << img_level, Hf = H << img_level;
            const float* img = images + (size_t)view * Hf * Wf * 3;
            float i0 = 0.f, i1 = 0.f, i2 = 0.f;
            for (int yy = 0; yy < s; ++yy)
                for (int xx = 0; xx < s; ++xx) {
                    const float* px = img + ((size_t)(qy * s + yy) * Wf + (qx * s + xx)) * 3;
                    i0 += __ldg(px);
                    i1 += __ldg(px + 1);
                    i2 += __ldg(px + 2);
                }
            const float inv_area = 1.f / (float)(s * s);
            // the image mean is rounded on its own (as the level images of the pyramid pass are)
            const float e0 = c0 - __fmul_rn(i0, inv_area), e1 = c1 - __fmul_rn(i1, inv_area),
                        e2 = c2 - __fmul_rn(i2, inv_area);
            lsum = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
            r0 = e0 * inv_n;
            r1 = e1 * inv_n;
            r2 = e2 * inv_n;
        } else {
            const float* go = grad_out + (((size_t)view * H + qy) * W + qx) * 3;
            r0 = __ldg(go);
            r1 = __ldg(go + 1);
            r2 = __ldg(go + 2);
        }
        float b0 = 0.f, b1 = 0.f, b2 = 0.f;
        const unsigned hw = (unsigned)(H * W);
        const unsigned ng = views.gplanes ? (unsigned)views.gplanes : (unsigned)D;  // checked in debug builds
#pragma unroll 1
        for (int d = 0; d < D; ++d) {
            const RLTaps t = w.taps(sA, d, views.rho[d], qx, qy);
            const float4 m = rl_sample_fast(M + d * plane, H, W, t);
            const float Td = sT[d * kGradThreads + tid];
            if (t.ok && Td != 0.f) {
                const float gc = Td * m.w;
                float4 g;
                g.x = gc * r0;
                g.y = gc * r1;
                g.z = gc * r2;
                g.w = Td * fmaf(m.x - b0, r0, fmaf(m.y - b1, r1, (m.z - b2) * r2));
                scatter4<SPARSE>(G, SPARSE ? slots + (size_t)d * hw : nullptr, d, hw, H, W, t, g, ng);
            }
            const float om = 1.f - m.w;
            b0 = fmaf(m.x, m.w, om * b0);
            b1 = fmaf(m.y, m.w, om * b1);
            b2 = fmaf(m.z, m.w, om * b2);
        }
    }
    if (LOSS) {
        __shared__ float red[kGradThreads / 32];
        lsum = rl_warp_sum(lsum);
        if ((tid & 31) == 0) red[tid >> 5] = lsum;
        __syncthreads();
        float blk = 0.f;
        if (tid == 0)
            for (int j = 0; j < kGradThreads / 32; ++j) blk += red[j];
        __syncthreads();
        rl_loss_epilogue(blk, partials, bid, nblocks, loss_out, counter, loss_scale, tid, kGradThreads, red);
    }
}

template <typename Tm, bool SPARSE, bool LOSS, bool ANCH>
__global__ void __launch_bounds__(kGradThreads, RL_GRAD_MIN_BLOCKS)
k_grad(const Tm* __restrict__ M, int D, int H, int W, const __grid_constant__ RLViews views, int tiles_x,
       const float* __restrict__ images, int img_level, const float* __restrict__ grad_out,
       const uint8_t* __restrict__ slots, float* __restrict__ G, float inv_n, float* __restrict__ partials,
       float* __restrict__ loss_out, unsigned* __restrict__ counter, float loss_scale) {
    extern __shared__ float sT[];  // [D][kGradThreads]
    // view-fastest block order: the N views of a tile run together and share M through L2
    grad_tile<Tm, SPARSE, LOSS, ANCH>(M, D, H, W, views, blockIdx.x, blockIdx.y * kGradBX + threadIdx.x,
                                blockIdx.z * kGradBY + threadIdx.y, threadIdx.y * kGradBX + threadIdx.x, sT, images,
                                img_level, grad_out, slots, G, inv_n, partials,
                                blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                                gridDim.x * gridDim.y * gridDim.z, loss_out, counter, loss_scale);
}

// Batched gradient, per-pixel gather family: one persistent launch walks the gradient units of
// the batch table's items that take this family (a unit is one 32 x 4 tile of one view of one
// item, in the order of k_grad's grid), each item with its own loss epilogue over its own
// units.  The dynamic shared memory holds `planes` planes; an item with more sets the batch bit
// of the status word and is skipped.
#ifndef RL_GRAD_BATCH_MIN_BLOCKS
#define RL_GRAD_BATCH_MIN_BLOCKS 8  // the table lookups need registers: at 10 blocks the kernel spills
#endif
template <typename Tm>
__global__ void __launch_bounds__(kGradThreads, RL_GRAD_BATCH_MIN_BLOCKS)
k_grad_batch(const RLBatchHeader* __restrict__ hdr, const RLBatchItem* __restrict__ items, int planes) {
    extern __shared__ float sT[];  // [planes][kGradThreads]
    const unsigned n = hdr->n, total = hdr->grad_units;
    if (hdr->dtype != (std::is_same<Tm, float>::value ? (unsigned)RL_F32 : (unsigned)RL_BF16)) return;
    const int tid = threadIdx.y * kGradBX + threadIdx.x;
    __shared__ unsigned next_slot;
    for (unsigned u = rl_batch_next(hdr, 1, &next_slot); u < total; u = rl_batch_next(hdr, 1, &next_slot)) {
        const RLBatchItem& it = items[rl_batch_find(items, n, u, &RLBatchItem::grad_begin)];
        if (it.D > planes) {
            if (tid == 0 && hdr->status) atomicOr(hdr->status, RL_DEVFLAG_BATCH);
            continue;
        }
        const unsigned local = u - it.grad_begin;
        const unsigned view = local % (unsigned)it.N, tile = local / (unsigned)it.N;
        const int tx = (int)(tile % it.grad_tiles_x), ty = (int)(tile / it.grad_tiles_x);
        const int h = it.H >> it.level, w = it.W >> it.level;
#define RL_GB(A) grad_tile<Tm, true, true, A>(static_cast<const Tm*>(it.Ml), it.D, h, w, it.views, (int)view,    \
                                             tx * kGradBX + threadIdx.x, ty * kGradBY + threadIdx.y, tid, sT,       \
                                             it.level ? it.Il : it.images, 0, nullptr, it.slots, it.G, it.inv_n,    \
                                             it.partials,                                                           \
                                             local, it.grad_units, it.loss_out, it.counter, it.loss_scale)
        if (it.views.anchored) RL_GB(true);
        else RL_GB(false);
#undef RL_GB
        __syncthreads();  // sT is reused by the next unit
    }
}

// Deterministic sum of the per-block partials (fixed order), times `scale`.
__global__ void __launch_bounds__(1024) k_loss_reduce(const float* __restrict__ partials, int n, float scale,
                                                     float* __restrict__ out) {
    __shared__ float red[32];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    s = rl_warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        v = rl_warp_sum(v);
        if (threadIdx.x == 0) out[0] = v * scale;
    }
}

template <typename Tm, bool SPARSE, bool LOSS>
void launch_grad_t(const void* M, int D, int H, int W, const RLViews& views, const float* images, int img_level,
                   const float* grad_out, const uint8_t* slots, float* G, float inv_n, float* partials, float* loss_out,
                   unsigned* counter, float loss_scale, int tiles_x, dim3 grid, size_t smem, cudaStream_t s) {
    auto kern = views.anchored ? k_grad<Tm, SPARSE, LOSS, true> : k_grad<Tm, SPARSE, LOSS, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, dim3(kGradBX, kGradBY), smem, s>>>((const Tm*)M, D, H, W, views, tiles_x, images, img_level, grad_out,
                                                    slots, G, inv_n, partials, loss_out, counter, loss_scale);
}

}  // namespace

size_t rl_grad_num_blocks(int H, int W, int N) {
    const size_t own = (size_t)((W + kGradBX - 1) / kGradBX) * ((H + kGradBY - 1) / kGradBY) * N;
    const size_t a = rl_grad_pp_num_blocks(H, W, N);
    return own > a ? own : a;
}

rl_status rl_launch_grad(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, bool mode_loss,
                         const float* images, int img_level, const float* grad_out, const uint8_t* slots, float* G,
                         float inv_n, float* partials, int* nblocks, cudaStream_t s, float* loss_out,
                         unsigned* counter, float loss_scale) {
    const int path = rl_kernel_path(H, W, views.n);
    if (path != 2)
        return rl_launch_grad_pp(M, dt, D, H, W, views, mode_loss, images, img_level, grad_out, slots, G, inv_n,
                                 partials, nblocks, s, loss_out, counter, loss_scale);
    const int tiles_x = (W + kGradBX - 1) / kGradBX, tiles_y = (H + kGradBY - 1) / kGradBY;
    const dim3 grid((unsigned)views.n, (unsigned)tiles_x, (unsigned)tiles_y);
    const size_t smem = (size_t)D * kGradThreads * sizeof(float);
    if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
    const bool sparse = slots != nullptr;
    const char* name = dt == RL_F32 ? (sparse ? "grad_sparse_f32" : "grad_dense_f32")
                                    : (sparse ? "grad_sparse_bf16" : "grad_dense_bf16");
    RLTraceScope ts(name, s);
#define RL_GRAD_CASE(TM, SP, LS) \
    launch_grad_t<TM, SP, LS>(M, D, H, W, views, images, img_level, grad_out, slots, G, inv_n, partials, loss_out, \
                              counter, loss_scale, tiles_x, grid, smem, s)
    if (dt == RL_F32) {
        if (sparse) { if (mode_loss) RL_GRAD_CASE(float, true, true); else RL_GRAD_CASE(float, true, false); }
        else        { if (mode_loss) RL_GRAD_CASE(float, false, true); else RL_GRAD_CASE(float, false, false); }
    } else {
        if (sparse) { if (mode_loss) RL_GRAD_CASE(__nv_bfloat16, true, true); else RL_GRAD_CASE(__nv_bfloat16, true, false); }
        else        { if (mode_loss) RL_GRAD_CASE(__nv_bfloat16, false, true); else RL_GRAD_CASE(__nv_bfloat16, false, false); }
    }
#undef RL_GRAD_CASE
    return rl_check_launch("grad");
}

unsigned rl_grad_gather_tiles_x(int w) { return (unsigned)((w + kGradBX - 1) / kGradBX); }
unsigned rl_grad_gather_tiles_y(int h) { return (unsigned)((h + kGradBY - 1) / kGradBY); }

rl_status rl_launch_grad_batch(const void* table, rl_dtype dt, int planes, cudaStream_t s) {
    const RLBatchHeader* hdr = static_cast<const RLBatchHeader*>(table);
    const RLBatchItem* items = rl_batch_items(table);
    planes = planes < 1 ? 1 : (planes > RL_DEV_MAX_PLANES ? RL_DEV_MAX_PLANES : planes);
    const size_t smem = (size_t)planes * kGradThreads * sizeof(float);
    // the resident blocks of the largest shared memory, so that any later capacity fits the grid
    const size_t smem_max = (size_t)RL_DEV_MAX_PLANES * kGradThreads * sizeof(float);
    const int grid = dt == RL_F32 ? rl_persistent_grid<k_grad_batch<float>>(kGradThreads, smem_max)
                                  : rl_persistent_grid<k_grad_batch<__nv_bfloat16>>(kGradThreads, smem_max);
    if (dt == RL_F32) {
        RLTraceScope ts("grad_batch_f32", s);
        k_grad_batch<float><<<grid, dim3(kGradBX, kGradBY), smem, s>>>(hdr, items, planes);
    } else {
        RLTraceScope ts("grad_batch_bf16", s);
        k_grad_batch<__nv_bfloat16><<<grid, dim3(kGradBX, kGradBY), smem, s>>>(hdr, items, planes);
    }
    return rl_check_launch("grad_batch");
}

rl_status rl_launch_loss_reduce(const float* partials, int n, float scale, float* out, cudaStream_t s) {
    RLTraceScope ts("loss_reduce", s);
    k_loss_reduce<<<1, 1024, 0, s>>>(partials, n, scale, out);
    return rl_check_launch("loss_reduce");
}

RL_DEBUG_READER(grad)
