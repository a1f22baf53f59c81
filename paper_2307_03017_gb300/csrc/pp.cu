// pp.cu -- plane-parallel warp kernels: novel-view rendering (Eq. eq_render, eq_over) and
// the fused warp + composite + residual + exact adjoint of one HSGD iteration.
//
// Layout.  A block is kGroups (4 or 8) warps over the same 32 view pixels (a 16 x 2 tile; grid =
// (views, tiles_x, tiles_y) so that the views of a tile run together); warp g
// owns planes [g C, g C + C), C = ceil(D / kGroups) rounded up to 1, 2, 4 or 8, so a warp's loads of one plane
// are 32 neighbouring voxels.  Each thread samples its C planes once and keeps them in
// registers, nearest first forming its chunk's composite Cc_g = sum c_d alpha_d T_d^loc
// and transmittance Tc_g = prod (1 - alpha_d).  The over operator is associative, so the
// chunks combine exactly:
//   T before chunk g (everything nearer):  Tb_g = prod_{g' > g} Tc_g'
//   pixel colour:                          C = sum_g Tb_g Cc_g
//   composite of everything farther:       Bb_g = f_{g-1}(... f_0(0)), f_g(x) = Cc_g + Tc_g x
// (shared-memory exchange of the per-chunk (Cc, Tc)).  The adjoint of plane d then uses
// T_d = Tb_g T_d^loc and the running below-composite B_d (B_{d+1} = c_d alpha_d + (1 -
// alpha_d) B_d, starting from Bb_g) -- no division by (1 - alpha), no second gather.
// Bilinear weights are applied with packed FP32x2 FMAs (same rounding as scalar FMAs).
#include <type_traits>

#include "rl_internal.h"

namespace {

constexpr int kTX = 16, kTY = 2, kPix = 32;  // pixels per block, one per lane

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Bilinear sample; interior samples use packed FMAs, border samples the checked path.
template <typename Tm>
__device__ __forceinline__ float4 sample_pp(const Tm* __restrict__ plane, int H, int W, const RLTaps& t) {
    if (t.ok && (unsigned)t.x0 < (unsigned)(W - 1) && (unsigned)t.y0 < (unsigned)(H - 1) &&
        RL_IN((long long)t.y0 * W + t.x0 + W + 1, (long long)H * W)) {
        const Tm* p = plane + (unsigned)(t.y0 * W + t.x0) * 4u;
        const float4 v00 = RLStore<Tm>::load4(p), v10 = RLStore<Tm>::load4(p + 4);
        const float4 v01 = RLStore<Tm>::load4(p + 4 * W), v11 = RLStore<Tm>::load4(p + 4 * W + 4);
        const float w00 = (1.f - t.fx) * (1.f - t.fy), w10 = t.fx * (1.f - t.fy);
        const float w01 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
        float2 lo = __fmul2_rn(f2(w00, w00), f2(v00.x, v00.y));
        float2 hi = __fmul2_rn(f2(w00, w00), f2(v00.z, v00.w));
        lo = __ffma2_rn(f2(w10, w10), f2(v10.x, v10.y), lo);
        hi = __ffma2_rn(f2(w10, w10), f2(v10.z, v10.w), hi);
        lo = __ffma2_rn(f2(w01, w01), f2(v01.x, v01.y), lo);
        hi = __ffma2_rn(f2(w01, w01), f2(v01.z, v01.w), hi);
        lo = __ffma2_rn(f2(w11, w11), f2(v11.x, v11.y), lo);
        hi = __ffma2_rn(f2(w11, w11), f2(v11.z, v11.w), hi);
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    return rl_sample(plane, H, W, t);
}

template <bool SPARSE>
__device__ __forceinline__ void scatter_tap_pp(float4* __restrict__ G4, const uint8_t* __restrict__ slots_d,
                                               unsigned d, unsigned hw, int H, int W, int x, int y, float wt,
                                               float4 g, unsigned ng) {
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return;
    const unsigned pix = (unsigned)(y * W + x);
    const unsigned slot = SPARSE ? (unsigned)__ldg(slots_d + pix) : d;
    if ((SPARSE && slot == RL_SLOT_NONE) || !RL_IN(slot, ng)) return;
    atomicAdd(G4 + (slot * hw + pix), make_float4(wt * g.x, wt * g.y, wt * g.z, wt * g.w));
}

// Bilinear transpose of one sample's gradient onto its four taps (kept voxels only).
template <bool SPARSE>
__device__ __forceinline__ void scatter_pp(float* __restrict__ G, const uint8_t* __restrict__ slots_d, unsigned d,
                                           unsigned hw, int H, int W, const RLTaps& t, float4 g, unsigned ng) {
    const float w00 = (1.f - t.fx) * (1.f - t.fy), w10 = t.fx * (1.f - t.fy);
    const float w01 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
    float4* G4 = reinterpret_cast<float4*>(G);
    if ((unsigned)t.x0 < (unsigned)(W - 1) && (unsigned)t.y0 < (unsigned)(H - 1)) {
        const unsigned p = (unsigned)(t.y0 * W + t.x0);
        unsigned s00 = d, s10 = d, s01 = d, s11 = d;
        if (SPARSE) {
            s00 = __ldg(slots_d + p);
            s10 = __ldg(slots_d + p + 1);
            s01 = __ldg(slots_d + p + W);
            s11 = __ldg(slots_d + p + W + 1);
        }
        const float2 gl = f2(g.x, g.y), gh = f2(g.z, g.w);
        if ((!SPARSE || s00 != RL_SLOT_NONE) && RL_IN(s00, ng)) {
            const float2 a = __fmul2_rn(f2(w00, w00), gl), b = __fmul2_rn(f2(w00, w00), gh);
            atomicAdd(G4 + (s00 * hw + p), make_float4(a.x, a.y, b.x, b.y));
        }
        if ((!SPARSE || s10 != RL_SLOT_NONE) && RL_IN(s10, ng)) {
            const float2 a = __fmul2_rn(f2(w10, w10), gl), b = __fmul2_rn(f2(w10, w10), gh);
            atomicAdd(G4 + (s10 * hw + p + 1), make_float4(a.x, a.y, b.x, b.y));
        }
        if ((!SPARSE || s01 != RL_SLOT_NONE) && RL_IN(s01, ng)) {
            const float2 a = __fmul2_rn(f2(w01, w01), gl), b = __fmul2_rn(f2(w01, w01), gh);
            atomicAdd(G4 + (s01 * hw + p + W), make_float4(a.x, a.y, b.x, b.y));
        }
        if ((!SPARSE || s11 != RL_SLOT_NONE) && RL_IN(s11, ng)) {
            const float2 a = __fmul2_rn(f2(w11, w11), gl), b = __fmul2_rn(f2(w11, w11), gh);
            atomicAdd(G4 + (s11 * hw + p + W + 1), make_float4(a.x, a.y, b.x, b.y));
        }
        return;
    }
    scatter_tap_pp<SPARSE>(G4, slots_d, d, hw, H, W, t.x0, t.y0, w00, g, ng);
    scatter_tap_pp<SPARSE>(G4, slots_d, d, hw, H, W, t.x0 + 1, t.y0, w10, g, ng);
    scatter_tap_pp<SPARSE>(G4, slots_d, d, hw, H, W, t.x0, t.y0 + 1, w01, g, ng);
    scatter_tap_pp<SPARSE>(G4, slots_d, d, hw, H, W, t.x0 + 1, t.y0 + 1, w11, g, ng);
}

struct PixelCoord {
    int qx, qy, view, g, lane;
    bool active;
};

__device__ __forceinline__ PixelCoord pixel_coord_at(int H, int W, int view, int tx, int ty) {
    PixelCoord c;
    c.view = view;
    c.g = threadIdx.x >> 5;
    c.lane = threadIdx.x & 31;
    c.qx = tx * kTX + (c.lane % kTX);
    c.qy = ty * kTY + (c.lane / kTX);
    c.active = c.qx < W && c.qy < H;
    return c;
}

// grid (views, tiles_x, tiles_y): the views of a tile run together and share M in L2
__device__ __forceinline__ PixelCoord pixel_coord(int H, int W) {
    return pixel_coord_at(H, W, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename Tm, int C, int kGroups, bool ANCH>
__global__ void __launch_bounds__(kGroups * kPix)
k_render_pp(const Tm* __restrict__ M, int D, int H, int W, const __grid_constant__ RLViews views, int tiles_x,
            float* __restrict__ out) {
    __shared__ float4 xch[kGroups][kPix];  // per chunk: (Cc.rgb, Tc)
    __shared__ RLAnchor sA;
    const PixelCoord pc = pixel_coord(H, W);
    if (ANCH)
        rl_anchor_build(&sA, views, pc.view, blockIdx.y * kTX + kTX / 2, blockIdx.z * kTY + kTY / 2, D, threadIdx.x,
                        kGroups * kPix);
    const int qx = min(pc.qx, W - 1), qy = min(pc.qy, H - 1);
    const RLPixWarp<ANCH> w = rl_pix_warp<ANCH>(sA, views.v[pc.view], qx, qy);
    const size_t plane = (size_t)H * W * 4;
    float Tl = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
    for (int i = C - 1; i >= 0; --i) {
        const int d = pc.g * C + i;
        if (d < D) {
            const RLTaps t = w.taps(sA, d, views.rho[d], qx, qy);
            const float4 m = sample_pp(M + d * plane, H, W, t);
            const float a = Tl * m.w;
            c0 = fmaf(a, m.x, c0);
            c1 = fmaf(a, m.y, c1);
            c2 = fmaf(a, m.z, c2);
            Tl = Tl * (1.f - m.w);
        }
    }
    xch[pc.g][pc.lane] = make_float4(c0, c1, c2, Tl);
    __syncthreads();
    if (pc.g == 0 && pc.active) {
        float T = 1.f, o0 = 0.f, o1 = 0.f, o2 = 0.f;
#pragma unroll
        for (int g = kGroups - 1; g >= 0; --g) {
            const float4 v = xch[g][pc.lane];
            o0 = fmaf(T, v.x, o0);
            o1 = fmaf(T, v.y, o1);
            o2 = fmaf(T, v.z, o2);
            T = T * v.w;
        }
        float* o = out + (((size_t)pc.view * H + pc.qy) * W + pc.qx) * 3;
        o[0] = o0;
        o[1] = o1;
        o[2] = o2;
    }
}

// One block's tile (kPix view pixels of one view, all planes): the body of k_grad_pp, with the
// tile, the exchange buffers and the block's index for the loss epilogue given explicitly.
template <typename Tm, int C, int kGroups, bool SPARSE, bool LOSS, bool ANCH>
__device__ __forceinline__ void grad_pp_tile(const Tm* __restrict__ M, int D, int H, int W, const RLViews& views,
                                             const PixelCoord pc, const float* __restrict__ images, int img_level,
                                             const float* __restrict__ grad_out, const uint8_t* __restrict__ slots,
                                             float* __restrict__ G, float inv_n, float* __restrict__ partials,
                                             unsigned bid, unsigned nblocks, float* __restrict__ loss_out,
                                             unsigned* __restrict__ counter, float loss_scale,
                                             float4 (*__restrict__ xch)[kPix], float* __restrict__ red) {
    __shared__ RLAnchor sA;
    if (ANCH)
        rl_anchor_build(&sA, views, pc.view, (pc.qx - pc.qx % kTX) + kTX / 2, (pc.qy - pc.qy % kTY) + kTY / 2, D,
                        threadIdx.x, kGroups * kPix);
    const int qx = min(pc.qx, W - 1), qy = min(pc.qy, H - 1);
    const RLPixWarp<ANCH> w = rl_pix_warp<ANCH>(sA, views.v[pc.view], qx, qy);
    const size_t plane = (size_t)H * W * 4;

    // a level image that is already averaged (img_level 0: one pixel a view) is read by one warp
    // before its gathers and handed to the others through shared memory at the chunk exchange
    __shared__ float ximg[kPix][3];
    const bool img_early = LOSS && img_level == 0;
    float li0 = 0.f, li1 = 0.f, li2 = 0.f;
    if (img_early && pc.g == kGroups - 1 && pc.active) {
        const float* px = images + (((size_t)pc.view * H + pc.qy) * W + pc.qx) * 3;
        li0 = __ldg(px);
        li1 = __ldg(px + 1);
        li2 = __ldg(px + 2);
    }

    // forward over this thread's chunk, nearest plane first; samples stay in registers
    float4 m[C];
    float Tloc[C];
    float Tl = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
    for (int i = C - 1; i >= 0; --i) {
        const int d = pc.g * C + i;
        m[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        Tloc[i] = Tl;
        if (d < D) {
            const RLTaps t = w.taps(sA, d, views.rho[d], qx, qy);
            m[i] = sample_pp(M + d * plane, H, W, t);
            const float a = Tl * m[i].w;
            c0 = fmaf(a, m[i].x, c0);
            c1 = fmaf(a, m[i].y, c1);
            c2 = fmaf(a, m[i].z, c2);
            Tl = Tl * (1.f - m[i].w);
        }
    }
    xch[pc.g][pc.lane] = make_float4(c0, c1, c2, Tl);
    if (img_early && pc.g == kGroups - 1) {
        ximg[pc.lane][0] = li0;
        ximg[pc.lane][1] = li1;
        ximg[pc.lane][2] = li2;
    }
    __syncthreads();
    // combine the chunks: pixel colour, transmittance in front of this chunk and the
    // composite of everything behind it
    float Tb = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    {
        float T = 1.f;
#pragma unroll
        for (int g = kGroups - 1; g >= 0; --g) {
            const float4 v = xch[g][pc.lane];
            if (g == pc.g) Tb = T;
            C0 = fmaf(T, v.x, C0);
            C1 = fmaf(T, v.y, C1);
            C2 = fmaf(T, v.z, C2);
            T = T * v.w;
        }
    }
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
    for (int g = 0; g < pc.g; ++g) {
        const float4 v = xch[g][pc.lane];
        b0 = fmaf(v.w, b0, v.x);
        b1 = fmaf(v.w, b1, v.y);
        b2 = fmaf(v.w, b2, v.z);
    }
    float r0 = 0.f, r1 = 0.f, r2 = 0.f, lsum = 0.f;
    if (pc.active) {
        if (LOSS) {
            const int s = 1 << img_level;
            const int Wf = W << img_level, Hf = H << img_level;
            const float* img = images + (size_t)pc.view * Hf * Wf * 3;
            float i0 = 0.f, i1 = 0.f, i2 = 0.f;
            if (img_early) {
                i0 = ximg[pc.lane][0];
                i1 = ximg[pc.lane][1];
                i2 = ximg[pc.lane][2];
            } else {
                for (int yy = 0; yy < s; ++yy)
                    for (int xx = 0; xx < s; ++xx) {
                        const float* px = img + ((size_t)(pc.qy * s + yy) * Wf + (pc.qx * s + xx)) * 3;
                        i0 += __ldg(px);
                        i1 += __ldg(px + 1);
                        i2 += __ldg(px + 2);
                    }
            }
            const float inv_area = 1.f / (float)(s * s);
            // the image mean is rounded on its own (as the level images of the pyramid pass are)
            const float e0 = C0 - __fmul_rn(i0, inv_area), e1 = C1 - __fmul_rn(i1, inv_area),
                        e2 = C2 - __fmul_rn(i2, inv_area);
            if (pc.g == 0) lsum = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
            r0 = e0 * inv_n;
            r1 = e1 * inv_n;
            r2 = e2 * inv_n;
        } else {
            const float* go = grad_out + (((size_t)pc.view * H + pc.qy) * W + pc.qx) * 3;
            r0 = __ldg(go);
            r1 = __ldg(go + 1);
            r2 = __ldg(go + 2);
        }
        // adjoint over the chunk, farthest plane first
        const unsigned hw = (unsigned)(H * W);
        const unsigned ng = views.gplanes ? (unsigned)views.gplanes : (unsigned)D;  // checked in debug builds
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int d = pc.g * C + i;
            if (d < D) {
                const float Td = Tb * Tloc[i];
                const float4 mi = m[i];
                if (Td != 0.f) {
                    const RLTaps t = w.taps(sA, d, views.rho[d], pc.qx, pc.qy);
                    if (t.ok) {
                        const float gc = Td * mi.w;
                        float4 g;
                        g.x = gc * r0;
                        g.y = gc * r1;
                        g.z = gc * r2;
                        g.w = Td * fmaf(mi.x - b0, r0, fmaf(mi.y - b1, r1, (mi.z - b2) * r2));
                        scatter_pp<SPARSE>(G, SPARSE ? slots + (size_t)d * hw : nullptr, (unsigned)d, hw, H, W, t, g,
                                           ng);
                    }
                }
                const float om = 1.f - mi.w;
                b0 = fmaf(mi.x, mi.w, om * b0);
                b1 = fmaf(mi.y, mi.w, om * b1);
                b2 = fmaf(mi.z, mi.w, om * b2);
            }
        }
    }
    if (LOSS) {
        lsum = rl_warp_sum(lsum);
        if (pc.lane == 0) red[pc.g] = lsum;
        __syncthreads();
        float blk = 0.f;
        if (threadIdx.x == 0)
            for (int i = 0; i < kGroups; ++i) blk += red[i];
        __syncthreads();
        rl_loss_epilogue(blk, partials, bid, nblocks, loss_out, counter, loss_scale, threadIdx.x, kGroups * kPix,
                         red);
    }
}

template <typename Tm, int C, int kGroups, bool SPARSE, bool LOSS, bool ANCH>
__global__ void __launch_bounds__(kGroups * kPix, C <= 4 ? 1024 / (kGroups * kPix) : 1)
k_grad_pp(const Tm* __restrict__ M, int D, int H, int W, const __grid_constant__ RLViews views, int tiles_x,
          const float* __restrict__ images, int img_level, const float* __restrict__ grad_out,
          const uint8_t* __restrict__ slots, float* __restrict__ G, float inv_n, float* __restrict__ partials,
          float* __restrict__ loss_out, unsigned* __restrict__ counter, float loss_scale) {
    __shared__ float4 xch[kGroups][kPix];
    __shared__ float red[kGroups];
    grad_pp_tile<Tm, C, kGroups, SPARSE, LOSS, ANCH>(M, D, H, W, views, pixel_coord(H, W), images, img_level, grad_out,
                                               slots, G, inv_n, partials,
                                               blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                                               gridDim.x * gridDim.y * gridDim.z, loss_out, counter, loss_scale, xch,
                                               red);
}

// Batched gradient, plane-parallel family: one persistent launch of 8-warp blocks walks the
// gradient units of the batch table's items that take this family (a unit is one 16 x 2 tile of
// one view of one item, in the order of k_grad_pp's grid; planes per thread from the item's D),
// each item with its own loss epilogue over its own units.
template <typename Tm>
__global__ void __launch_bounds__(8 * kPix, 3)
k_grad_pp_batch(const RLBatchHeader* __restrict__ hdr, const RLBatchItem* __restrict__ items) {
    __shared__ float4 xch[8][kPix];
    __shared__ float red[8];
    const unsigned n = hdr->n, total = hdr->pp_units;
    if (hdr->dtype != (std::is_same<Tm, float>::value ? (unsigned)RL_F32 : (unsigned)RL_BF16)) return;
    __shared__ unsigned next_slot;
    for (unsigned u = rl_batch_next(hdr, 2, &next_slot); u < total; u = rl_batch_next(hdr, 2, &next_slot)) {
        const RLBatchItem& it = items[rl_batch_find(items, n, u, &RLBatchItem::pp_begin)];
        const unsigned local = u - it.pp_begin;
        const unsigned view = local % (unsigned)it.N, tile = local / (unsigned)it.N;
        const int h = it.H >> it.level, w = it.W >> it.level;
        const PixelCoord pc =
            pixel_coord_at(h, w, (int)view, (int)(tile % it.pp_tiles_x), (int)(tile / it.pp_tiles_x));
        const Tm* Ml = static_cast<const Tm*>(it.Ml);
#define RL_PPB(CC, A) grad_pp_tile<Tm, CC, 8, true, true, A>(Ml, it.D, h, w, it.views, pc,                       \
                                                             it.level ? it.Il : it.images, 0,                       \
                                                             nullptr, it.slots, it.G, it.inv_n, it.partials, local, \
                                                             it.pp_units, it.loss_out, it.counter, it.loss_scale,   \
                                                             xch, red)
        const int c = (it.D + 7) / 8;
        if (it.views.anchored) {
            if (c <= 1) RL_PPB(1, true);
            else if (c <= 2) RL_PPB(2, true);
            else if (c <= 4) RL_PPB(4, true);
            else RL_PPB(8, true);
        } else {
            if (c <= 1) RL_PPB(1, false);
            else if (c <= 2) RL_PPB(2, false);
            else if (c <= 4) RL_PPB(4, false);
            else RL_PPB(8, false);
        }
#undef RL_PPB
        __syncthreads();  // the exchange buffers are reused by the next unit
    }
}

// planes per thread for D planes over G warps: the next of 1, 2, 4, 8 >= ceil(D / G)
int chunk_for(int D, int G) {
    const int c = (D + G - 1) / G;
    return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : 8;
}

// Warps per block: 8 (measured faster than 4 at D = 32 despite the chunk combination being
// amortised over fewer planes); kernel path 4 forces 4 where D <= 32 (at most 8 planes per
// thread).
int groups_for(int D, int path) {
    return (path == 4 && D <= 32) ? 4 : 8;
}

template <typename Tm, bool SPARSE, bool LOSS>
void launch_grad_pp_t(int G, int C, const void* M, int D, int H, int W, const RLViews& views, int tiles_x, dim3 grid,
                      const float* images, int img_level, const float* grad_out, const uint8_t* slots, float* G_,
                      float inv_n, float* partials, float* loss_out, unsigned* counter, float loss_scale,
                      cudaStream_t s) {
#define RL_PP_ARGS (const Tm*)M, D, H, W, views, tiles_x, images, img_level, grad_out, slots, G_, inv_n, partials, \
                   loss_out, counter, loss_scale
#define RL_PP_LAUNCH(CC, GG) k_grad_pp<Tm, CC, GG, SPARSE, LOSS, false><<<grid, GG * kPix, 0, s>>>(RL_PP_ARGS)
#define RL_PP_LAUNCH_A(CC) k_grad_pp<Tm, CC, 8, SPARSE, LOSS, true><<<grid, 8 * kPix, 0, s>>>(RL_PP_ARGS)
    if (views.anchored) {  // 8 warps a block (the 4-warp option keeps the FP32 coordinates only)
        switch (C) {
            case 1: RL_PP_LAUNCH_A(1); break;
            case 2: RL_PP_LAUNCH_A(2); break;
            case 4: RL_PP_LAUNCH_A(4); break;
            default: RL_PP_LAUNCH_A(8); break;
        }
    } else if (G == 4) {
        switch (C) {
            case 1: RL_PP_LAUNCH(1, 4); break;
            case 2: RL_PP_LAUNCH(2, 4); break;
            case 4: RL_PP_LAUNCH(4, 4); break;
            default: RL_PP_LAUNCH(8, 4); break;
        }
    } else {
        switch (C) {
            case 1: RL_PP_LAUNCH(1, 8); break;
            case 2: RL_PP_LAUNCH(2, 8); break;
            case 4: RL_PP_LAUNCH(4, 8); break;
            default: RL_PP_LAUNCH(8, 8); break;
        }
    }
#undef RL_PP_LAUNCH_A
#undef RL_PP_LAUNCH
#undef RL_PP_ARGS
}

template <typename Tm>
void launch_render_pp_t(int G, int C, const void* M, int D, int H, int W, const RLViews& views, int tiles_x,
                        dim3 grid, float* out, cudaStream_t s) {
#define RL_PP_LAUNCH(CC, GG) \
    k_render_pp<Tm, CC, GG, false><<<grid, GG * kPix, 0, s>>>((const Tm*)M, D, H, W, views, tiles_x, out)
#define RL_PP_LAUNCH_A(CC) \
    k_render_pp<Tm, CC, 8, true><<<grid, 8 * kPix, 0, s>>>((const Tm*)M, D, H, W, views, tiles_x, out)
    if (views.anchored) {
        switch (C) {
            case 1: RL_PP_LAUNCH_A(1); break;
            case 2: RL_PP_LAUNCH_A(2); break;
            case 4: RL_PP_LAUNCH_A(4); break;
            default: RL_PP_LAUNCH_A(8); break;
        }
    } else if (G == 4) {
        switch (C) {
            case 1: RL_PP_LAUNCH(1, 4); break;
            case 2: RL_PP_LAUNCH(2, 4); break;
            case 4: RL_PP_LAUNCH(4, 4); break;
            default: RL_PP_LAUNCH(8, 4); break;
        }
    } else {
        switch (C) {
            case 1: RL_PP_LAUNCH(1, 8); break;
            case 2: RL_PP_LAUNCH(2, 8); break;
            case 4: RL_PP_LAUNCH(4, 8); break;
            default: RL_PP_LAUNCH(8, 8); break;
        }
    }
#undef RL_PP_LAUNCH
}

}  // namespace

size_t rl_grad_pp_num_blocks(int H, int W, int N) {
    return (size_t)((W + kTX - 1) / kTX) * ((H + kTY - 1) / kTY) * N;
}

rl_status rl_launch_grad_pp(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, bool mode_loss,
                            const float* images, int img_level, const float* grad_out, const uint8_t* slots,
                            float* G_out, float inv_n, float* partials, int* nblocks, cudaStream_t s,
                            float* loss_out, unsigned* counter, float loss_scale) {
    const int tiles_x = (W + kTX - 1) / kTX;
    const dim3 grid((unsigned)views.n, (unsigned)tiles_x, (unsigned)((H + kTY - 1) / kTY));
    if (nblocks) *nblocks = (int)rl_grad_pp_num_blocks(H, W, views.n);
    const int G = views.anchored ? 8 : groups_for(D, rl_kernel_path_setting());
    const int C = chunk_for(D, G);
    const bool sparse = slots != nullptr;
    const char* name = dt == RL_F32 ? (sparse ? "grad_sparse_f32" : "grad_dense_f32")
                                    : (sparse ? "grad_sparse_bf16" : "grad_dense_bf16");
    RLTraceScope ts(name, s);
#define RL_CASE(TM, SP, LS) \
    launch_grad_pp_t<TM, SP, LS>(G, C, M, D, H, W, views, tiles_x, grid, images, img_level, grad_out, slots, G_out, \
                                 inv_n, partials, loss_out, counter, loss_scale, s)
    if (dt == RL_F32) {
        if (sparse) { if (mode_loss) RL_CASE(float, true, true); else RL_CASE(float, true, false); }
        else        { if (mode_loss) RL_CASE(float, false, true); else RL_CASE(float, false, false); }
    } else {
        if (sparse) { if (mode_loss) RL_CASE(__nv_bfloat16, true, true); else RL_CASE(__nv_bfloat16, true, false); }
        else        { if (mode_loss) RL_CASE(__nv_bfloat16, false, true); else RL_CASE(__nv_bfloat16, false, false); }
    }
#undef RL_CASE
    return rl_check_launch("grad_pp");
}

rl_status rl_launch_render_pp(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, float* out,
                              cudaStream_t s) {
    const int tiles_x = (W + kTX - 1) / kTX;
    const dim3 grid((unsigned)views.n, (unsigned)tiles_x, (unsigned)((H + kTY - 1) / kTY));
    const int G = views.anchored ? 8 : groups_for(D, rl_kernel_path_setting());
    const int C = chunk_for(D, G);
    if (dt == RL_F32) {
        RLTraceScope ts("render_f32", s);
        launch_render_pp_t<float>(G, C, M, D, H, W, views, tiles_x, grid, out, s);
    } else {
        RLTraceScope ts("render_bf16", s);
        launch_render_pp_t<__nv_bfloat16>(G, C, M, D, H, W, views, tiles_x, grid, out, s);
    }
    return rl_check_launch("render_pp");
}

unsigned rl_grad_pp_tiles_x(int w) { return (unsigned)((w + kTX - 1) / kTX); }
unsigned rl_grad_pp_tiles_y(int h) { return (unsigned)((h + kTY - 1) / kTY); }

rl_status rl_launch_grad_pp_batch(const void* table, rl_dtype dt, cudaStream_t s) {
    const RLBatchHeader* hdr = static_cast<const RLBatchHeader*>(table);
    const RLBatchItem* items = rl_batch_items(table);
    const int grid = dt == RL_F32 ? rl_persistent_grid<k_grad_pp_batch<float>>(8 * kPix, 0)
                                  : rl_persistent_grid<k_grad_pp_batch<__nv_bfloat16>>(8 * kPix, 0);
    if (dt == RL_F32) {
        RLTraceScope ts("grad_pp_batch_f32", s);
        k_grad_pp_batch<float><<<grid, 8 * kPix, 0, s>>>(hdr, items);
    } else {
        RLTraceScope ts("grad_pp_batch_bf16", s);
        k_grad_pp_batch<__nv_bfloat16><<<grid, 8 * kPix, 0, s>>>(hdr, items);
    }
    return rl_check_launch("grad_pp_batch");
}

RL_DEBUG_READER(pp)
