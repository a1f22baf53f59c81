// grad_tma.cu -- fused warp + composite + residual + exact adjoint with TMA-staged plane
// windows and shared-memory adjoint accumulation (the arithmetic is that of grad.cu).
//
// Block = 32 x 8 pixels of one view; blocks of the N views of a tile are adjacent in the
// launch so that their overlapping windows meet in L2.  The block walks 2D plane windows
// through a two-stage TMA pipeline: first the planes nearest to farthest (composite, T_d
// kept in shared memory), then farthest to nearest (adjoint).  In the adjoint, every
// sample adds its four bilinear contributions into a shared-memory copy of the plane
// window (one FP32 plane per channel, so lanes hit distinct banks); after the plane, the
// window is flushed with one slot-map lookup and at most one global float4 atomic per
// voxel (sparse mode: only voxels kept by the selection, at their compact slot).
#include "rl_internal.h"
#include "rl_tma.cuh"

namespace {

using namespace rltma;

template <bool SPARSE>
__device__ __forceinline__ void scatter_tap_g(float* __restrict__ G, const uint8_t* __restrict__ slots_d, int d,
                                              int H, int W, int x, int y, float wt, float4 g) {
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H || wt == 0.f) return;
    const size_t pix = (size_t)y * W + x;
    const unsigned slot = SPARSE ? (unsigned)__ldg(slots_d + pix) : (unsigned)d;
    if (SPARSE && slot == RL_SLOT_NONE) return;
    atomicAdd(reinterpret_cast<float4*>(G + ((size_t)slot * H * W + pix) * 4),
              make_float4(wt * g.x, wt * g.y, wt * g.z, wt * g.w));
}

template <typename Tm>
__host__ __device__ constexpr size_t stage_bytes() {
    return (size_t)BW * BH * 4 * sizeof(Tm);
}

template <typename Tm>
size_t grad_smem_bytes(int D) {
    return 2 * stage_bytes<Tm>() + (size_t)4 * BW * BH * sizeof(float) + (size_t)D * NT * sizeof(float) + 128 + 256;
}

template <typename Tm, bool SPARSE, bool LOSS>
__global__ void __launch_bounds__(NT, 3)
k_grad_tma(const __grid_constant__ CUtensorMap tmap, const Tm* __restrict__ M, int D, int H, int W,
           const __grid_constant__ RLViews views, int tiles_x, const float* __restrict__ images, int img_level,
           const float* __restrict__ grad_out, const uint8_t* __restrict__ slots, float* __restrict__ G, float inv_n,
           float* __restrict__ partials, unsigned int* __restrict__ status, float* __restrict__ loss_out,
           unsigned* __restrict__ counter, float loss_scale) {
    extern __shared__ __align__(128) unsigned char smem[];
    Tm* stage0 = reinterpret_cast<Tm*>(smem);
    Tm* stage1 = reinterpret_cast<Tm*>(smem + stage_bytes<Tm>());
    float* acc = reinterpret_cast<float*>(smem + 2 * stage_bytes<Tm>());  // [4][BH][BW]
    float* sT = acc + 4 * BW * BH;                                        // [D][NT]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sT + (size_t)D * NT);    // [2]
    float* scratch = reinterpret_cast<float*>(bars + 2);                  // [64]

    const int tid = threadIdx.x;
    const int nv = views.n;
    const int view = blockIdx.x % nv;
    const int tile = blockIdx.x / nv;
    const int qx = (tile % tiles_x) * TX + (tid % TX);
    const int qy = (tile / tiles_x) * TY + (tid / TX);
    const bool active = qx < W && qy < H;
    const RLWarp w = rl_warp_coeffs(views.v[view], (float)min(qx, W - 1), (float)min(qy, H - 1));
    const TileBounds tb = tile_bounds((float)min(qx, W - 1) + w.ax, (float)min(qy, H - 1) + w.ay, w.bx, w.by,
                                      w.dir_ok, scratch);

    for (int i = tid; i < 4 * BW * BH; i += NT) acc[i] = 0.f;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int nseq = 2 * D;  // planes D-1..0 (forward), then 0..D-1 (adjoint)
    auto plane_of = [&](int j) { return j < D ? D - 1 - j : j - D; };
    auto issue = [&](int j) {
        const int d = plane_of(j);
        const Window win = window_for(tb, views.rho[d]);
        uint64_t* bar = &bars[j & 1];
        fence_proxy_async();
        mbar_expect_tx(bar, (uint32_t)stage_bytes<Tm>());
        tma_load_3d((j & 1) ? (void*)stage1 : (void*)stage0, &tmap, bar, win.xlo * 4, win.ylo, d);
    };
    if (tid == 0) {
        issue(0);
        if (nseq > 1) issue(1);
    }
    uint32_t phase0 = 0, phase1 = 0;

    const size_t plane = (size_t)H * W * 4;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    float r0 = 0.f, r1 = 0.f, r2 = 0.f, lsum = 0.f;
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
    bool aborted = false;

    for (int j = 0; j < nseq; ++j) {
        const int d = plane_of(j);
        const bool adj = j >= D;
        const float rho = views.rho[d];
        const Window win = window_for(tb, rho);
        const Tm* st = (j & 1) ? stage1 : stage0;
        if (j == D && active) {
            if (LOSS) {
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
                const float e0 = c0 - i0 * inv_area, e1 = c1 - i1 * inv_area, e2 = c2 - i2 * inv_area;
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
        }
        // wait for this plane's window
        const bool ok_wait = mbar_wait(&bars[j & 1], (j & 1) ? phase1 : phase0);
        if (ok_wait) {
            if (j & 1) phase1 ^= 1u; else phase0 ^= 1u;
        } else {
            atomicOr(status, RL_DEVFLAG_TIMEOUT);
        }

        RLTaps t;
        t.ok = false;
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
        int lx = 0, ly = 0;
        bool inwin = false;
        if (active) {
            t = rl_taps(w, rho, qx, qy);
            if (t.ok) {
                lx = t.x0 - win.xlo;
                ly = t.y0 - win.ylo;
                inwin = lx >= 0 && ly >= 0 && lx + 1 < win.nx && ly + 1 < win.ny;
                m = inwin ? window_sample(st, lx, ly, t.fx, t.fy) : rl_sample(M + d * plane, H, W, t);
            }
        }
        if (!adj) {
            if (active) {
                sT[d * NT + tid] = T;
                const float a = T * m.w;
                c0 = fmaf(a, m.x, c0);
                c1 = fmaf(a, m.y, c1);
                c2 = fmaf(a, m.z, c2);
                T = T * (1.f - m.w);
            }
        } else if (active) {
            const float Td = sT[d * NT + tid];
            if (t.ok && Td != 0.f) {
                const float gc = Td * m.w;
                float4 g;
                g.x = gc * r0;
                g.y = gc * r1;
                g.z = gc * r2;
                g.w = Td * fmaf(m.x - b0, r0, fmaf(m.y - b1, r1, (m.z - b2) * r2));
                const float w00 = (1.f - t.fx) * (1.f - t.fy), w10 = t.fx * (1.f - t.fy);
                const float w01 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
                if (inwin) {
                    float* a0 = acc + ly * BW + lx;
                    const int cs = BW * BH;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float gv = c == 0 ? g.x : c == 1 ? g.y : c == 2 ? g.z : g.w;
                        float* ac = a0 + c * cs;
                        atomicAdd(ac, w00 * gv);
                        atomicAdd(ac + 1, w10 * gv);
                        atomicAdd(ac + BW, w01 * gv);
                        atomicAdd(ac + BW + 1, w11 * gv);
                    }
                } else {
                    const uint8_t* sd = SPARSE ? slots + (size_t)d * H * W : nullptr;
                    scatter_tap_g<SPARSE>(G, sd, d, H, W, t.x0, t.y0, w00, g);
                    scatter_tap_g<SPARSE>(G, sd, d, H, W, t.x0 + 1, t.y0, w10, g);
                    scatter_tap_g<SPARSE>(G, sd, d, H, W, t.x0, t.y0 + 1, w01, g);
                    scatter_tap_g<SPARSE>(G, sd, d, H, W, t.x0 + 1, t.y0 + 1, w11, g);
                }
            }
            const float om = 1.f - m.w;
            b0 = fmaf(m.x, m.w, om * b0);
            b1 = fmaf(m.y, m.w, om * b1);
            b2 = fmaf(m.z, m.w, om * b2);
        }
        // every thread is done with this stage (and, in the adjoint, the window sums are complete)
        aborted = __syncthreads_or(!ok_wait) != 0;
        if (aborted) break;
        if (adj) {
            // flush the window: one mask lookup and at most one global atomic per voxel
            const int cs = BW * BH;
            for (int yy = tid / 32; yy < win.ny; yy += NT / 32) {
                const int gy = win.ylo + yy;
                for (int xx = tid % 32; xx < win.nx; xx += 32) {
                    const int i = yy * BW + xx;
                    const float4 v = make_float4(acc[i], acc[i + cs], acc[i + 2 * cs], acc[i + 3 * cs]);
                    if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
                    acc[i] = 0.f;
                    acc[i + cs] = 0.f;
                    acc[i + 2 * cs] = 0.f;
                    acc[i + 3 * cs] = 0.f;
                    const int gx = win.xlo + xx;
                    if ((unsigned)gx >= (unsigned)W || (unsigned)gy >= (unsigned)H) continue;
                    const size_t pix = (size_t)gy * W + gx;
                    const unsigned slot = SPARSE ? (unsigned)__ldg(slots + (size_t)d * H * W + pix) : (unsigned)d;
                    if (SPARSE && slot == RL_SLOT_NONE) continue;
                    atomicAdd(reinterpret_cast<float4*>(G + ((size_t)slot * H * W + pix) * 4), v);
                }
            }
        }
        if (tid == 0 && j + 2 < nseq) issue(j + 2);
        if (adj) __syncthreads();  // window sums cleared before the next plane adds into them
    }
    if (aborted) {
        // let copies still in flight land before the block's shared memory is released
        if (tid == 0) {
            mbar_wait(&bars[0], phase0);
            mbar_wait(&bars[1], phase1);
        }
        __syncthreads();
        return;
    }
    if (LOSS) {
        lsum = rl_warp_sum(lsum);
        if ((tid & 31) == 0) scratch[tid >> 5] = lsum;
        __syncthreads();
        float blk = 0.f;
        if (tid == 0)
            for (int i = 0; i < NT / 32; ++i) blk += scratch[i];
        __syncthreads();
        rl_loss_epilogue(blk, partials, blockIdx.x, gridDim.x, loss_out, counter, loss_scale, tid, NT, scratch);
    }
}

template <typename Tm, bool SPARSE, bool LOSS>
void launch_t(const CUtensorMap& tmap, const void* M, int D, int H, int W, const RLViews& views, const float* images,
              int img_level, const float* grad_out, const uint8_t* slots, float* G, float inv_n, float* partials,
              unsigned int* status, float* loss_out, unsigned* counter, float loss_scale, cudaStream_t s) {
    auto kern = k_grad_tma<Tm, SPARSE, LOSS>;
    const size_t smem = grad_smem_bytes<Tm>(D);
    static size_t configured = 0;
    if (smem > configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem_bytes<Tm>(RL_DEV_MAX_PLANES));
        configured = grad_smem_bytes<Tm>(RL_DEV_MAX_PLANES);
    }
    const int tiles_x = (W + TX - 1) / TX, tiles_y = (H + TY - 1) / TY;
    const unsigned blocks = (unsigned)(tiles_x * tiles_y * views.n);
    kern<<<blocks, NT, smem, s>>>(tmap, (const Tm*)M, D, H, W, views, tiles_x, images, img_level, grad_out, slots, G,
                                  inv_n, partials, status, loss_out, counter, loss_scale);
}

}  // namespace

size_t rl_grad_tma_num_blocks(int H, int W, int N) {
    return (size_t)((W + TX - 1) / TX) * ((H + TY - 1) / TY) * N;
}

rl_status rl_launch_grad_tma(const CUtensorMap& tmap, const void* M, rl_dtype dt, int D, int H, int W,
                             const RLViews& views, bool mode_loss, const float* images, int img_level,
                             const float* grad_out, const uint8_t* slots, float* G, float inv_n, float* partials,
                             int* nblocks, cudaStream_t s, float* loss_out, unsigned* counter, float loss_scale) {
    unsigned int* status = rl_device_status_ptr();
    if (!status) return rl_fail(RL_ECUDA, "device status word unavailable");
    if (nblocks) *nblocks = (int)rl_grad_tma_num_blocks(H, W, views.n);
    const bool sparse = slots != nullptr;
    const char* name = dt == RL_F32 ? (sparse ? "grad_sparse_f32" : "grad_dense_f32")
                                    : (sparse ? "grad_sparse_bf16" : "grad_dense_bf16");
    RLTraceScope ts(name, s);
#define RL_CASE(TM, SP, LS) \
    launch_t<TM, SP, LS>(tmap, M, D, H, W, views, images, img_level, grad_out, slots, G, inv_n, partials, status, \
                         loss_out, counter, loss_scale, s)
    if (dt == RL_F32) {
        if (sparse) { if (mode_loss) RL_CASE(float, true, true); else RL_CASE(float, true, false); }
        else        { if (mode_loss) RL_CASE(float, false, true); else RL_CASE(float, false, false); }
    } else {
        if (sparse) { if (mode_loss) RL_CASE(__nv_bfloat16, true, true); else RL_CASE(__nv_bfloat16, true, false); }
        else        { if (mode_loss) RL_CASE(__nv_bfloat16, false, true); else RL_CASE(__nv_bfloat16, false, false); }
    }
#undef RL_CASE
    return rl_check_launch("grad_tma");
}
