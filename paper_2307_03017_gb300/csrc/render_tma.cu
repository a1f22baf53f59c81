// render_tma.cu -- novel-view rendering (Eq. eq_render, Eq. eq_over) with TMA-staged plane
// windows; the arithmetic is that of render.cu.
//
// Block = 32 x 8 pixels of one target view, the blocks of all views of a tile adjacent in
// the launch.  Planes are walked nearest first through a two-stage TMA pipeline; a block
// stops early once every one of its pixels has reached transmittance exactly zero.
#include "rl_internal.h"
#include "rl_tma.cuh"

namespace {

using namespace rltma;

template <typename Tm>
__host__ __device__ constexpr size_t rstage_bytes() {
    return (size_t)BW * BH * 4 * sizeof(Tm);
}

template <typename Tm>
__host__ __device__ constexpr size_t render_smem_bytes() {
    return 2 * rstage_bytes<Tm>() + 16 + 256;
}

template <typename Tm>
__global__ void __launch_bounds__(NT)
k_render_tma(const __grid_constant__ CUtensorMap tmap, const Tm* __restrict__ M, int D, int H, int W,
             const __grid_constant__ RLViews views, int tiles_x, float* __restrict__ out,
             unsigned int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    Tm* stage0 = reinterpret_cast<Tm*>(smem);
    Tm* stage1 = reinterpret_cast<Tm*>(smem + rstage_bytes<Tm>());
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * rstage_bytes<Tm>());
    float* scratch = reinterpret_cast<float*>(bars + 2);

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
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int j) {
        const int d = D - 1 - j;
        const Window win = window_for(tb, views.rho[d]);
        uint64_t* bar = &bars[j & 1];
        fence_proxy_async();
        mbar_expect_tx(bar, (uint32_t)rstage_bytes<Tm>());
        tma_load_3d((j & 1) ? (void*)stage1 : (void*)stage0, &tmap, bar, win.xlo * 4, win.ylo, d);
    };
    if (tid == 0) {
        issue(0);
        if (D > 1) issue(1);
    }
    uint32_t phase0 = 0, phase1 = 0;
    int issued = D > 1 ? 2 : 1;
    const size_t plane = (size_t)H * W * 4;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    bool aborted = false;
    int j = 0;
    for (; j < D; ++j) {
        const int d = D - 1 - j;
        const float rho = views.rho[d];
        const Window win = window_for(tb, rho);
        const Tm* st = (j & 1) ? stage1 : stage0;
        const bool ok_wait = mbar_wait(&bars[j & 1], (j & 1) ? phase1 : phase0);
        if (ok_wait) {
            if (j & 1) phase1 ^= 1u; else phase0 ^= 1u;
        } else {
            atomicOr(status, RL_DEVFLAG_TIMEOUT);
        }
        if (active && T != 0.f) {
            const RLTaps t = rl_taps(w, rho, qx, qy);
            if (t.ok) {
                const int lx = t.x0 - win.xlo, ly = t.y0 - win.ylo;
                const bool inwin = lx >= 0 && ly >= 0 && lx + 1 < win.nx && ly + 1 < win.ny;
                const float4 m = inwin ? window_sample(st, lx, ly, t.fx, t.fy) : rl_sample(M + d * plane, H, W, t);
                const float a = T * m.w;
                c0 = fmaf(a, m.x, c0);
                c1 = fmaf(a, m.y, c1);
                c2 = fmaf(a, m.z, c2);
                T = T * (1.f - m.w);
            }
        }
        const bool done = !active || T == 0.f;
        // all threads are done with this stage; stop early when every pixel is opaque
        const int votes = __syncthreads_count(done) + (__syncthreads_or(!ok_wait) ? (1 << 20) : 0);
        if (votes >= (1 << 20)) {
            aborted = true;
            break;
        }
        if (votes == NT) break;
        if (tid == 0 && j + 2 < D) {
            issue(j + 2);
            ++issued;
        }
    }
    // copies issued but not consumed must land before shared memory is released
    if (tid == 0) {
        const int consumed = aborted ? j : j + 1;
        for (int k = consumed; k < issued; ++k) {
            if (!mbar_wait(&bars[k & 1], (k & 1) ? phase1 : phase0)) atomicOr(status, RL_DEVFLAG_TIMEOUT);
            if (k & 1) phase1 ^= 1u; else phase0 ^= 1u;
        }
    }
    __syncthreads();
    if (active) {
        float* o = out + (((size_t)view * H + qy) * W + qx) * 3;
        o[0] = c0;
        o[1] = c1;
        o[2] = c2;
    }
}

template <typename Tm>
void launch_render_t(const CUtensorMap& tmap, const void* M, int D, int H, int W, const RLViews& views, float* out,
                     unsigned int* status, cudaStream_t s) {
    const int tiles_x = (W + TX - 1) / TX, tiles_y = (H + TY - 1) / TY;
    k_render_tma<Tm><<<(unsigned)(tiles_x * tiles_y * views.n), NT, render_smem_bytes<Tm>(), s>>>(
        tmap, (const Tm*)M, D, H, W, views, tiles_x, out, status);
}

}  // namespace

rl_status rl_launch_render_tma(const CUtensorMap& tmap, const void* M, rl_dtype dt, int D, int H, int W,
                               const RLViews& views, float* out, cudaStream_t s) {
    unsigned int* status = rl_device_status_ptr();
    if (!status) return rl_fail(RL_ECUDA, "device status word unavailable");
    if (dt == RL_F32) {
        RLTraceScope ts("render_f32", s);
        launch_render_t<float>(tmap, M, D, H, W, views, out, status, s);
    } else {
        RLTraceScope ts("render_bf16", s);
        launch_render_t<__nv_bfloat16>(tmap, M, D, H, W, views, out, status, s);
    }
    return rl_check_launch("render_tma");
}
