// metrics.cu -- quality metrics of renders (Sec. 5.1: PSNR, SSIM) and the kept-mass fraction
// of a selection (the share of the reference view's alpha weights that the kept planes carry,
// Eq. eq_gradient, Sec. 3.3).
//
// SSIM follows Wang et al. (2004): per colour channel, over every 11 x 11 window that lies
// inside the image, with Gaussian weights (sigma 1.5, normalised), weighted means mu, variances
// and covariance, C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1), averaged over windows, channels
// and images.  A block stages a 26 x 26 pixel tile (3 channels of both images) in shared
// memory and each thread forms one window's moments twice: first the means, then the moments
// of the values minus those means (no cancellation of E[x^2] - mu^2 in FP32).  Sums leave each
// block as FP64 partials that one block adds in index order, so the results are deterministic.
#include <cmath>

#include "rl_internal.h"

namespace {

constexpr int kTile = 16, kRad = 5, kWin = 2 * kRad + 1, kSpan = kTile + 2 * kRad;
constexpr int kMseBlocks = 1024, kMetricThreads = 256;

struct SsimWeights {
    float g[kWin];  // separable Gaussian, normalised so that the 11 x 11 outer product sums to 1
};

// Block sum (thread tid of nthreads, a multiple of 32); the total is returned to thread 0.
__device__ __forceinline__ double block_sum_f64(double v, double* red, int tid, int nthreads) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int i = 0; i < (nthreads >> 5); ++i) s += red[i];  // fixed order
    __syncthreads();
    return s;
}

// grid (tiles_x, tiles_y, N); block kTile x kTile.  partials[block] = sum over the block's
// windows and the three channels of SSIM.
__global__ void __launch_bounds__(kTile* kTile)
k_ssim(const float* __restrict__ x, const float* __restrict__ y, int H, int W, const __grid_constant__ SsimWeights sw,
       double* __restrict__ partials) {
    __shared__ float sx[3][kSpan][kSpan + 1];
    __shared__ float sy[3][kSpan][kSpan + 1];
    __shared__ double red[kTile * kTile / 32];
    const int n = blockIdx.z;
    const int ox = blockIdx.x * kTile, oy = blockIdx.y * kTile;  // top-left window of the tile
    const size_t img = (size_t)n * H * W * 3;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    for (int i = tid; i < kSpan * kSpan; i += kTile * kTile) {
        const int ty = i / kSpan, tx = i % kSpan;
        const int gx = ox + tx, gy = oy + ty;
        const bool in = gx < W && gy < H;
        const size_t e = img + ((size_t)gy * W + gx) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sx[c][ty][tx] = in ? __ldg(x + e + c) : 0.f;
            sy[c][ty][tx] = in ? __ldg(y + e + c) : 0.f;
        }
    }
    __syncthreads();
    const int wx = ox + threadIdx.x, wy = oy + threadIdx.y;  // window's top-left pixel
    float acc = 0.f;
    if (wx + kWin <= W && wy + kWin <= H) {
        const float C1 = 1.0e-4f, C2 = 9.0e-4f;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            float mx = 0.f, my = 0.f;
            for (int i = 0; i < kWin; ++i) {
                float rx = 0.f, ry = 0.f;
#pragma unroll
                for (int j = 0; j < kWin; ++j) {
                    rx = fmaf(sw.g[j], sx[c][threadIdx.y + i][threadIdx.x + j], rx);
                    ry = fmaf(sw.g[j], sy[c][threadIdx.y + i][threadIdx.x + j], ry);
                }
                mx = fmaf(sw.g[i], rx, mx);
                my = fmaf(sw.g[i], ry, my);
            }
            float vxx = 0.f, vyy = 0.f, vxy = 0.f;
            for (int i = 0; i < kWin; ++i) {
                float rxx = 0.f, ryy = 0.f, rxy = 0.f;
#pragma unroll
                for (int j = 0; j < kWin; ++j) {
                    const float a = sx[c][threadIdx.y + i][threadIdx.x + j] - mx;
                    const float b = sy[c][threadIdx.y + i][threadIdx.x + j] - my;
                    rxx = fmaf(sw.g[j] * a, a, rxx);
                    ryy = fmaf(sw.g[j] * b, b, ryy);
                    rxy = fmaf(sw.g[j] * a, b, rxy);
                }
                vxx = fmaf(sw.g[i], rxx, vxx);
                vyy = fmaf(sw.g[i], ryy, vyy);
                vxy = fmaf(sw.g[i], rxy, vxy);
            }
            const float num = (2.f * mx * my + C1) * (2.f * vxy + C2);
            const float den = (mx * mx + my * my + C1) * (vxx + vyy + C2);
            acc += num / den;
        }
    }
    const double s = block_sum_f64((double)acc, red, tid, kTile * kTile);
    if (tid == 0) partials[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
}

// Sum of squared differences over n floats: grid-stride, FP32 per thread, FP64 per block.
__global__ void __launch_bounds__(kMetricThreads)
k_sq_diff(const float* __restrict__ x, const float* __restrict__ y, size_t n, double* __restrict__ partials) {
    __shared__ double red[kMetricThreads / 32];
    float s = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = __ldg(x + i) - __ldg(y + i);
        s = fmaf(d, d, s);
    }
    const double b = block_sum_f64((double)s, red, threadIdx.x, kMetricThreads);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// Kept mass: one thread per reference pixel, planes nearest first; A_d = T alpha_d in FP32
// (the selection's own keys), T *= 1 - alpha_d.  partials[2 block] = kept, [2 block + 1] = all.
template <typename Tm>
__global__ void __launch_bounds__(kMetricThreads)
k_kept_mass(const Tm* __restrict__ M, int D, int hw, const uint64_t* __restrict__ mask,
            double* __restrict__ partials) {
    __shared__ double red[kMetricThreads / 32];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float kept = 0.f, all = 0.f;
    if (p < hw) {
        const uint64_t mk = __ldg(reinterpret_cast<const unsigned long long*>(mask) + p);
        float T = 1.f;
        for (int d = D - 1; d >= 0; --d) {
            const float a = RLStore<Tm>::load1(M + ((size_t)d * hw + p) * 4 + 3);
            const float A = T * a;
            all += A;
            if ((mk >> d) & 1ull) kept += A;
            T = T * (1.f - a);
        }
    }
    const double k = block_sum_f64((double)kept, red, threadIdx.x, kMetricThreads);
    const double t = block_sum_f64((double)all, red, threadIdx.x, kMetricThreads);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = k;
        partials[2 * blockIdx.x + 1] = t;
    }
}

// out[0] = scale * sum of partials[i * stride + offset] over i < n, in index order per thread
// and a fixed tree across threads (deterministic).
__global__ void __launch_bounds__(kMetricThreads)
k_sum_partials(const double* __restrict__ partials, int n, int stride, int offset, double scale,
               double* __restrict__ out) {
    __shared__ double red[kMetricThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[(size_t)i * stride + offset];
    s = block_sum_f64(s, red, threadIdx.x, kMetricThreads);
    if (threadIdx.x == 0) out[0] = s * scale;
}

SsimWeights ssim_weights() {
    SsimWeights w;
    double g[kWin], sum = 0.0;
    for (int i = 0; i < kWin; ++i) {
        const double r = (double)(i - kRad);
        g[i] = std::exp(-r * r / (2.0 * 1.5 * 1.5));
        sum += g[i];
    }
    for (int i = 0; i < kWin; ++i) w.g[i] = (float)(g[i] / sum);
    return w;
}

}  // namespace

size_t rl_ssim_blocks(int N, int H, int W) {
    if (H < kWin || W < kWin) return 0;
    return (size_t)N * ((W - kWin + 1 + kTile - 1) / kTile) * ((H - kWin + 1 + kTile - 1) / kTile);
}

size_t rl_metrics_partials(int N, int H, int W) {
    const size_t img = rl_ssim_blocks(N, H, W) + kMseBlocks;
    const size_t kept = 2 * (((size_t)H * W + kMetricThreads - 1) / kMetricThreads);
    return img > kept ? img : kept;
}

rl_status rl_launch_image_metrics(const float* x, const float* y, int N, int H, int W, double* out, double* partials,
                                  cudaStream_t s) {
    const size_t nssim = rl_ssim_blocks(N, H, W);
    const dim3 grid((unsigned)((W - kWin + 1 + kTile - 1) / kTile), (unsigned)((H - kWin + 1 + kTile - 1) / kTile),
                    (unsigned)N);
    {
        RLTraceScope ts("ssim", s);
        k_ssim<<<grid, dim3(kTile, kTile), 0, s>>>(x, y, H, W, ssim_weights(), partials);
    }
    const size_t n = (size_t)N * H * W * 3;
    {
        RLTraceScope ts("sq_diff", s);
        k_sq_diff<<<kMseBlocks, kMetricThreads, 0, s>>>(x, y, n, partials + nssim);
    }
    const double nwin = (double)N * 3.0 * (double)(H - kWin + 1) * (double)(W - kWin + 1);
    RLTraceScope ts("metric_sums", s);
    k_sum_partials<<<1, kMetricThreads, 0, s>>>(partials + nssim, kMseBlocks, 1, 0, 1.0 / (double)n, out);
    k_sum_partials<<<1, kMetricThreads, 0, s>>>(partials, (int)nssim, 1, 0, 1.0 / nwin, out + 1);
    return rl_check_launch("image_metrics");
}

rl_status rl_launch_kept_mass(const void* M, rl_dtype dt, int D, int H, int W, const uint64_t* mask, double* out,
                              double* partials, cudaStream_t s) {
    const int hw = H * W;
    const int blocks = (hw + kMetricThreads - 1) / kMetricThreads;
    {
        RLTraceScope ts("kept_mass", s);
        if (dt == RL_F32)
            k_kept_mass<float><<<blocks, kMetricThreads, 0, s>>>((const float*)M, D, hw, mask, partials);
        else
            k_kept_mass<__nv_bfloat16><<<blocks, kMetricThreads, 0, s>>>((const __nv_bfloat16*)M, D, hw, mask,
                                                                         partials);
    }
    RLTraceScope ts("metric_sums", s);
    k_sum_partials<<<1, kMetricThreads, 0, s>>>(partials, blocks, 2, 0, 1.0, out);
    k_sum_partials<<<1, kMetricThreads, 0, s>>>(partials, blocks, 2, 1, 1.0, out + 1);
    return rl_check_launch("kept_mass");
}
