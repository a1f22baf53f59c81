/*
 * reallife.h -- C ABI of the GB300 (sm_103a) RealLiFe hot path: Hierarchical Sparse
 * Gradient Descent (HSGD) refinement of a multi-plane image (MPI) and MPI rendering.
 *
 * Paper: "RealLiFe: Real-Time Light Field Reconstruction via Hierarchical Sparse
 * Gradient Descent" (arXiv 2307.03017).  Problem statement (Sec. 3, 3.2): sparse posed
 * source images in, an MPI in the reference frustum out, novel views rendered from it.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - MPI layout: [D][H][W][4] (R, G, B, alpha) row-major, plane d = 0 farthest and
 *    d = D-1 nearest, so the over operator of Eq. (eq_over) puts the unoccluded plane at
 *    the top index.  Storage is FP32 (RL_F32) or BF16 (RL_BF16, round-to-nearest-even
 *    on every store); all arithmetic is FP32.
 *  - Plane depths are uniform in inverse depth: rho_d = 1/far + d/(D-1) (1/near - 1/far)
 *    (rho_0 = 1/far when D = 1).
 *  - Cameras are world->camera, x_cam = R X + t, pixel = K x_cam / z with pixel centres
 *    on integer coordinates; K must have zero skew and last row (0, 0, 1).  Source and
 *    target images have the MPI's resolution H x W.
 *  - Images: [N][H][W][3] FP32.  Selections S: [k][H_l][W_l] uint8 plane indices in
 *    ascending order; masks: [H_l][W_l] uint64 with bit d set for each kept plane.
 *  - Pyramid level l works at H_l = H / 2^l, W_l = W / 2^l: images and MPI are 2x2 box
 *    averaged l times, intrinsics become f / 2^l and (c + 0.5) / 2^l - 0.5.
 *
 * Ownership and execution
 * -----------------------
 *  - The caller owns every buffer (MPI, images, outputs, workspace); the library
 *    allocates no device memory.  Pointers named "device" must be device memory of the
 *    current CUDA device; camera/parameter structs are host memory read before return.
 *  - Every call is asynchronous on `stream` (0 = legacy default stream) and enqueues
 *    kernels only, so it can be captured into a CUDA graph.  Results are valid once the
 *    stream reaches them.  Calls that share a workspace must be ordered on one stream.
 *  - Validation happens on the host before anything is launched: a call that returns
 *    RL_EINVAL launched nothing.  A launch failure returns RL_ECUDA (details from
 *    reallife_last_error()).  No C++ exception crosses this boundary.
 *  - Gradients are accumulated with FP32 atomics, so results agree run to run within
 *    FP32 rounding of the summation order, not bit for bit.
 */
#ifndef REALLIFE_H
#define REALLIFE_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RL_OK = 0,
    RL_EINVAL = 1,    /* invalid argument; nothing was launched */
    RL_ENOMEM = 2,    /* workspace too small */
    RL_ECUDA = 3,     /* a CUDA call or launch failed */
    RL_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    RL_ENOTIMPL = 5,
    RL_EBOUNDS = 6    /* a bounds check of the debug build failed (reallife_device_status) */
} rl_status;

typedef enum { RL_F32 = 0, RL_BF16 = 1 } rl_dtype;

/* Pinhole camera, world->camera, row-major. */
typedef struct {
    double K[9];
    double R[9];
    double t[3];
} rl_camera;

/* A multi-plane image in the frustum of camera `ref` (Sec. 3.1).  `data` is device
 * memory [D][H][W][4] of `dtype`, owned by the caller. */
typedef struct {
    int D, H, W;
    double near_, far_;
    rl_dtype dtype;
    void* data;
    rl_camera ref;
} rl_mpi;

/* Selection criteria (Sec. 3.3 "Gradient Sparsification" and the ablation of Sec. 5.5). */
typedef enum {
    RL_SELECT_TOPK = 0, /* the k largest reference-view alpha weights A_d, ties to the lower d */
    RL_SELECT_MVS = 1   /* MVS-sampling: the argmax of A_d (ties to the lower d) and its (k-1)/2
                           neighbours on each side, i.e. k consecutive planes starting at
                           argmax - floor((k-1)/2), shifted to stay within [0, D) */
} rl_selection;

/* One HSGD iteration: keep k planes per pixel chosen by `selection`, step `lambda` (the
 * analytic update of Sec. 3.1 read as descent), clamp the updated values to [0,1] when
 * clamp01 != 0, work at pyramid level `level`.  lambda_s > 0 adds the sparsity prior of
 * Sec. 3.4 as the prior phi of Sec. 3.1: lambda_s dL_s/dalpha, L_s = mean over the D x H_l x
 * W_l voxels of log(1.5 - |0.5 - alpha|), on the alphas of the level MPI. */
typedef struct {
    int k;
    float lambda;
    int clamp01;
    int level;
    int selection;  /* rl_selection */
    float lambda_s;
} rl_hsgd_params;

/* Upper bounds checked on the host (also D*H*W < 2^29 voxels). */
#define RL_MAX_PLANES 64
#define RL_MAX_VIEWS 16

/* ------------------------------------------------------------------ top level */

/* Bytes of workspace that reallife_hsgd_step / reallife_refine need for an MPI of
 * D x H x W with N source views and k kept planes (any level of the schedule). */
size_t reallife_workspace_bytes(int N, int D, int H, int W, int k, rl_dtype dtype);

/* Novel views (Eq. eq_render with the over operator of Eq. eq_over): warp every plane
 * into each target camera by its plane-induced homography (Eq. eq_homo), bilinear
 * sampling with zero padding, composite front to back with no background.
 *   tgt:  host array of T cameras.
 *   out:  device [T][H][W][3] FP32.
 * No workspace.  RL_EINVAL for T < 1, null pointers or invalid MPI/cameras (including views
 * whose rays at the image corners run nearly parallel to the planes). */
rl_status reallife_render(const rl_mpi* m, const rl_camera* tgt, int T, float* out, cudaStream_t stream);

/* One HSGD iteration on `m` in place (Sec. 3.3 with the analytic gradient of Sec. 3.1):
 *   M_l = Down^l(M); S = top-k of the reference-view alpha weight A_d of M_l
 *   (Eq. eq_gradient, ties to the lower plane); G = dL/dM_l on the kept voxels, where
 *   L = 1/(2N) sum_i sum_q |O(w_i(M_l))(q) - I_i^l(q)|^2 (warp, composite, loss and the
 *   exact adjoint, transmittance recomputed); M[S] <- clamp(M[S] - lambda U_l(G)) with
 *   U_l nearest-neighbour replication (the restore operator R(., S)).
 *   images:   device [N][H][W][3] FP32 at full resolution (the call averages to level l).
 *   src:      host array of N source cameras.
 *   loss_out: device float[1] (loss at level l) or NULL.
 *   S_out:    device uint8 [k][H_l][W_l] receiving the selection, or NULL.
 *   ws:       device workspace of at least reallife_workspace_bytes(...) bytes.
 * RL_ENOMEM if ws_bytes is too small; RL_EINVAL for 1 <= k <= D <= 64, 1 <= N <= 16,
 * H and W divisible by 2^level violated, or null pointers. */
rl_status reallife_hsgd_step(rl_mpi* m, const float* images, const rl_camera* src, int N, const rl_hsgd_params* p,
                             float* loss_out, uint8_t* S_out, void* ws, size_t ws_bytes, cudaStream_t stream);

/* HSGD refinement: reallife_hsgd_step at levels schedule[0..iters-1] (coarse to fine,
 * e.g. {2,1,0}; Fig. 3 and Sec. 5.2), p->level ignored.
 *   loss_per_iter: device float[iters] or NULL.
 * Errors as reallife_hsgd_step, checked for every level before the first launch. */
rl_status reallife_refine(rl_mpi* m, const float* images, const rl_camera* src, int N, const rl_hsgd_params* p,
                          const int* schedule, int iters, float* loss_per_iter, void* ws, size_t ws_bytes,
                          cudaStream_t stream);

/* HSGD iteration for callers that cannot allocate device memory (no counterpart in the
 * paper; an interface for hosts such as plugins inside an application that owns the GPU
 * heap and gives them no allocator, or frame loops that must not call cudaMalloc).  It
 * computes exactly what reallife_hsgd_step computes, but takes no workspace: the
 * library keeps a fixed scratch array of RL_NOALLOC_SCRATCH_BYTES in every GPU that
 * loads it, held until the process exits, and this call allocates nothing.
 *   - Arguments and outputs as reallife_hsgd_step.
 *   - RL_ENOMEM (with a message) when the problem needs more scratch than the array
 *     holds (reallife_workspace_bytes > RL_NOALLOC_SCRATCH_BYTES); e.g. 512x384, D=32,
 *     N=4, k=5 needs 48 MB and fits, 1920x1080 D=64 does not.
 *   - Every call made outside stream capture looks up the array's device address for the
 *     current device (cudaGetSymbolAddress), so the address stays right after a
 *     cudaDeviceReset; a call being captured reuses the address of the device's last
 *     uncaptured call.  Make the first call on a device before any stream capture.
 *   - All calls on a device share the one array, and it keeps what the last call left
 *     in it (every value a call reads is written earlier in the same call).  Calls that
 *     overlap on the GPU -- on different streams, or from different threads -- race on
 *     it: order them.
 *   - RL_EINVAL while kernel tracing is enabled (tracing creates CUDA events). */
#define RL_NOALLOC_SCRATCH_BYTES (64u << 20)
rl_status reallife_hsgd_step_noalloc(rl_mpi* m, const float* images, const rl_camera* src, int N,
                                     const rl_hsgd_params* p, float* loss_out, uint8_t* S_out, cudaStream_t stream);

/* ------------------------------------------------------------- batched step */

/* One HSGD iteration of each of many independent requests in one launch per stage, for the
 * serving pattern in which requests of different sizes are refined concurrently (the paper's
 * real-time generation for displays, Sec. 1 and Sec. 5.1 "3D display efficiency").  Each item
 * is one request's iteration with exactly the arguments of reallife_hsgd_step; the results
 * are those of reallife_hsgd_step on every item, up to FP32 rounding order: the gradient of
 * every item takes the per-pixel gather kernel family.
 *
 * The batch is described by a work table: reallife_batch_prepare writes it (host only) into
 * page-locked host memory, and reallife_hsgd_step_batch copies it to the device table and
 * enqueues three persistent launches (selection, gradient, update) whose grids do not depend
 * on the table.  A CUDA graph captured from one reallife_hsgd_step_batch call therefore serves
 * any later table of the same storage type and capacity: rewrite the host table with
 * reallife_batch_prepare (once the previous replay's copy has run) and replay.
 *
 *   items:       host array of n items; the MPI structs and cameras are read during the call.
 *   table_host:  page-locked host memory of table_bytes >= reallife_batch_table_bytes(n).
 *   table_dev:   device memory of table_bytes, 256-byte aligned.
 * RL_EINVAL: n outside [1, RL_BATCH_MAX_ITEMS], any item failing the checks of
 * reallife_hsgd_step (its index in reallife_last_error), items of different storage types,
 * two items sharing an MPI or overlapping workspaces, a table_host that is not page-locked.
 * RL_ENOMEM: table_bytes too small, or an item's ws_bytes too small.  Device-side: a table of
 * another storage type than the captured kernels' sets bit 2 of the device status word
 * (reallife_device_status) and leaves the MPIs unchanged. */
#define RL_BATCH_MAX_ITEMS 256
typedef struct {
    rl_mpi* mpi;             /* refined in place; caller-owned */
    const float* images;     /* device [N][H][W][3] FP32, full resolution */
    const rl_camera* src;    /* host array of N source cameras */
    int N;
    rl_hsgd_params params;   /* this iteration's k, lambda, clamp01, level, selection, lambda_s */
    float* loss_out;         /* device float[1] (loss at the level) or NULL */
    void* ws;                /* the request's workspace: reallife_workspace_bytes(N, D, H, W, k, dtype) */
    size_t ws_bytes;
} rl_batch_item;
size_t reallife_batch_table_bytes(int max_items);
rl_status reallife_batch_prepare(const rl_batch_item* items, int n, void* table_host, size_t table_bytes);
rl_status reallife_hsgd_step_batch(const void* table_host, void* table_dev, size_t table_bytes, cudaStream_t stream);

/* --------------------------------------------------------- gradient volume */

/* Bytes of workspace that reallife_gradient_volume needs for an MPI of D x H x W with N
 * views and k kept planes, at any level (a multiple of 256). */
size_t reallife_gradient_volume_workspace_bytes(int N, int D, int H, int W, int k, rl_dtype dtype);

/* The sparsified gradient volume V_s of one HSGD iteration at level `level` (Sec. 3.3,
 * Eq. eq_simplifiedGradients and eq_V): the input of the paper's learned update.  With
 * M_l = Down^l(M), S the selection on M_l (top-k of the reference alpha weights or the
 * MVS window, `selection`), h = H/2^l and w = W/2^l, for slot j < k of level pixel p and
 * d = S[j][p]:
 *   V[3i + c][j][p]  c < 3   PSV of source view i (Sec. 3.2): the full-resolution image i
 *                            bilinearly sampled (zero padding) where the inverse homography
 *                            of Eq. eq_homo carries each of p's 2^l x 2^l full-resolution
 *                            child pixels on plane d, averaged over the children;
 *   V[3N + i][j][p]          A^{w^-1}_i: the alpha weights alpha_d prod_{j>d}(1 - alpha_j) of
 *                            M_l warped into view i at level l (Eq. eq_gradient), sampled
 *                            bilinearly where the inverse homography carries p on plane d;
 *   V[4N + c][j][p]  c < 4   M_l[d][p] (R, G, B, alpha).
 * images: device [N][H][W][3] FP32 (full resolution).  V: device [4N+4][k][h][w] FP32,
 * overwritten.  S_out: device [k][h][w] uint8 (ascending d) or NULL.  The MPI is not
 * modified.  ws: device workspace, 256-byte aligned, at least
 * reallife_gradient_volume_workspace_bytes(...) bytes (RL_ENOMEM when smaller).
 * Asynchronous on `stream`; RL_EINVAL for the argument errors of reallife_hsgd_step. */
rl_status reallife_gradient_volume(const rl_mpi* m, const float* images, const rl_camera* src, int N, int k,
                                   int level, int selection, uint8_t* S_out, float* V, void* ws, size_t ws_bytes,
                                   cudaStream_t stream);

/* ---------------------------------------------------------- learned update */

/* Parameters of the learned-update network N_w of Sec. 3.3 ("Sparse Gradient Update"), as
 * trained: five blocks of 3x3x3 convolution (zero padding 1), batch norm and ReLU, then a
 * 1x1x1 convolution to the 4-channel (R, G, B, alpha) residual (Sec. 4 names the block
 * structure; kernel size, 32 channels per block and inference-mode batch norm are this
 * library's reading).  All pointers are device FP32:
 *   conv_w[l] [32][c_l][3][3][3] (c_0 = c_in, else 32), conv_b[l], bn_*[l] [32];
 *   out_w [4][32], out_b [4].  c_in = 4N + 4 <= 32 for the volume of N views. */
typedef struct {
    int c_in;
    float eps;
    const float* conv_w[5];
    const float* conv_b[5];
    const float* bn_gamma[5];
    const float* bn_beta[5];
    const float* bn_mean[5];
    const float* bn_var[5];
    const float* out_w;
    const float* out_b;
} rl_lgd_params;

/* Bytes of a packed network (BF16 weights with batch norm folded, FP32 biases). */
size_t reallife_lgd_net_bytes(void);

/* Folds batch norm into each block (w' = w gamma / sqrt(var + eps), b' = (b - mean) gamma /
 * sqrt(var + eps) + beta), rounds the weights to BF16 (nearest even) and packs them for the
 * tensor-core kernels.  net: device, 256-byte aligned, reallife_lgd_net_bytes() bytes;
 * written asynchronously on `stream`.  RL_EINVAL for NULL parameters or c_in outside [1, 32]. */
rl_status reallife_lgd_prepare(const rl_lgd_params* p, void* net, cudaStream_t stream);

/* Workspace of reallife_lgd_forward: two BF16 activation volumes of k x h x w x 32 and the
 * network's grid-barrier counter. */
size_t reallife_lgd_workspace_bytes(int k, int h, int w);

/* N_w(V): V device [C][k][h][w] FP32 (C <= 32; e.g. the volume of reallife_gradient_volume),
 * residual device [k][h][w][4] FP32 (16-byte aligned, overwritten).  The input is rounded to
 * BF16, every block accumulates in FP32 on the tensor cores and stores BF16 activations; the
 * last block's output feeds the 1x1x1 layer in FP32.  ws: device, 256-byte aligned, at least
 * reallife_lgd_workspace_bytes(k, h, w) bytes (RL_ENOMEM when smaller); calls that run at the
 * same time need separate workspaces.  The five blocks run in one cooperative launch (one CTA
 * per SM at most); RL_ECUDA when the device cannot make its CTAs resident together. */
rl_status reallife_lgd_forward(const void* net, const float* V, int C, int k, int h, int w, float* residual,
                               void* ws, size_t ws_bytes, cudaStream_t stream);

/* Workspace of reallife_lgd_step (any level). */
size_t reallife_lgd_step_workspace_bytes(int N, int D, int H, int W, int k, rl_dtype dtype);

/* One learned HSGD iteration at `level` (Sec. 3.3, M_{n+1} = M_n + R(N_w(V_s), S)):
 * reallife_gradient_volume, reallife_lgd_forward, then for every full-resolution pixel (y, x)
 * and slot j, d = S[j][y>>l][x>>l]: M[d][y][x] += residual[j][y>>l][x>>l], clamped to [0, 1]
 * when clamp01, rounded to the storage type.  N <= 7 (4N + 4 <= 32 channels).  S_out: device
 * [k][h][w] or NULL.  Same argument checks as reallife_gradient_volume. */
rl_status reallife_lgd_step(rl_mpi* m, const float* images, const rl_camera* src, int N, int k, int level,
                            int selection, int clamp01, const void* net, uint8_t* S_out, void* ws, size_t ws_bytes,
                            cudaStream_t stream);

/* -------------------------------------------------------- steps of the iteration */

/* Down^l of P stacked [H][W][C] FP32 slices (2x2 box average applied l times, computed
 * as one 2^l x 2^l average): x device [P][H][W][C] -> y device [P][H/2^l][W/2^l][C].
 * Sec. 3.2 "Hierarchical PSV construction". */
rl_status reallife_downsample_f32(const float* x, int P, int H, int W, int C, int level, float* y,
                                  cudaStream_t stream);

/* Selection on an MPI `m` (at whatever resolution it has): A_d = alpha_d prod_{j>d}
 * (1 - alpha_j) in FP32 at the reference view (Eq. eq_gradient), then k planes per pixel by
 * `selection` (rl_selection; Sec. 3.3).  S device [k][H][W] uint8 (ascending), mask device
 * [H][W] uint64; either may be NULL. */
rl_status reallife_select(const rl_mpi* m, int k, int selection, uint8_t* S, uint64_t* mask, cudaStream_t stream);

/* Same selection from caller-supplied FP32 keys `keys` device [D][H][W]. */
rl_status reallife_select_keys(const float* keys, int D, int H, int W, int k, int selection, uint8_t* S,
                               uint64_t* mask, cudaStream_t stream);

/* Photometric loss of N views of `m` against `images` (both at m's resolution) and its
 * gradient (warp + composite + loss + exact adjoint, Sec. 3.1/3.3):
 *   mask == NULL: dense G device [D][H][W][4] FP32;
 *   mask != NULL: compact G device [k][H][W][4] FP32, slot j of pixel p holding the
 *                 j-th kept plane of p in ascending order (mask device [H][W] uint64; bits
 *                 at or above D are ignored, and of a pixel with more than k bits set only
 *                 the k lowest planes are kept).
 *   loss_out: device float[1] or NULL.  G is overwritten.
 *   ws: device workspace (256-byte aligned), at least reallife_workspace_bytes(N, D, H, W,
 *       1, dtype) bytes; RL_ENOMEM when smaller. */
rl_status reallife_loss_grad(const rl_mpi* m, const float* images, const rl_camera* src, int N,
                             const uint64_t* mask, int k, float* G, float* loss_out, void* ws, size_t ws_bytes,
                             cudaStream_t stream);

/* Masked update (restore operator R(., S) of Sec. 3.3 followed by nearest-neighbour
 * upsampling to full resolution): for every full-resolution pixel (y, x) and j < k,
 *   d = S[j][y>>level][x>>level];
 *   M[d][y][x] <- clamp01 ? clamp(M - lambda G[j][y>>level][x>>level], 0, 1) : M - lambda G.
 * S device [k][H_l][W_l] uint8, G device [k][H_l][W_l][4] FP32.  No sparsity prior here
 * (reallife_hsgd_step applies it). */
rl_status reallife_sparse_update(rl_mpi* m, const uint8_t* S, const float* G, int k, int level, float lambda,
                                 int clamp01, cudaStream_t stream);

/* Backward of warp + composite (the differentiable forward is reallife_render with the
 * source cameras): given dL/dC device [N][H][W][3], write dL/dM device [D][H][W][4]
 * FP32 (dense, overwritten).  Transmittance is recomputed, not stored. */
rl_status reallife_render_backward(const rl_mpi* m, const rl_camera* views, int N, const float* grad_out,
                                   float* grad_mpi, cudaStream_t stream);

/* Diagnostic: warp offsets of view `view`: out device [D][H][W][2] FP32 holding
 * p - q, where p is the reference pixel sampled for plane d at the view's pixel q
 * (Eq. eq_homo inverted); NaN where the plane is not met in front of the view. */
rl_status reallife_warp_offsets(const rl_mpi* m, const rl_camera* view, float* out, cudaStream_t stream);

/* ----------------------------------------------------------------- metrics */

/* Bytes of device workspace that reallife_image_metrics (N images of H x W) and
 * reallife_kept_mass (N = 1, an H x W MPI) need; 0 for non-positive sizes. */
size_t reallife_metrics_workspace_bytes(int N, int H, int W);

/* Quality of renders (Sec. 5.1 names PSNR and SSIM): x, y device [N][H][W][3] FP32 in [0, 1].
 * out device double[2]: out[0] = mean squared difference over all N H W 3 values (PSNR =
 * 10 log10(1 / out[0])); out[1] = mean SSIM in the form of Wang et al. (2004): per colour
 * channel, over every 11 x 11 window inside the image, Gaussian window weights (sigma 1.5,
 * normalised), weighted means, variances and covariance, C1 = 0.01^2, C2 = 0.03^2, averaged
 * over windows, channels and images.  FP32 per window, FP64 sums in a fixed order
 * (deterministic).  ws: at least reallife_metrics_workspace_bytes(N, H, W) bytes, 8-byte
 * aligned.  RL_EINVAL unless 1 <= N <= 65535 and 11 <= H, W <= 65535; RL_ENOMEM when ws is
 * smaller. */
rl_status reallife_image_metrics(const float* x, const float* y, int N, int H, int W, double* out, void* ws,
                                 size_t ws_bytes, cudaStream_t stream);

/* Kept mass of a selection (Sec. 3.3; the selection keeps the planes with the largest alpha
 * weights A_d = alpha_d prod_{j>d} (1 - alpha_j) of Eq. eq_gradient at the reference view,
 * formed in FP32 as the selection forms them): out device double[2] = {sum of A over the
 * voxels whose bit d is set in mask device [H][W] uint64, sum of A over all voxels}, FP64
 * sums in a fixed order.  The fraction out[0] / out[1] is the share of the reference view's
 * alpha weight that the k kept planes carry.  ws as for reallife_image_metrics with N = 1. */
rl_status reallife_kept_mass(const rl_mpi* m, const uint64_t* mask, double* out, void* ws, size_t ws_bytes,
                             cudaStream_t stream);

/* ------------------------------------------------------------------ utilities */

/* Kernel family for the warp kernels (render, gradient):
 *   0 (default) automatic: plane-parallel for launches of fewer than 2^19 pixel-views,
 *     per-pixel gather otherwise;
 *   1 not used (a family of TMA-staged plane windows, measured slower and removed): RL_EINVAL;
 *   2 per-pixel gather (one thread per view pixel walks all planes);
 *   3 plane-parallel (warps own chunks of planes; chunks combined through the
 *     associativity of the over operator), 8 warps per block;
 *   4 plane-parallel with 4 warps per block where D <= 32; 5 same as 3.
 * All compute the same values up to FP32 rounding of the accumulation order.
 * Process-wide; RL_EINVAL for other values. */
rl_status reallife_set_kernel_path(int path);

/* Device-side status: synchronises the device and reports the status word that kernels
 * set when a bounded wait (about one second) gives up; *flags_out receives its bits
 * (1 = timeout; 2 = a batched step was given a table it cannot serve, see
 * reallife_hsgd_step_batch; 4 = a bounds check of the debug build failed).  Returns
 * RL_ETIMEOUT when the timeout bit is set, else RL_EBOUNDS when the bounds bit is set, RL_OK
 * otherwise; clear != 0 resets the word.  Results of launches that timed out are invalid.
 *
 * Debug build.  Compiled with -DRL_DEBUG (libreallife_debug.so), the warp, selection,
 * gradient-volume and update kernels check the index of each data-dependent global access
 * (bilinear taps, gradient slots taken from the slot map, plane indices written to S, batch
 * items, loss partials, the voxels of an update) against the extent of its buffer before the
 * access.  A failed check sets bit 4 and skips that access: no trap, the context stays usable.
 * The release build compiles the checks out. */
rl_status reallife_device_status(int clear, unsigned int* flags_out);

/* 1 in the debug build (-DRL_DEBUG), 0 in the release build. */
int reallife_debug_build(void);

/* Self-test of the bounds reporting of the debug build (no fault): one launch whose threads
 * 0 .. 32 store to a 32-element device buffer, each behind the bounds check; thread 32 fails
 * it, sets bit 4 of the status word and stores nothing.  After the stream has run it,
 * reallife_device_status reports RL_EBOUNDS.  The release build returns RL_ENOTIMPL and
 * launches nothing. */
rl_status reallife_selftest_bounds(cudaStream_t stream);

/* Self-test of the failure reporting (no fault, no hang): one thread waits on a
 * shared-memory barrier that nothing completes, for at most wait_us microseconds of the
 * global timer, then sets the timeout bit of the device status word and returns.  After the
 * stream has run it, reallife_device_status reports RL_ETIMEOUT; once the word is cleared,
 * the context is usable.  RL_EINVAL unless 1 <= wait_us <= 1000000. */
rl_status reallife_selftest_wait_timeout(unsigned int wait_us, cudaStream_t stream);

/* Host-side kernel tracing: when enabled, every kernel launch of this library is
 * bracketed by CUDA events on its stream and counted per kernel name.  Launches made
 * while the stream is being captured into a CUDA graph are bracketed by external event
 * nodes instead, which record on every replay of the graph. */
rl_status reallife_trace_enable(int on);
/* Synchronises the recorded events and reports, for up to `max` kernel names: name,
 * launch count and summed device milliseconds.  Resets the counters.  Captured launches
 * contribute the durations of the most recent replay (read after every replay). */
typedef struct {
    char name[48];
    long long launches;
    double total_ms;
} rl_trace_entry;
rl_status reallife_trace_read(rl_trace_entry* out, int max, int* n_out);
/* Returns the events of captured launches to the tracer (call once their graphs are gone). */
rl_status reallife_trace_release_captured(void);

const char* reallife_strerror(rl_status s);
/* Message of the most recent failure on the calling thread ("" if none). */
const char* reallife_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* REALLIFE_H */
