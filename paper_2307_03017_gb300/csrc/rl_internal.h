// rl_internal.h -- host-side declarations shared by the translation units of libreallife.
#pragma once
#include <cuda.h>
#include <cuda_runtime_api.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/reallife.h"
#include "rl_common.cuh"

// Kernel launch tracing (implemented in reallife_api.cu).  rl_trace_begin returns a
// token (-1 when tracing is off) that rl_trace_end closes on the same stream.
int rl_trace_begin(const char* name, cudaStream_t s);
void rl_trace_end(int token, cudaStream_t s);
// Records a failure message for reallife_last_error() and returns `st`.
rl_status rl_fail(rl_status st, const char* fmt, ...);
// Checks the last launch; RL_ECUDA with the CUDA message on failure.
rl_status rl_check_launch(const char* what);

struct RLTraceScope {
    int tok;
    cudaStream_t s;
    RLTraceScope(const char* name, cudaStream_t st) : tok(rl_trace_begin(name, st)), s(st) {}
    ~RLTraceScope() { rl_trace_end(tok, s); }
};

// Device status word (bit RL_DEVFLAG_TIMEOUT: a bounded wait gave up); address on the
// current device, or NULL if it cannot be resolved.
unsigned int* rl_device_status_ptr();
// Warp-kernel family for a launch over H x W pixels of n views: 2 per-pixel gather,
// 3 plane-parallel.  The automatic setting picks plane-parallel for launches of fewer than
// 2^19 pixel-views (coarse pyramid levels, small requests), where per-pixel threads are too
// few to hide gather latency, and per-pixel gather otherwise.
int rl_kernel_path(int H, int W, int nviews);
// The raw process-wide setting of reallife_set_kernel_path (0, 2 to 5).
int rl_kernel_path_setting();

// TMA descriptor of a BF16 activation volume [K][H][W][32] (16-byte aligned) with a box of
// {32 channels, halo voxels along W} and 64-byte swizzling; false when it cannot be encoded.
bool rl_encode_act_tmap(CUtensorMap* map, const void* act, int K, int H, int W, int halo);

// True when every view's warp offset p - q is the same for all pixels of a plane: no
// rotation relative to the reference (R_rel - I exactly 0 in FP32), no depth offset of the
// centre and the reference's focal lengths.
inline bool rl_views_are_shifts(const RLViews& v) {
    for (int i = 0; i < v.n; ++i) {
        const RLViewParam& p = v.v[i];
        for (int j = 0; j < 9; ++j)
            if (p.E[j] != 0.f) return false;
        if (p.C[2] != 0.f || p.dfx != 0.f || p.dfy != 0.f) return false;
    }
    return v.n > 0;
}

// ----------------------------------------------------------------- launchers
// All take device pointers and enqueue on `s`; arguments are validated by the caller.

rl_status rl_launch_render(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, float* out,
                           cudaStream_t s);
rl_status rl_launch_warp_offsets(int D, int H, int W, const RLViews& views, float* out, cudaStream_t s);

// Fused warp + composite + residual + adjoint.  mode_loss: residual from images (full-res
// images at level img_level, averaged on the fly) else from grad_out.  slots != NULL
// (slot map [D][H][W], RL_SLOT_NONE where not kept): compact gradient [k][H][W][4]; else
// dense [D][H][W][4].  partials: one float per block
// (loss mode); returns the number of blocks through *nblocks.  With loss_out != NULL the
// last block also writes loss_out[0] = loss_scale * (sum of the partials), counting blocks
// on *counter (0 at launch, left at 0).
rl_status rl_launch_grad(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, bool mode_loss,
                         const float* images, int img_level, const float* grad_out, const uint8_t* slots, float* G,
                         float inv_n, float* partials, int* nblocks, cudaStream_t s, float* loss_out = nullptr,
                         unsigned* counter = nullptr, float loss_scale = 0.f);
// Largest number of loss partials any gradient kernel family writes.
size_t rl_grad_num_blocks(int H, int W, int N);
rl_status rl_launch_grad_pp(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, bool mode_loss,
                            const float* images, int img_level, const float* grad_out, const uint8_t* slots, float* G,
                            float inv_n, float* partials, int* nblocks, cudaStream_t s, float* loss_out,
                            unsigned* counter, float loss_scale);
size_t rl_grad_pp_num_blocks(int H, int W, int N);
rl_status rl_launch_render_pp(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, float* out,
                              cudaStream_t s);
rl_status rl_launch_loss_reduce(const float* partials, int n, float scale, float* out, cudaStream_t s);

// Top-k selection on the MPI M [D][h][w][4] (or on keys [D][h][w] when keys != NULL).
// Outputs (each optional): S [k][h][w], mask [h][w], slot map [D][h][w]; Gzero
// [k][h][w][4] is zeroed.
rl_status rl_launch_select(const void* M, rl_dtype dt, const float* keys, int D, int h, int w, int k, uint8_t* S,
                           uint64_t* mask, uint8_t* slots, float* Gzero, cudaStream_t s,
                           unsigned* counter_zero = nullptr, int mode = 0);
// Level-l MPI Ml [D][H>>l][W>>l][4] = Down^l(M) (level >= 1) and the selection on it in one pass: outputs as
// rl_launch_select without the mask, identical values.  With images and Il != NULL it also writes the
// level-l source images Il [N][H>>l][W>>l][3] (2^l x 2^l means of images [N][H][W][3], formed exactly as
// the gradient kernels form them on the fly), which the gradient then reads at img_level 0.
rl_status rl_launch_pyramid_select(const void* M, rl_dtype dt, int D, int H, int W, int level, void* Ml, int k,
                                   uint8_t* S, uint8_t* slots, float* Gzero, unsigned* counter_zero, int mode,
                                   cudaStream_t s, const float* images = nullptr, int N = 0, float* Il = nullptr);
// Slot map [D][h][w] from a selection mask [h][w]: the kept planes of a pixel in ascending order
// take slots 0 .. k-1; kept planes beyond the first k get no slot.
rl_status rl_launch_mask_to_slots(const uint64_t* mask, int D, int k, int hw, uint8_t* slots, cudaStream_t s);
rl_status rl_launch_downsample_f32(const float* x, int P, int H, int W, int C, int level, float* y,
                                   cudaStream_t s);
// With Ml (level MPI) and lambda_s != 0 the sparsity prior joins the alpha step.
rl_status rl_launch_update(void* M, rl_dtype dt, int D, int H, int W, int level, const uint8_t* S, const float* G,
                           int k, float lambda, int clamp01, cudaStream_t s, const void* Ml = nullptr,
                           float lambda_s = 0.f);

// Batched stages of one HSGD iteration over a batch table in device memory (header and items
// of rl_common.cuh), each one persistent launch of one wave of resident blocks.  The gradient
// stage is two launches: the items that rl_kernel_path sends to the per-pixel gather family
// (shared memory for `planes` planes) and those it sends to the plane-parallel family.
rl_status rl_launch_select_batch(const void* table, rl_dtype dt, cudaStream_t s);
rl_status rl_launch_grad_batch(const void* table, rl_dtype dt, int planes, cudaStream_t s);
rl_status rl_launch_grad_pp_batch(const void* table, rl_dtype dt, cudaStream_t s);
rl_status rl_launch_update_batch(const void* table, rl_dtype dt, cudaStream_t s);
unsigned rl_grad_gather_tiles_x(int w);
unsigned rl_grad_gather_tiles_y(int h);
unsigned rl_grad_pp_tiles_x(int w);
unsigned rl_grad_pp_tiles_y(int h);

// Blocks of a persistent launch of `kernel`: the resident blocks per SM on the current device
// times its SMs (at least one); computed once per device and kernel instantiation.
template <auto kernel>
inline int rl_persistent_grid(int threads, size_t smem) {
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cacheable = dev >= 0 && dev < 64;
    if (cacheable && cached[dev]) return cached[dev];
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess) cudaGetLastError();
    const int grid = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    if (cacheable) cached[dev] = grid;
    return grid;
}
unsigned rl_grad_batch_tiles_x(int w);
unsigned rl_grad_batch_tiles_y(int h);

// Metrics (metrics.cu): FP64 partial sums of the SSIM windows, squared differences and kept
// mass, and the number of partials the two metric calls need.
size_t rl_ssim_blocks(int N, int H, int W);
size_t rl_metrics_partials(int N, int H, int W);
// out[0] = mean squared difference, out[1] = mean SSIM of x, y [N][H][W][3] (H, W >= 11).
rl_status rl_launch_image_metrics(const float* x, const float* y, int N, int H, int W, double* out, double* partials,
                                  cudaStream_t s);
// out[0] = sum of the kept alpha weights, out[1] = sum of all alpha weights.
rl_status rl_launch_kept_mass(const void* M, rl_dtype dt, int D, int H, int W, const uint64_t* mask, double* out,
                              double* partials, cudaStream_t s);

// Alpha weights of the MPI warped into each view (Eq. eq_gradient): A device [N][D][H][W].
rl_status rl_launch_view_alpha(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, float* A,
                               cudaStream_t s);
// Sparsified gradient volume V [4N+4][k][h][w] from the level MPI Ml [D][h][w][4], the
// selection S [k][h][w], the view alpha weights A [N][D][h][w] and full-resolution images.
// With act != NULL the same channels go to act [k][h][w][32] BF16 channels-last (the learned
// network's input, channels >= 4N+4 zero) instead, and V is not written.
rl_status rl_launch_volume(const void* Ml, rl_dtype dt, int D, int h, int w, int level, const uint8_t* S, int k,
                           const float* A, const float* images, const RLInvViews& iv, float* V, cudaStream_t s,
                           void* act = nullptr);

// Gradient volume of Sec. 3.3 at `level`: selection S, view alpha weights and V_s, with the
// checks of reallife_gradient_volume; with act != NULL it writes the network's packed input
// instead of V (V may then be NULL).
rl_status rl_gradient_volume(const rl_mpi* m, const float* images, const rl_camera* src, int N, int k, int level,
                             int selection, uint8_t* S_out, float* V, void* act, void* ws, size_t ws_bytes,
                             cudaStream_t stream);

// Learned update network (lgd.cu): packed parameter bytes, parameter packing, activation
// buffer bytes and the forward pass (V [C][K][H][W] FP32 -> residual [K][H][W][4] FP32,
// two activation buffers of rl_lgd_act_bytes each and a 4-byte grid-barrier counter that the
// call resets on the stream).
size_t rl_lgd_net_bytes();
rl_status rl_lgd_prepare(const rl_lgd_params* p, void* net, cudaStream_t s);
size_t rl_lgd_act_bytes(int K, int H, int W);
rl_status rl_lgd_forward(const void* net, const float* V, int C, int K, int H, int W, float* residual, void* act0,
                         void* act1, unsigned* grid_bar, cudaStream_t s);
// The network alone, on an input already packed into act0 (act1 and the counter as above).
rl_status rl_lgd_network(const void* net, int K, int H, int W, float* residual, void* act0, void* act1,
                         unsigned* grid_bar, cudaStream_t s);
