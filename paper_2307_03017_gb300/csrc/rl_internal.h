// rl_internal.h -- host-side declarations shared by the translation units of libreallife.
#pragma once
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

// ----------------------------------------------------------------- launchers
// All take device pointers and enqueue on `s`; arguments are validated by the caller.

rl_status rl_launch_render(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, float* out,
                           cudaStream_t s);
rl_status rl_launch_warp_offsets(int D, int H, int W, const RLViews& views, float* out, cudaStream_t s);

// Fused warp + composite + residual + adjoint.  mode_loss: residual from images (full-res
// images at level img_level, averaged on the fly) else from grad_out.  mask != NULL:
// compact gradient [k][H][W][4]; else dense [D][H][W][4].  partials: one float per block
// (loss mode); returns the number of blocks through *nblocks.
rl_status rl_launch_grad(const void* M, rl_dtype dt, int D, int H, int W, const RLViews& views, bool mode_loss,
                         const float* images, int img_level, const float* grad_out, const uint64_t* mask, float* G,
                         float inv_n, float* partials, int* nblocks, cudaStream_t s);
size_t rl_grad_num_blocks(int H, int W, int N);
rl_status rl_launch_loss_reduce(const float* partials, int n, float scale, float* out, cudaStream_t s);

// Level-l downsample of the full MPI (optional output Ml) fused with top-k selection.
// keys != NULL selects from keys [D][H][W] instead (M, level, Ml ignored).
rl_status rl_launch_select(const void* M, rl_dtype dt, const float* keys, int D, int Hf, int Wf, int level,
                           void* Ml, int k, uint8_t* S, uint64_t* mask, float* Gzero, cudaStream_t s);
rl_status rl_launch_downsample_f32(const float* x, int P, int H, int W, int C, int level, float* y,
                                   cudaStream_t s);
rl_status rl_launch_update(void* M, rl_dtype dt, int D, int H, int W, int level, const uint8_t* S, const float* G,
                           int k, float lambda, int clamp01, cudaStream_t s);
