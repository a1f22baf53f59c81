// tma_host.cu -- host-side TMA descriptors of the learned update's activations, the device
// status word and the kernel-path switch.
#include <atomic>
#include <mutex>

#include <cudaTypedefs.h>

#include "rl_internal.h"
#include "rl_tma.cuh"

// Set by kernels (atomicOr) when a bounded wait gives up; read by reallife_device_status.
__device__ unsigned int g_rl_status_word;

namespace {
std::atomic<int> g_path{0};
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
std::mutex g_status_mu;
unsigned int* g_status_ptr[256] = {};

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return g_encode;
}
}  // namespace

int rl_kernel_path(int H, int W, int nviews) {
    const int p = g_path.load(std::memory_order_relaxed);
    if (p >= 3) return 3;  // plane-parallel; the group count is read in pp.cu
    if (p != 0) return p;
    return (long long)H * W * nviews < (1ll << 19) ? 3 : 2;
}

unsigned int* rl_device_status_ptr() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_rl_status_word) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_status_ptr[dev] = static_cast<unsigned int*>(p);
    }
    return g_status_ptr[dev];
}

bool rl_encode_act_tmap(CUtensorMap* map, const void* act, int K, int H, int W, int halo) {
    if (((uintptr_t)act & 15) != 0 || K < 1 || H < 1 || W < 1 || halo < 1 || halo > 256) return false;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn) return false;
    // [z][y][x][32] BF16, innermost first: channel, x, y, z; 64-byte rows swizzled in 512-byte atoms
    const cuuint64_t dims[4] = {32, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)K};
    const cuuint64_t row = 64;  // bytes of one voxel
    const cuuint64_t strides[3] = {row, row * W, row * W * H};
    const cuuint32_t box[4] = {32, (cuuint32_t)halo, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(act), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int rl_kernel_path_setting() { return g_path.load(std::memory_order_relaxed); }

extern "C" rl_status reallife_set_kernel_path(int path) {
    if (path < 0 || path == 1 || path > 5) return rl_fail(RL_EINVAL, "kernel path must be 0 or 2 to 5");
    g_path.store(path);
    return RL_OK;
}

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread waits on a shared-memory barrier that nothing completes, for at most limit_ns
// of the global timer, then reports the timeout through the status word and returns: the
// same bounded-wait path every waiting kernel takes.
__global__ void k_selftest_wait(unsigned long long limit_ns, unsigned int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    rltma::mbar_init(&bar, 1);
    rltma::fence_mbar_init();
    const unsigned long long t0 = global_ns();
    while (!rltma::mbar_try_wait(&bar, 0u)) {
        if (global_ns() - t0 > limit_ns) {
            atomicOr(status, RL_DEVFLAG_TIMEOUT);
            return;
        }
    }
}

}  // namespace

extern "C" rl_status reallife_selftest_wait_timeout(unsigned int wait_us, cudaStream_t stream) {
    if (wait_us < 1 || wait_us > 1000000u) return rl_fail(RL_EINVAL, "selftest: wait_us=%u outside [1, 1e6]", wait_us);
    unsigned int* status = rl_device_status_ptr();
    if (!status) return rl_fail(RL_ECUDA, "device status word unavailable");
    k_selftest_wait<<<1, 32, 0, stream>>>((unsigned long long)wait_us * 1000ull, status);
    return rl_check_launch("selftest_wait");
}

// Debug words of the translation units that carry bounds checks (zero in the release build).
unsigned int rl_dbg_read_grad(int clear);
unsigned int rl_dbg_read_pp(int clear);
unsigned int rl_dbg_read_render(int clear);
unsigned int rl_dbg_read_select(int clear);
unsigned int rl_dbg_read_update(int clear);
unsigned int rl_dbg_read_volume(int clear);
RL_DEBUG_READER(status)

#ifdef RL_DEBUG
namespace {
__device__ unsigned int g_rl_selftest_buf[32];

// Threads 0 .. 32 each store to element i of a 32-element buffer, each behind the bounds check:
// thread 32 fails it, sets the bounds bit and stores nothing.
__global__ void k_selftest_bounds() {
    const unsigned i = threadIdx.x;
    if (i <= 32u && RL_IN(i, 32u)) g_rl_selftest_buf[i] = i;
}
}  // namespace
#endif

extern "C" rl_status reallife_selftest_bounds(cudaStream_t stream) {
#ifdef RL_DEBUG
    k_selftest_bounds<<<1, 64, 0, stream>>>();
    return rl_check_launch("selftest_bounds");
#else
    (void)stream;
    return rl_fail(RL_ENOTIMPL, "bounds checks are compiled into the debug build only");
#endif
}

extern "C" int reallife_debug_build(void) {
#ifdef RL_DEBUG
    return 1;
#else
    return 0;
#endif
}

extern "C" rl_status reallife_device_status(int clear, unsigned int* flags_out) {
    unsigned int* p = rl_device_status_ptr();
    if (!p) return rl_fail(RL_ECUDA, "device status word unavailable");
    cudaError_t e = cudaDeviceSynchronize();
    unsigned int v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && clear) e = cudaMemset(p, 0, sizeof(v));
    if (e != cudaSuccess) return rl_fail(RL_ECUDA, "device status: %s", cudaGetErrorString(e));
    v |= rl_dbg_read_grad(clear) | rl_dbg_read_pp(clear) | rl_dbg_read_render(clear) | rl_dbg_read_select(clear) |
         rl_dbg_read_update(clear) | rl_dbg_read_volume(clear) | rl_dbg_read_status(clear);
    if (flags_out) *flags_out = v;
    if (v & RL_DEVFLAG_TIMEOUT) return rl_fail(RL_ETIMEOUT, "a device-side wait timed out (flags 0x%x)", v);
    if (v & RL_DEVFLAG_BOUNDS) return rl_fail(RL_EBOUNDS, "a bounds check of the debug build failed (flags 0x%x)", v);
    return RL_OK;
}
