// lgd.cu -- the learned update of Sec. 3.3 ("Sparse Gradient Update"): the network N_w over
// the sparsified volume V_s [C][k][h][w] -- five blocks of 3x3x3 convolution (inference batch
// norm folded into weights and bias) with ReLU, then a 1x1x1 convolution to the 4-channel
// (R, G, B, alpha) residual -- as implicit GEMMs on the tcgen05 tensor cores, and the learned
// HSGD iteration M <- clamp(M + R(N_w(V_s), S)).
//
// Activations: BF16, channels-last act[z][y][x][32] (64 bytes a voxel).  One TMA tile copy of
// box {32 channels, 144 voxels} at (0, x0 - 8, y, z) with 64-byte swizzling lands in shared
// memory as the K-major SWIZZLE_64B operand layout of tcgen05.mma (a row of 64 bytes per voxel,
// 16-byte chunks permuted within 512-byte atoms; 8-row groups 512 bytes apart).  The copy
// engine zero-fills voxels, lines and planes outside the volume: the convolution's zero
// padding.  The taps dx = -1, 0, +1 read the same halo from rows 7, 8 and 9 on, and the two
// 16-channel K steps from byte 0 and 32 of each row (the descriptor's start address moved).
// Output: lines of 128 consecutive voxels of one (z, y) x 32 channels, accumulated in FP32 in
// tensor memory.  Persistent CTAs (one per SM) each take a contiguous run of output lines in
// (z, x-tile, y) order and walk it along y.  Every input row (the halos of planes z-1, z, z+1
// at one y) is copied once into a ring of five staged rows and multiplied once: the weights of
// one (dz, dx) tap pair are stacked over dy as a 96-row B operand, so that one 128x96x16 MMA
// forms the row's products for the three output lines y+1, y, y-1 that read it.  Each staged
// row has its own 96-column accumulator window (four windows taken in turn), initialised by
// its first MMA, so no two MMAs in flight write the same columns; the epilogue adds a line's
// three partial products from three consecutive windows.  A row inside a run is a fixed,
// branch-free sequence of 9 (dz, dx) x 2 K steps = 18 MMAs with constant descriptor offsets
// (a single issuing thread keeps the tensor core fed only with such a lean sequence); the two
// rows at each end of a run take their taps one by one.  Warp-specialised: warp 0 issues the
// TMA copies, warp 1 the MMAs (one lane), warps 2-5 drain the windows and finish completed
// lines: bias, ReLU, BF16 rounding and the store of the next layer's activations; after the
// last block they also apply the 1x1x1 layer and store the FP32 residual [z][y][x][4].
//
// All five blocks run in one cooperative launch over the same CTAs.  Tensor memory, barriers
// and the 1x1x1 layer are set up once, and the barriers' phases carry from block to block.
// Between blocks each CTA waits for its own MMAs, starts copying the next block's weights, and
// then meets the others at a grid-wide barrier (a counter in the workspace, bounded wait).
// Past the barrier a proxy fence orders the other CTAs' stored activations before this CTA's
// tensor copies of them.
//
// Every mbarrier wait is bounded; a wait that gives up sets RL_DEVFLAG_TIMEOUT, the roles
// stop, the producer waits (bounded) for its copies in flight and the MMA lane for its MMAs,
// and tensor memory is freed before the CTA exits.
#include "rl_internal.h"
#include "rl_tma.cuh"

namespace {

using namespace rltma;

constexpr int kF = 32;                           // channels of every block
constexpr int kTileM = 128;                      // voxels per output tile
constexpr int kHalo = kTileM + 16;               // 144 rows: x0 - 8 .. x0 + 135
constexpr int kRowBytes = kF * 2;                // 64: one voxel's channels
constexpr int kStageBytes = kHalo * kRowBytes;   // 9216: one halo (one input line of one plane)
constexpr int kSlotBytes = 3 * kStageBytes;      // one input row y of the three planes z-1, z, z+1
constexpr int kRowSlots = 5;                     // ring of staged input rows
constexpr int kGroupRows = 3 * kF;               // the dy-stacked weights of one (dz, dx)
constexpr int kGroupBytes = kGroupRows * kRowBytes;  // [96][32] BF16, 64-byte swizzled
constexpr int kWBytes = 9 * kGroupBytes;         // 55296
constexpr int kThreads = 192;
constexpr int kBlocks = 5;                       // 3x3x3 blocks of the network
constexpr int kSets = 4;                         // accumulator windows, taken by staged rows in turn
constexpr uint32_t kSetCols = 128;               // one window: tap dy in columns 32 dy .. 32 dy + 31
constexpr uint32_t kTmemCols = kSets * kSetCols;  // 512: all of it (one CTA per SM)
// instruction descriptor: D FP32, A and B BF16, both K-major, M = 128; N in bits 17-22
constexpr uint32_t kIdescBase = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileM >> 4) << 24);
static_assert((kIdescBase | (4u << 17)) == 0x08080490u, "instruction descriptor (N = 32)");

// Packed network: per block [9 (dz, dx)][3 dy x 32 out][32 in] BF16 in the 64-byte swizzled
// K-major layout, then biases, then the 1x1x1 layer.
constexpr size_t kNetW = 0;
constexpr size_t kNetBias = 5 * (size_t)kWBytes;              // 5 x 32 FP32
constexpr size_t kNetOutW = kNetBias + 5 * kF * 4;            // 4 x 32 FP32
constexpr size_t kNetOutB = kNetOutW + 4 * kF * 4;            // 4 FP32
constexpr size_t kNetBytes = (kNetOutB + 16 + 255) & ~(size_t)255;

struct SmemLayout {
    static constexpr int W = 0;
    static constexpr int A = W + kWBytes;
    static constexpr int BAR = A + kRowSlots * kSlotBytes;
    static constexpr int NBAR = 2 * kRowSlots + kSets + 2;
    static constexpr int TSLOT = BAR + NBAR * 8;
    static constexpr int BIAS = TSLOT + 16;
    static constexpr int OUTW = BIAS + kF * 4;
    static constexpr int OUTB = OUTW + 4 * kF * 4;
    static constexpr int TOTAL = OUTB + 16;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major with 64-byte swizzling: start address, 8-row group
// stride 512 bytes, leading offset unused (1), fixed field 0b001, base offset 0 (the swizzle
// follows the absolute address bits, as the TMA writes it), layout type 4 (SWIZZLE_64B).  The
// start address is the low field, so a descriptor of addr + off is this one plus off / 16
// (shared addresses stay below 256 KB: no carry out of the field).
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= 1ull << 46;
    d |= 4ull << 61;
    return d;
}

__device__ __forceinline__ uint32_t idesc_n(int n) { return kIdescBase | ((uint32_t)n >> 3 << 17); }

// Descriptor steps (16-byte units) of tap pair g = (dz, dx) and K step kk: the A operand is the
// halo of plane z + dz - 1 from row 7 + dx on, the B operand the weights of group g.
__device__ __forceinline__ constexpr uint64_t a_step(int g, int kk) {
    return (uint32_t)((g / 3) * kStageBytes + (7 + g % 3) * kRowBytes + kk * 32) >> 4;
}
__device__ __forceinline__ constexpr uint64_t b_step(int g, int kk) {
    return (uint32_t)(g * kGroupBytes + kk * 32) >> 4;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 consecutive FP32 columns: thread t of the warp gets lane (base + t).  The
// registers are valid only after tmem_wait_ld() and tmem_regs_ready() on them: the empty
// statement ties every later use of the registers to a point after the wait.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_regs_ready(uint32_t (&r)[32]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

__device__ __forceinline__ void flag_timeout(unsigned int* status) { atomicOr(status, RL_DEVFLAG_TIMEOUT); }

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The whole network in one cooperative launch: the five 3x3x3 blocks run in turn over the
// same persistent CTAs (block l reads activations l & 1 and writes the other buffer; the
// last block writes the residual), separated by a grid-wide barrier on *grid_bar (zero at
// launch), so that every line of block l is stored before any CTA copies it for block l + 1.
__global__ void __launch_bounds__(kThreads, 1)
k_conv_net(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
           const unsigned char* __restrict__ net, int K, int H, int W, __nv_bfloat16* __restrict__ act0,
           __nv_bfloat16* __restrict__ act1, float* __restrict__ out_res, unsigned int* __restrict__ grid_bar,
           unsigned int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the swizzled operands assume 1024-byte aligned atoms: align the base (1 KB of slack allocated)
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sW = smem + SmemLayout::W;
    unsigned char* sA = smem + SmemLayout::A;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SmemLayout::BAR);
    uint64_t* full = bars;
    uint64_t* empty = bars + kRowSlots;
    // empty[slot] also tells the epilogue that the row's products are in its window: row jr + 5
    // (the slot's next completion) waits for the epilogue to drain row jr + 1, so the epilogue
    // cannot miss a phase
    uint64_t* tdrain = bars + 2 * kRowSlots;  // [kSets]: the epilogue has read the window
    uint64_t* wbar = tdrain + kSets;        // a block's weights have landed (one phase a block)
    uint64_t* mma_done = wbar + 1;          // every MMA of a block has completed (one phase a block)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SmemLayout::TSLOT);
    float* sBias = reinterpret_cast<float*>(smem + SmemLayout::BIAS);
    float* sOutW = reinterpret_cast<float*>(smem + SmemLayout::OUTW);
    float* sOutB = reinterpret_cast<float*>(smem + SmemLayout::OUTB);
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (W + kTileM - 1) / kTileM;
    // this CTA's output lines: [r_begin, r_end) of the (z, x-tile, y) order, the same in every block
    const long long R = (long long)K * tiles_x * H;
    const long long r_begin = R * blockIdx.x / gridDim.x, r_end = R * (blockIdx.x + 1) / gridDim.x;
    const float* bias_g = reinterpret_cast<const float*>(net + kNetBias);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kRowSlots; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < kSets; ++b) {
            mbar_init(&tdrain[b], 4);
        }
        mbar_init(wbar, 1);
        mbar_init(mma_done, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    if (threadIdx.x < kF) sBias[threadIdx.x] = bias_g[threadIdx.x];
    if (threadIdx.x < 4 * kF) sOutW[threadIdx.x] = reinterpret_cast<const float*>(net + kNetOutW)[threadIdx.x];
    if (threadIdx.x < 4) sOutB[threadIdx.x] = reinterpret_cast<const float*>(net + kNetOutB)[threadIdx.x];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (threadIdx.x == 0) {  // block 0's weights
        mbar_expect_tx(wbar, kWBytes);
        bulk_load(sW, net + kNetW, kWBytes, wbar);
    }

    // role state carried from block to block: staged rows and ring slots keep counting, so
    // every barrier's phases stay in step across the blocks
    int p_irow = 0;                      // producer: input rows staged
    int m_jr = 0, m_slot = 0;            // MMA lane: staged rows, ring slot of the next row
    uint32_t m_slot_phase = 0;
    int e_irow = 0;                      // epilogue: staged rows drained
    float sn[32], sm[32];                // epilogue: running sums of the two open lines
#pragma unroll
    for (int c = 0; c < kF; ++c) sn[c] = sm[c] = 0.f;

    for (int layer = 0; layer < kBlocks; ++layer) {
        const CUtensorMap* in_map = (layer & 1) ? &map1 : &map0;
        __nv_bfloat16* out_act = (layer & 1) ? act0 : act1;
        const bool last_block = layer == kBlocks - 1;
        if (warp == 0 && lane == 0) {
            // ------------------------------------------------------------- producer
            int& irow = p_irow;
            bool ok = true;
            for (long long seg = r_begin; seg < r_end && ok;) {
                const long long col = seg / H;
                const int y0 = (int)(seg % H);
                const long long seg_end = min(r_end, (col + 1) * H);
                const int n = (int)(seg_end - seg);
                const int tx = (int)(col % tiles_x), z = (int)(col / tiles_x);
                for (int r = y0 - 1; r <= y0 + n && ok; ++r, ++irow) {  // input rows of outputs y0 .. y0+n-1
                    const int slot = irow % kRowSlots, round = irow / kRowSlots;
                    if (round > 0 && !mbar_wait(&empty[slot], (uint32_t)((round - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    if (*(volatile int*)&s_abort) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[slot], kSlotBytes);
                    unsigned char* dst = sA + slot * kSlotBytes;
                    for (int dz = 0; dz < 3; ++dz)
                        tma_load_4d(dst + dz * kStageBytes, in_map, &full[slot], 0, tx * kTileM - 8, r, z + dz - 1);
                }
                seg = seg_end;
            }
            if (!ok) {
                flag_timeout(status);
                s_abort = 1;
            }
            // copies in flight: the last row of every slot must have landed before exit; on the
            // normal path also its release by the MMAs (the tensor core's arrival on empty[slot])
            for (int slot = 0; slot < kRowSlots && slot < irow; ++slot) {
                const int last = irow - 1 - ((irow - 1 - slot) % kRowSlots);
                if (!mbar_wait(&full[slot], (uint32_t)((last / kRowSlots) & 1))) flag_timeout(status);
                if (ok && !mbar_wait(&empty[slot], (uint32_t)((last / kRowSlots) & 1))) flag_timeout(status);
            }
            // block 0's weight copy has landed (later blocks' copies are waited for at the boundary)
            if (layer == 0 && !mbar_wait(wbar, 0)) flag_timeout(status);
        } else if (warp == 1 && lane == 0) {
            // ------------------------------------------------------------- MMA issuer
            // Staged row jr (the CTA's count) writes window jr mod kSets, tap dy into columns
            // 32 dy of it: row j of a run adds tap dy in [lo, hi] to output line t0 + j - dy.  Every
            // row initialises what it writes, so no two MMAs in flight share accumulator columns;
            // the epilogue adds a line's three partial products.  The rows inside a run take all
            // three taps in one 128x96x16 MMA per (dz, dx, K step), issued as a branch-free
            // sequence with constant offsets; only the two rows at each end of a run go tap by tap.
            bool ok = mbar_wait(wbar, (uint32_t)(layer & 1));
            const uint32_t abase = smem_u32(sA);
            const uint64_t bdesc0 = umma_desc_sw64(smem_u32(sW));
            int& jr = m_jr;
            int& slot = m_slot;
            uint32_t& slot_phase = m_slot_phase;
            for (long long seg = r_begin; seg < r_end && ok;) {
                const long long col = seg / H;
                const long long seg_end = min(r_end, (col + 1) * H);
                const int n = (int)(seg_end - seg);
                for (int j = 0; j < n + 2; ++j, ++jr) {  // input rows y0 - 1 .. y0 + n
                    const int lo = max(0, j - (n - 1)), hi = min(2, j);
                    const int set = jr & (kSets - 1);
                    // the window was read by the epilogue after row jr - kSets
                    if (jr >= kSets && !mbar_wait(&tdrain[set], (uint32_t)(((jr >> 2) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    if (!mbar_wait(&full[slot], slot_phase) || *(volatile int*)&s_abort) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t win = tmem + (uint32_t)set * kSetCols;
                    const uint64_t adesc0 = umma_desc_sw64(abase + (uint32_t)(slot * kSlotBytes));
                    if (lo == 0 && hi == 2) {
#pragma unroll
                        for (int g = 0; g < 9; ++g)
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                umma_bf16(win, adesc0 + a_step(g, kk), bdesc0 + b_step(g, kk), idesc_n(3 * kF),
                                          (g | kk) != 0 ? 1u : 0u);
                            }
                    } else {
                        for (int dy = lo; dy <= hi; ++dy) {
                            const uint32_t d = win + (uint32_t)(dy * kF);
                            const uint64_t bdy = bdesc0 + (uint64_t)((uint32_t)(dy * kF * kRowBytes) >> 4);
#pragma unroll
                            for (int g = 0; g < 9; ++g)
#pragma unroll
                                for (int kk = 0; kk < 2; ++kk) {
                                    umma_bf16(d, adesc0 + a_step(g, kk), bdy + b_step(g, kk), idesc_n(kF),
                                              (g | kk) != 0 ? 1u : 0u);
                                }
                        }
                    }
                    // the row is read by no later MMA, and its window holds its products
                    umma_commit(&empty[slot]);
                    if (++slot == kRowSlots) {
                        slot = 0;
                        slot_phase ^= 1u;
                    }
                }
                seg = seg_end;
            }
            if (!ok) {
                flag_timeout(status);
                s_abort = 1;
            }
            // every MMA of the block has completed before its weights are replaced or tensor memory
            // is released (on the normal path the epilogue has already seen them all)
            umma_commit(mma_done);
            if (!mbar_wait(mma_done, (uint32_t)(layer & 1))) flag_timeout(status);
        } else if (warp >= 2) {
            // ------------------------------------------------------------- epilogue
            // After staged row j of a run its window holds the tap-0 product of line t0 + j, the
            // tap-1 product of line t0 + j - 1 and the tap-2 product of line t0 + j - 2, which is
            // then complete.  The two open lines' running sums stay in registers (sn: the newest).
            const int q = warp & 3;  // tensor-memory lane quarter this warp may access
            const uint32_t lanes = (uint32_t)(32 * q) << 16;
            int& irow = e_irow;
            bool run = true;
            for (long long seg = r_begin; seg < r_end && run;) {
                const long long col = seg / H;
                const int y0 = (int)(seg % H);
                const long long seg_end = min(r_end, (col + 1) * H);
                const int n = (int)(seg_end - seg);
                const int px = (int)(col % tiles_x), z = (int)(col / tiles_x);
                for (int j = 0; j < n + 2; ++j) {
                    const int jr = irow + j, set = jr % kSets;
                    const int lo = max(0, j - (n - 1)), hi = min(2, j);
                    bool ok = true;
                    if (lane == 0)
                        ok = mbar_wait(&empty[jr % kRowSlots], (uint32_t)((jr / kRowSlots) & 1)) &&
                             !*(volatile int*)&s_abort;
                    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                    if (!ok) {
                        if (lane == 0) {
                            flag_timeout(status);
                            s_abort = 1;
                        }
                        run = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t win = tmem + lanes + (uint32_t)set * kSetCols;
                    uint32_t r0[32], r1[32], r2[32];
                    tmem_ld32_async(win, r0);
                    tmem_ld32_async(win + kF, r1);
                    tmem_ld32_async(win + 2 * kF, r2);
                    tmem_wait_ld();
                    tmem_regs_ready(r0);
                    tmem_regs_ready(r1);
                    tmem_regs_ready(r2);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tdrain[set]);
                    const bool fin = hi == 2;  // line t0 + j - 2 completes
                    float acc[32];
#pragma unroll
                    for (int c = 0; c < kF; ++c) {
                        acc[c] = __uint_as_float(r2[c]) + sm[c];
                        if (lo <= 1 && hi >= 1) sm[c] = sn[c] + __uint_as_float(r1[c]);
                        if (lo == 0) sn[c] = __uint_as_float(r0[c]);
                    }
                    if (!fin) continue;
                    const int y = y0 + j - 2;
                    const int x = px * kTileM + 32 * q + lane;
                    if (x >= W) continue;
#pragma unroll
                    for (int c = 0; c < kF; ++c) acc[c] = fmaxf(acc[c] + sBias[c], 0.f);
                    if (last_block) {
                        float4 r;
                        r.x = sOutB[0]; r.y = sOutB[1]; r.z = sOutB[2]; r.w = sOutB[3];
#pragma unroll
                        for (int c = 0; c < kF; ++c) {
                            r.x = fmaf(sOutW[0 * kF + c], acc[c], r.x);
                            r.y = fmaf(sOutW[1 * kF + c], acc[c], r.y);
                            r.z = fmaf(sOutW[2 * kF + c], acc[c], r.z);
                            r.w = fmaf(sOutW[3 * kF + c], acc[c], r.w);
                        }
                        *reinterpret_cast<float4*>(out_res + (((size_t)z * H + y) * W + x) * 4) = r;
                    } else {
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch) {
                            uint4 pk;
                            __nv_bfloat162 p0 = __floats2bfloat162_rn(acc[ch * 8 + 0], acc[ch * 8 + 1]);
                            __nv_bfloat162 p1 = __floats2bfloat162_rn(acc[ch * 8 + 2], acc[ch * 8 + 3]);
                            __nv_bfloat162 p2 = __floats2bfloat162_rn(acc[ch * 8 + 4], acc[ch * 8 + 5]);
                            __nv_bfloat162 p3 = __floats2bfloat162_rn(acc[ch * 8 + 6], acc[ch * 8 + 7]);
                            pk.x = *reinterpret_cast<uint32_t*>(&p0);
                            pk.y = *reinterpret_cast<uint32_t*>(&p1);
                            pk.z = *reinterpret_cast<uint32_t*>(&p2);
                            pk.w = *reinterpret_cast<uint32_t*>(&p3);
                            *reinterpret_cast<uint4*>(out_act + (((size_t)z * H + y) * W + x) * kF + ch * 8) = pk;
                        }
                    }
                }
                irow += n + 2;
                seg = seg_end;
            }
        }
        __syncwarp();  // the single-lane roles rejoin their warps
        tc_fence_before();
        __syncthreads();
        if (*(volatile int*)&s_abort || last_block) break;
        // block boundary: the MMAs of this block have completed (the MMA lane waited for them),
        // so the weights can be replaced; the epilogue has stored its lines
        if (threadIdx.x == 0) {
            mbar_expect_tx(wbar, kWBytes);
            bulk_load(sW, net + kNetW + (size_t)(layer + 1) * kWBytes, kWBytes, wbar);
            // grid barrier: this CTA's stores are made visible at GPU scope, then it waits until
            // every CTA has arrived (bounded)
            __threadfence();
            atomicAdd(grid_bar, 1u);
            const unsigned target = (unsigned)(layer + 1) * gridDim.x;
            if (ld_acquire_gpu(grid_bar) < target) {
                const long long t0 = clock64();
                while (ld_acquire_gpu(grid_bar) < target) {
                    if (clock64() - t0 > kWaitCycles) {
                        flag_timeout(status);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            // the next block's copies (async proxy) read what the generic stores wrote
            asm volatile("fence.proxy.async.global;" ::: "memory");
            // the weight copy is not left in flight if the CTA stops here
            if (!mbar_wait(wbar, (uint32_t)((layer + 1) & 1))) {
                flag_timeout(status);
                s_abort = 1;
            }
        }
        if (threadIdx.x < kF) sBias[threadIdx.x] = bias_g[(layer + 1) * kF + threadIdx.x];
        __syncthreads();
        if (*(volatile int*)&s_abort) break;
        tc_fence_after();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// V_s [C][K][H][W] FP32 -> act [K][H][W][32] BF16 (round to nearest even); channels >= C zero.
__global__ void k_pack_input(const float* __restrict__ V, int C, int K, int H, int W, __nv_bfloat16* __restrict__ act) {
    const long long n = (long long)K * H * W;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int c = ch * 8 + e;
            v[e] = c < C ? __ldg(V + (size_t)c * n + i) : 0.f;
        }
        uint4 pk;
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
        pk.x = *reinterpret_cast<uint32_t*>(&p0);
        pk.y = *reinterpret_cast<uint32_t*>(&p1);
        pk.z = *reinterpret_cast<uint32_t*>(&p2);
        pk.w = *reinterpret_cast<uint32_t*>(&p3);
        *reinterpret_cast<uint4*>(act + i * kF + ch * 8) = pk;
    }
}

// Batch-norm folding and packing of one block: w [32][cin][3][3][3] FP32 ->
// [9 (dz, dx)][3 dy x 32 out][32 in] BF16, 64-byte swizzled (inputs >= cin zero), and the
// folded bias.
__global__ void k_prepare_block(const float* __restrict__ w, const float* __restrict__ b,
                                const float* __restrict__ gamma, const float* __restrict__ beta,
                                const float* __restrict__ mean, const float* __restrict__ var, float eps, int cin,
                                __nv_bfloat16* __restrict__ wp, float* __restrict__ bias) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 27 * 32 * 32
    if (i < kF) {
        const float s = gamma[i] / sqrtf(var[i] + eps);
        bias[i] = (b[i] - mean[i]) * s + beta[i];
    }
    if (i >= 27 * kF * kF) return;
    const int ci = i % kF, co = (i / kF) % kF, tap = i / (kF * kF);  // tap = (dz * 3 + dy) * 3 + dx
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const float s = gamma[co] / sqrtf(var[co] + eps);
    const float v = ci < cin ? w[((size_t)co * cin + ci) * 27 + tap] * s : 0.f;
    // row n of group (dz, dx) holds output channel co of tap dy; its 16-byte chunk ci / 8 sits at
    // chunk (ci / 8) ^ ((n / 2) % 4): the 64-byte swizzle of a 1024-byte aligned group
    const int n = dy * kF + co;
    const int chunk = (ci / 8) ^ ((n >> 1) & 3);
    wp[((size_t)(dz * 3 + dx) * kGroupRows + n) * kF + chunk * 8 + ci % 8] = __float2bfloat16_rn(v);
}

}  // namespace

size_t rl_lgd_net_bytes() { return kNetBytes; }

rl_status rl_lgd_prepare(const rl_lgd_params* p, void* net, cudaStream_t s) {
    unsigned char* base = (unsigned char*)net;
    for (int l = 0; l < 5; ++l) {
        const int cin = l == 0 ? p->c_in : kF;
        k_prepare_block<<<(27 * kF * kF + 255) / 256, 256, 0, s>>>(
            p->conv_w[l], p->conv_b[l], p->bn_gamma[l], p->bn_beta[l], p->bn_mean[l], p->bn_var[l], p->eps, cin,
            (__nv_bfloat16*)(base + kNetW + (size_t)l * kWBytes), (float*)(base + kNetBias) + l * kF);
    }
    cudaMemcpyAsync(base + kNetOutW, p->out_w, 4 * kF * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(base + kNetOutB, p->out_b, 4 * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return rl_check_launch("lgd_prepare");
}

size_t rl_lgd_act_bytes(int K, int H, int W) { return ((size_t)K * H * W * kF * 2 + 1023) & ~(size_t)1023; }

rl_status rl_lgd_forward(const void* net, const float* V, int C, int K, int H, int W, float* residual, void* act0,
                         void* act1, unsigned* grid_bar, cudaStream_t s) {
    const long long n = (long long)K * H * W;
    {
        RLTraceScope ts("lgd_pack", s);
        k_pack_input<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, C, K, H, W, (__nv_bfloat16*)act0);
    }
    rl_status st = rl_check_launch("lgd_pack");
    if (st) return st;
    return rl_lgd_network(net, K, H, W, residual, act0, act1, grid_bar, s);
}

rl_status rl_lgd_network(const void* net, int K, int H, int W, float* residual, void* act0, void* act1,
                         unsigned* grid_bar, cudaStream_t s) {
    CUtensorMap maps[2];
    if (!rl_encode_act_tmap(&maps[0], act0, K, H, W, kHalo) || !rl_encode_act_tmap(&maps[1], act1, K, H, W, kHalo))
        return rl_fail(RL_ECUDA, "lgd: activation tensor maps could not be encoded");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long lines = (long long)K * H * ((W + kTileM - 1) / kTileM);
    // one CTA per SM at most: every CTA is resident, as the grid barrier between blocks needs
    // (the cooperative launch fails rather than run a grid that cannot be)
    const unsigned grid = (unsigned)std::min<long long>(lines, sms > 0 ? sms : 1);
    const size_t smem = SmemLayout::TOTAL + 1024;
    cudaFuncSetAttribute(k_conv_net, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    unsigned int* status = rl_device_status_ptr();
    if (!status) return rl_fail(RL_ECUDA, "device status word unavailable");
    if (cudaMemsetAsync(grid_bar, 0, sizeof(unsigned), s) != cudaSuccess)
        return rl_fail(RL_ECUDA, "lgd: grid barrier reset failed");
    const unsigned char* netp = (const unsigned char*)net;
    __nv_bfloat16* a0 = (__nv_bfloat16*)act0;
    __nv_bfloat16* a1 = (__nv_bfloat16*)act1;
    void* args[] = {(void*)&maps[0], (void*)&maps[1], (void*)&netp, (void*)&K, (void*)&H, (void*)&W,
                    (void*)&a0, (void*)&a1, (void*)&residual, (void*)&grid_bar, (void*)&status};
    {
        RLTraceScope ts("lgd_conv_net", s);
        const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_conv_net, dim3(grid), dim3(kThreads), args,
                                                          smem, s);
        if (e != cudaSuccess) return rl_fail(RL_ECUDA, "lgd: cooperative launch: %s", cudaGetErrorString(e));
    }
    return rl_check_launch("lgd_conv");
}

// ------------------------------------------------------------------ C ABI

namespace {
struct LgdStepLayout {
    size_t vol, res, S, act0, act1, gbar, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

LgdStepLayout lgd_step_layout(int N, int D, int H, int W, int k, rl_dtype dt) {
    LgdStepLayout L;
    size_t off = 0;
    L.vol = off;
    off += a256(reallife_gradient_volume_workspace_bytes(N, D, H, W, k, dt));
    L.res = off;
    off += a256((size_t)k * H * W * 4 * sizeof(float));
    L.S = off;
    off += a256((size_t)k * H * W);
    L.act0 = off;
    off += rl_lgd_act_bytes(k, H, W);
    L.act1 = off;
    off += rl_lgd_act_bytes(k, H, W);
    L.gbar = off;  // the network's grid-barrier counter
    off += 256;
    L.total = off;
    return L;
}
}  // namespace

extern "C" size_t reallife_lgd_net_bytes(void) { return rl_lgd_net_bytes(); }

extern "C" rl_status reallife_lgd_prepare(const rl_lgd_params* p, void* net, cudaStream_t stream) {
    if (!p || !net || ((uintptr_t)net & 255) != 0) return rl_fail(RL_EINVAL, "lgd_prepare: NULL or misaligned");
    if (p->c_in < 1 || p->c_in > 32) return rl_fail(RL_EINVAL, "lgd_prepare: c_in=%d outside [1,32]", p->c_in);
    if (!(p->eps >= 0.f)) return rl_fail(RL_EINVAL, "lgd_prepare: eps must be >= 0");
    for (int l = 0; l < 5; ++l)
        if (!p->conv_w[l] || !p->conv_b[l] || !p->bn_gamma[l] || !p->bn_beta[l] || !p->bn_mean[l] || !p->bn_var[l])
            return rl_fail(RL_EINVAL, "lgd_prepare: block %d has a NULL parameter", l);
    if (!p->out_w || !p->out_b) return rl_fail(RL_EINVAL, "lgd_prepare: NULL output layer");
    return rl_lgd_prepare(p, net, stream);
}

extern "C" size_t reallife_lgd_workspace_bytes(int k, int h, int w) {
    if (k < 1 || h < 1 || w < 1) return 0;
    return 2 * rl_lgd_act_bytes(k, h, w) + 256;  // two activation buffers, the grid-barrier counter
}

extern "C" rl_status reallife_lgd_forward(const void* net, const float* V, int C, int k, int h, int w,
                                          float* residual, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!net || ((uintptr_t)net & 255) != 0 || !V || !residual || ((uintptr_t)residual & 15) != 0 || !ws ||
        ((uintptr_t)ws & 255) != 0)
        return rl_fail(RL_EINVAL, "lgd_forward: NULL or misaligned pointer");
    if (C < 1 || C > 32 || k < 1 || h < 1 || w < 1 || (long long)k * h * w >= (1ll << 31))
        return rl_fail(RL_EINVAL, "lgd_forward: C=%d (<= 32), k=%d, h=%d, w=%d", C, k, h, w);
    const size_t need = reallife_lgd_workspace_bytes(k, h, w);
    if (ws_bytes < need) return rl_fail(RL_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    char* b = (char*)ws;
    const size_t act = rl_lgd_act_bytes(k, h, w);
    return rl_lgd_forward(net, V, C, k, h, w, residual, b, b + act, (unsigned*)(b + 2 * act), stream);
}

extern "C" size_t reallife_lgd_step_workspace_bytes(int N, int D, int H, int W, int k, rl_dtype dtype) {
    if (N < 1 || D < 1 || H < 1 || W < 1 || k < 1) return 0;
    return lgd_step_layout(N, D, H, W, k, dtype).total;
}

extern "C" rl_status reallife_lgd_step(rl_mpi* m, const float* images, const rl_camera* src, int N, int k, int level,
                                       int selection, int clamp01, const void* net, uint8_t* S_out, void* ws,
                                       size_t ws_bytes, cudaStream_t stream) {
    if (N < 1 || 4 * N + 4 > 32) return rl_fail(RL_EINVAL, "lgd_step: N=%d views give more than 32 channels", N);
    if (!net || ((uintptr_t)net & 255) != 0) return rl_fail(RL_EINVAL, "lgd_step: net NULL or misaligned");
    if (!m || !ws || ((uintptr_t)ws & 255) != 0) return rl_fail(RL_EINVAL, "lgd_step: NULL or misaligned");
    if (m->D < 1 || m->H < 1 || m->W < 1) return rl_fail(RL_EINVAL, "lgd_step: bad MPI shape");
    const LgdStepLayout L = lgd_step_layout(N, m->D, m->H, m->W, k, m->dtype);
    if (ws_bytes < L.total) return rl_fail(RL_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
    char* b = (char*)ws;
    uint8_t* S = S_out ? S_out : (uint8_t*)(b + L.S);
    float* res = (float*)(b + L.res);
    // V_s and S (validates the MPI, views, k, level and selection), written as the network's
    // BF16 channels-last input
    rl_status st = rl_gradient_volume(m, images, src, N, k, level, selection, S, nullptr, b + L.act0, b + L.vol,
                                      L.res - L.vol, stream);
    if (st) return st;
    const int h = m->H >> level, w = m->W >> level;
    st = rl_lgd_network(net, k, h, w, res, b + L.act0, b + L.act1, (unsigned*)(b + L.gbar), stream);
    if (st) return st;
    // M <- M + R(residual, S): the masked update with step -1 (and the level's upsampling)
    return rl_launch_update(m->data, m->dtype, m->D, m->H, m->W, level, S, res, k, -1.0f, clamp01, stream);
}
