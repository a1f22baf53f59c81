// rl_common.cuh -- device-side building blocks shared by the RealLiFe kernels (sm_103a).
//
// Warp geometry.  For a view camera v and the reference camera r, let R_rel = R_v R_r^T and
// C the view's centre in the reference frame.  The ray of view pixel q = (u, v) has
// reference-frame direction dir = R_rel^T K_v^{-1} (u, v, 1); it meets the fronto-parallel
// plane z = 1/rho at the reference pixel
//     p = q + a(q) + rho * b(q),
//     a_x = (cx_r - cx_v) + (fx_r - fx_v) m_x + fx_r (dir_x/dir_z - m_x),
//     b_x = fx_r (C_x - C_z dir_x/dir_z),         (same for y)
// with m = K_v^{-1} q.  This is the inverse of the plane-induced homography of Eq. (eq_homo)
// written per pixel: exact, linear in inverse depth, and evaluated as small offsets from q
// so that FP32 keeps ~1e-6 px of accuracy at 2k-pixel coordinates.  The plane is met in
// front of the view iff dir_z > 0 and 1 - rho C_z > 0.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define RL_DEV_MAX_PLANES 64
#define RL_DEV_MAX_VIEWS 16

// Bounds checks of the debug build (-DRL_DEBUG, built by build.py as libreallife_debug.so):
// the hot kernels check the computed index of each global access against its buffer before
// the access; a failed check sets RL_DEVFLAG_BOUNDS in the translation unit's debug word and
// skips the access, never a trap.  reallife_device_status reports the words of every
// translation unit.  In the release build RL_IN is `true` and costs nothing.
#define RL_DEVFLAG_BOUNDS 4u
#ifdef RL_DEBUG
static __device__ unsigned int rl_dbg_word;  // one per translation unit
__device__ __forceinline__ bool rl_dbg_in(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicOr(&rl_dbg_word, RL_DEVFLAG_BOUNDS);
    return false;
}
#define RL_IN(i, n) rl_dbg_in((long long)(i), (long long)(n))
// Host reader of this translation unit's debug word (defined once per .cu by the macro).
#define RL_DEBUG_READER(name)                                                       \
    unsigned int rl_dbg_read_##name(int clear) {                                    \
        unsigned int v = 0;                                                         \
        if (cudaMemcpyFromSymbol(&v, rl_dbg_word, sizeof(v)) != cudaSuccess) {      \
            cudaGetLastError();                                                     \
            return 0;                                                               \
        }                                                                           \
        if (clear) {                                                                \
            const unsigned int z = 0;                                               \
            if (cudaMemcpyToSymbol(rl_dbg_word, &z, sizeof(z)) != cudaSuccess) cudaGetLastError(); \
        }                                                                           \
        return v;                                                                   \
    }
#else
#define RL_IN(i, n) true
#define RL_DEBUG_READER(name) \
    unsigned int rl_dbg_read_##name(int) { return 0; }
#endif

struct RLViewParam {
    float E[9];          // R_rel^T - I (row-major)
    float C[3];          // view centre in the reference frame
    float inv_fxv, inv_fyv, cxv, cyv;
    float fxr, fyr;      // reference focal lengths
    float dcx, dcy;      // cx_r - cx_v, cy_r - cy_v
    float dfx, dfy;      // fx_r - fx_v, fy_r - fy_v
};

// The same parameters in FP64, for the per-block anchors below.
struct RLViewParam64 {
    double E[9], C[3];
    double inv_fxv, inv_fyv, cxv, cyv, fxr, fyr, dcx, dcy, dfx, dfy;
};

// Views and plane inverse depths of one launch, passed by value as a kernel parameter.
struct RLViews {
    int n;
    int anchored;  // 1: the kernels take the anchored coordinates below (offsets beyond ~128 px)
    float rho[RL_DEV_MAX_PLANES];
    RLViewParam v[RL_DEV_MAX_VIEWS];
    double rho64[RL_DEV_MAX_PLANES];
    RLViewParam64 v64[RL_DEV_MAX_VIEWS];
    int gplanes;  // planes of the gradient buffer a launch scatters into (0: D); debug-build bounds checks
};

// ------------------------------------------------------------------ batch work tables
//
// A batch table serves one HSGD iteration of many requests in one launch per stage
// (selection, gradient, update).  It is a header followed by one item per request, in device
// memory; the persistent batched kernels take fixed grids and walk the work units of all items
// (a unit is one block's worth of work of one item), so one captured launch serves any table.

#define RL_DEVFLAG_BATCH 2u  // a batched kernel was given a table of another storage type

struct RLBatchHeader {
    unsigned n;                                // items
    unsigned dtype;                            // rl_dtype of every item's MPI
    unsigned sel_units, grad_units, upd_units;  // work units of the stages (gradient: gather family)
    unsigned pp_units;                         // gradient units of the plane-parallel family
    unsigned int* status;                      // device status word
    unsigned max_gather_D;                     // largest D among the gather family's items
    unsigned next[4];                          // next unit of each launch (0 in the copied table)
    unsigned pad1[3];
};

// The next work unit of a persistent batched launch for the calling block: taken from the
// launch's counter in the table header, so that blocks finishing early take more units.
// Every thread of the block calls it; `slot` is block-shared scratch.
__device__ __forceinline__ unsigned rl_batch_next(const RLBatchHeader* hdr, int which, unsigned* slot) {
    __syncthreads();  // the previous unit's readers of *slot are done
    if (threadIdx.x == 0 && threadIdx.y == 0)
        *slot = atomicAdd(const_cast<unsigned*>(&hdr->next[which]), 1u);
    __syncthreads();
    return *slot;
}

struct RLBatchItem {
    void* M;                 // full-resolution MPI [D][H][W][4], refined in place
    void* Ml;                // level-l MPI (M itself at level 0)
    const float* images;     // full-resolution source images [N][H][W][3]
    uint8_t* S;              // selection [k][h][w]
    uint8_t* slots;          // slot map [D][h][w]
    float* G;                // compact gradient [k][h][w][4]
    float* partials;         // loss partials, one per gradient unit
    unsigned* counter;       // last-block counter of the loss epilogue
    float* loss_out;         // device [1] or NULL
    float* Il;               // level-l source images [N][h][w][3] (levels >= 1; written by the selection)
    int D, H, W, level, k, mode, clamp01, N;
    float lambda, prior_scale, inv_n, loss_scale;
    unsigned sel_begin, sel_units;    // first unit and unit count of each stage
    unsigned grad_begin, grad_units, grad_tiles_x;   // gather family (units 0 for the other items)
    unsigned pp_begin, pp_units, pp_tiles_x;         // plane-parallel family (units 0 for the others)
    unsigned upd_begin, upd_units, upd_tiles_x, pad;
    RLViews views;           // level-l warp parameters of the N views and the plane inverse depths
};

__host__ __device__ inline const RLBatchItem* rl_batch_items(const void* table) {
    return reinterpret_cast<const RLBatchItem*>(static_cast<const char*>(table) + sizeof(RLBatchHeader));
}

// Item owning work unit u of a stage whose first units are items[i].*begin (ascending).
__device__ __forceinline__ unsigned rl_batch_find(const RLBatchItem* __restrict__ items, unsigned n, unsigned u,
                                                  unsigned RLBatchItem::*begin) {
    unsigned lo = 0, hi = n - 1;
    while (lo < hi) {
        const unsigned mid = (lo + hi + 1) >> 1;
        if (items[mid].*begin <= u) lo = mid;
        else hi = mid - 1;
    }
    return RL_IN(lo, n) ? lo : 0;
}

// Per-pixel warp coefficients of one view.
struct RLWarp {
    float ax, ay, bx, by, cz;
    bool dir_ok;
};

__device__ __forceinline__ RLWarp rl_warp_coeffs(const RLViewParam& P, float u, float v) {
    RLWarp w;
    float mx = (u - P.cxv) * P.inv_fxv;
    float my = (v - P.cyv) * P.inv_fyv;
    float ex = fmaf(P.E[0], mx, fmaf(P.E[1], my, P.E[2]));
    float ey = fmaf(P.E[3], mx, fmaf(P.E[4], my, P.E[5]));
    float ez = fmaf(P.E[6], mx, fmaf(P.E[7], my, P.E[8]));
    float dz = 1.0f + ez;
    float inv_dz = 1.0f / dz;
    // r - m = (e - m e_z) / dir_z : small, computed without cancellation
    float rmx = fmaf(-mx, ez, ex) * inv_dz;
    float rmy = fmaf(-my, ez, ey) * inv_dz;
    float rx = mx + rmx, ry = my + rmy;
    w.ax = P.dcx + fmaf(P.dfx, mx, P.fxr * rmx);
    w.ay = P.dcy + fmaf(P.dfy, my, P.fyr * rmy);
    w.bx = P.fxr * fmaf(-P.C[2], rx, P.C[0]);
    w.by = P.fyr * fmaf(-P.C[2], ry, P.C[1]);
    w.cz = P.C[2];
    w.dir_ok = dz > 0.0f;
    return w;
}

// Bilinear footprint of one sample: top-left tap (x0, y0) and fractional offsets.
struct RLTaps {
    int x0, y0;
    float fx, fy;
    bool ok;  // plane met in front of the view
};

__device__ __forceinline__ RLTaps rl_taps(const RLWarp& w, float rho, int qx, int qy) {
    RLTaps t;
    float dx = fmaf(rho, w.bx, w.ax);
    float dy = fmaf(rho, w.by, w.ay);
    float flx = floorf(dx), fly = floorf(dy);
    t.fx = dx - flx;  // exact
    t.fy = dy - fly;
    t.x0 = qx + (int)flx;
    t.y0 = qy + (int)fly;
    t.ok = w.dir_ok && (fmaf(-rho, w.cz, 1.0f) > 0.0f) && fabsf(dx) < 1.0e7f && fabsf(dy) < 1.0e7f;
    return t;
}

// ------------------------------------------------------------------ anchored warp coordinates
//
// The offset p - q = a(q) + rho_d b(q) reaches hundreds of pixels for wide baselines and
// rotated views (|a|, |b| up to ~400 px at 1920 x 1080), where FP32 spacing is ~3e-5 px.  So
// each block evaluates the warp once at an anchor pixel q_c in FP64 and keeps, for every
// plane, the offset at the anchor split into an integer and an FP32 fraction; a pixel of the
// block adds the small FP32 differences a(q) - a(q_c) and b(q) - b(q_c), formed without
// cancellation (exact algebra, small terms only):
//   dm = K_v^{-1} (q - q_c),  de = (R_rel^T - I) dm,
//   dN = de_xy - m_c de_z - dm (e_zc + de_z),   N = e_xy - m e_z,  Dn = 1 + e_z,
//   r_m(q) - r_m(q_c) = (dN Dc - N_c de_z) / (Dn Dc),
//   a(q) - a(q_c) = (f_r - f_v) dm + f_r (r_m(q) - r_m(q_c)),
//   b(q) - b(q_c) = -f_r C_z (dm + r_m(q) - r_m(q_c)).
// The sample position's error stays near 1e-7 px at any image size.  The plane is met in
// front of the view iff 1 - rho_d C_z > 0 (per plane) and the pixel's ray points into the
// reference frame's half-space, 1 + e_z > 0; the host rejects views whose rays at the image
// corners run nearly parallel to the planes, so the anchors are always valid.
//
// The per-pixel FP32 coefficients of rl_warp_coeffs carry an error near 1.2e-7 times the
// offset (measured against the FP64 ray/plane intersection): ~1e-5 px at 100 px.  The host
// therefore takes the anchored path only for launches whose offsets exceed 128 px anywhere
// (RLViews::anchored), where the per-block FP64 set-up pays for itself in accuracy; the
// kernels are compiled for both paths.

struct RLPlaneK {
    float fx, fy;  // fraction of the anchor's offset on plane d
    int ix, iy;    // integer part (plane not met in front of the view: ix = RL_PLANE_NONE)
};
#define RL_PLANE_NONE (-0x40000000)

struct RLAnchor {
    float mx, my, ez, Nx, Ny, Dc;  // anchor quantities (FP32) for the per-pixel differences
    int u, v;                      // anchor pixel
    RLPlaneK k[RL_DEV_MAX_PLANES];
};

// Fills A (shared memory) for view `view` of V at anchor pixel (u, v).  Every thread of the
// block calls it (it synchronises the block twice); nthreads threads, index tid.
__device__ __forceinline__ void rl_anchor_build(RLAnchor* A, const RLViews& V, int view, int u, int v, int D,
                                                int tid, int nthreads) {
    __shared__ double s_ab[4];
    const RLViewParam64& P = V.v64[view];
    if (tid == 0) {
        const double mx = ((double)u - P.cxv) * P.inv_fxv, my = ((double)v - P.cyv) * P.inv_fyv;
        const double ex = P.E[0] * mx + P.E[1] * my + P.E[2];
        const double ey = P.E[3] * mx + P.E[4] * my + P.E[5];
        const double ez = P.E[6] * mx + P.E[7] * my + P.E[8];
        const double dz = 1.0 + ez;
        const double Nx = ex - mx * ez, Ny = ey - my * ez;
        // 1 / dz: the FP32 reciprocal refined by two Newton steps in FP64 (relative error far
        // below FP64's 1e-16 after the second), cheaper than an FP64 division on this GPU
        double inv = (double)__frcp_rn((float)dz);
        inv = inv * (2.0 - dz * inv);
        inv = inv * (2.0 - dz * inv);
        const double rmx = Nx * inv, rmy = Ny * inv;
        s_ab[0] = P.dcx + P.dfx * mx + P.fxr * rmx;
        s_ab[1] = P.dcy + P.dfy * my + P.fyr * rmy;
        s_ab[2] = P.fxr * (P.C[0] - P.C[2] * (mx + rmx));
        s_ab[3] = P.fyr * (P.C[1] - P.C[2] * (my + rmy));
        A->mx = (float)mx;
        A->my = (float)my;
        A->ez = (float)ez;
        A->Nx = (float)Nx;
        A->Ny = (float)Ny;
        A->Dc = (float)dz;
        A->u = u;
        A->v = v;
    }
    __syncthreads();
    for (int d = tid; d < D; d += nthreads) {
        const double rho = V.rho64[d];
        const double kx = s_ab[0] + rho * s_ab[2], ky = s_ab[1] + rho * s_ab[3];
        RLPlaneK k;
        if (1.0 - rho * P.C[2] > 0.0 && fabs(kx) < 1e9 && fabs(ky) < 1e9) {
            const double fx = floor(kx), fy = floor(ky);
            k.ix = (int)fx;
            k.iy = (int)fy;
            k.fx = (float)(kx - fx);
            k.fy = (float)(ky - fy);
        } else {
            k.ix = k.iy = RL_PLANE_NONE;
            k.fx = k.fy = 0.f;
        }
        A->k[d] = k;
    }
    __syncthreads();
}

// Per-pixel differences from the anchor.
struct RLAnchorPix {
    float dax, day, dbx, dby;
    bool ok;  // the pixel's ray points into the reference half-space and its offsets are bounded
};

__device__ __forceinline__ RLAnchorPix rl_anchor_pixel(const RLAnchor& A, const RLViewParam& P, int qx, int qy) {
    RLAnchorPix w;
    const float dmx = (float)(qx - A.u) * P.inv_fxv, dmy = (float)(qy - A.v) * P.inv_fyv;
    const float dex = fmaf(P.E[0], dmx, P.E[1] * dmy);
    const float dey = fmaf(P.E[3], dmx, P.E[4] * dmy);
    const float dez = fmaf(P.E[6], dmx, P.E[7] * dmy);
    const float ez = A.ez + dez;
    const float dNx = dex - fmaf(A.mx, dez, dmx * ez);
    const float dNy = dey - fmaf(A.my, dez, dmy * ez);
    const float Dn = A.Dc + dez;
    const float inv = 1.0f / (Dn * A.Dc);
    const float drx = fmaf(dNx, A.Dc, -A.Nx * dez) * inv;
    const float dry = fmaf(dNy, A.Dc, -A.Ny * dez) * inv;
    w.dax = fmaf(P.dfx, dmx, P.fxr * drx);
    w.day = fmaf(P.dfy, dmy, P.fyr * dry);
    w.dbx = -P.fxr * P.C[2] * (dmx + drx);
    w.dby = -P.fyr * P.C[2] * (dmy + dry);
    w.ok = Dn > 0.f && fabsf(w.dax) + fabsf(w.dbx) < 1.0e6f && fabsf(w.day) + fabsf(w.dby) < 1.0e6f;
    return w;
}

// Taps of plane d (inverse depth rho, its FP32 value) at view pixel (qx, qy).
__device__ __forceinline__ RLTaps rl_anchor_taps(const RLAnchor& A, const RLAnchorPix& w, int d, float rho, int qx,
                                                 int qy) {
    const RLPlaneK k = A.k[d];
    RLTaps t;
    const float sx = k.fx + fmaf(rho, w.dbx, w.dax), sy = k.fy + fmaf(rho, w.dby, w.day);
    const float flx = floorf(sx), fly = floorf(sy);
    t.fx = sx - flx;
    t.fy = sy - fly;
    t.x0 = qx + k.ix + (int)flx;
    t.y0 = qy + k.iy + (int)fly;
    t.ok = w.ok && k.ix != RL_PLANE_NONE;
    return t;
}

// Warp state of one view pixel for either coordinate path (ANCH: the block's anchor A).
template <bool ANCH>
struct RLPixWarp;

template <>
struct RLPixWarp<false> {
    RLWarp w;
    __device__ __forceinline__ RLTaps taps(const RLAnchor&, int, float rho, int qx, int qy) const {
        return rl_taps(w, rho, qx, qy);
    }
};

template <>
struct RLPixWarp<true> {
    RLAnchorPix w;
    __device__ __forceinline__ RLTaps taps(const RLAnchor& A, int d, float rho, int qx, int qy) const {
        return rl_anchor_taps(A, w, d, rho, qx, qy);
    }
};

template <bool ANCH>
__device__ __forceinline__ RLPixWarp<ANCH> rl_pix_warp(const RLAnchor& A, const RLViewParam& P, int qx, int qy) {
    RLPixWarp<ANCH> r;
    if constexpr (ANCH)
        r.w = rl_anchor_pixel(A, P, qx, qy);
    else
        r.w = rl_warp_coeffs(P, (float)qx, (float)qy);
    return r;
}

// Inverse warp (reference -> view, the direction of Eq. eq_homo's H^{-1}).  The reference
// pixel (u, v) on the plane of inverse depth rho has reference-frame direction
// m = K_r^{-1}(u, v, 1); in the view camera it lies along R_rel m + rho t_rel, with
// R_rel = R_v R_r^T and t_rel = t_v - R_rel t_r.  Writing R_rel = I + F and e = F m:
//     x = u + (cx_v - cx_r) + (fx_v - fx_r) m_x + fx_v (e_x - m_x e_z + rho (t_x - m_x t_z)) / Z,
//     Z = 1 + e_z + rho t_z,                                            (same for y)
// and the point is in front of the view iff Z > 0.  As for the forward warp, the offset
// from u is formed from small terms only.
struct RLInvParam {
    float F[9];          // R_rel - I (row-major)
    float t[3];          // t_rel
    float inv_fxr, inv_fyr, cxr, cyr;
    float fxv, fyv;
    float dcx, dcy;      // cx_v - cx_r, cy_v - cy_r
    float dfx, dfy;      // fx_v - fx_r, fy_v - fy_r
};

// Inverse-warp parameters of one launch (level-l and full-resolution cameras of each view).
struct RLInvViews {
    int n;
    float rho[RL_DEV_MAX_PLANES];
    RLInvParam lv[RL_DEV_MAX_VIEWS];
    RLInvParam full[RL_DEV_MAX_VIEWS];
};

// Per-pixel inverse-warp coefficients: offset = a + f_v (g + rho h) / (z0 + rho tz).
struct RLInvWarp {
    float gx, gy, hx, hy, z0, tz, ax, ay;
};

__device__ __forceinline__ RLInvWarp rl_inv_coeffs(const RLInvParam& P, float u, float v) {
    RLInvWarp c;
    const float mx = (u - P.cxr) * P.inv_fxr;
    const float my = (v - P.cyr) * P.inv_fyr;
    const float ex = fmaf(P.F[0], mx, fmaf(P.F[1], my, P.F[2]));
    const float ey = fmaf(P.F[3], mx, fmaf(P.F[4], my, P.F[5]));
    const float ez = fmaf(P.F[6], mx, fmaf(P.F[7], my, P.F[8]));
    c.gx = fmaf(-mx, ez, ex);
    c.gy = fmaf(-my, ez, ey);
    c.hx = fmaf(-mx, P.t[2], P.t[0]);
    c.hy = fmaf(-my, P.t[2], P.t[1]);
    c.z0 = 1.0f + ez;
    c.tz = P.t[2];
    c.ax = fmaf(P.dfx, mx, P.dcx);
    c.ay = fmaf(P.dfy, my, P.dcy);
    return c;
}

__device__ __forceinline__ RLTaps rl_inv_taps(const RLInvWarp& c, const RLInvParam& P, float rho, int u, int v) {
    RLTaps t;
    const float Z = fmaf(rho, c.tz, c.z0);
    const float inv = 1.0f / Z;
    const float dx = fmaf(P.fxv, fmaf(rho, c.hx, c.gx) * inv, c.ax);
    const float dy = fmaf(P.fyv, fmaf(rho, c.hy, c.gy) * inv, c.ay);
    const float flx = floorf(dx), fly = floorf(dy);
    t.fx = dx - flx;
    t.fy = dy - fly;
    t.x0 = u + (int)flx;
    t.y0 = v + (int)fly;
    t.ok = Z > 0.0f && fabsf(dx) < 1.0e7f && fabsf(dy) < 1.0e7f;
    return t;
}

// ---------------------------------------------------------------- storage types

template <typename T> struct RLStore;

template <> struct RLStore<float> {
    static __device__ __forceinline__ float4 load4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
    static __device__ __forceinline__ float4 load4_nc(const float* p) { return *reinterpret_cast<const float4*>(p); }
    static __device__ __forceinline__ void store4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
    static __device__ __forceinline__ float load1(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float round1(float v) { return v; }
};

template <> struct RLStore<__nv_bfloat16> {
    static __device__ __forceinline__ float4 cvt(uint2 r) {
        float4 o;
        o.x = __uint_as_float(r.x << 16);
        o.y = __uint_as_float(r.x & 0xffff0000u);
        o.z = __uint_as_float(r.y << 16);
        o.w = __uint_as_float(r.y & 0xffff0000u);
        return o;
    }
    static __device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
        return cvt(__ldg(reinterpret_cast<const uint2*>(p)));
    }
    static __device__ __forceinline__ float4 load4_nc(const __nv_bfloat16* p) {
        return cvt(*reinterpret_cast<const uint2*>(p));
    }
    static __device__ __forceinline__ void store4(__nv_bfloat16* p, float4 v) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);  // round to nearest even
        __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
        uint2 r;
        r.x = *reinterpret_cast<uint32_t*>(&lo);
        r.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(p) = r;
    }
    static __device__ __forceinline__ float load1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    // the value a store of v would hold
    static __device__ __forceinline__ float round1(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

// Bilinear sample (zero padding per tap) of plane `plane` (base pointer of [H][W][4]).
template <typename Tm>
__device__ __forceinline__ float4 rl_sample(const Tm* __restrict__ plane, int H, int W, const RLTaps& t) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!t.ok) return acc;
    const float w00 = (1.f - t.fx) * (1.f - t.fy), w10 = t.fx * (1.f - t.fy);
    const float w01 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
    const bool x0in = (unsigned)t.x0 < (unsigned)W, x1in = (unsigned)(t.x0 + 1) < (unsigned)W;
    const bool y0in = (unsigned)t.y0 < (unsigned)H, y1in = (unsigned)(t.y0 + 1) < (unsigned)H;
    const size_t r0 = (size_t)t.y0 * W, r1 = r0 + W, hw = (size_t)H * W;
    if (y0in) {
        if (x0in && RL_IN(r0 + t.x0, hw)) { float4 v = RLStore<Tm>::load4(plane + (r0 + t.x0) * 4); acc.x = fmaf(w00, v.x, acc.x); acc.y = fmaf(w00, v.y, acc.y); acc.z = fmaf(w00, v.z, acc.z); acc.w = fmaf(w00, v.w, acc.w); }
        if (x1in && RL_IN(r0 + t.x0 + 1, hw)) { float4 v = RLStore<Tm>::load4(plane + (r0 + t.x0 + 1) * 4); acc.x = fmaf(w10, v.x, acc.x); acc.y = fmaf(w10, v.y, acc.y); acc.z = fmaf(w10, v.z, acc.z); acc.w = fmaf(w10, v.w, acc.w); }
    }
    if (y1in) {
        if (x0in && RL_IN(r1 + t.x0, hw)) { float4 v = RLStore<Tm>::load4(plane + (r1 + t.x0) * 4); acc.x = fmaf(w01, v.x, acc.x); acc.y = fmaf(w01, v.y, acc.y); acc.z = fmaf(w01, v.z, acc.z); acc.w = fmaf(w01, v.w, acc.w); }
        if (x1in && RL_IN(r1 + t.x0 + 1, hw)) { float4 v = RLStore<Tm>::load4(plane + (r1 + t.x0 + 1) * 4); acc.x = fmaf(w11, v.x, acc.x); acc.y = fmaf(w11, v.y, acc.y); acc.z = fmaf(w11, v.z, acc.z); acc.w = fmaf(w11, v.w, acc.w); }
    }
    return acc;
}

// Same sample as rl_sample; when all four taps are inside the plane (the common case) it
// skips the per-tap checks and addresses the taps with 32-bit offsets (D*H*W*4 < 2^31).
template <typename Tm>
__device__ __forceinline__ float4 rl_sample_fast(const Tm* __restrict__ plane, int H, int W, const RLTaps& t) {
    if (t.ok && (unsigned)t.x0 < (unsigned)(W - 1) && (unsigned)t.y0 < (unsigned)(H - 1) &&
        RL_IN((long long)t.y0 * W + t.x0 + W + 1, (long long)H * W)) {
        const Tm* p = plane + (unsigned)(t.y0 * W + t.x0) * 4u;
        const float4 v00 = RLStore<Tm>::load4(p), v10 = RLStore<Tm>::load4(p + 4);
        const float4 v01 = RLStore<Tm>::load4(p + 4 * W), v11 = RLStore<Tm>::load4(p + 4 * W + 4);
        const float w00 = (1.f - t.fx) * (1.f - t.fy), w10 = t.fx * (1.f - t.fy);
        const float w01 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
        // packed FP32x2 FMAs: each lane of a pair is rounded as a scalar fmaf would round it
        float2 lo = __fmul2_rn(make_float2(w00, w00), make_float2(v00.x, v00.y));
        float2 hi = __fmul2_rn(make_float2(w00, w00), make_float2(v00.z, v00.w));
        lo = __ffma2_rn(make_float2(w10, w10), make_float2(v10.x, v10.y), lo);
        hi = __ffma2_rn(make_float2(w10, w10), make_float2(v10.z, v10.w), hi);
        lo = __ffma2_rn(make_float2(w01, w01), make_float2(v01.x, v01.y), lo);
        hi = __ffma2_rn(make_float2(w01, w01), make_float2(v01.z, v01.w), hi);
        lo = __ffma2_rn(make_float2(w11, w11), make_float2(v11.x, v11.y), lo);
        hi = __ffma2_rn(make_float2(w11, w11), make_float2(v11.z, v11.w), hi);
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    return rl_sample(plane, H, W, t);
}

// Slot-map value of a voxel that the selection did not keep.
#define RL_SLOT_NONE 0xFF

__device__ __forceinline__ float rl_warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Loss epilogue shared by the gradient kernels.  Thread `tid` 0 of every block passes the
// block's partial sum `s`; it is stored at partials[bid].  When out != NULL the last block
// to finish (counted on *counter, which must be 0 at launch and is reset to 0 here) adds
// all nblocks partials in index order -- a fixed order, so the loss is deterministic -- and
// writes out[0] = sum * scale.  `red` is shared scratch of nthreads / 32 floats.
__device__ __forceinline__ void rl_loss_epilogue(float s, float* __restrict__ partials, unsigned bid, unsigned nblocks,
                                                 float* __restrict__ out, unsigned* __restrict__ counter, float scale,
                                                 int tid, int nthreads, float* red) {
    __shared__ int rl_am_last;
    if (tid == 0) {
        if (RL_IN(bid, nblocks)) partials[bid] = s;
        rl_am_last = 0;
        if (out) {
            __threadfence();
            rl_am_last = atomicAdd(counter, 1u) == nblocks - 1;
        }
    }
    __syncthreads();
    if (!rl_am_last) return;
    __threadfence();
    float acc = 0.f;
    for (unsigned i = tid; i < nblocks; i += nthreads) acc += __ldcg(partials + i);
    acc = rl_warp_sum(acc);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        float total = 0.f;
        for (int wi = 0; wi < nthreads / 32; ++wi) total += red[wi];
        out[0] = total * scale;
        *counter = 0u;
    }
}
