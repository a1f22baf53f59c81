// reallife_api.cu -- the C ABI of libreallife (include/reallife.h): host-side validation,
// camera geometry in FP64, workspace layout, kernel sequencing and launch tracing.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rl_internal.h"

// ------------------------------------------------------------------ errors

static thread_local char g_err[512] = "";

rl_status rl_fail(rl_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

rl_status rl_check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rl_fail(RL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return RL_OK;
}

extern "C" const char* reallife_strerror(rl_status s) {
    switch (s) {
        case RL_OK: return "ok";
        case RL_EINVAL: return "invalid argument";
        case RL_ENOMEM: return "workspace too small";
        case RL_ECUDA: return "CUDA error";
        case RL_ETIMEOUT: return "device wait timed out";
        case RL_ENOTIMPL: return "not implemented";
        case RL_EBOUNDS: return "bounds check failed";
    }
    return "unknown status";
}

extern "C" const char* reallife_last_error(void) { return g_err; }

// ------------------------------------------------------------------ tracing

namespace {
struct TracePending {
    int name;
    cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_trace_on = false;
std::vector<TracePending> g_pending;   // launches made outside stream capture, read once
std::vector<TracePending> g_captured;  // launches captured into a graph, read after every replay
std::vector<cudaEvent_t> g_free_events;
std::vector<std::string> g_names;
std::vector<long long> g_counts;

cudaEvent_t take_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int name_index(const char* name) {
    for (size_t i = 0; i < g_names.size(); ++i)
        if (g_names[i] == name) return (int)i;
    g_names.emplace_back(name);
    g_counts.push_back(0);
    return (int)g_names.size() - 1;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusActive;
}

constexpr int kCapturedTag = 1 << 30;
}  // namespace

int rl_trace_begin(const char* name, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_tmu);
    if (!g_trace_on) return -1;
    TracePending p;
    p.name = name_index(name);
    p.a = take_event();
    p.b = take_event();
    if (capturing(s)) {
        // becomes an event-record node of the graph: it records on every replay
        cudaEventRecordWithFlags(p.a, s, cudaEventRecordExternal);
        g_captured.push_back(p);
        return kCapturedTag | ((int)g_captured.size() - 1);
    }
    g_counts[p.name] += 1;
    cudaEventRecord(p.a, s);
    g_pending.push_back(p);
    return (int)g_pending.size() - 1;
}

void rl_trace_end(int token, cudaStream_t s) {
    if (token < 0) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    if (token & kCapturedTag) {
        const int i = token & ~kCapturedTag;
        if (i < (int)g_captured.size()) cudaEventRecordWithFlags(g_captured[i].b, s, cudaEventRecordExternal);
    } else if (token < (int)g_pending.size()) {
        cudaEventRecord(g_pending[token].b, s);
    }
}

extern "C" rl_status reallife_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_trace_on = on != 0;
    return RL_OK;
}

extern "C" rl_status reallife_trace_read(rl_trace_entry* out, int max, int* n_out) {
    std::lock_guard<std::mutex> lk(g_tmu);
    std::vector<double> ms(g_names.size(), 0.0);
    rl_status st = RL_OK;
    for (const TracePending& p : g_pending) {
        float t = 0.f;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&t, p.a, p.b) != cudaSuccess)
            st = rl_fail(RL_ECUDA, "trace: %s", cudaGetErrorString(cudaGetLastError()));
        ms[p.name] += t;
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
    // captured launches: the events hold the most recent replay's timestamps
    for (const TracePending& p : g_captured) {
        float t = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
            ms[p.name] += t;
            g_counts[p.name] += 1;
        } else {
            cudaGetLastError();  // not replayed yet
        }
    }
    int n = 0;
    for (size_t i = 0; i < g_names.size(); ++i) {
        if (g_counts[i] == 0) continue;
        if (out && n < max) {
            std::memset(out[n].name, 0, sizeof(out[n].name));
            std::strncpy(out[n].name, g_names[i].c_str(), sizeof(out[n].name) - 1);
            out[n].launches = g_counts[i];
            out[n].total_ms = ms[i];
        }
        ++n;
        g_counts[i] = 0;
    }
    if (n_out) *n_out = n;
    return st;
}

extern "C" rl_status reallife_trace_release_captured(void) {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (const TracePending& p : g_captured) {
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_captured.clear();
    return RL_OK;
}

// ------------------------------------------------------------------ geometry

namespace {

bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Zero-skew pinhole with last row (0,0,1), finite pose, R orthonormal to 1e-6.
bool camera_ok(const rl_camera& c) {
    if (!finite_all(c.K, 9) || !finite_all(c.R, 9) || !finite_all(c.t, 3)) return false;
    if (c.K[1] != 0.0 || c.K[3] != 0.0 || c.K[6] != 0.0 || c.K[7] != 0.0 || c.K[8] != 1.0) return false;
    if (!(c.K[0] > 0.0) || !(c.K[4] > 0.0)) return false;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += c.R[a * 3 + j] * c.R[b * 3 + j];
            if (std::fabs(s - (a == b ? 1.0 : 0.0)) > 1e-6) return false;
        }
    return true;
}

rl_camera camera_at_level(const rl_camera& c, int level) {
    rl_camera o = c;
    const double s = std::ldexp(1.0, -level);
    o.K[0] = c.K[0] * s;
    o.K[4] = c.K[4] * s;
    o.K[2] = (c.K[2] + 0.5) * s - 0.5;
    o.K[5] = (c.K[5] + 0.5) * s - 0.5;
    return o;
}

// Relative pose of `view` w.r.t. the reference camera (Eq. eq_homo's R_i R_r^{-1} and
// t_i - R_i R_r^{-1} t_r), reduced to the per-pixel warp parameters of rl_common.cuh, in
// FP64 (the kernels' per-block anchors) and rounded to FP32 (their per-pixel differences).
RLViewParam64 view_param64(const rl_camera& ref, const rl_camera& view) {
    double Rrel[9];  // R_v R_r^T
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += view.R[a * 3 + j] * ref.R[b * 3 + j];
            Rrel[a * 3 + b] = s;
        }
    RLViewParam64 P;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P.E[a * 3 + b] = Rrel[b * 3 + a] - (a == b ? 1.0 : 0.0);
    // centre of the view in the reference frame: -R_rel^T t_v + t_r
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += Rrel[j * 3 + a] * view.t[j];
        P.C[a] = ref.t[a] - s;
    }
    P.inv_fxv = 1.0 / view.K[0];
    P.inv_fyv = 1.0 / view.K[4];
    P.cxv = view.K[2];
    P.cyv = view.K[5];
    P.fxr = ref.K[0];
    P.fyr = ref.K[4];
    P.dcx = ref.K[2] - view.K[2];
    P.dcy = ref.K[5] - view.K[5];
    P.dfx = ref.K[0] - view.K[0];
    P.dfy = ref.K[4] - view.K[4];
    return P;
}

RLViewParam view_param(const RLViewParam64& Q) {
    RLViewParam P;
    for (int j = 0; j < 9; ++j) P.E[j] = (float)Q.E[j];
    for (int j = 0; j < 3; ++j) P.C[j] = (float)Q.C[j];
    P.inv_fxv = (float)Q.inv_fxv;
    P.inv_fyv = (float)Q.inv_fyv;
    P.cxv = (float)Q.cxv;
    P.cyv = (float)Q.cyv;
    P.fxr = (float)Q.fxr;
    P.fyr = (float)Q.fyr;
    P.dcx = (float)Q.dcx;
    P.dcy = (float)Q.dcy;
    P.dfx = (float)Q.dfx;
    P.dfy = (float)Q.dfy;
    return P;
}

// Largest |p - q| = |a(q) + rho b(q)| over the image's corners and centre and the nearest and
// farthest planes (FP64): the offsets are smooth in q and linear in rho.
double max_offset(const RLViewParam64& P, int H, int W, double rho_lo, double rho_hi) {
    double hi = 0.0;
    for (int c = 0; c < 5; ++c) {
        const double u = c == 4 ? 0.5 * W : ((c & 1) ? W - 1.0 : 0.0);
        const double v = c == 4 ? 0.5 * H : ((c & 2) ? H - 1.0 : 0.0);
        const double mx = (u - P.cxv) * P.inv_fxv, my = (v - P.cyv) * P.inv_fyv;
        const double ex = P.E[0] * mx + P.E[1] * my + P.E[2], ey = P.E[3] * mx + P.E[4] * my + P.E[5];
        const double dz = 1.0 + P.E[6] * mx + P.E[7] * my + P.E[8];
        const double rmx = (ex - mx * (dz - 1.0)) / dz, rmy = (ey - my * (dz - 1.0)) / dz;
        const double ax = P.dcx + P.dfx * mx + P.fxr * rmx, ay = P.dcy + P.dfy * my + P.fyr * rmy;
        const double bx = P.fxr * (P.C[0] - P.C[2] * (mx + rmx)), by = P.fyr * (P.C[1] - P.C[2] * (my + rmy));
        for (double r : {rho_lo, rho_hi}) hi = std::max(hi, std::max(std::fabs(ax + r * bx), std::fabs(ay + r * by)));
    }
    return hi;
}

// Offsets beyond which the kernels take the anchored coordinates (rl_common.cuh).
constexpr double kAnchorOffsetPx = 128.0;

// Smallest 1 + e_z (the cosine-like factor of the view's ray direction in the reference
// frame) over the image of W x H pixels and a margin of half a block: it is linear in the
// pixel, so the extremes lie at the corners.
double min_ray_dz(const RLViewParam64& P, int H, int W) {
    double lo = 1e300;
    for (int c = 0; c < 4; ++c) {
        const double u = (c & 1) ? W + 16.0 : -16.0, v = (c & 2) ? H + 4.0 : -4.0;
        const double mx = (u - P.cxv) * P.inv_fxv, my = (v - P.cyv) * P.inv_fyv;
        lo = std::min(lo, 1.0 + P.E[6] * mx + P.E[7] * my + P.E[8]);
    }
    return lo;
}

// Inverse warp parameters (reference -> view) of rl_common.cuh for one view.
RLInvParam inv_view_param(const rl_camera& ref, const rl_camera& view) {
    double Rrel[9];  // R_v R_r^T
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += view.R[a * 3 + j] * ref.R[b * 3 + j];
            Rrel[a * 3 + b] = s;
        }
    RLInvParam P;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P.F[a * 3 + b] = (float)(Rrel[a * 3 + b] - (a == b ? 1.0 : 0.0));
    for (int a = 0; a < 3; ++a) {  // t_rel = t_v - R_rel t_r
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += Rrel[a * 3 + j] * ref.t[j];
        P.t[a] = (float)(view.t[a] - s);
    }
    P.inv_fxr = (float)(1.0 / ref.K[0]);
    P.inv_fyr = (float)(1.0 / ref.K[4]);
    P.cxr = (float)ref.K[2];
    P.cyr = (float)ref.K[5];
    P.fxv = (float)view.K[0];
    P.fyv = (float)view.K[4];
    P.dcx = (float)(view.K[2] - ref.K[2]);
    P.dcy = (float)(view.K[5] - ref.K[5]);
    P.dfx = (float)(view.K[0] - ref.K[0]);
    P.dfy = (float)(view.K[4] - ref.K[4]);
    return P;
}

void fill_rho(RLViews& v, int D, double near_, double far_) {
    for (int d = 0; d < RL_DEV_MAX_PLANES; ++d) {
        v.rho[d] = 0.f;
        v.rho64[d] = 0.0;
    }
    for (int d = 0; d < D; ++d) {
        const double r = (D == 1) ? 1.0 / far_ : 1.0 / far_ + ((double)d / (double)(D - 1)) * (1.0 / near_ - 1.0 / far_);
        v.rho[d] = (float)r;
        v.rho64[d] = r;
    }
}

rl_status check_mpi(const rl_mpi* m) {
    if (!m) return rl_fail(RL_EINVAL, "mpi is NULL");
    if (m->D < 1 || m->D > RL_MAX_PLANES) return rl_fail(RL_EINVAL, "D=%d outside [1,%d]", m->D, RL_MAX_PLANES);
    if (m->H < 1 || m->W < 1) return rl_fail(RL_EINVAL, "H=%d W=%d must be positive", m->H, m->W);
    if ((long long)m->D * m->H * m->W >= (1ll << 29))
        return rl_fail(RL_EINVAL, "D*H*W = %lld voxels exceeds the 2^29 limit", (long long)m->D * m->H * m->W);
    if (m->dtype != RL_F32 && m->dtype != RL_BF16) return rl_fail(RL_EINVAL, "unknown dtype %d", (int)m->dtype);
    if (!m->data) return rl_fail(RL_EINVAL, "mpi data is NULL");
    if (((uintptr_t)m->data & 15) != 0) return rl_fail(RL_EINVAL, "mpi data must be 16-byte aligned");
    if (!(m->near_ > 0.0) || !(m->far_ > m->near_) || !std::isfinite(m->far_))
        return rl_fail(RL_EINVAL, "need 0 < near < far < inf (near=%g far=%g)", m->near_, m->far_);
    if (!camera_ok(m->ref)) return rl_fail(RL_EINVAL, "reference camera invalid (zero-skew K, orthonormal R)");
    return RL_OK;
}

rl_status make_views(const rl_mpi* m, const rl_camera* cams, int n, int level, RLViews& v) {
    if (!cams) return rl_fail(RL_EINVAL, "camera array is NULL");
    if (n < 1 || n > RL_DEV_MAX_VIEWS) return rl_fail(RL_EINVAL, "%d views outside [1,%d]", n, RL_DEV_MAX_VIEWS);
    std::memset(&v, 0, sizeof(v));
    v.n = n;
    fill_rho(v, m->D, m->near_, m->far_);
    const rl_camera ref = camera_at_level(m->ref, level);
    const int H = m->H >> level, W = m->W >> level;
    for (int i = 0; i < n; ++i) {
        if (!camera_ok(cams[i])) return rl_fail(RL_EINVAL, "camera %d invalid (zero-skew K, orthonormal R)", i);
        v.v64[i] = view_param64(ref, camera_at_level(cams[i], level));
        v.v[i] = view_param(v.v64[i]);
        if (max_offset(v.v64[i], H, W, v.rho64[0], v.rho64[m->D - 1]) > kAnchorOffsetPx) v.anchored = 1;
        if (!(min_ray_dz(v.v64[i], H, W) > 0.05))
            return rl_fail(RL_EINVAL,
                           "camera %d: its rays at the image corners run nearly parallel to the reference planes "
                           "(1 + e_z <= 0.05); such views are not supported",
                           i);
    }
    return RL_OK;
}

size_t elt_size(rl_dtype dt) { return dt == RL_F32 ? 4 : 2; }

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
    size_t Ml, S, slots, G, partials, counter, Il, total;
};

// One workspace serves every level of a schedule: level 0 has the largest selection and
// gradient buffers, level 1 the largest downsampled MPI and source images.
WsLayout ws_layout(int N, int D, int H, int W, int k, rl_dtype dt) {
    WsLayout L;
    size_t off = 0;
    L.Ml = off;
    if (H % 2 == 0 && W % 2 == 0) off += align_up((size_t)D * (H / 2) * (W / 2) * 4 * elt_size(dt));
    L.S = off;
    off += align_up((size_t)k * H * W);
    L.slots = off;
    off += align_up((size_t)D * H * W);
    L.G = off;
    off += align_up((size_t)k * H * W * 16);
    L.partials = off;
    off += align_up(rl_grad_num_blocks(H, W, N) * sizeof(float));
    L.counter = off;
    off += align_up(sizeof(unsigned));
    L.Il = off;  // the level-l source images of a coarse level [N][h][w][3]
    if (H % 2 == 0 && W % 2 == 0) off += align_up((size_t)N * (H / 2) * (W / 2) * 3 * sizeof(float));
    L.total = off;
    return L;
}

rl_status check_hsgd(const rl_mpi* m, const float* images, const rl_camera* src, int N, const rl_hsgd_params* p,
                     int level, void* ws, size_t ws_bytes) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (!p) return rl_fail(RL_EINVAL, "params is NULL");
    if (p->k < 1 || p->k > m->D) return rl_fail(RL_EINVAL, "k=%d outside [1, D=%d]", p->k, m->D);
    if (!std::isfinite(p->lambda)) return rl_fail(RL_EINVAL, "lambda not finite");
    if (p->selection != RL_SELECT_TOPK && p->selection != RL_SELECT_MVS)
        return rl_fail(RL_EINVAL, "unknown selection %d", p->selection);
    if (!std::isfinite(p->lambda_s) || p->lambda_s < 0.f) return rl_fail(RL_EINVAL, "lambda_s must be >= 0");
    if (level < 0 || level > 10 || (m->H % (1 << level)) || (m->W % (1 << level)))
        return rl_fail(RL_EINVAL, "level %d: H=%d and W=%d must be divisible by 2^level", level, m->H, m->W);
    if (!images) return rl_fail(RL_EINVAL, "images is NULL");
    if (N < 1 || N > RL_MAX_VIEWS) return rl_fail(RL_EINVAL, "N=%d outside [1,%d]", N, RL_MAX_VIEWS);
    if (!src) return rl_fail(RL_EINVAL, "source cameras NULL");
    for (int i = 0; i < N; ++i)
        if (!camera_ok(src[i])) return rl_fail(RL_EINVAL, "source camera %d invalid", i);
    if (!ws) return rl_fail(RL_EINVAL, "workspace is NULL");
    const size_t need = ws_layout(N, m->D, m->H, m->W, p->k, m->dtype).total;
    if (ws_bytes < need) return rl_fail(RL_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (((uintptr_t)ws & 255) != 0) return rl_fail(RL_EINVAL, "workspace must be 256-byte aligned");
    return RL_OK;
}

// Enqueue one HSGD iteration (arguments already validated).
rl_status enqueue_hsgd(rl_mpi* m, const float* images, const rl_camera* src, int N, int k, float lambda, int clamp01,
                       int level, int selection, float lambda_s, float* loss_out, uint8_t* S_out, void* ws,
                       cudaStream_t s) {
    const WsLayout L = ws_layout(N, m->D, m->H, m->W, k, m->dtype);
    char* base = (char*)ws;
    const int h = m->H >> level, w = m->W >> level;
    void* Ml = level == 0 ? m->data : (void*)(base + L.Ml);
    uint8_t* S = S_out ? S_out : (uint8_t*)(base + L.S);
    uint8_t* slots = (uint8_t*)(base + L.slots);
    float* G = (float*)(base + L.G);
    float* partials = (float*)(base + L.partials);
    unsigned* counter = (unsigned*)(base + L.counter);
    RLViews views;
    rl_status st = make_views(m, src, N, level, views);
    if (st) return st;
    views.gplanes = k;
    // coarse levels: the pyramid, the level source images and the selection share one pass
    float* Il = level ? (float*)(base + L.Il) : nullptr;
    st = level ? rl_launch_pyramid_select(m->data, m->dtype, m->D, m->H, m->W, level, Ml, k, S, slots, G, counter,
                                          selection, s, images, N, Il)
               : rl_launch_select(Ml, m->dtype, nullptr, m->D, h, w, k, S, nullptr, slots, G, s, counter, selection);
    if (st) return st;
    int nb = 0;
    // the gradient kernel's last block reduces the loss partials (fixed order) into loss_out
    // (measured 1.2% faster per step than a separate reduction launch)
    st = rl_launch_grad(Ml, m->dtype, m->D, h, w, views, true, level ? Il : images, 0, nullptr, slots, G,
                        1.0f / (float)N, partials, &nb, s, loss_out, counter, 0.5f / (float)N);
    if (st) return st;
    return rl_launch_update(m->data, m->dtype, m->D, m->H, m->W, level, S, G, k, lambda, clamp01, s, Ml, lambda_s);
}

// Workspace of reallife_gradient_volume: the level MPI (levels >= 1), the selection and
// the view alpha weights [N][D][h][w] (largest at level 0).
struct VolLayout {
    size_t Ml, S, A, total;
};

VolLayout vol_layout(int N, int D, int H, int W, int k, rl_dtype dt) {
    VolLayout L;
    size_t off = 0;
    L.Ml = off;
    if (H % 2 == 0 && W % 2 == 0) off += align_up((size_t)D * (H / 2) * (W / 2) * 4 * elt_size(dt));
    L.S = off;
    off += align_up((size_t)k * H * W);
    L.A = off;
    off += align_up((size_t)N * D * H * W * sizeof(float));
    L.total = off;
    return L;
}

__global__ void k_zero(float4* __restrict__ p, size_t n4) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

rl_status launch_zero(float* p, size_t nfloats, cudaStream_t s) {
    RLTraceScope ts("zero_fill", s);
    const size_t n4 = nfloats / 4;  // callers pass multiples of 4 floats
    const unsigned blocks = (unsigned)std::min<size_t>((n4 + 255) / 256, 152 * 16);
    if (n4) k_zero<<<blocks ? blocks : 1, 256, 0, s>>>((float4*)p, n4);
    return rl_check_launch("zero_fill");
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" size_t reallife_workspace_bytes(int N, int D, int H, int W, int k, rl_dtype dtype) {
    if (N < 1 || D < 1 || H < 1 || W < 1 || k < 1) return 0;
    return ws_layout(N, D, H, W, k, dtype).total;
}

extern "C" rl_status reallife_render(const rl_mpi* m, const rl_camera* tgt, int T, float* out, cudaStream_t stream) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (!tgt || T < 1) return rl_fail(RL_EINVAL, "need T >= 1 target cameras");
    if (!out) return rl_fail(RL_EINVAL, "out is NULL");
    for (int i = 0; i < T; ++i)
        if (!camera_ok(tgt[i])) return rl_fail(RL_EINVAL, "target camera %d invalid", i);
    for (int i0 = 0; i0 < T; i0 += RL_DEV_MAX_VIEWS) {
        const int n = std::min(RL_DEV_MAX_VIEWS, T - i0);
        RLViews views;
        st = make_views(m, tgt + i0, n, 0, views);
        if (st) return st;
        st = rl_launch_render(m->data, m->dtype, m->D, m->H, m->W, views, out + (size_t)i0 * m->H * m->W * 3, stream);
        if (st) return st;
    }
    return RL_OK;
}

extern "C" rl_status reallife_hsgd_step(rl_mpi* m, const float* images, const rl_camera* src, int N,
                                        const rl_hsgd_params* p, float* loss_out, uint8_t* S_out, void* ws,
                                        size_t ws_bytes, cudaStream_t stream) {
    rl_status st = check_hsgd(m, images, src, N, p, p ? p->level : 0, ws, ws_bytes);
    if (st) return st;
    return enqueue_hsgd(m, images, src, N, p->k, p->lambda, p->clamp01, p->level, p->selection, p->lambda_s, loss_out,
                        S_out, ws, stream);
}

extern "C" rl_status reallife_refine(rl_mpi* m, const float* images, const rl_camera* src, int N,
                                     const rl_hsgd_params* p, const int* schedule, int iters, float* loss_per_iter,
                                     void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!schedule || iters < 1) return rl_fail(RL_EINVAL, "need a schedule of >= 1 levels");
    for (int it = 0; it < iters; ++it) {
        rl_status st = check_hsgd(m, images, src, N, p, schedule[it], ws, ws_bytes);
        if (st) return st;
    }
    for (int it = 0; it < iters; ++it) {
        rl_status st = enqueue_hsgd(m, images, src, N, p->k, p->lambda, p->clamp01, schedule[it], p->selection,
                                    p->lambda_s, loss_per_iter ? loss_per_iter + it : nullptr, nullptr, ws, stream);
        if (st) return st;
    }
    return RL_OK;
}

extern "C" size_t reallife_gradient_volume_workspace_bytes(int N, int D, int H, int W, int k, rl_dtype dtype) {
    if (N < 1 || D < 1 || H < 1 || W < 1 || k < 1) return 0;
    return vol_layout(N, D, H, W, k, dtype).total;
}

extern "C" rl_status reallife_gradient_volume(const rl_mpi* m, const float* images, const rl_camera* src, int N,
                                              int k, int level, int selection, uint8_t* S_out, float* V, void* ws,
                                              size_t ws_bytes, cudaStream_t stream) {
    return rl_gradient_volume(m, images, src, N, k, level, selection, S_out, V, nullptr, ws, ws_bytes, stream);
}

rl_status rl_gradient_volume(const rl_mpi* m, const float* images, const rl_camera* src, int N, int k, int level,
                             int selection, uint8_t* S_out, float* V, void* act, void* ws, size_t ws_bytes,
                             cudaStream_t stream) {
    rl_hsgd_params p;
    std::memset(&p, 0, sizeof(p));
    p.k = k;
    p.lambda = 1.0f;
    p.selection = selection;
    const size_t need = (m && N >= 1) ? vol_layout(N, m->D, m->H, m->W, k, m->dtype).total : 0;
    // the step's checks (MPI, k, selection, level, images, cameras); its workspace is not used
    rl_status st = check_hsgd(m, images, src, N, &p, level, ws, ~(size_t)0);
    if (st) return st;
    if (act ? ((uintptr_t)act & 15) != 0 : (!V || ((uintptr_t)V & 3) != 0))
        return rl_fail(RL_EINVAL, "V must be a non-NULL, 4-byte aligned device buffer");
    if (ws_bytes < need) return rl_fail(RL_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    const VolLayout L = vol_layout(N, m->D, m->H, m->W, k, m->dtype);
    char* base = (char*)ws;
    const int h = m->H >> level, w = m->W >> level;
    void* Ml = level == 0 ? m->data : (void*)(base + L.Ml);
    uint8_t* S = S_out ? S_out : (uint8_t*)(base + L.S);
    float* A = (float*)(base + L.A);
    RLViews views;
    st = make_views(m, src, N, level, views);
    if (st) return st;
    RLInvViews iv;
    std::memset(&iv, 0, sizeof(iv));
    iv.n = N;
    for (int d = 0; d < RL_DEV_MAX_PLANES; ++d) iv.rho[d] = views.rho[d];
    const rl_camera refl = camera_at_level(m->ref, level);
    for (int i = 0; i < N; ++i) {
        iv.lv[i] = inv_view_param(refl, camera_at_level(src[i], level));
        iv.full[i] = inv_view_param(m->ref, src[i]);
    }
    st = level ? rl_launch_pyramid_select(m->data, m->dtype, m->D, m->H, m->W, level, Ml, k, S, nullptr, nullptr,
                                          nullptr, selection, stream)
               : rl_launch_select(Ml, m->dtype, nullptr, m->D, h, w, k, S, nullptr, nullptr, nullptr, stream,
                                  nullptr, selection);
    if (st) return st;
    st = rl_launch_view_alpha(Ml, m->dtype, m->D, h, w, views, A, stream);
    if (st) return st;
    return rl_launch_volume(Ml, m->dtype, m->D, h, w, level, S, k, A, images, iv, V, stream, act);
}

extern "C" rl_status reallife_downsample_f32(const float* x, int P, int H, int W, int C, int level, float* y,
                                             cudaStream_t stream) {
    if (!x || !y || P < 1 || H < 1 || W < 1 || C < 1 || level < 0 || level > 10 || (H % (1 << level)) ||
        (W % (1 << level)))
        return rl_fail(RL_EINVAL, "downsample: bad arguments (H, W must be divisible by 2^level)");
    return rl_launch_downsample_f32(x, P, H, W, C, level, y, stream);
}

extern "C" rl_status reallife_select(const rl_mpi* m, int k, int selection, uint8_t* S, uint64_t* mask,
                                     cudaStream_t stream) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (k < 1 || k > m->D) return rl_fail(RL_EINVAL, "k=%d outside [1, D=%d]", k, m->D);
    if (selection != RL_SELECT_TOPK && selection != RL_SELECT_MVS)
        return rl_fail(RL_EINVAL, "unknown selection %d", selection);
    if (!S && !mask) return rl_fail(RL_EINVAL, "select: no output");
    return rl_launch_select(m->data, m->dtype, nullptr, m->D, m->H, m->W, k, S, mask, nullptr, nullptr, stream,
                            nullptr, selection);
}

extern "C" rl_status reallife_select_keys(const float* keys, int D, int H, int W, int k, int selection, uint8_t* S,
                                          uint64_t* mask, cudaStream_t stream) {
    if (!keys || D < 1 || D > RL_MAX_PLANES || H < 1 || W < 1 || k < 1 || k > D || (!S && !mask) ||
        (selection != RL_SELECT_TOPK && selection != RL_SELECT_MVS))
        return rl_fail(RL_EINVAL, "select_keys: bad arguments");
    return rl_launch_select(nullptr, RL_F32, keys, D, H, W, k, S, mask, nullptr, nullptr, stream, nullptr, selection);
}

extern "C" rl_status reallife_loss_grad(const rl_mpi* m, const float* images, const rl_camera* src, int N,
                                        const uint64_t* mask, int k, float* G, float* loss_out, void* ws,
                                        size_t ws_bytes, cudaStream_t stream) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (!images || !G) return rl_fail(RL_EINVAL, "loss_grad: images and G must be non-NULL");
    if (((uintptr_t)G & 15) != 0) return rl_fail(RL_EINVAL, "G must be 16-byte aligned");
    if (mask && (k < 1 || k > m->D)) return rl_fail(RL_EINVAL, "k=%d outside [1, D=%d]", k, m->D);
    if (!ws) return rl_fail(RL_EINVAL, "workspace is NULL");
    RLViews views;
    st = make_views(m, src, N, 0, views);
    if (st) return st;
    const size_t part = align_up(rl_grad_num_blocks(m->H, m->W, N) * sizeof(float));
    const size_t need = part + (mask ? align_up((size_t)m->D * m->H * m->W) : 0);
    if (ws_bytes < need) return rl_fail(RL_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (((uintptr_t)ws & 255) != 0) return rl_fail(RL_EINVAL, "workspace must be 256-byte aligned");
    uint8_t* slots = mask ? (uint8_t*)ws + part : nullptr;
    const int nslots = mask ? k : m->D;
    views.gplanes = nslots;
    st = launch_zero(G, (size_t)nslots * m->H * m->W * 4, stream);
    if (st) return st;
    if (mask) {
        st = rl_launch_mask_to_slots(mask, m->D, k, m->H * m->W, slots, stream);
        if (st) return st;
    }
    int nb = 0;
    st = rl_launch_grad(m->data, m->dtype, m->D, m->H, m->W, views, true, images, 0, nullptr, slots, G,
                        1.0f / (float)N, (float*)ws, &nb, stream);
    if (st) return st;
    if (loss_out) return rl_launch_loss_reduce((float*)ws, nb, 0.5f / (float)N, loss_out, stream);
    return RL_OK;
}

extern "C" rl_status reallife_sparse_update(rl_mpi* m, const uint8_t* S, const float* G, int k, int level,
                                            float lambda, int clamp01, cudaStream_t stream) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (!S || !G) return rl_fail(RL_EINVAL, "sparse_update: S and G must be non-NULL");
    if (((uintptr_t)G & 15) != 0) return rl_fail(RL_EINVAL, "G must be 16-byte aligned");
    if (k < 1 || k > m->D) return rl_fail(RL_EINVAL, "k=%d outside [1, D=%d]", k, m->D);
    if (level < 0 || level > 10 || (m->H % (1 << level)) || (m->W % (1 << level)))
        return rl_fail(RL_EINVAL, "level %d incompatible with H=%d W=%d", level, m->H, m->W);
    if (!std::isfinite(lambda)) return rl_fail(RL_EINVAL, "lambda not finite");
    return rl_launch_update(m->data, m->dtype, m->D, m->H, m->W, level, S, G, k, lambda, clamp01, stream);
}

extern "C" rl_status reallife_render_backward(const rl_mpi* m, const rl_camera* views_in, int N, const float* grad_out,
                                              float* grad_mpi, cudaStream_t stream) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (!grad_out || !grad_mpi) return rl_fail(RL_EINVAL, "render_backward: NULL buffer");
    if (((uintptr_t)grad_mpi & 15) != 0) return rl_fail(RL_EINVAL, "grad_mpi must be 16-byte aligned");
    RLViews views;
    st = make_views(m, views_in, N, 0, views);
    if (st) return st;
    st = launch_zero(grad_mpi, (size_t)m->D * m->H * m->W * 4, stream);
    if (st) return st;
    return rl_launch_grad(m->data, m->dtype, m->D, m->H, m->W, views, false, nullptr, 0, grad_out, nullptr, grad_mpi,
                          1.0f, nullptr, nullptr, stream);
}

extern "C" rl_status reallife_warp_offsets(const rl_mpi* m, const rl_camera* view, float* out, cudaStream_t stream) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (!out) return rl_fail(RL_EINVAL, "out is NULL");
    RLViews views;
    st = make_views(m, view, 1, 0, views);
    if (st) return st;
    return rl_launch_warp_offsets(m->D, m->H, m->W, views, out, stream);
}

// ------------------------------------------------------------- batched step

extern "C" size_t reallife_metrics_workspace_bytes(int N, int H, int W) {
    if (N < 1 || H < 1 || W < 1) return 0;
    return align_up(rl_metrics_partials(N, H, W) * sizeof(double));
}

extern "C" rl_status reallife_image_metrics(const float* x, const float* y, int N, int H, int W, double* out,
                                            void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!x || !y || !out || N < 1 || N > 65535 || H < 11 || W < 11 || H > 65535 || W > 65535)
        return rl_fail(RL_EINVAL, "image_metrics: need x, y, out, 1 <= N <= 65535 and 11 <= H, W <= 65535 (N=%d H=%d "
                       "W=%d)", N, H, W);
    if (!ws || ((uintptr_t)ws & 7) != 0) return rl_fail(RL_EINVAL, "image_metrics: workspace NULL or not 8-byte aligned");
    const size_t need = rl_metrics_partials(N, H, W) * sizeof(double);
    if (ws_bytes < need) return rl_fail(RL_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    return rl_launch_image_metrics(x, y, N, H, W, out, static_cast<double*>(ws), stream);
}

extern "C" rl_status reallife_kept_mass(const rl_mpi* m, const uint64_t* mask, double* out, void* ws, size_t ws_bytes,
                                        cudaStream_t stream) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (!mask || !out) return rl_fail(RL_EINVAL, "kept_mass: mask and out are required");
    if (((uintptr_t)mask & 7) != 0) return rl_fail(RL_EINVAL, "kept_mass: mask must be 8-byte aligned");
    if (!ws || ((uintptr_t)ws & 7) != 0) return rl_fail(RL_EINVAL, "kept_mass: workspace NULL or not 8-byte aligned");
    const size_t need = rl_metrics_partials(1, m->H, m->W) * sizeof(double);
    if (ws_bytes < need) return rl_fail(RL_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
    return rl_launch_kept_mass(m->data, m->dtype, m->D, m->H, m->W, mask, out, static_cast<double*>(ws), stream);
}

extern "C" size_t reallife_batch_table_bytes(int max_items) {
    if (max_items < 1 || max_items > RL_BATCH_MAX_ITEMS) return 0;
    return align_up(sizeof(RLBatchHeader) + (size_t)max_items * sizeof(RLBatchItem));
}

namespace {
bool ranges_overlap(uintptr_t a, size_t na, uintptr_t b, size_t nb) { return a < b + nb && b < a + na; }
}  // namespace

extern "C" rl_status reallife_batch_prepare(const rl_batch_item* items, int n, void* table_host, size_t table_bytes) {
    if (!items || n < 1 || n > RL_BATCH_MAX_ITEMS)
        return rl_fail(RL_EINVAL, "batch: n=%d outside [1, %d]", n, RL_BATCH_MAX_ITEMS);
    if (!table_host) return rl_fail(RL_EINVAL, "batch: table_host is NULL");
    if (table_bytes < reallife_batch_table_bytes(n))
        return rl_fail(RL_ENOMEM, "batch: table of %zu bytes < %zu needed", table_bytes, reallife_batch_table_bytes(n));
    RLBatchHeader* hdr = static_cast<RLBatchHeader*>(table_host);
    RLBatchItem* out = const_cast<RLBatchItem*>(rl_batch_items(table_host));
    std::memset(hdr, 0, sizeof(*hdr));
    unsigned sel = 0, grad = 0, pp = 0, upd = 0, max_gather_D = 0;
    for (int i = 0; i < n; ++i) {
        const rl_batch_item& b = items[i];
        const rl_hsgd_params* p = &b.params;
        rl_status st = check_hsgd(b.mpi, b.images, b.src, b.N, p, p->level, b.ws, b.ws_bytes);
        if (st) return rl_fail(st, "batch item %d: %s", i, reallife_last_error());
        const rl_mpi* m = b.mpi;
        if (m->dtype != items[0].mpi->dtype) return rl_fail(RL_EINVAL, "batch item %d: storage type differs", i);
        const size_t mb = (size_t)m->D * m->H * m->W * 4 * elt_size(m->dtype);
        const WsLayout L = ws_layout(b.N, m->D, m->H, m->W, p->k, m->dtype);
        for (int j = 0; j < i; ++j) {
            const rl_mpi* o = items[j].mpi;
            const size_t ob = (size_t)o->D * o->H * o->W * 4 * elt_size(o->dtype);
            const size_t ow = ws_layout(items[j].N, o->D, o->H, o->W, items[j].params.k, o->dtype).total;
            if (ranges_overlap((uintptr_t)m->data, mb, (uintptr_t)o->data, ob) ||
                ranges_overlap((uintptr_t)b.ws, L.total, (uintptr_t)items[j].ws, ow) ||
                ranges_overlap((uintptr_t)m->data, mb, (uintptr_t)items[j].ws, ow) ||
                ranges_overlap((uintptr_t)b.ws, L.total, (uintptr_t)o->data, ob))
                return rl_fail(RL_EINVAL, "batch items %d and %d share an MPI or workspace", j, i);
        }
        RLBatchItem& it = out[i];
        std::memset(&it, 0, sizeof(it));
        st = make_views(m, b.src, b.N, p->level, it.views);
        if (st) return rl_fail(st, "batch item %d: %s", i, reallife_last_error());
        it.views.gplanes = p->k;
        char* base = static_cast<char*>(b.ws);
        const int l = p->level, h = m->H >> l, w = m->W >> l;
        it.M = m->data;
        it.Ml = l == 0 ? m->data : (void*)(base + L.Ml);
        it.images = b.images;
        it.Il = l == 0 ? nullptr : (float*)(base + L.Il);
        it.S = (uint8_t*)(base + L.S);
        it.slots = (uint8_t*)(base + L.slots);
        it.G = (float*)(base + L.G);
        it.partials = (float*)(base + L.partials);
        it.counter = (unsigned*)(base + L.counter);
        it.loss_out = b.loss_out;
        it.D = m->D;
        it.H = m->H;
        it.W = m->W;
        it.level = l;
        it.k = p->k;
        it.mode = p->selection;
        it.clamp01 = p->clamp01;
        it.N = b.N;
        it.lambda = p->lambda;
        it.prior_scale = p->lambda_s != 0.f ? (float)((double)p->lambda_s / ((double)h * w * m->D)) : 0.f;
        it.inv_n = 1.0f / (float)b.N;
        it.loss_scale = 0.5f / (float)b.N;
        const unsigned hw = (unsigned)(h * w);
        it.sel_begin = sel;
        it.sel_units = l == 0 ? (hw + 255) / 256 : (hw + 31) / 32;
        const bool gather = rl_kernel_path(h, w, b.N) == 2;
        it.grad_begin = grad;
        it.pp_begin = pp;
        if (gather) {
            it.grad_tiles_x = rl_grad_gather_tiles_x(w);
            it.grad_units = (unsigned)b.N * it.grad_tiles_x * rl_grad_gather_tiles_y(h);
            max_gather_D = std::max(max_gather_D, (unsigned)m->D);
        } else {
            it.pp_tiles_x = rl_grad_pp_tiles_x(w);
            it.pp_units = (unsigned)b.N * it.pp_tiles_x * rl_grad_pp_tiles_y(h);
        }
        it.upd_begin = upd;
        it.upd_tiles_x = (unsigned)((m->W + 127) / 128);
        it.upd_units = it.upd_tiles_x * (unsigned)m->H;
        sel += it.sel_units;
        grad += it.grad_units;
        pp += it.pp_units;
        upd += it.upd_units;
    }
    hdr->n = (unsigned)n;
    hdr->dtype = (unsigned)items[0].mpi->dtype;
    hdr->sel_units = sel;
    hdr->grad_units = grad;
    hdr->pp_units = pp;
    hdr->max_gather_D = max_gather_D;
    hdr->upd_units = upd;
    hdr->status = rl_device_status_ptr();
    return RL_OK;
}

extern "C" rl_status reallife_hsgd_step_batch(const void* table_host, void* table_dev, size_t table_bytes,
                                              cudaStream_t stream) {
    if (!table_host || !table_dev) return rl_fail(RL_EINVAL, "batch: NULL table");
    if (((uintptr_t)table_dev & 255) != 0) return rl_fail(RL_EINVAL, "batch: table_dev must be 256-byte aligned");
    const RLBatchHeader* hdr = static_cast<const RLBatchHeader*>(table_host);
    if (hdr->n < 1 || hdr->n > RL_BATCH_MAX_ITEMS || (hdr->dtype != RL_F32 && hdr->dtype != RL_BF16))
        return rl_fail(RL_EINVAL, "batch: the table was not written by reallife_batch_prepare");
    if (table_bytes < reallife_batch_table_bytes((int)hdr->n))
        return rl_fail(RL_ENOMEM, "batch: table of %zu bytes < %zu needed", table_bytes,
                       reallife_batch_table_bytes((int)hdr->n));
    if (!capturing(stream)) {  // while capturing, a copy from pageable memory fails at the copy itself
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, table_host) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return rl_fail(RL_EINVAL, "batch: table_host must be page-locked host memory");
        }
    }
    const rl_dtype dt = (rl_dtype)hdr->dtype;
    cudaError_t e = cudaMemcpyAsync(table_dev, table_host, table_bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return rl_fail(RL_ECUDA, "batch: table copy: %s", cudaGetErrorString(e));
    rl_status st = rl_launch_select_batch(table_dev, dt, stream);
    if (st) return st;
    // a captured launch may later serve a table of larger planes: reserve the most then
    const int planes = capturing(stream) ? RL_DEV_MAX_PLANES : (int)hdr->max_gather_D;
    if (hdr->grad_units || capturing(stream)) {
        st = rl_launch_grad_batch(table_dev, dt, planes, stream);
        if (st) return st;
    }
    if (hdr->pp_units || capturing(stream)) {
        st = rl_launch_grad_pp_batch(table_dev, dt, stream);
        if (st) return st;
    }
    return rl_launch_update_batch(table_dev, dt, stream);
}

// ------------------------------------------------------ fixed-scratch HSGD step
//
// Some callers cannot allocate device memory at all: a plugin running inside a host
// application that owns the GPU heap and hands its plugins no allocator, or a frame loop
// that must not call cudaMalloc because the call can synchronise the device and stall
// the frame.  reallife_hsgd_step_noalloc runs the same iteration as reallife_hsgd_step
// without asking them for a workspace: its scratch is the array below, a fixed
// RL_NOALLOC_SCRATCH_BYTES per device that every GPU loading this library keeps until
// the process exits.  The array's name is only a host-side stand-in in host code, so its
// device address is looked up with cudaGetSymbolAddress (on every call made outside stream
// capture, with the call's device current) and passed to the kernels.

static __device__ __align__(256) unsigned char g_rl_noalloc_scratch[RL_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};

// Device address of the fixed scratch on the current device.  Looked up again on every call
// made outside stream capture (cheap, and right after a cudaDeviceReset has reloaded the
// library's device code); a call being captured uses the address of the device's last
// uncaptured call, or looks it up if there was none.
rl_status noalloc_scratch(void** out, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rl_fail(RL_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return rl_fail(RL_ECUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev] || !capturing(s)) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rl_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return rl_fail(RL_ECUDA, "cudaGetSymbolAddress of the fixed scratch: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return RL_OK;
}
}  // namespace

extern "C" rl_status reallife_hsgd_step_noalloc(rl_mpi* m, const float* images, const rl_camera* src, int N,
                                                const rl_hsgd_params* p, float* loss_out, uint8_t* S_out,
                                                cudaStream_t stream) {
    rl_status st = check_mpi(m);
    if (st) return st;
    if (!p) return rl_fail(RL_EINVAL, "params is NULL");
    if (p->k < 1 || p->k > m->D) return rl_fail(RL_EINVAL, "k=%d outside [1, D=%d]", p->k, m->D);
    if (N < 1 || N > RL_MAX_VIEWS) return rl_fail(RL_EINVAL, "N=%d outside [1,%d]", N, RL_MAX_VIEWS);
    const size_t need = ws_layout(N, m->D, m->H, m->W, p->k, m->dtype).total;
    if (need > (size_t)RL_NOALLOC_SCRATCH_BYTES)
        return rl_fail(RL_ENOMEM, "this problem needs %zu bytes of scratch; the fixed scratch holds %zu bytes", need,
                       (size_t)RL_NOALLOC_SCRATCH_BYTES);
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        if (g_trace_on) return rl_fail(RL_EINVAL, "kernel tracing creates CUDA events; disable it for this call");
    }
    void* ws = nullptr;
    st = noalloc_scratch(&ws, stream);
    if (st) return st;
    st = check_hsgd(m, images, src, N, p, p->level, ws, (size_t)RL_NOALLOC_SCRATCH_BYTES);
    if (st) return st;
    // every part of the scratch this iteration reads is written earlier in the same
    // iteration (level MPI, selection, slot map; the select kernel zeroes the gradient slots)
    return enqueue_hsgd(m, images, src, N, p->k, p->lambda, p->clamp01, p->level, p->selection, p->lambda_s, loss_out,
                        S_out, ws, stream);
}
