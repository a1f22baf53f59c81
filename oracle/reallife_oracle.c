/*
 * reallife_oracle.c -- plain, slow FP64 CPU oracle of the RealLiFe HSGD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the test-suite, the package smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library; every function is written from the paper's equations, in the
 * paper's order, with straightforward loops and no blocking or fusion.
 *
 * Conventions (the readings of the paper this oracle fixes):
 *   - MPI M[d][y][x][c], c = (R,G,B,alpha), d = 0 farthest ... D-1 nearest, so the
 *     over operator of Eq. (eq_over) puts the unoccluded plane at the top index.
 *   - Plane depths are uniform in inverse depth: rho_d = 1/far + d/(D-1) (1/near - 1/far)
 *     (rho_0 = 1/far when D = 1).  The paper does not state the spacing.
 *   - Cameras are world->camera, x_cam = R X + t; a pixel is K x_cam / z, pixel centres
 *     at integer coordinates.  Under this convention Eq. (eq_homo) is exactly the
 *     plane-induced homography of the plane z = z_d in the reference frame.
 *   - Warping the MPI into a view (Eq. eq_render) samples plane d at the reference
 *     pixel where the ray of the view's pixel meets that plane (ray-plane intersection,
 *     computed geometrically here, not through Eq. eq_homo's matrix), with bilinear
 *     interpolation and zero padding per tap (grid_sample with zero padding, Sec. 3.2).
 *     A ray that meets the plane behind the camera samples nothing.
 *   - Composite: C = sum_d c_d alpha_d prod_{j>d} (1 - alpha_j), no background (Eq. eq_over).
 *   - Photometric loss: L = 1/(2N) sum_i sum_q sum_ch (C_i(q) - I_i(q))^2; the analytic
 *     gradient step of Sec. 3.1 is read as descent, M <- M - lambda dL/dM.
 *   - Selection key: the reference-view alpha weight A_d = alpha_d prod_{j>d}(1-alpha_j)
 *     (Eq. eq_gradient / eq_overA); keep the k largest per pixel, ties to the lower d,
 *     indices stored in ascending depth order (Sec. 3.3, "Gradient Sparsification").
 *   - Levels: an iteration at level l works on Down^l(M) and Down^l(I) (2x2 box
 *     averages, Sec. 3.2 "Hierarchical PSV construction"), intrinsics scaled by 2^-l,
 *     and adds the nearest-neighbour upsampled masked step to the full MPI (the
 *     restore operator R(., S) of Sec. 3.3 followed by the coarse-to-fine upsampling).
 *   - Update: M[d] <- clamp(M[d] - lambda g[d], 0, 1) for selected d (clamp optional).
 *   - Gradient volume (Sec. 3.3): the PSV samples each source image at the reference pixel
 *     carried into the view by Eq. (eq_homo)'s inverse homography (computed geometrically);
 *     the level-l PSV is Down^l of the full-resolution PSV, as Sec. 3.2 downsamples the
 *     volume itself.  The inverse-warped alpha weights of view i come from the level MPI
 *     M_l warped into view i at level l (Eq. eq_gradient at every view pixel), sampled back at
 *     the reference pixels the same way.  Channels: P (3N, view-major), A (N), M_l (4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double K[9]; /* row-major intrinsics */
    double R[9]; /* row-major world->camera rotation */
    double t[3]; /* world->camera translation */
} orc_camera;

/* Threads the build runs its parallel loops on (1 for the serial build). */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- geometry */

/* Plane inverse depths (uniform in inverse depth between far and near). */
void orc_plane_inverse_depths(int D, double near_, double far_, double* rho) {
    for (int d = 0; d < D; ++d)
        rho[d] = (D == 1) ? 1.0 / far_ : 1.0 / far_ + ((double)d / (double)(D - 1)) * (1.0 / near_ - 1.0 / far_);
}

static void inv3(const double* A, double* B) {
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    B[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

/* Camera scaled to pyramid level l: focal lengths / 2^l, principal point (c + 0.5)/2^l - 0.5. */
void orc_camera_at_level(const orc_camera* in, int level, orc_camera* out) {
    *out = *in;
    double s = ldexp(1.0, -level);
    out->K[0] = in->K[0] * s;
    out->K[1] = in->K[1] * s;
    out->K[4] = in->K[4] * s;
    out->K[2] = (in->K[2] + 0.5) * s - 0.5;
    out->K[5] = (in->K[5] + 0.5) * s - 0.5;
}

/*
 * Geometric warp (Eq. eq_render's omega, Eq. eq_homo by construction): pixel (u,v) of
 * camera `view`, plane z_ref = z of the reference frustum -> reference pixel (px,py).
 * Casts the view's ray through (u,v), intersects it with the plane, projects into the
 * reference camera.  Returns 0 when the plane is not met in front of the view.
 */
int orc_view_to_ref(const orc_camera* ref, const orc_camera* view, double z, double u, double v,
                    double* px, double* py) {
    double Kinv[9];
    inv3(view->K, Kinv);
    double m[3] = {Kinv[0] * u + Kinv[1] * v + Kinv[2], Kinv[3] * u + Kinv[4] * v + Kinv[5],
                   Kinv[6] * u + Kinv[7] * v + Kinv[8]};
    /* world-frame ray: origin = camera centre -R^T t, direction R^T m */
    double Cw[3], dw[3];
    for (int a = 0; a < 3; ++a) {
        Cw[a] = -(view->R[0 * 3 + a] * view->t[0] + view->R[1 * 3 + a] * view->t[1] + view->R[2 * 3 + a] * view->t[2]);
        dw[a] = view->R[0 * 3 + a] * m[0] + view->R[1 * 3 + a] * m[1] + view->R[2 * 3 + a] * m[2];
    }
    /* into the reference camera frame */
    double Cr[3], dr[3];
    for (int a = 0; a < 3; ++a) {
        Cr[a] = ref->R[a * 3 + 0] * Cw[0] + ref->R[a * 3 + 1] * Cw[1] + ref->R[a * 3 + 2] * Cw[2] + ref->t[a];
        dr[a] = ref->R[a * 3 + 0] * dw[0] + ref->R[a * 3 + 1] * dw[1] + ref->R[a * 3 + 2] * dw[2];
    }
    if (!(dr[2] > 0.0) || !(z - Cr[2] > 0.0)) return 0;
    double s = (z - Cr[2]) / dr[2];
    double X[3] = {Cr[0] + s * dr[0], Cr[1] + s * dr[1], z};
    const double* K = ref->K;
    double hx = K[0] * X[0] + K[1] * X[1] + K[2] * X[2];
    double hy = K[3] * X[0] + K[4] * X[1] + K[5] * X[2];
    double hz = K[6] * X[0] + K[7] * X[1] + K[8] * X[2];
    *px = hx / hz;
    *py = hy / hz;
    return 1;
}

/* Bilinear taps at (x,y): integer corners and weights; taps outside the image get weight 0. */
static void bilinear_taps(double x, double y, int W, int H, int tx[4], int ty[4], double w[4]) {
    double x0 = floor(x), y0 = floor(y);
    double fx = x - x0, fy = y - y0;
    int ix = (int)x0, iy = (int)y0;
    tx[0] = ix;     ty[0] = iy;     w[0] = (1.0 - fx) * (1.0 - fy);
    tx[1] = ix + 1; ty[1] = iy;     w[1] = fx * (1.0 - fy);
    tx[2] = ix;     ty[2] = iy + 1; w[2] = (1.0 - fx) * fy;
    tx[3] = ix + 1; ty[3] = iy + 1; w[3] = fx * fy;
    for (int k = 0; k < 4; ++k)
        if (tx[k] < 0 || tx[k] >= W || ty[k] < 0 || ty[k] >= H) w[k] = 0.0;
}

/* ------------------------------------------------------------ forward model */

typedef struct {
    int tx[4], ty[4];
    double w[4];
    double m[4]; /* sampled (R,G,B,alpha) */
} sample_t;

static void sample_plane(const double* M, int d, int H, int W, int valid, double px, double py, sample_t* s) {
    memset(s, 0, sizeof(*s));
    if (!valid) return;
    bilinear_taps(px, py, W, H, s->tx, s->ty, s->w);
    for (int k = 0; k < 4; ++k) {
        if (s->w[k] == 0.0) continue;
        const double* v = M + (((size_t)d * H + s->ty[k]) * W + s->tx[k]) * 4;
        for (int c = 0; c < 4; ++c) s->m[c] += s->w[k] * v[c];
    }
}

/* Composite of one view pixel (u, v): Eq. (eq_render) with the over operator of Eq. (eq_over). */
static void render_pixel(const double* M, int D, int H, int W, const double* rho, const orc_camera* ref,
                         const orc_camera* view, double u, double v, double C[3]) {
    C[0] = C[1] = C[2] = 0.0;
    /* sum_d c_d alpha_d prod_{j>d}(1-alpha_j), accumulated from the nearest plane */
    double T = 1.0;
    for (int d = D - 1; d >= 0; --d) {
        double px, py;
        int ok = orc_view_to_ref(ref, view, 1.0 / rho[d], u, v, &px, &py);
        sample_t s;
        sample_plane(M, d, H, W, ok, px, py, &s);
        for (int c = 0; c < 3; ++c) C[c] += s.m[c] * s.m[3] * T;
        T *= (1.0 - s.m[3]);
    }
}

/* Render one view of size H x W (same size as the MPI): out[y][x][3]. */
void orc_render(const double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                const orc_camera* view, double* out) {
    double* rho = (double*)malloc(sizeof(double) * D);
    orc_plane_inverse_depths(D, near_, far_, rho);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) render_pixel(M, D, H, W, rho, ref, view, x, y, out + ((size_t)y * W + x) * 3);
    free(rho);
}

/* Render only the n view pixels (xs[j], ys[j]): out[n][3]. */
void orc_render_pixels(const double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                       const orc_camera* view, int n, const int* xs, const int* ys, double* out) {
    double* rho = (double*)malloc(sizeof(double) * D);
    orc_plane_inverse_depths(D, near_, far_, rho);
    for (int j = 0; j < n; ++j) render_pixel(M, D, H, W, rho, ref, view, xs[j], ys[j], out + (size_t)j * 3);
    free(rho);
}

/*
 * Vector-Jacobian product of warp + composite for N views: given dL/dC_i (g_out[N][H][W][3]),
 * accumulate dL/dM into grad[D][H][W][4] (which the caller zeroes).  For each view pixel:
 *   dC/dc_d     = alpha_d T_d                         (Eq. eq_gradient)
 *   dC/dalpha_d = T_d (c_d - B_d),   B_d = over-composite of the planes below d
 * with T_d = prod_{j>d}(1 - alpha_j); then the bilinear transpose scatters the per-sample
 * gradient onto the four taps.  No division by (1 - alpha).
 */
/* Per-sample gradient of plane d at one view pixel: dC/dc_d and dC/dalpha_d contracted with r. */
static void sample_gradient(const double* m, double Td, const double* B, const double* r, double g[4]) {
    for (int c = 0; c < 3; ++c) g[c] = Td * m[3] * r[c];
    g[3] = 0.0;
    for (int c = 0; c < 3; ++c) g[3] += Td * (m[c] - B[c]) * r[c];
}

#ifndef _OPENMP
void orc_vjp(const double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
             const orc_camera* views, int N, const double* g_out, double* grad) {
    double* rho = (double*)malloc(sizeof(double) * D);
    sample_t* smp = (sample_t*)malloc(sizeof(sample_t) * D);
    double* T = (double*)malloc(sizeof(double) * D);
    orc_plane_inverse_depths(D, near_, far_, rho);
    for (int i = 0; i < N; ++i)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const double* r = g_out + (((size_t)i * H + y) * W + x) * 3;
                double Tr = 1.0;
                for (int d = D - 1; d >= 0; --d) {
                    double px, py;
                    int ok = orc_view_to_ref(ref, &views[i], 1.0 / rho[d], x, y, &px, &py);
                    sample_plane(M, d, H, W, ok, px, py, &smp[d]);
                    T[d] = Tr;
                    Tr *= (1.0 - smp[d].m[3]);
                }
                double B[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d) {
                    const double* m = smp[d].m;
                    double g[4];
                    sample_gradient(m, T[d], B, r, g);
                    for (int c = 0; c < 3; ++c) B[c] = m[c] * m[3] + (1.0 - m[3]) * B[c];
                    for (int k = 0; k < 4; ++k) {
                        if (smp[d].w[k] == 0.0) continue;
                        double* gp = grad + (((size_t)d * H + smp[d].ty[k]) * W + smp[d].tx[k]) * 4;
                        for (int c = 0; c < 4; ++c) gp[c] += smp[d].w[k] * g[c];
                    }
                }
            }
    free(T);
    free(smp);
    free(rho);
}
#else
/*
 * The same vector-Jacobian product on the host's cores (the OpenMP build, used to time the
 * oracle on all cores).  Bit-identical to the serial loop above: a voxel of plane d receives
 * contributions only from samples of plane d, so for each view and each band of rows, phase 1
 * forms every sample and its per-sample gradient (rows in parallel, the serial arithmetic),
 * and phase 2 adds them plane by plane (planes in parallel), each plane in the serial order of
 * (row, column, tap).  Views and bands are taken in order.
 */
#define ORC_VJP_BAND 16
void orc_vjp(const double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
             const orc_camera* views, int N, const double* g_out, double* grad) {
    double* rho = (double*)malloc(sizeof(double) * D);
    orc_plane_inverse_depths(D, near_, far_, rho);
    const size_t band_px = (size_t)ORC_VJP_BAND * W;
    sample_t* smp = (sample_t*)malloc(sizeof(sample_t) * D * band_px); /* [d][band row][x] */
    double* gs = (double*)malloc(sizeof(double) * 4 * D * band_px);    /* per-sample gradients */
    for (int i = 0; i < N; ++i)
        for (int y0 = 0; y0 < H; y0 += ORC_VJP_BAND) {
            const int rows = H - y0 < ORC_VJP_BAND ? H - y0 : ORC_VJP_BAND;
#pragma omp parallel for schedule(static)
            for (int yy = 0; yy < rows; ++yy) {
                double* T = (double*)malloc(sizeof(double) * D);
                const int y = y0 + yy;
                for (int x = 0; x < W; ++x) {
                    const double* r = g_out + (((size_t)i * H + y) * W + x) * 3;
                    const size_t q = (size_t)yy * W + x;
                    double Tr = 1.0;
                    for (int d = D - 1; d >= 0; --d) {
                        double px, py;
                        int ok = orc_view_to_ref(ref, &views[i], 1.0 / rho[d], x, y, &px, &py);
                        sample_plane(M, d, H, W, ok, px, py, &smp[d * band_px + q]);
                        T[d] = Tr;
                        Tr *= (1.0 - smp[d * band_px + q].m[3]);
                    }
                    double B[3] = {0, 0, 0};
                    for (int d = 0; d < D; ++d) {
                        const double* m = smp[d * band_px + q].m;
                        sample_gradient(m, T[d], B, r, gs + (d * band_px + q) * 4);
                        for (int c = 0; c < 3; ++c) B[c] = m[c] * m[3] + (1.0 - m[3]) * B[c];
                    }
                }
                free(T);
            }
#pragma omp parallel for schedule(static)
            for (int d = 0; d < D; ++d)
                for (size_t q = 0; q < (size_t)rows * W; ++q) {
                    const sample_t* s = &smp[d * band_px + q];
                    const double* g = gs + (d * band_px + q) * 4;
                    for (int k = 0; k < 4; ++k) {
                        if (s->w[k] == 0.0) continue;
                        double* gp = grad + (((size_t)d * H + s->ty[k]) * W + s->tx[k]) * 4;
                        for (int c = 0; c < 4; ++c) gp[c] += s->w[k] * g[c];
                    }
                }
        }
    free(gs);
    free(smp);
    free(rho);
}
#endif

/*
 * Photometric loss of N views and, if grad != NULL, its gradient dL/dM (dense, overwritten).
 * renders (optional) receives the N rendered views.  Returns L.
 */
double orc_loss_grad(const double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                     const double* images, const orc_camera* views, int N, double* grad, double* renders) {
    size_t npx = (size_t)H * W * 3;
    double* Ct = (double*)malloc(sizeof(double) * npx * N);
    for (int i = 0; i < N; ++i) orc_render(M, D, H, W, near_, far_, ref, &views[i], Ct + i * npx);
    double L = 0.0;
    double* r = (double*)malloc(sizeof(double) * npx * N);
    for (size_t j = 0; j < npx * (size_t)N; ++j) {
        double e = Ct[j] - images[j];
        L += e * e;
        r[j] = e / N;
    }
    L /= (2.0 * N);
    if (grad) {
        memset(grad, 0, sizeof(double) * (size_t)D * H * W * 4);
        orc_vjp(M, D, H, W, near_, far_, ref, views, N, r, grad);
    }
    if (renders) memcpy(renders, Ct, sizeof(double) * npx * N);
    free(r);
    free(Ct);
    return L;
}

/*
 * dL/dM of the photometric loss (the gradient orc_loss_grad returns) at n chosen voxels
 * (ds[j], ys[j], xs[j]), out[n][4], by brute force over the view pixels: a view pixel q adds
 * w_tap * dL/dm_d (Eq. eq_gradient, as in orc_vjp) when the voxel is one of the four taps of
 * its sample of plane d.  The candidates are the view pixels within `radius` of the point
 * where the voxel's centre on plane d projects into the view (Eq. eq_homo's inverse warp);
 * every other view pixel's sample of plane d lies more than a pixel away from the voxel for
 * the near-identity warps of forward-facing views.  Views, then candidates in row-major order,
 * as orc_vjp visits them, so each voxel's sum is formed in the same order.  For outputs the
 * dense gradient would be too large to form (one voxel needs N (2 radius + 1)^2 composites).
 */
int orc_ref_to_view(const orc_camera* ref, const orc_camera* view, double z, double u, double v, double* x,
                    double* y);

void orc_grad_voxels(const double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                     const double* images, const orc_camera* views, int N, int n, const int* ds, const int* ys,
                     const int* xs, int radius, double* out) {
    double* rho = (double*)malloc(sizeof(double) * D);
    orc_plane_inverse_depths(D, near_, far_, rho);
#pragma omp parallel for schedule(dynamic, 8)
    for (int j = 0; j < n; ++j) {
        sample_t* smp = (sample_t*)malloc(sizeof(sample_t) * D);
        double* T = (double*)malloc(sizeof(double) * D);
        const int d = ds[j], y = ys[j], x = xs[j];
        double acc[4] = {0, 0, 0, 0};
        for (int i = 0; i < N; ++i) {
            double u0, v0;
            if (!orc_ref_to_view(ref, &views[i], 1.0 / rho[d], x, y, &u0, &v0)) continue;
            if (!(fabs(u0) < 1e7) || !(fabs(v0) < 1e7)) continue;
            const int cu = (int)floor(u0), cv = (int)floor(v0);
            for (int qy = cv - radius; qy <= cv + radius + 1; ++qy) {
                if (qy < 0 || qy >= H) continue;
                for (int qx = cu - radius; qx <= cu + radius + 1; ++qx) {
                    if (qx < 0 || qx >= W) continue;
                    double px, py;
                    int ok = orc_view_to_ref(ref, &views[i], 1.0 / rho[d], qx, qy, &px, &py);
                    sample_t s;
                    sample_plane(M, d, H, W, ok, px, py, &s);
                    int kk = -1;
                    for (int k = 0; k < 4; ++k)
                        if (s.w[k] != 0.0 && s.tx[k] == x && s.ty[k] == y) kk = k;
                    if (kk < 0) continue;
                    /* the view pixel's composite, residual, transmittances and below-composite */
                    double C[3];
                    render_pixel(M, D, H, W, rho, ref, &views[i], qx, qy, C);
                    double r[3];
                    for (int c = 0; c < 3; ++c)
                        r[c] = (C[c] - images[(((size_t)i * H + qy) * W + qx) * 3 + c]) / N;
                    double Tr = 1.0;
                    for (int e = D - 1; e >= 0; --e) {
                        double ex, ey;
                        int oke = orc_view_to_ref(ref, &views[i], 1.0 / rho[e], qx, qy, &ex, &ey);
                        sample_plane(M, e, H, W, oke, ex, ey, &smp[e]);
                        T[e] = Tr;
                        Tr *= (1.0 - smp[e].m[3]);
                    }
                    double B[3] = {0, 0, 0};
                    for (int e = 0; e < d; ++e)
                        for (int c = 0; c < 3; ++c) B[c] = smp[e].m[c] * smp[e].m[3] + (1.0 - smp[e].m[3]) * B[c];
                    double g[4];
                    sample_gradient(smp[d].m, T[d], B, r, g);
                    for (int c = 0; c < 4; ++c) acc[c] += smp[d].w[kk] * g[c];
                }
            }
        }
        for (int c = 0; c < 4; ++c) out[(size_t)j * 4 + c] = acc[c];
        free(T);
        free(smp);
    }
    free(rho);
}

/* ------------------------------------------------------------ sparsification */

/* Reference-view alpha weights A_d = alpha_d prod_{j>d}(1 - alpha_j)  (Eq. eq_gradient, eq_overA). */
void orc_alpha_weights(const double* M, int D, int H, int W, double* A) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int d = 0; d < D; ++d) {
                double a = M[(((size_t)d * H + y) * W + x) * 4 + 3];
                double T = 1.0;
                for (int j = d + 1; j < D; ++j) T *= (1.0 - M[(((size_t)j * H + y) * W + x) * 4 + 3]);
                A[((size_t)d * H + y) * W + x] = a * T;
            }
}

/*
 * Top-k along depth: the k planes with the largest key, ties to the lower plane index;
 * S[j][y][x] lists them in ascending plane order, mask[y][x] has bit d set for each.
 * Written as the definition: sort the D (key, d) pairs by (key descending, d ascending)
 * and keep the first k.
 */
void orc_select_topk(const double* A, int D, int H, int W, int k, uint8_t* S, uint64_t* mask) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        int* order = (int*)malloc(sizeof(int) * D);
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            for (int d = 0; d < D; ++d) order[d] = d;
            /* insertion sort by (A desc, d asc) */
            for (int a = 1; a < D; ++a) {
                int cur = order[a];
                double ka = A[(size_t)cur * H * W + p];
                int b = a - 1;
                while (b >= 0) {
                    int o = order[b];
                    double kb = A[(size_t)o * H * W + p];
                    int before = (ka > kb) || (ka == kb && cur < o);
                    if (!before) break;
                    order[b + 1] = o;
                    --b;
                }
                order[b + 1] = cur;
            }
            uint64_t mk = 0;
            for (int j = 0; j < k; ++j) mk |= (uint64_t)1 << order[j];
            mask[p] = mk;
            int j = 0;
            for (int d = 0; d < D; ++d)
                if (mk >> d & 1) S[(size_t)j++ * H * W + p] = (uint8_t)d;
        }
        free(order);
    }
}

/*
 * MVS-sampling selection (the ablation alternative of Sec. 3.3 and Sec. 5.5): the plane
 * with the largest key (ties to the lower index) and its (k-1)/2 neighbours on each side,
 * i.e. the k consecutive planes starting at argmax - floor((k-1)/2), shifted to stay in
 * [0, D).  S ascending, mask with bit d per kept plane.
 */
void orc_select_mvs(const double* A, int D, int H, int W, int k, uint8_t* S, uint64_t* mask) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            int best = 0;
            for (int d = 1; d < D; ++d)
                if (A[(size_t)d * H * W + p] > A[(size_t)best * H * W + p]) best = d;
            int start = best - (k - 1) / 2;
            if (start > D - k) start = D - k;
            if (start < 0) start = 0;
            uint64_t mk = 0;
            for (int j = 0; j < k; ++j) {
                mk |= (uint64_t)1 << (start + j);
                S[(size_t)j * H * W + p] = (uint8_t)(start + j);
            }
            mask[p] = mk;
        }
}

/*
 * Gradient of the sparsity loss of Sec. 3.4, L_s = mean_{h,w,d} log(1.5 - |0.5 - alpha|),
 * with respect to one alpha of an MPI of D x H x W voxels:
 *   dL_s/dalpha = sign(0.5 - alpha) / ((1.5 - |0.5 - alpha|) H W D)   (0 at alpha = 0.5).
 */
double orc_sparsity_grad(double alpha, int D, int H, int W) {
    double s = (alpha < 0.5) ? 1.0 : (alpha > 0.5 ? -1.0 : 0.0);
    return s / ((1.5 - fabs(0.5 - alpha)) * (double)H * W * D);
}

/* L_s itself (mean of log(1.5 - |0.5 - alpha|) over all voxels). */
double orc_sparsity_loss(const double* M, int D, int H, int W) {
    double acc = 0.0;
    for (size_t v = 0; v < (size_t)D * H * W; ++v) acc += log(1.5 - fabs(0.5 - M[v * 4 + 3]));
    return acc / ((double)D * H * W);
}

/* ------------------------------------------------------------------ pyramid */

/* 2x2 box average of P stacked [H][W][C] slices -> [H/2][W/2][C]. */
void orc_downsample2(const double* x, int P, int H, int W, int C, double* y) {
    int h = H / 2, w = W / 2;
    for (int s = 0; s < P; ++s)
        for (int yy = 0; yy < h; ++yy)
            for (int xx = 0; xx < w; ++xx)
                for (int c = 0; c < C; ++c) {
                    const double* b = x + (size_t)s * H * W * C;
                    double v = b[((size_t)(2 * yy) * W + 2 * xx) * C + c] + b[((size_t)(2 * yy) * W + 2 * xx + 1) * C + c] +
                               b[((size_t)(2 * yy + 1) * W + 2 * xx) * C + c] + b[((size_t)(2 * yy + 1) * W + 2 * xx + 1) * C + c];
                    y[((size_t)s * h * w + (size_t)yy * w + xx) * C + c] = 0.25 * v;
                }
}

/* Down^l: l successive 2x2 box averages.  Returns a malloc'd buffer (caller frees). */
static double* down_levels(const double* x, int P, int H, int W, int C, int level) {
    size_t n = (size_t)P * H * W * C;
    double* cur = (double*)malloc(sizeof(double) * n);
    memcpy(cur, x, sizeof(double) * n);
    for (int l = 0; l < level; ++l) {
        double* nxt = (double*)malloc(sizeof(double) * (size_t)P * (H >> (l + 1)) * (W >> (l + 1)) * C);
        orc_downsample2(cur, P, H >> l, W >> l, C, nxt);
        free(cur);
        cur = nxt;
    }
    return cur;
}

void orc_down_levels(const double* x, int P, int H, int W, int C, int level, double* y) {
    double* r = down_levels(x, P, H, W, C, level);
    memcpy(y, r, sizeof(double) * (size_t)P * (H >> level) * (W >> level) * C);
    free(r);
}

/* ---------------------------------------------------- gradient volume (Sec. 3.3) */

/*
 * Inverse homographic warp of Eq. (eq_homo): reference pixel (u,v) on the plane z_ref = z
 * -> pixel (x,y) of camera `view`.  Back-projects the reference pixel to depth z in the
 * reference frame, takes the point to the world frame and into the view camera, projects.
 * Returns 0 when the point is not in front of the view.
 */
int orc_ref_to_view(const orc_camera* ref, const orc_camera* view, double z, double u, double v, double* x,
                    double* y) {
    double Kinv[9];
    inv3(ref->K, Kinv);
    double Xr[3];
    for (int a = 0; a < 3; ++a) Xr[a] = z * (Kinv[a * 3 + 0] * u + Kinv[a * 3 + 1] * v + Kinv[a * 3 + 2]);
    /* world point X_w = R_r^T (X_r - t_r) */
    double Xw[3];
    for (int a = 0; a < 3; ++a)
        Xw[a] = ref->R[0 * 3 + a] * (Xr[0] - ref->t[0]) + ref->R[1 * 3 + a] * (Xr[1] - ref->t[1]) +
                ref->R[2 * 3 + a] * (Xr[2] - ref->t[2]);
    double Xv[3];
    for (int a = 0; a < 3; ++a)
        Xv[a] = view->R[a * 3 + 0] * Xw[0] + view->R[a * 3 + 1] * Xw[1] + view->R[a * 3 + 2] * Xw[2] + view->t[a];
    if (!(Xv[2] > 0.0)) return 0;
    const double* K = view->K;
    double hx = K[0] * Xv[0] + K[1] * Xv[1] + K[2] * Xv[2];
    double hy = K[3] * Xv[0] + K[4] * Xv[1] + K[5] * Xv[2];
    double hz = K[6] * Xv[0] + K[7] * Xv[1] + K[8] * Xv[2];
    *x = hx / hz;
    *y = hy / hz;
    return 1;
}

/* Bilinear sample (zero padding per tap) of a [H][W][C] image at (x, y): out[C]. */
static void sample_image(const double* img, int H, int W, int C, int valid, double x, double y, double* out) {
    for (int c = 0; c < C; ++c) out[c] = 0.0;
    if (!valid) return;
    int tx[4], ty[4];
    double w[4];
    bilinear_taps(x, y, W, H, tx, ty, w);
    for (int k = 0; k < 4; ++k) {
        if (w[k] == 0.0) continue;
        const double* v = img + ((size_t)ty[k] * W + tx[k]) * C;
        for (int c = 0; c < C; ++c) out[c] += w[k] * v[c];
    }
}

/*
 * Alpha weights of the MPI warped into a view (Eq. eq_gradient applied to M_i):
 * A[d][y][x] = alpha_d(q) prod_{j>d} (1 - alpha_j(q)), alpha_j(q) the alpha of plane j
 * sampled along the ray of view pixel q = (x, y) (the same warp as the render).  The view
 * has the MPI's size H x W.
 */
void orc_view_alpha_weights(const double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                            const orc_camera* view, double* A) {
    double* rho = (double*)malloc(sizeof(double) * D);
    double* alpha = (double*)malloc(sizeof(double) * D);
    orc_plane_inverse_depths(D, near_, far_, rho);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            for (int d = 0; d < D; ++d) {
                double px, py;
                int ok = orc_view_to_ref(ref, view, 1.0 / rho[d], x, y, &px, &py);
                sample_t s;
                sample_plane(M, d, H, W, ok, px, py, &s);
                alpha[d] = s.m[3];
            }
            for (int d = 0; d < D; ++d) {
                double T = 1.0;
                for (int j = d + 1; j < D; ++j) T *= (1.0 - alpha[j]);
                A[((size_t)d * H + y) * W + x] = alpha[d] * T;
            }
        }
    free(alpha);
    free(rho);
}

/*
 * Plane sweep volume of one source view (Sec. 3.2): P[d][y][x][3] = grid_sample of the
 * view's image [H][W][3] at the inverse-warped reference pixel (x, y) of plane d
 * (orc_ref_to_view), bilinear with zero padding.
 */
void orc_psv_view(const double* image, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                  const orc_camera* view, double* P) {
    double* rho = (double*)malloc(sizeof(double) * D);
    orc_plane_inverse_depths(D, near_, far_, rho);
    for (int d = 0; d < D; ++d)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double vx, vy;
                int ok = orc_ref_to_view(ref, view, 1.0 / rho[d], x, y, &vx, &vy);
                sample_image(image, H, W, 3, ok, vx, vy, P + (((size_t)d * H + y) * W + x) * 3);
            }
    free(rho);
}

/*
 * Inverse warp of a per-plane stack of view-frame maps X[D][H][W] (one channel) into the
 * reference frame: out[d][y][x] = bilinear(X[d], orc_ref_to_view(ref, view, z_d, x, y)).
 */
void orc_inverse_warp_stack(const double* X, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                            const orc_camera* view, double* out) {
    double* rho = (double*)malloc(sizeof(double) * D);
    orc_plane_inverse_depths(D, near_, far_, rho);
    for (int d = 0; d < D; ++d)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double vx, vy;
                int ok = orc_ref_to_view(ref, view, 1.0 / rho[d], x, y, &vx, &vy);
                sample_image(X + (size_t)d * H * W, H, W, 1, ok, vx, vy, out + ((size_t)d * H + y) * W + x);
            }
    free(rho);
}

/*
 * Sparsified gradient volume of one HSGD iteration at level l (Sec. 3.3, Eq.
 * eq_simplifiedGradients and eq_V): V = [P_l, A^{w^-1}_1 .. A^{w^-1}_N, M_l] with
 *   P_l        = Down^l of the full-resolution plane sweep volume of the N source views
 *                (Sec. 3.2, "we downsample it hierarchically"), 3N channels, view-major;
 *   A^{w^-1}_i = the alpha weights of M_l warped into view i at level l, inverse-warped
 *                back to the reference frame, N channels;
 *   M_l        = Down^l(M), 4 channels (R, G, B, alpha);
 * compacted along depth to the k planes of S (Sec. 3.3, "Gradient Sparsification"):
 *   Vs[c][j][y][x] = V[c][S[j][y][x]][y][x],  C = 4N + 4 channels.
 * S is the selection of orc_hsgd_step2 on M_l (top-k or MVS window) or S_pin; S_out gets it.
 */
int orc_gradient_volume(const double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                        const double* images, const orc_camera* views, int N, int k, int level, int selection,
                        const uint8_t* S_pin, uint8_t* S_out, double* Vs) {
    if (k < 1 || k > D || D > 64 || (H % (1 << level)) || (W % (1 << level))) return 1;
    const int h = H >> level, w = W >> level, C = 4 * N + 4;
    const size_t hw = (size_t)h * w;
    double* Ml = down_levels(M, D, H, W, 4, level);
    orc_camera refl;
    orc_camera_at_level(ref, level, &refl);
    uint8_t* S = (uint8_t*)malloc((size_t)k * hw);
    if (S_pin) {
        memcpy(S, S_pin, (size_t)k * hw);
    } else {
        double* A = (double*)malloc(sizeof(double) * (size_t)D * hw);
        uint64_t* mk = (uint64_t*)malloc(sizeof(uint64_t) * hw);
        orc_alpha_weights(Ml, D, h, w, A);
        if (selection == 1)
            orc_select_mvs(A, D, h, w, k, S, mk);
        else
            orc_select_topk(A, D, h, w, k, S, mk);
        free(mk);
        free(A);
    }
    double* Pfull = (double*)malloc(sizeof(double) * (size_t)D * H * W * 3);
    double* Aview = (double*)malloc(sizeof(double) * (size_t)D * hw);
    double* Ainv = (double*)malloc(sizeof(double) * (size_t)D * hw);
    for (int i = 0; i < N; ++i) {
        orc_psv_view(images + (size_t)i * H * W * 3, D, H, W, near_, far_, ref, &views[i], Pfull);
        double* Pl = down_levels(Pfull, D, H, W, 3, level);
        orc_camera vl;
        orc_camera_at_level(&views[i], level, &vl);
        orc_view_alpha_weights(Ml, D, h, w, near_, far_, &refl, &vl, Aview);
        orc_inverse_warp_stack(Aview, D, h, w, near_, far_, &refl, &vl, Ainv);
        for (int j = 0; j < k; ++j)
            for (size_t p = 0; p < hw; ++p) {
                const int d = S[(size_t)j * hw + p];
                for (int c = 0; c < 3; ++c)
                    Vs[((size_t)(3 * i + c) * k + j) * hw + p] = Pl[((size_t)d * hw + p) * 3 + c];
                Vs[((size_t)(3 * N + i) * k + j) * hw + p] = Ainv[(size_t)d * hw + p];
            }
        free(Pl);
    }
    for (int j = 0; j < k; ++j)
        for (size_t p = 0; p < hw; ++p) {
            const int d = S[(size_t)j * hw + p];
            for (int c = 0; c < 4; ++c) Vs[((size_t)(4 * N + c) * k + j) * hw + p] = Ml[((size_t)d * hw + p) * 4 + c];
        }
    if (S_out) memcpy(S_out, S, (size_t)k * hw);
    free(Ainv);
    free(Aview);
    free(Pfull);
    free(S);
    free(Ml);
    return 0;
}

/* ------------------------------------------------------------------- update */

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/*
 * One HSGD iteration at pyramid level `level` (Sec. 3.3), updating the full-resolution
 * MPI in place:
 *   M_l = Down^l(M), I_l = Down^l(I), cameras at level l;
 *   S   = top-k of A(M_l) (selection 0), the MVS-sampling window (selection 1), or S_pin;
 *   g  += lambda_s dL_s/dalpha on the alphas of M_l (the sparsity prior, when lambda_s != 0);
 *   g   = dL/dM_l (dense);
 *   M[d][Y][X] <- clamp(M[d][Y][X] - lambda g[d][Y>>l][X>>l]) for d in S[.][Y>>l][X>>l].
 * S_out (optional) receives the selection [k][H_l][W_l]; loss_out the loss at level l.
 */
int orc_hsgd_step2(double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                   const double* images, const orc_camera* views, int N, int k, double lambda, int clamp,
                   int level, int selection, double lambda_s, const uint8_t* S_pin, uint8_t* S_out,
                   double* loss_out) {
    if (k < 1 || k > D || D > 64 || (H % (1 << level)) || (W % (1 << level))) return 1;
    int h = H >> level, w = W >> level;
    double* Ml = down_levels(M, D, H, W, 4, level);
    double* Il = down_levels(images, N, H, W, 3, level);
    orc_camera refl;
    orc_camera_at_level(ref, level, &refl);
    orc_camera* vl = (orc_camera*)malloc(sizeof(orc_camera) * N);
    for (int i = 0; i < N; ++i) orc_camera_at_level(&views[i], level, &vl[i]);

    uint8_t* S = (uint8_t*)malloc((size_t)k * h * w);
    if (S_pin) {
        memcpy(S, S_pin, (size_t)k * h * w);
    } else {
        double* A = (double*)malloc(sizeof(double) * (size_t)D * h * w);
        uint64_t* mk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)h * w);
        orc_alpha_weights(Ml, D, h, w, A);
        if (selection == 1)
            orc_select_mvs(A, D, h, w, k, S, mk);
        else
            orc_select_topk(A, D, h, w, k, S, mk);
        free(mk);
        free(A);
    }
    double* g = (double*)malloc(sizeof(double) * (size_t)D * h * w * 4);
    double L = orc_loss_grad(Ml, D, h, w, near_, far_, &refl, Il, vl, N, g, NULL);
    /* prior phi = lambda_s L_s on the level-l MPI (Sec. 3.1's dphi/df with L_s of Sec. 3.4) */
    if (lambda_s != 0.0)
        for (size_t v = 0; v < (size_t)D * h * w; ++v)
            g[v * 4 + 3] += lambda_s * orc_sparsity_grad(Ml[v * 4 + 3], D, h, w);
#pragma omp parallel for schedule(static)
    for (int yy = 0; yy < h; ++yy)
        for (int xx = 0; xx < w; ++xx)
            for (int j = 0; j < k; ++j) {
                int d = S[(size_t)j * h * w + (size_t)yy * w + xx];
                const double* gd = g + (((size_t)d * h + yy) * w + xx) * 4;
                for (int Y = yy << level; Y < (yy + 1) << level; ++Y)
                    for (int X = xx << level; X < (xx + 1) << level; ++X)
                        for (int c = 0; c < 4; ++c) {
                            double* mv = M + (((size_t)d * H + Y) * W + X) * 4 + c;
                            double nv = *mv - lambda * gd[c];
                            *mv = clamp ? clamp01(nv) : nv;
                        }
            }
    if (S_out) memcpy(S_out, S, (size_t)k * h * w);
    if (loss_out) *loss_out = L;
    free(g);
    free(S);
    free(vl);
    free(Il);
    free(Ml);
    return 0;
}

int orc_hsgd_step(double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                  const double* images, const orc_camera* views, int N, int k, double lambda, int clamp,
                  int level, const uint8_t* S_pin, uint8_t* S_out, double* loss_out) {
    return orc_hsgd_step2(M, D, H, W, near_, far_, ref, images, views, N, k, lambda, clamp, level, 0, 0.0, S_pin,
                          S_out, loss_out);
}

/*
 * Dense analytic gradient descent step (Sec. 3.1) at level `level`, no sparsification:
 * every plane of every pixel takes the step.  The keep-everything case of HSGD must
 * reduce to this.
 */
int orc_gd_step(double* M, int D, int H, int W, double near_, double far_, const orc_camera* ref,
                const double* images, const orc_camera* views, int N, double lambda, int clamp, int level,
                double* loss_out) {
    if ((H % (1 << level)) || (W % (1 << level))) return 1;
    int h = H >> level, w = W >> level;
    double* Ml = down_levels(M, D, H, W, 4, level);
    double* Il = down_levels(images, N, H, W, 3, level);
    orc_camera refl;
    orc_camera_at_level(ref, level, &refl);
    orc_camera* vl = (orc_camera*)malloc(sizeof(orc_camera) * N);
    for (int i = 0; i < N; ++i) orc_camera_at_level(&views[i], level, &vl[i]);
    double* g = (double*)malloc(sizeof(double) * (size_t)D * h * w * 4);
    double L = orc_loss_grad(Ml, D, h, w, near_, far_, &refl, Il, vl, N, g, NULL);
    for (int d = 0; d < D; ++d)
        for (int Y = 0; Y < H; ++Y)
            for (int X = 0; X < W; ++X)
                for (int c = 0; c < 4; ++c) {
                    double* mv = M + (((size_t)d * H + Y) * W + X) * 4 + c;
                    double nv = *mv - lambda * g[(((size_t)d * h + (Y >> level)) * w + (X >> level)) * 4 + c];
                    *mv = clamp ? clamp01(nv) : nv;
                }
    if (loss_out) *loss_out = L;
    free(g);
    free(vl);
    free(Il);
    free(Ml);
    return 0;
}
