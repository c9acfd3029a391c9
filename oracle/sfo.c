/*
 * sfo.c -- FP64 single-threaded CPU oracle of the halfway-domain scene-flow
 * solve of Thies et al., "Real-time Halfway Domain Reconstruction of Motion
 * and Geometry" (arXiv 1610.07159).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the parity reference for the CUDA
 * library: it is called by the tests, by the package's smoke check and by the
 * benchmark's CPU-baseline leg, and by nothing on the product path. It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * It is written for a reader who checks it against the paper by eye: plain
 * loops, one step after another in the paper's order, no blocking, no fusion,
 * every accumulation in double precision.
 *
 * Conventions (the paper's notation, Section 3):
 *   images   imgs[c] for c = 0: I_0^0 (left, t0), 1: I_1^0 (right, t0),
 *            2: I_0^1 (left, t1), 3: I_1^1 (right, t1); row-major w*h.
 *   planes   per level and image: 3 planes (I, dI/dx, dI/dy), layout
 *            planes[((img*3 + plane)*h + y)*w + x].
 *   fields   per node 6 unknowns (s_x, s_y, m_x, m_y, d_x, d_y), stored
 *            component-major: F[comp*G + j*nx + i], G = nx*ny.
 *   system   block form A[n][q][r][c] (n node, q = 3*(dy+1) + (dx+1) the
 *            neighbour slot, 6x6 row-major block), b[n*6 + r].
 *
 * Readings where the paper is silent or ambiguous are marked [Cn] and match
 * the list of readings in the design notes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define SFO_MAX_LEVELS 8
#define SFO_MAX_GN 16
#define SFO_STEP_STATS 10
#define SFO_STATS_LEN (16 + SFO_MAX_LEVELS * SFO_MAX_GN * SFO_STEP_STATS)

enum { SFO_IRLS = 0, SFO_SQRT_PAPER = 1 };
enum { SFO_GRAD_BROX = 0, SFO_GRAD_LITERAL = 1 };
enum { SFO_WFEAT_EIG = 0, SFO_WFEAT_OFF = 1 };
enum { SFO_TEMPORAL_PROPAGATE = 0, SFO_TEMPORAL_COPY = 1, SFO_TEMPORAL_ZERO = 2 };
enum { SFO_SOLVER_PCG = 0, SFO_SOLVER_SCHWARZ = 1 };

typedef struct sfo_params {
    /* Table 1 (Appendix A) */
    double w_reg, w_photo, w_grad, w_epi, w_smooth, w_mag;
    double w_s, w_m, w_d, m_s, m_m, m_d;
    double eps;   /* pseudo-Huber epsilon, Eq. 12 */
    double eps_p; /* outlier threshold of W, Section 4.1; <= 0 disables W */
    double F[9];  /* fundamental matrix, finest-level pixels, row-major */
    int gn_iters[SFO_MAX_LEVELS];  /* per level, index 0 = finest */
    int pcg_iters[SFO_MAX_LEVELS];
    int robust_mode, grad_mode, wfeat_mode;
    double wfeat_gain, wfeat_tau;
    int temporal_mode, max_backtracks;
    /* linear solver of each Gauss-Newton step (Section 5.2) [C24]: global
     * Jacobi-PCG with pcg_iters iterations, or alternating Schwarz with
     * pcg_iters sweeps over square subdomains of schwarz_tile x schwarz_tile
     * nodes plus schwarz_overlap nodes of overlap, each subdomain solved by
     * patch_iters local PCG iterations */
    int solver;
    int patch_iters[SFO_MAX_LEVELS];
    int schwarz_tile, schwarz_overlap;
    /* per-level maps of Algorithm 1, computed after a level's solve and
     * prolongated to the next finer level: occlusion maps V (Section 4.1,
     * Section 5.3) [C25] with the closeness tolerance occ_tau (level pixels
     * of disparity), and illumination correction maps (Section 5.3) [C26]
     * with the Gaussian's sigma (level pixels) */
    int occlusion;
    double occ_tau;
    int illumination;
    double illum_sigma;
} sfo_params;

/* The maps a level's data terms use (NULL members: V = 1, no correction):
 * V[h][w] visibility, L[2][h][w] the illumination difference of the right
 * camera at times 0 and 1, in the level's reference frame. */
typedef struct sfo_maps {
    const unsigned char* V;
    const double* L;
} sfo_maps;

/* Sign of stereo, motion and difference flow in each image's sample position
 * (Eqs. 1-6): image 0 at x-s-m+d, 1 at x+s-m-d, 2 at x-s+m-d, 3 at x+s+m+d. */
static const double SIGN[4][3] = {
    {-1.0, -1.0, +1.0},
    {+1.0, -1.0, -1.0},
    {-1.0, +1.0, -1.0},
    {+1.0, +1.0, +1.0},
};
/* The six consistency checks d_k = I_first(p_first) - I_second(p_second),
 * Eqs. 1-6 in order. */
static const int CHECK[6][2] = {{1, 0}, {3, 2}, {2, 0}, {3, 1}, {3, 0}, {2, 1}};

/* ------------------------------------------------------------------------ */
/* Image hierarchy (Section 5.3: mip-map pyramid, factor 2) [C5, C6]         */
/* ------------------------------------------------------------------------ */

void sfo_level_dims(int w0, int h0, int level, int* w, int* h)
{
    int a = w0, b = h0;
    for (int l = 0; l < level; ++l) {
        a = (a + 1) / 2;
        b = (b + 1) / 2;
    }
    *w = a;
    *h = b;
}

/* One mip-map step: 2x2 box average, ceil(w/2) x ceil(h/2), edge clamped. */
void sfo_downsample(int w, int h, const double* src, double* dst)
{
    int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
    for (int y = 0; y < h2; ++y)
        for (int x = 0; x < w2; ++x) {
            double acc = 0.0;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int xx = 2 * x + a, yy = 2 * y + b;
                    if (xx > w - 1) xx = w - 1;
                    if (yy > h - 1) yy = h - 1;
                    acc += src[yy * w + xx];
                }
            dst[y * w2 + x] = 0.25 * acc;
        }
}

/* Central differences with edge clamping. */
void sfo_gradients(int w, int h, const double* img, double* gx, double* gy)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int xm = x > 0 ? x - 1 : 0, xp = x < w - 1 ? x + 1 : w - 1;
            int ym = y > 0 ? y - 1 : 0, yp = y < h - 1 ? y + 1 : h - 1;
            gx[y * w + x] = 0.5 * (img[y * w + xp] - img[y * w + xm]);
            gy[y * w + x] = 0.5 * (img[yp * w + x] - img[ym * w + x]);
        }
}

/* Builds the planes (I, Gx, Gy) of the four images at one level from that
 * level's four intensity images. */
void sfo_level_planes(int w, int h, const double* imgs4, double* planes)
{
    size_t n = (size_t)w * h;
    for (int c = 0; c < 4; ++c) {
        const double* I = imgs4 + c * n;
        double* P = planes + (size_t)c * 3 * n;
        memcpy(P, I, n * sizeof(double));
        sfo_gradients(w, h, I, P + n, P + 2 * n);
    }
}

/* ------------------------------------------------------------------------ */
/* Bilinear sampling with derivative [C5, C7]                                */
/* ------------------------------------------------------------------------ */

/* Bilinear interpolation of plane P (w x h) at (px, py); the position is
 * clamped to [0, w-1] x [0, h-1]; the cell is min(floor(p), w-2). The
 * derivative is that of the bilinear interpolant, 0 along a clamped axis.
 *
 * The cell decision of one axis: position p on [0, n-1] -> clamped position,
 * cell min(floor(p), n-2) and whether p was clamped. */
static void axis_decision(int n, double p, double* cp, int* cell, int* clamped)
{
    *clamped = 0;
    *cp = p;
    if (p < 0.0) { *cp = 0.0; *clamped = 1; }
    if (p > n - 1) { *cp = n - 1; *clamped = 1; }
    *cell = (int)floor(*cp);
    if (*cell > n - 2) *cell = n - 2;
}

/* A cell decision given from outside (a record of another implementation,
 * see sfo_solve_frame): code = cell << 1 | clamped, or -1 for none. With a
 * given decision the interpolant of that cell is used: a clamped axis takes
 * the cell's edge value and derivative 0; otherwise the fraction p - cell
 * (slightly outside [0, 1] when the two decisions part). */
static double sample_decided(int w, int h, const double* P, double px, double py, int gx, int gy, double* dpx,
                             double* dpy)
{
    int clx, cly, ix, iy;
    double cx, cy;
    axis_decision(w, px, &cx, &ix, &clx);
    axis_decision(h, py, &cy, &iy, &cly);
    double fx = cx - ix, fy = cy - iy;
    if (gx >= 0) {
        ix = gx >> 1;
        clx = gx & 1;
        fx = clx ? (ix == 0 && px < 0.5 * (w - 1) ? 0.0 : 1.0) : px - ix;
    }
    if (gy >= 0) {
        iy = gy >> 1;
        cly = gy & 1;
        fy = cly ? (iy == 0 && py < 0.5 * (h - 1) ? 0.0 : 1.0) : py - iy;
    }
    double p00 = P[iy * w + ix], p10 = P[iy * w + ix + 1];
    double p01 = P[(iy + 1) * w + ix], p11 = P[(iy + 1) * w + ix + 1];
    double v = (1 - fx) * (1 - fy) * p00 + fx * (1 - fy) * p10 + (1 - fx) * fy * p01 + fx * fy * p11;
    if (dpx) *dpx = clx ? 0.0 : (1 - fy) * (p10 - p00) + fy * (p11 - p01);
    if (dpy) *dpy = cly ? 0.0 : (1 - fx) * (p01 - p00) + fx * (p11 - p10);
    return v;
}

double sfo_sample(int w, int h, const double* P, double px, double py, double* dpx, double* dpy)
{
    return sample_decided(w, h, P, px, py, -1, -1, dpx, dpy);
}

/* Same rule on a node grid (nx x ny): used by prolongation and the temporal
 * transfer, no derivative. */
static double grid_sample(int nx, int ny, const double* Fc, double u, double v)
{
    return sfo_sample(nx, ny, Fc, u, v, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Warp grid (Section 3.3, Eq. 7) [C8]                                       */
/* ------------------------------------------------------------------------ */

/* The four nodes and bilinear weights of pixel (x, y); node (i, j) sits at
 * level pixel (i*s, j*s); pixels past the last node clamp to it. */
void sfo_grid_weights(int x, int y, int s, int nx, int ny, int nodes[4], double wts[4])
{
    double u = (double)x / s, v = (double)y / s;
    if (u > nx - 1) u = nx - 1;
    if (v > ny - 1) v = ny - 1;
    int i0 = (int)floor(u), j0 = (int)floor(v);
    if (i0 > nx - 2) i0 = nx - 2;
    if (j0 > ny - 2) j0 = ny - 2;
    double a = u - i0, b = v - j0;
    nodes[0] = j0 * nx + i0;
    nodes[1] = j0 * nx + i0 + 1;
    nodes[2] = (j0 + 1) * nx + i0;
    nodes[3] = (j0 + 1) * nx + i0 + 1;
    wts[0] = (1 - a) * (1 - b);
    wts[1] = a * (1 - b);
    wts[2] = (1 - a) * b;
    wts[3] = a * b;
}

/* Per-pixel fields f[6] = sum_k alpha_k T_k (Eq. 7). */
static void pixel_fields(int x, int y, int s, int nx, int ny, const double* T, double f[6])
{
    int nd[4];
    double al[4];
    int G = nx * ny;
    sfo_grid_weights(x, y, s, nx, ny, nd, al);
    for (int c = 0; c < 6; ++c) {
        f[c] = 0.0;
        for (int k = 0; k < 4; ++k) f[c] += al[k] * T[c * G + nd[k]];
    }
}

/* ------------------------------------------------------------------------ */
/* Consistency checks (Section 3.2, Eqs. 1-6) and their analytic Jacobian    */
/* ------------------------------------------------------------------------ */

/* For pixel (x, y) with fields f = (s, m, d): the six brightness checks e[k],
 * the six gradient-constancy 2-vectors g[2k], g[2k+1] (difference of the
 * warped image gradients [C2]) and their Jacobians w.r.t. the six pixel
 * fields (Je[k][u], Jg[2k+a][u], u = sx, sy, mx, my, dx, dy). dec is NULL or
 * gives, per image c, a cell decision for x (dec[2c]) and y (dec[2c+1]) as
 * sample_decided takes it (-1: the oracle's own). corr is NULL or the
 * illumination difference (time 0, time 1) at this pixel, subtracted from the
 * right images' intensities (a constant of the level: the Jacobians keep). */
static void pixel_terms_decided(int w, int h, const double* planes, double x, double y, const double f[6],
                                const int dec[8], const double* corr, double e[6], double g[12], double Je[36],
                                double Jg[72])
{
    size_t n = (size_t)w * h;
    double val[4][3], dx[4][3], dy[4][3];
    for (int c = 0; c < 4; ++c) {
        double px = x + SIGN[c][0] * f[0] + SIGN[c][1] * f[2] + SIGN[c][2] * f[4];
        double py = y + SIGN[c][0] * f[1] + SIGN[c][1] * f[3] + SIGN[c][2] * f[5];
        int gx = dec ? dec[2 * c] : -1, gy = dec ? dec[2 * c + 1] : -1;
        for (int p = 0; p < 3; ++p)
            val[c][p] = sample_decided(w, h, planes + (size_t)(c * 3 + p) * n, px, py, gx, gy, &dx[c][p], &dy[c][p]);
    }
    if (corr) {
        /* illumination correction [C26]: the right images (1 at time 0, 3 at
         * time 1) less the right camera's illumination difference */
        val[1][0] -= corr[0];
        val[3][0] -= corr[1];
    }
    for (int k = 0; k < 6; ++k) {
        int F = CHECK[k][0], S = CHECK[k][1];
        e[k] = val[F][0] - val[S][0];
        g[2 * k] = val[F][1] - val[S][1];
        g[2 * k + 1] = val[F][2] - val[S][2];
        for (int fld = 0; fld < 3; ++fld) {
            double sF = SIGN[F][fld], sS = SIGN[S][fld];
            /* d p_X.x / d field_x = sign, and likewise for y */
            if (Je) {
                Je[k * 6 + 2 * fld + 0] = sF * dx[F][0] - sS * dx[S][0];
                Je[k * 6 + 2 * fld + 1] = sF * dy[F][0] - sS * dy[S][0];
            }
            if (Jg) {
                for (int a = 0; a < 2; ++a) {
                    Jg[(2 * k + a) * 6 + 2 * fld + 0] = sF * dx[F][1 + a] - sS * dx[S][1 + a];
                    Jg[(2 * k + a) * 6 + 2 * fld + 1] = sF * dy[F][1 + a] - sS * dy[S][1 + a];
                }
            }
        }
    }
}

void sfo_pixel_terms(int w, int h, const double* planes, double x, double y, const double f[6],
                     double e[6], double g[12], double Je[36], double Jg[72])
{
    pixel_terms_decided(w, h, planes, x, y, f, NULL, NULL, e, g, Je, Jg);
}

/* The correction of pixel p from the maps (NULL without illumination maps). */
static const double* pixel_corr(const sfo_maps* mp, int w, int h, int p, double buf[2])
{
    if (!mp || !mp->L) return NULL;
    buf[0] = mp->L[p];
    buf[1] = mp->L[(size_t)w * h + p];
    return buf;
}

/* Halfway image: mean of the four warped samples (used by the feature weight). */
static double halfway_value(int w, int h, const double* planes, int x, int y, const double f[6])
{
    size_t n = (size_t)w * h;
    double acc = 0.0;
    for (int c = 0; c < 4; ++c) {
        double px = x + SIGN[c][0] * f[0] + SIGN[c][1] * f[2] + SIGN[c][2] * f[4];
        double py = y + SIGN[c][0] * f[1] + SIGN[c][1] * f[3] + SIGN[c][2] * f[5];
        acc += sfo_sample(w, h, planes + (size_t)(c * 3) * n, px, py, NULL, NULL);
    }
    return 0.25 * acc;
}

/* ------------------------------------------------------------------------ */
/* Robust penalties (Eq. 12, Eq. 11, Eq. 13) [C1, C3]                        */
/* ------------------------------------------------------------------------ */

static double phi(double x, double eps) { return sqrt(x * x + eps * eps); }

/* Gradient-term penalty of |g|^2: Brox convention sqrt(|g|^2 + eps^2) by
 * default, the literal reading sqrt(|g|^4 + eps^2) on request. */
static double psi_grad(double q, double eps, int mode)
{
    return mode == SFO_GRAD_LITERAL ? sqrt(q * q + eps * eps) : sqrt(q + eps * eps);
}

/* d psi / d g = coef * g; returns coef. */
static double psi_grad_coef(double q, double eps, int mode)
{
    return mode == SFO_GRAD_LITERAL ? 2.0 * q / sqrt(q * q + eps * eps) : 1.0 / sqrt(q + eps * eps);
}

/* W (Section 4.1): 1 if the largest brightness check is below eps_p [C11]. */
static int outlier_weight(const double e[6], double eps_p)
{
    if (eps_p <= 0.0) return 1;
    double mx = 0.0;
    for (int k = 0; k < 6; ++k)
        if (fabs(e[k]) > mx) mx = fabs(e[k]);
    return mx < eps_p ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Per-level helpers                                                          */
/* ------------------------------------------------------------------------ */

/* Fundamental matrix in level-l pixels: S F S rescaled to the Frobenius norm
 * of F, S = diag(2^l, 2^l, 1) [C14]. */
void sfo_level_F(const double F[9], int level, double Fl[9])
{
    double sc[3] = {ldexp(1.0, level), ldexp(1.0, level), 1.0};
    double n0 = 0.0, n1 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Fl[a * 3 + b] = sc[a] * F[a * 3 + b] * sc[b];
            n0 += F[a * 3 + b] * F[a * 3 + b];
            n1 += Fl[a * 3 + b] * Fl[a * 3 + b];
        }
    if (n1 > 0.0)
        for (int a = 0; a < 9; ++a) Fl[a] *= sqrt(n0 / n1);
}

/* Epipolar residuals of node position (X, Y) with totals t[6] (Eqs. 15-17):
 * r[t] = l_t^T F r_t, and their gradients J[t][6] w.r.t. the node totals. */
static void epipolar_terms(const double Fl[9], double X, double Y, const double t[6], double r[2], double J[12])
{
    /* signs (s, m, d) of l^0, r^0, l^1, r^1: those of images 0, 1, 2, 3 */
    for (int tt = 0; tt < 2; ++tt) {
        int il = tt == 0 ? 0 : 2, ir = tt == 0 ? 1 : 3;
        double l[3], rr[3];
        l[0] = X + SIGN[il][0] * t[0] + SIGN[il][1] * t[2] + SIGN[il][2] * t[4];
        l[1] = Y + SIGN[il][0] * t[1] + SIGN[il][1] * t[3] + SIGN[il][2] * t[5];
        l[2] = 1.0;
        rr[0] = X + SIGN[ir][0] * t[0] + SIGN[ir][1] * t[2] + SIGN[ir][2] * t[4];
        rr[1] = Y + SIGN[ir][0] * t[1] + SIGN[ir][1] * t[3] + SIGN[ir][2] * t[5];
        rr[2] = 1.0;
        double Fr[3], Ftl[3];
        for (int a = 0; a < 3; ++a) {
            Fr[a] = Fl[a * 3 + 0] * rr[0] + Fl[a * 3 + 1] * rr[1] + Fl[a * 3 + 2] * rr[2];
            Ftl[a] = Fl[0 * 3 + a] * l[0] + Fl[1 * 3 + a] * l[1] + Fl[2 * 3 + a] * l[2];
        }
        r[tt] = l[0] * Fr[0] + l[1] * Fr[1] + l[2] * Fr[2];
        for (int fld = 0; fld < 3; ++fld)
            for (int a = 0; a < 2; ++a)
                J[tt * 6 + 2 * fld + a] = SIGN[il][fld] * Fr[a] + SIGN[ir][fld] * Ftl[a];
    }
}

/* Halfway image of a level at totals T (Section 3.1: the reference frame
 * halfway between the four views): H(x) = mean of the four warped samples. */
void sfo_halfway_image(int w, int h, int s, int nx, int ny, const double* planes, const double* T, double* H)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double f[6];
            pixel_fields(x, y, s, nx, ny, T, f);
            H[y * w + x] = halfway_value(w, h, planes, x, y, f);
        }
}

/* Feature weight w_i of every node (Section 4.3) [C10]: structure tensor of
 * the halfway image over the 3x3 pixels at the node, w = 1 + g exp(-lmin/tau). */
void sfo_feature_weights(int w, int h, int s, int nx, int ny, const double* planes, const double* T,
                         const sfo_params* p, double* wf)
{
    int G = nx * ny;
    if (p->wfeat_mode == SFO_WFEAT_OFF) {
        for (int n = 0; n < G; ++n) wf[n] = 1.0;
        return;
    }
    double* H = (double*)malloc(sizeof(double) * w * h);
    sfo_halfway_image(w, h, s, nx, ny, planes, T, H);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double a = 0.0, b = 0.0, c = 0.0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int qx = i * s + dx, qy = j * s + dy;
                    qx = qx < 0 ? 0 : (qx > w - 1 ? w - 1 : qx);
                    qy = qy < 0 ? 0 : (qy > h - 1 ? h - 1 : qy);
                    int xm = qx > 0 ? qx - 1 : 0, xp = qx < w - 1 ? qx + 1 : w - 1;
                    int ym = qy > 0 ? qy - 1 : 0, yp = qy < h - 1 ? qy + 1 : h - 1;
                    double hx = 0.5 * (H[qy * w + xp] - H[qy * w + xm]);
                    double hy = 0.5 * (H[yp * w + qx] - H[ym * w + qx]);
                    a += hx * hx;
                    b += hx * hy;
                    c += hy * hy;
                }
            double lmin = 0.5 * (a + c) - sqrt(0.25 * (a - c) * (a - c) + b * b);
            if (lmin < 0.0) lmin = 0.0;
            wf[j * nx + i] = 1.0 + p->wfeat_gain * exp(-lmin / p->wfeat_tau);
        }
    free(H);
}

/* ------------------------------------------------------------------------ */
/* Energy (Eqs. 8-18) with W frozen                                           */
/* ------------------------------------------------------------------------ */

/* terms[0..4] = E_photo, E_grad, E_smooth, E_epi, E_mag (unweighted sums as
 * in Eqs. 11, 13, 14, 15, 18); returns the weighted total of Eqs. 8-10.
 * If W is NULL it is computed at this state (and written to Wout if given). */
static double energy_impl(int w, int h, int s, int nx, int ny, int level, const double* planes,
                          const double* base, const double* delta, const double* wf, const unsigned char* W,
                          const sfo_params* p, double terms[5], unsigned char* Wout, const sfo_maps* mp)
{
    int G = nx * ny;
    double* T = (double*)malloc(sizeof(double) * 6 * G);
    for (int a = 0; a < 6 * G; ++a) T[a] = base[a] + delta[a];
    double Ep = 0.0, Eg = 0.0, Es = 0.0, Ee = 0.0, Em = 0.0;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double f[6], e[6], g[12], cb[2];
            pixel_fields(x, y, s, nx, ny, T, f);
            pixel_terms_decided(w, h, planes, x, y, f, NULL, pixel_corr(mp, w, h, y * w + x, cb), e, g, NULL, NULL);
            int Wi = W ? W[y * w + x] : outlier_weight(e, p->eps_p);
            if (Wout) Wout[y * w + x] = (unsigned char)Wi;
            if (!Wi) continue;
            if (mp && mp->V && !mp->V[y * w + x]) continue; /* V of Eqs. 11 and 13 [C25] */
            for (int k = 0; k < 6; ++k) {
                Ep += phi(e[k], p->eps);
                Eg += psi_grad(g[2 * k] * g[2 * k] + g[2 * k + 1] * g[2 * k + 1], p->eps, p->grad_mode);
            }
        }
    const double wfl[3] = {p->w_s, p->w_m, p->w_d};
    const double mfl[3] = {p->m_s, p->m_m, p->m_d};
    double Fl[9];
    sfo_level_F(p->F, level, Fl);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int n = j * nx + i;
            /* Eq. 14: both directed pairs of every 4-neighbour edge [C9] */
            for (int nb = 0; nb < 2; ++nb) {
                int i2 = i + (nb == 0), j2 = j + (nb == 1);
                if (i2 >= nx || j2 >= ny) continue;
                int m = j2 * nx + i2;
                for (int fld = 0; fld < 3; ++fld)
                    for (int a = 0; a < 2; ++a) {
                        double d = T[(2 * fld + a) * G + n] - T[(2 * fld + a) * G + m];
                        Es += (wf[n] + wf[m]) * wfl[fld] * d * d;
                    }
            }
            double t6[6], r[2], J[12];
            for (int c = 0; c < 6; ++c) t6[c] = T[c * G + n];
            epipolar_terms(Fl, (double)(i * s), (double)(j * s), t6, r, J);
            Ee += r[0] * r[0] + r[1] * r[1];
            /* Eq. 18 on the deltas (Section 5.1) [C9] */
            for (int fld = 0; fld < 3; ++fld)
                for (int a = 0; a < 2; ++a) {
                    double d = delta[(2 * fld + a) * G + n];
                    Em += mfl[fld] * d * d;
                }
        }
    free(T);
    if (terms) {
        terms[0] = Ep;
        terms[1] = Eg;
        terms[2] = Es;
        terms[3] = Ee;
        terms[4] = Em;
    }
    return p->w_photo * Ep + p->w_grad * Eg + p->w_reg * (p->w_smooth * Es + p->w_epi * Ee + p->w_mag * Em);
}

double sfo_energy(int w, int h, int s, int nx, int ny, int level, const double* planes,
                  const double* base, const double* delta, const double* wf, const unsigned char* W,
                  const sfo_params* p, double terms[5], unsigned char* Wout)
{
    return energy_impl(w, h, s, nx, ny, level, planes, base, delta, wf, W, p, terms, Wout, NULL);
}

/* The energy with a level's maps (V: h*w bytes or NULL; L: 2*h*w or NULL). */
double sfo_energy_maps(int w, int h, int s, int nx, int ny, int level, const double* planes,
                       const double* base, const double* delta, const double* wf, const unsigned char* W,
                       const sfo_params* p, const unsigned char* V, const double* L, double terms[5],
                       unsigned char* Wout)
{
    sfo_maps mp = {V, L};
    return energy_impl(w, h, s, nx, ny, level, planes, base, delta, wf, W, p, terms, Wout, &mp);
}

/* ------------------------------------------------------------------------ */
/* Gauss-Newton normal equations (Section 5.1, Eqs. 19-24) [C3]               */
/* ------------------------------------------------------------------------ */

static int slot_of(int di, int dj) { return 3 * (dj + 1) + (di + 1); }

static void add_block(double* A, int n, int slot, int r, int c, double v) { A[((size_t)n * 9 + slot) * 36 + r * 6 + c] += v; }

/* Sample position of image c along axis a (0: x, 1: y) for fields f
 * (Eqs. 1-6). */
static double sample_position(int c, int a, double x, double y, const double f[6])
{
    return (a == 0 ? x : y) + SIGN[c][0] * f[a] + SIGN[c][1] * f[2 + a] + SIGN[c][2] * f[4 + a];
}

/* Assembles A dx = b at the state base + delta, with W taken at this state
 * (written to Wout) unless W is given. Returns the energy at the state.
 * recs/nrec: cell decisions given for some samples (record format of
 * sfo_solve_frame, sorted by pixel), or NULL; *ndis and *margin then count
 * the given decisions that differ from this oracle's own and the largest
 * distance of such a sample's own position from the nearest integer. */
static double assemble_impl(int w, int h, int s, int nx, int ny, int level, const double* planes,
                            const double* base, const double* delta, const double* wf, const unsigned char* Win,
                            const sfo_params* p, double* A, double* b, unsigned char* Wout, const unsigned* recs,
                            long nrec, int* ndis, double* margin, const sfo_maps* mp)
{
    long cur = 0;
    int G = nx * ny;
    memset(A, 0, sizeof(double) * (size_t)G * 9 * 36);
    memset(b, 0, sizeof(double) * (size_t)G * 6);
    double* T = (double*)malloc(sizeof(double) * 6 * G);
    for (int a = 0; a < 6 * G; ++a) T[a] = base[a] + delta[a];

    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double f[6], e[6], g[12], Je[36], Jg[72];
            int nd[4];
            double al[4];
            sfo_grid_weights(x, y, s, nx, ny, nd, al);
            pixel_fields(x, y, s, nx, ny, T, f);
            int dec[8] = {-1, -1, -1, -1, -1, -1, -1, -1}, have = 0;
            const unsigned pix = (unsigned)(y * w + x);
            while (recs && cur < nrec && recs[2 * cur] < pix) ++cur;
            while (recs && cur < nrec && recs[2 * cur] == pix) {
                const unsigned code = recs[2 * cur + 1];
                const int img = (code >> 1) & 3, ax = code & 1;
                dec[2 * img + ax] = (int)((code >> 4) << 1 | ((code >> 3) & 1));
                have = 1;
                /* does the oracle's own decision differ? */
                double pos = sample_position(img, ax, x, y, f), cp;
                int cell, cl;
                axis_decision(ax == 0 ? w : h, pos, &cp, &cell, &cl);
                if ((cell << 1 | cl) != dec[2 * img + ax]) {
                    double dist = fabs(pos - floor(pos + 0.5));
                    ++*ndis;
                    if (dist > *margin) *margin = dist;
                }
                ++cur;
            }
            double cb[2];
            pixel_terms_decided(w, h, planes, x, y, f, have ? dec : NULL, pixel_corr(mp, w, h, (int)pix, cb), e, g, Je,
                                Jg);
            int Wi = Win ? Win[y * w + x] : outlier_weight(e, p->eps_p);
            if (Wout) Wout[y * w + x] = (unsigned char)Wi;
            if (!Wi) continue;
            if (mp && mp->V && !mp->V[pix]) continue; /* V [C25] */
            /* pixel-level 6x6 H_p and 6-vector b_p */
            double Hp[36] = {0}, bp[6] = {0};
            if (p->robust_mode == SFO_IRLS) {
                /* each robust term c*rho(r) -> weight c*rho'(r)/(2r) on (r + J dx)^2 */
                for (int k = 0; k < 6; ++k) {
                    double om = p->w_photo / (2.0 * phi(e[k], p->eps));
                    for (int r = 0; r < 6; ++r) {
                        bp[r] -= om * e[k] * Je[k * 6 + r];
                        for (int c = 0; c < 6; ++c) Hp[r * 6 + c] += om * Je[k * 6 + r] * Je[k * 6 + c];
                    }
                    double q = g[2 * k] * g[2 * k] + g[2 * k + 1] * g[2 * k + 1];
                    double og = 0.5 * p->w_grad * psi_grad_coef(q, p->eps, p->grad_mode);
                    for (int a = 0; a < 2; ++a)
                        for (int r = 0; r < 6; ++r) {
                            bp[r] -= og * g[2 * k + a] * Jg[(2 * k + a) * 6 + r];
                            for (int c = 0; c < 6; ++c)
                                Hp[r * 6 + c] += og * Jg[(2 * k + a) * 6 + r] * Jg[(2 * k + a) * 6 + c];
                        }
                }
            } else {
                /* paper-literal: one residual sqrt(rho) per pixel and term (Eq. 19) */
                double rho_p = 0.0, rho_g = 0.0, gp[6] = {0}, gg[6] = {0};
                for (int k = 0; k < 6; ++k) {
                    double ph = phi(e[k], p->eps);
                    rho_p += p->w_photo * ph;
                    for (int r = 0; r < 6; ++r) gp[r] += p->w_photo * e[k] / ph * Je[k * 6 + r];
                    double q = g[2 * k] * g[2 * k] + g[2 * k + 1] * g[2 * k + 1];
                    rho_g += p->w_grad * psi_grad(q, p->eps, p->grad_mode);
                    double cf = p->w_grad * psi_grad_coef(q, p->eps, p->grad_mode);
                    for (int a = 0; a < 2; ++a)
                        for (int r = 0; r < 6; ++r) gg[r] += cf * g[2 * k + a] * Jg[(2 * k + a) * 6 + r];
                }
                for (int r = 0; r < 6; ++r) {
                    bp[r] -= 0.5 * (gp[r] + gg[r]);
                    for (int c = 0; c < 6; ++c) {
                        if (rho_p > 0) Hp[r * 6 + c] += gp[r] * gp[c] / (4.0 * rho_p);
                        if (rho_g > 0) Hp[r * 6 + c] += gg[r] * gg[c] / (4.0 * rho_g);
                    }
                }
            }
            /* chain rule through the bilinear weights to the four nodes (Eq. 7) */
            for (int k = 0; k < 4; ++k) {
                int ik = nd[k] % nx, jk = nd[k] / nx;
                for (int r = 0; r < 6; ++r) b[nd[k] * 6 + r] += al[k] * bp[r];
                for (int l = 0; l < 4; ++l) {
                    int il = nd[l] % nx, jl = nd[l] / nx;
                    int sl = slot_of(il - ik, jl - jk);
                    for (int r = 0; r < 6; ++r)
                        for (int c = 0; c < 6; ++c) add_block(A, nd[k], sl, r, c, al[k] * al[l] * Hp[r * 6 + c]);
                }
            }
        }

    /* priors on the nodes: exact Gauss-Newton rows */
    const double wfl[3] = {p->w_s, p->w_m, p->w_d};
    const double mfl[3] = {p->m_s, p->m_m, p->m_d};
    double Fl[9];
    sfo_level_F(p->F, level, Fl);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int n = j * nx + i;
            for (int nb = 0; nb < 2; ++nb) {
                int i2 = i + (nb == 0), j2 = j + (nb == 1);
                if (i2 >= nx || j2 >= ny) continue;
                int m = j2 * nx + i2;
                for (int fld = 0; fld < 3; ++fld) {
                    double c = p->w_reg * p->w_smooth * (wf[n] + wf[m]) * wfl[fld];
                    for (int a = 0; a < 2; ++a) {
                        int u = 2 * fld + a;
                        double d = T[u * G + n] - T[u * G + m];
                        add_block(A, n, 4, u, u, c);
                        add_block(A, m, 4, u, u, c);
                        add_block(A, n, slot_of(i2 - i, j2 - j), u, u, -c);
                        add_block(A, m, slot_of(i - i2, j - j2), u, u, -c);
                        b[n * 6 + u] -= c * d;
                        b[m * 6 + u] += c * d;
                    }
                }
            }
            double t6[6], r[2], J[12];
            for (int c = 0; c < 6; ++c) t6[c] = T[c * G + n];
            epipolar_terms(Fl, (double)(i * s), (double)(j * s), t6, r, J);
            double ce = p->w_reg * p->w_epi;
            for (int tt = 0; tt < 2; ++tt)
                for (int u = 0; u < 6; ++u) {
                    b[n * 6 + u] -= ce * r[tt] * J[tt * 6 + u];
                    for (int v = 0; v < 6; ++v) add_block(A, n, 4, u, v, ce * J[tt * 6 + u] * J[tt * 6 + v]);
                }
            for (int fld = 0; fld < 3; ++fld) {
                double cm = p->w_reg * p->w_mag * mfl[fld];
                for (int a = 0; a < 2; ++a) {
                    int u = 2 * fld + a;
                    add_block(A, n, 4, u, u, cm);
                    b[n * 6 + u] -= cm * delta[u * G + n];
                }
            }
        }
    free(T);
    return energy_impl(w, h, s, nx, ny, level, planes, base, delta, wf, Win ? Win : Wout, p, NULL, NULL, mp);
}

double sfo_assemble(int w, int h, int s, int nx, int ny, int level, const double* planes,
                    const double* base, const double* delta, const double* wf, const unsigned char* Win,
                    const sfo_params* p, double* A, double* b, unsigned char* Wout)
{
    int ndis = 0;
    double margin = 0.0;
    return assemble_impl(w, h, s, nx, ny, level, planes, base, delta, wf, Win, p, A, b, Wout, NULL, 0, &ndis,
                         &margin, NULL);
}

/* The Gauss-Newton system with a level's maps (V: h*w bytes or NULL; L: 2*h*w
 * or NULL). */
double sfo_assemble_maps(int w, int h, int s, int nx, int ny, int level, const double* planes,
                         const double* base, const double* delta, const double* wf, const unsigned char* Win,
                         const sfo_params* p, const unsigned char* V, const double* L, double* A, double* b,
                         unsigned char* Wout)
{
    int ndis = 0;
    double margin = 0.0;
    sfo_maps mp = {V, L};
    return assemble_impl(w, h, s, nx, ny, level, planes, base, delta, wf, Win, p, A, b, Wout, NULL, 0, &ndis,
                         &margin, &mp);
}

/* y = A x for the block system; vectors interleaved per node (n*6 + r). */
void sfo_apply(int nx, int ny, const double* A, const double* x, double* y)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int n = j * nx + i;
            for (int r = 0; r < 6; ++r) y[n * 6 + r] = 0.0;
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    int i2 = i + di, j2 = j + dj;
                    if (i2 < 0 || i2 >= nx || j2 < 0 || j2 >= ny) continue;
                    int m = j2 * nx + i2;
                    const double* B = A + ((size_t)n * 9 + slot_of(di, dj)) * 36;
                    for (int r = 0; r < 6; ++r)
                        for (int c = 0; c < 6; ++c) y[n * 6 + r] += B[r * 6 + c] * x[m * 6 + c];
                }
        }
}

static double dot(int n, const double* a, const double* b)
{
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += a[i] * b[i];
    return acc;
}

/* Jacobi-preconditioned conjugate gradients on A x = b from x = 0 (Section
 * 5.1) [C17]; exactly `iters` iterations unless p^T A p or r^T z drops to
 * 1e-30. model[k] = 0.5 x^T A x - b^T x after iteration k (may be NULL).
 * Returns the number of iterations run. */
int sfo_pcg(int nx, int ny, const double* A, const double* b, int iters, double* x, double* model)
{
    int N = nx * ny * 6;
    double* r = (double*)malloc(sizeof(double) * N);
    double* z = (double*)malloc(sizeof(double) * N);
    double* pv = (double*)malloc(sizeof(double) * N);
    double* q = (double*)malloc(sizeof(double) * N);
    double* Minv = (double*)malloc(sizeof(double) * N);
    for (int n = 0; n < nx * ny; ++n)
        for (int u = 0; u < 6; ++u) {
            double d = A[((size_t)n * 9 + 4) * 36 + u * 6 + u];
            Minv[n * 6 + u] = d > 0.0 ? 1.0 / d : 1.0;
        }
    for (int a = 0; a < N; ++a) {
        x[a] = 0.0;
        r[a] = b[a];
        z[a] = Minv[a] * r[a];
        pv[a] = z[a];
    }
    double rz = dot(N, r, z);
    int it = 0;
    for (; it < iters; ++it) {
        if (rz <= 1e-30) break;
        sfo_apply(nx, ny, A, pv, q);
        double pq = dot(N, pv, q);
        if (pq <= 1e-30) break;
        double alpha = rz / pq;
        for (int a = 0; a < N; ++a) {
            x[a] += alpha * pv[a];
            r[a] -= alpha * q[a];
            z[a] = Minv[a] * r[a];
        }
        double rz_new = dot(N, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int a = 0; a < N; ++a) pv[a] = z[a] + beta * pv[a];
        if (model) {
            sfo_apply(nx, ny, A, x, q);
            model[it] = 0.5 * dot(N, x, q) - dot(N, b, x);
        }
    }
    free(r);
    free(z);
    free(pv);
    free(q);
    free(Minv);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Domain decomposition (Section 5.2): alternating Schwarz [C24]            */
/* ------------------------------------------------------------------------ */

/* Solves A x = b from x = 0 by `sweeps` data-parallel Schwarz iterations. The
 * grid is cut into square tiles of `tile` x `tile` nodes (the last row and
 * column of tiles ragged); a subdomain is a tile grown by `overlap` nodes on
 * every side (clipped to the grid). In each sweep, from the same iterate x:
 * the residual r = b - A x; for every subdomain, the local system (the rows
 * and columns of A of the subdomain's nodes; couplings to nodes outside it
 * dropped, those nodes held at x) is solved for a correction e by
 * `patch_iters` Jacobi-PCG iterations from e = 0 (sfo_pcg on the local block
 * grid); then every node takes x + e from the subdomain whose tile holds it
 * (restricted additive Schwarz). The exchange between subdomains is the
 * global iterate. Returns 0, or -1 for an invalid tiling. */
int sfo_schwarz(int nx, int ny, const double* A, const double* b, int sweeps, int patch_iters, int tile, int overlap,
                double* x)
{
    if (tile < 1 || overlap < 0) return -1;
    int N = nx * ny * 6;
    double* r = (double*)malloc(sizeof(double) * N);
    double* xn = (double*)malloc(sizeof(double) * N);
    int ext = tile + 2 * overlap;
    double* Al = (double*)malloc(sizeof(double) * (size_t)ext * ext * 9 * 36);
    double* rl = (double*)malloc(sizeof(double) * ext * ext * 6);
    double* el = (double*)malloc(sizeof(double) * ext * ext * 6);
    for (int a = 0; a < N; ++a) x[a] = 0.0;
    for (int sw = 0; sw < sweeps; ++sw) {
        sfo_apply(nx, ny, A, x, r);
        for (int a = 0; a < N; ++a) r[a] = b[a] - r[a];
        memcpy(xn, x, sizeof(double) * N);
        for (int tj = 0; tj * tile < ny; ++tj)
            for (int ti = 0; ti * tile < nx; ++ti) {
                /* the subdomain: nodes [i0, i1) x [j0, j1) */
                int i0 = ti * tile - overlap, j0 = tj * tile - overlap;
                int i1 = (ti + 1) * tile + overlap, j1 = (tj + 1) * tile + overlap;
                if (i0 < 0) i0 = 0;
                if (j0 < 0) j0 = 0;
                if (i1 > nx) i1 = nx;
                if (j1 > ny) j1 = ny;
                int lx = i1 - i0, ly = j1 - j0;
                /* local block grid: the couplings inside the subdomain */
                memset(Al, 0, sizeof(double) * (size_t)lx * ly * 9 * 36);
                for (int j = j0; j < j1; ++j)
                    for (int i = i0; i < i1; ++i) {
                        int nl = (j - j0) * lx + (i - i0), n = j * nx + i;
                        for (int q = 0; q < 9; ++q) {
                            int di = q % 3 - 1, dj = q / 3 - 1;
                            if (i + di < i0 || i + di >= i1 || j + dj < j0 || j + dj >= j1) continue;
                            memcpy(Al + ((size_t)nl * 9 + q) * 36, A + ((size_t)n * 9 + q) * 36, sizeof(double) * 36);
                        }
                        for (int u = 0; u < 6; ++u) rl[nl * 6 + u] = r[n * 6 + u];
                    }
                sfo_pcg(lx, ly, Al, rl, patch_iters, el, NULL);
                /* restricted update: the tile's own nodes only */
                for (int j = tj * tile; j < (tj + 1) * tile && j < ny; ++j)
                    for (int i = ti * tile; i < (ti + 1) * tile && i < nx; ++i) {
                        int nl = (j - j0) * lx + (i - i0), n = j * nx + i;
                        for (int u = 0; u < 6; ++u) xn[n * 6 + u] = x[n * 6 + u] + el[nl * 6 + u];
                    }
            }
        memcpy(x, xn, sizeof(double) * N);
    }
    free(r);
    free(xn);
    free(Al);
    free(rl);
    free(el);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Delta hierarchy (Section 5.3) and temporal transfer [C19]                 */
/* ------------------------------------------------------------------------ */

/* base = 2 * Up(Tc): fine node (i, j) reads the coarse grid at (i/2, j/2),
 * bilinear, clamped; displacements double with the pixel size. */
void sfo_upsample(int nxc, int nyc, const double* Tc, int nx, int ny, double* base)
{
    int Gc = nxc * nyc, G = nx * ny;
    for (int c = 0; c < 6; ++c)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                base[c * G + j * nx + i] = 2.0 * grid_sample(nxc, nyc, Tc + c * Gc, 0.5 * i, 0.5 * j);
}

/* Constant-velocity transfer of one level's delta to the next frame: the node
 * at pixel X takes the previous delta at X - 2 m(X), m the previous total
 * motion at that node (grid coordinates = pixels / s). */
void sfo_temporal(int s, int nx, int ny, const double* delta_prev, const double* T_prev, int mode, double* delta)
{
    int G = nx * ny;
    if (mode == SFO_TEMPORAL_ZERO) {
        memset(delta, 0, sizeof(double) * 6 * G);
        return;
    }
    if (mode == SFO_TEMPORAL_COPY) {
        memcpy(delta, delta_prev, sizeof(double) * 6 * G);
        return;
    }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int n = j * nx + i;
            double X = (double)(i * s) - 2.0 * T_prev[2 * G + n];
            double Y = (double)(j * s) - 2.0 * T_prev[3 * G + n];
            for (int c = 0; c < 6; ++c) delta[c * G + n] = grid_sample(nx, ny, delta_prev + c * G, X / s, Y / s);
        }
}

/* ------------------------------------------------------------------------ */
/* Occlusion maps (Section 5.3, V of Eqs. 11 and 13) [C25]                   */
/* ------------------------------------------------------------------------ */

/* Closeness of the surface point with fields f at time t (0 or 1): the
 * horizontal disparity of that time's stereo pair, the left camera's sample
 * position less the right camera's (Eqs. 1-6: 2 d_x - 2 s_x at time 0,
 * -2 s_x - 2 d_x at time 1). Depth falls as it grows: a larger value is
 * nearer the cameras. */
static double closeness(int t, const double f[6])
{
    int il = t == 0 ? 0 : 2, ir = il + 1;
    double ol = SIGN[il][0] * f[0] + SIGN[il][1] * f[2] + SIGN[il][2] * f[4];
    double orr = SIGN[ir][0] * f[0] + SIGN[ir][1] * f[2] + SIGN[ir][2] * f[4];
    return ol - orr;
}

/* Twice the signed area of (a, b, p): > 0 when p lies left of a -> b. */
static double edge_fn(double ax, double ay, double bx, double by, double px, double py)
{
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

/* Occlusion map O (h*w bytes, 1 = visible) of a level at totals T: the
 * triangulated warp grid (every cell split into the triangles (i,j) (i+1,j)
 * (i+1,j+1) and (i,j) (i+1,j+1) (i,j+1)) is rendered into each of the four
 * images at its nodes' sample positions (Eqs. 1-6), keeping per image pixel
 * the largest closeness (a z-buffer; a pixel centre on a triangle's edge
 * counts as covered; degenerate triangles draw nothing). A reference pixel
 * is visible when, in every image, its sample position rounded to the
 * nearest pixel lies in the image and its own closeness is at least that
 * pixel's z-buffer value less tau. */
void sfo_occlusion_map(int w, int h, int s, int nx, int ny, const double* T, double tau, unsigned char* O)
{
    int G = nx * ny;
    size_t N = (size_t)w * h;
    double* Z = (double*)malloc(sizeof(double) * 4 * N);
    for (size_t a = 0; a < 4 * N; ++a) Z[a] = -INFINITY;
    for (int c = 0; c < 4; ++c) {
        int t = c / 2;
        for (int j = 0; j + 1 < ny; ++j)
            for (int i = 0; i + 1 < nx; ++i)
                for (int tri = 0; tri < 2; ++tri) {
                    int vi[3] = {i, i + 1, tri == 0 ? i + 1 : i};
                    int vj[3] = {j, tri == 0 ? j : j + 1, j + 1};
                    double X[3], Y[3], K[3];
                    for (int v = 0; v < 3; ++v) {
                        int n = vj[v] * nx + vi[v];
                        double f[6];
                        for (int q = 0; q < 6; ++q) f[q] = T[q * G + n];
                        X[v] = vi[v] * s + SIGN[c][0] * f[0] + SIGN[c][1] * f[2] + SIGN[c][2] * f[4];
                        Y[v] = vj[v] * s + SIGN[c][0] * f[1] + SIGN[c][1] * f[3] + SIGN[c][2] * f[5];
                        K[v] = closeness(t, f);
                    }
                    double area = edge_fn(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
                    if (area == 0.0) continue;
                    double xmin = fmin(X[0], fmin(X[1], X[2])), xmax = fmax(X[0], fmax(X[1], X[2]));
                    double ymin = fmin(Y[0], fmin(Y[1], Y[2])), ymax = fmax(Y[0], fmax(Y[1], Y[2]));
                    int x0 = (int)ceil(fmax(xmin, 0.0)), x1 = (int)floor(fmin(xmax, w - 1.0));
                    int y0 = (int)ceil(fmax(ymin, 0.0)), y1 = (int)floor(fmin(ymax, h - 1.0));
                    for (int py = y0; py <= y1; ++py)
                        for (int px = x0; px <= x1; ++px) {
                            double b0 = edge_fn(X[1], Y[1], X[2], Y[2], px, py);
                            double b1 = edge_fn(X[2], Y[2], X[0], Y[0], px, py);
                            double b2 = edge_fn(X[0], Y[0], X[1], Y[1], px, py);
                            if (area < 0.0) {
                                b0 = -b0;
                                b1 = -b1;
                                b2 = -b2;
                            }
                            if (b0 < 0.0 || b1 < 0.0 || b2 < 0.0) continue;
                            double k = (b0 * K[0] + b1 * K[1] + b2 * K[2]) / fabs(area);
                            double* z = Z + (size_t)c * N + (size_t)py * w + px;
                            if (k > *z) *z = k;
                        }
                }
    }
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double f[6];
            pixel_fields(x, y, s, nx, ny, T, f);
            int vis = 1;
            for (int c = 0; c < 4 && vis; ++c) {
                double px = x + SIGN[c][0] * f[0] + SIGN[c][1] * f[2] + SIGN[c][2] * f[4];
                double py = y + SIGN[c][0] * f[1] + SIGN[c][1] * f[3] + SIGN[c][2] * f[5];
                double qx = floor(px + 0.5), qy = floor(py + 0.5);
                if (qx < 0.0 || qx > w - 1.0 || qy < 0.0 || qy > h - 1.0) {
                    vis = 0;
                    break;
                }
                double z = Z[(size_t)c * N + (size_t)qy * w + (size_t)qx];
                if (!(closeness(c / 2, f) >= z - tau)) vis = 0;
            }
            O[y * w + x] = (unsigned char)vis;
        }
    free(Z);
}

/* Prolongation of a coarse occlusion map to the next finer level: fine pixel
 * (x, y) interpolates the coarse map bilinearly at (x/2, y/2) and is visible
 * when the result is at least 1/2. */
void sfo_vis_upsample(int wc, int hc, const unsigned char* Oc, int w, int h, unsigned char* V)
{
    double* P = (double*)malloc(sizeof(double) * wc * hc);
    for (int a = 0; a < wc * hc; ++a) P[a] = Oc[a] ? 1.0 : 0.0;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) V[y * w + x] = sfo_sample(wc, hc, P, 0.5 * x, 0.5 * y, NULL, NULL) >= 0.5;
    free(P);
}

/* ------------------------------------------------------------------------ */
/* Illumination correction maps (Section 5.3) [C26]                          */
/* ------------------------------------------------------------------------ */

/* Stereo intensity residuals of a level at totals T in the reference frame:
 * r[t][y][x] = I_1^t(p) - I_0^t(p') at the pixel's sample positions in the
 * right and left image of time t (Eqs. 1-6, checks d_0 and d_1). */
void sfo_illum_residual(int w, int h, int s, int nx, int ny, const double* planes, const double* T, double* r)
{
    size_t N = (size_t)w * h;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double f[6], e[6], g[12];
            pixel_fields(x, y, s, nx, ny, T, f);
            sfo_pixel_terms(w, h, planes, x, y, f, e, g, NULL, NULL);
            r[(size_t)y * w + x] = e[0];
            r[N + (size_t)y * w + x] = e[1];
        }
}

/* Gaussian low-pass of an image: weights exp(-k^2 / (2 sigma^2)) for
 * |k| <= R = ceil(3 sigma) along each axis, normalised to sum 1, edges
 * clamped; written as the plain 2D sum over the (2R+1)^2 window. */
void sfo_gauss_blur(int w, int h, const double* src, double sigma, double* dst)
{
    int R = (int)ceil(3.0 * sigma);
    double* g = (double*)malloc(sizeof(double) * (2 * R + 1));
    double sum = 0.0;
    for (int k = -R; k <= R; ++k) {
        g[k + R] = exp(-(double)k * k / (2.0 * sigma * sigma));
        sum += g[k + R];
    }
    for (int k = 0; k <= 2 * R; ++k) g[k] /= sum;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double acc = 0.0;
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    int xx = x + dx, yy = y + dy;
                    xx = xx < 0 ? 0 : (xx > w - 1 ? w - 1 : xx);
                    yy = yy < 0 ? 0 : (yy > h - 1 ? h - 1 : yy);
                    acc += g[dx + R] * g[dy + R] * src[(size_t)yy * w + xx];
                }
            dst[(size_t)y * w + x] = acc;
        }
    free(g);
}

/* Box prolongation to the next finer level: fine pixel (x, y) takes coarse
 * pixel (x/2, y/2) (integer division), for both times. */
void sfo_illum_upsample(int wc, int hc, const double* Rc, int w, int h, double* L)
{
    for (int t = 0; t < 2; ++t)
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                int xc = x / 2, yc = y / 2;
                if (xc > wc - 1) xc = wc - 1;
                if (yc > hc - 1) yc = hc - 1;
                L[(size_t)t * w * h + (size_t)y * w + x] = Rc[(size_t)t * wc * hc + (size_t)yc * wc + xc];
            }
}

/* Compares a given outlier mask with the one this oracle takes at the state
 * base + delta: returns the number of pixels that differ and, in *margin, the
 * largest distance | max_k |e_k| - eps_p | among them (how far from the
 * threshold the two decisions part). */
static int w_disagreement(int w, int h, int s, int nx, int ny, const double* planes, const double* base,
                          const double* delta, const unsigned char* Wg, const sfo_params* p, double* margin,
                          const sfo_maps* mp)
{
    int G = nx * ny, n = 0;
    double* T = (double*)malloc(sizeof(double) * 6 * G);
    for (int a = 0; a < 6 * G; ++a) T[a] = base[a] + delta[a];
    *margin = 0.0;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double f[6], e[6], g[12], cb[2];
            pixel_fields(x, y, s, nx, ny, T, f);
            pixel_terms_decided(w, h, planes, x, y, f, NULL, pixel_corr(mp, w, h, y * w + x, cb), e, g, NULL, NULL);
            if (outlier_weight(e, p->eps_p) != Wg[y * w + x]) {
                double mx = 0.0;
                for (int k = 0; k < 6; ++k)
                    if (fabs(e[k]) > mx) mx = fabs(e[k]);
                if (fabs(mx - p->eps_p) > *margin) *margin = fabs(mx - p->eps_p);
                ++n;
            }
        }
    free(T);
    return n;
}

/* ------------------------------------------------------------------------ */
/* One frame: Algorithm 1                                                     */
/* ------------------------------------------------------------------------ */

/* Packed per-level node arrays: level l starts at 6 * sum_{k<l} G_k. */
long sfo_packed_size(int w0, int h0, int s, int levels)
{
    long tot = 0;
    for (int l = 0; l < levels; ++l) {
        int w, h;
        sfo_level_dims(w0, h0, l, &w, &h);
        tot += 6L * ((w + s - 1) / s) * ((h + s - 1) / s);
    }
    return tot;
}

/* Solves one frame.
 *   imgs          4 * w0 * h0 doubles (image order of the file header)
 *   prev_delta,   packed per-level deltas and totals of the previous frame,
 *   prev_total    or NULL for the first frame (zero initialisation)
 *   init_coarsest optional 6 * G_{L-1} initial delta of the coarsest level
 *                 (overrides the temporal rule there), or NULL
 *   out_delta,    packed per-level final deltas and totals
 *   out_total
 *   W_given       optional outlier masks to use instead of taking W here:
 *                 for l = 0..L-1 and g = 0..gn_iters[l]-1 one w_l*h_l byte
 *                 mask each, in that order; NULL to take W at each state
 *   cell_recs,    optional bilinear cell decisions to use instead of taking
 *   cell_offs     them here, for the assembly of each Gauss-Newton step:
 *                 records of two unsigned each, (pixel y*w + x, code) with
 *                 code = cell << 4 | clamped << 3 | image << 1 | axis
 *                 (axis 0 = x), sorted by pixel; the records of level l and
 *                 step g are [cell_offs[l*16+g], cell_offs[l*16+g+1]); NULL
 *                 to take every decision here. A decision is an integer
 *                 taken in floating point (the cell min(floor(p), w-2) of
 *                 reading C7), like W; replaying another implementation's
 *                 decisions for samples at a cell edge isolates the
 *                 continuous error of the rest.
 *   V_given       optional occlusion maps to use instead of prolongating this
 *                 oracle's own (p->occlusion): for l = 0..L-1 one w_l*h_l
 *                 byte map each (level L-1's is all ones); NULL to compute
 *   stats         SFO_STATS_LEN doubles: [0] final energy, [1..5] its terms,
 *                 [6] pixels with W = 0 in the last step; at 16 + (l*16+g)*8:
 *                 E at the linearisation point, E accepted, step t (0 if
 *                 rejected), pixels with W = 0, PCG iterations run, with
 *                 W_given the pixels whose given W differs from the one taken
 *                 here and the largest | max_k |e_k| - eps_p | among them,
 *                 and with cell_recs the given cell decisions that differ from
 *                 the ones taken here and the largest distance of such a
 *                 sample's position from the nearest integer (SFO_STEP_STATS
 *                 values per step at 16 + (l*16+g)*SFO_STEP_STATS); with
 *                 V_given, stats[8 + l] counts the pixels of level l whose
 *                 given V differs from this oracle's own prolongated map.
 * Returns 0, or -1 for invalid sizes. */
int sfo_solve_frame(int w0, int h0, int s, int L, const sfo_params* p, const double* imgs,
                    const double* prev_delta, const double* prev_total, const double* init_coarsest,
                    const unsigned char* W_given, const unsigned* cell_recs, const long* cell_offs,
                    const unsigned char* V_given, double* out_delta, double* out_total, double* stats)
{
    if (L < 1 || L > SFO_MAX_LEVELS || s < 1) return -1;
    int W[SFO_MAX_LEVELS], H[SFO_MAX_LEVELS], NX[SFO_MAX_LEVELS], NY[SFO_MAX_LEVELS];
    long off[SFO_MAX_LEVELS], woff[SFO_MAX_LEVELS], poff[SFO_MAX_LEVELS];
    long acc = 0, wacc = 0, pacc = 0;
    for (int l = 0; l < L; ++l) {
        sfo_level_dims(w0, h0, l, &W[l], &H[l]);
        NX[l] = (W[l] + s - 1) / s;
        NY[l] = (H[l] + s - 1) / s;
        if (W[l] < 2 || H[l] < 2 || NX[l] < 2 || NY[l] < 2) return -1;
        off[l] = acc;
        acc += 6L * NX[l] * NY[l];
        woff[l] = wacc;
        wacc += (long)p->gn_iters[l] * W[l] * H[l];
        poff[l] = pacc;
        pacc += (long)W[l] * H[l];
    }
    if (stats) memset(stats, 0, sizeof(double) * SFO_STATS_LEN);

    /* pyramid of intensities, then per-level planes */
    double* lvl_imgs[SFO_MAX_LEVELS];
    for (int l = 0; l < L; ++l) lvl_imgs[l] = (double*)malloc(sizeof(double) * 4 * W[l] * H[l]);
    memcpy(lvl_imgs[0], imgs, sizeof(double) * 4 * W[0] * H[0]);
    for (int l = 1; l < L; ++l)
        for (int c = 0; c < 4; ++c)
            sfo_downsample(W[l - 1], H[l - 1], lvl_imgs[l - 1] + (size_t)c * W[l - 1] * H[l - 1],
                           lvl_imgs[l] + (size_t)c * W[l] * H[l]);

    /* the maps each level takes from the next coarser one (Algorithm 1):
     * none at the coarsest level, then prolongated after every solve */
    unsigned char* Vown = (unsigned char*)malloc(pacc);   /* this oracle's own prolongated V, per level */
    double* Lmap = (double*)malloc(sizeof(double) * 2 * pacc); /* illumination differences, per level */
    memset(Vown, 1, pacc);
    memset(Lmap, 0, sizeof(double) * 2 * pacc);
    for (int l = L - 1; l >= 0; --l) {
        int w = W[l], h = H[l], nx = NX[l], ny = NY[l], G = nx * ny;
        double* planes = (double*)malloc(sizeof(double) * 12 * w * h);
        sfo_level_planes(w, h, lvl_imgs[l], planes);
        sfo_maps maps = {NULL, NULL};
        if (p->occlusion) {
            maps.V = V_given ? V_given + poff[l] : Vown + poff[l];
            if (V_given && stats) {
                int nd = 0;
                for (long a = 0; a < (long)w * h; ++a) nd += (V_given[poff[l] + a] != 0) != (Vown[poff[l] + a] != 0);
                stats[8 + l] = nd;
            }
        }
        if (p->illumination) maps.L = Lmap + 2 * poff[l];
        double* base = out_total + off[l]; /* reuse the output as scratch for the base */
        double* delta = out_delta + off[l];
        if (l == L - 1) {
            memset(base, 0, sizeof(double) * 6 * G);
        } else {
            sfo_upsample(NX[l + 1], NY[l + 1], out_total + off[l + 1], nx, ny, base);
        }
        if (l == L - 1 && init_coarsest) {
            memcpy(delta, init_coarsest, sizeof(double) * 6 * G);
        } else if (prev_delta && prev_total) {
            sfo_temporal(s, nx, ny, prev_delta + off[l], prev_total + off[l], p->temporal_mode, delta);
        } else {
            memset(delta, 0, sizeof(double) * 6 * G);
        }
        double* T = (double*)malloc(sizeof(double) * 6 * G);
        for (int a = 0; a < 6 * G; ++a) T[a] = base[a] + delta[a];
        double* wf = (double*)malloc(sizeof(double) * G);
        sfo_feature_weights(w, h, s, nx, ny, planes, T, p, wf);

        double* A = (double*)malloc(sizeof(double) * (size_t)G * 9 * 36);
        double* b = (double*)malloc(sizeof(double) * G * 6);
        double* x = (double*)malloc(sizeof(double) * G * 6);
        double* trial = (double*)malloc(sizeof(double) * G * 6);
        unsigned char* Wm = (unsigned char*)malloc((size_t)w * h);
        int have_W = 0;
        for (int g = 0; g < p->gn_iters[l] && g < SFO_MAX_GN; ++g) {
            const unsigned char* Wg = W_given ? W_given + woff[l] + (long)g * w * h : NULL;
            int ndis = 0;
            double margin = 0.0;
            if (Wg) ndis = w_disagreement(w, h, s, nx, ny, planes, base, delta, Wg, p, &margin, &maps);
            const unsigned* rg = NULL;
            long nrg = 0;
            if (cell_recs && cell_offs) {
                rg = cell_recs + 2 * cell_offs[l * SFO_MAX_GN + g];
                nrg = cell_offs[l * SFO_MAX_GN + g + 1] - cell_offs[l * SFO_MAX_GN + g];
            }
            int ncdis = 0;
            double cmargin = 0.0;
            double Ecur = assemble_impl(w, h, s, nx, ny, l, planes, base, delta, wf, Wg, p, A, b, Wm, rg, nrg,
                                        &ncdis, &cmargin, &maps);
            have_W = 1;
            int nexcl = 0;
            for (int a = 0; a < w * h; ++a) nexcl += Wm[a] == 0;
            int its = p->pcg_iters[l];
            if (p->solver == SFO_SOLVER_SCHWARZ) {
                if (sfo_schwarz(nx, ny, A, b, p->pcg_iters[l], p->patch_iters[l], p->schwarz_tile,
                                p->schwarz_overlap, x) != 0)
                    memset(x, 0, sizeof(double) * G * 6);
            } else {
                its = sfo_pcg(nx, ny, A, b, p->pcg_iters[l], x, NULL);
            }
            /* backtracking safeguard [C18]: first t in {1, 1/2, ...} that does
             * not raise the energy (W frozen at this step's value) */
            double t = 1.0, Eacc = Ecur, tacc = 0.0;
            for (int bt = 0; bt <= p->max_backtracks; ++bt, t *= 0.5) {
                for (int n = 0; n < G; ++n)
                    for (int c = 0; c < 6; ++c) trial[c * G + n] = delta[c * G + n] + t * x[n * 6 + c];
                double Et = energy_impl(w, h, s, nx, ny, l, planes, base, trial, wf, Wm, p, NULL, NULL, &maps);
                if (Et <= Ecur) {
                    memcpy(delta, trial, sizeof(double) * 6 * G);
                    Eacc = Et;
                    tacc = t;
                    break;
                }
            }
            if (stats) {
                double* st = stats + 16 + (l * SFO_MAX_GN + g) * SFO_STEP_STATS;
                st[0] = Ecur;
                st[1] = Eacc;
                st[2] = tacc;
                st[3] = nexcl;
                st[4] = its;
                st[5] = ndis;
                st[6] = margin;
                st[7] = ncdis;
                st[8] = cmargin;
            }
        }
        if (l == 0 && stats) {
            /* final energy: with the last step's W, or W at this state */
            double terms[5];
            double E = energy_impl(w, h, s, nx, ny, l, planes, base, delta, wf, have_W ? Wm : NULL, p, terms,
                                   have_W ? NULL : Wm, &maps);
            stats[0] = E;
            stats[1] = p->w_photo * terms[0];
            stats[2] = p->w_grad * terms[1];
            stats[3] = p->w_reg * p->w_smooth * terms[2];
            stats[4] = p->w_reg * p->w_epi * terms[3];
            stats[5] = p->w_reg * p->w_mag * terms[4];
            int nexcl = 0;
            for (int a = 0; a < w * h; ++a) nexcl += Wm[a] == 0;
            stats[6] = nexcl;
        }
        for (int a = 0; a < 6 * G; ++a) base[a] += delta[a]; /* the slot now holds the total T_l */
        if (l > 0 && p->occlusion) {
            /* occlusion map of this level, prolongated to the next finer one */
            unsigned char* O = (unsigned char*)malloc((size_t)w * h);
            sfo_occlusion_map(w, h, s, nx, ny, base, p->occ_tau, O);
            sfo_vis_upsample(w, h, O, W[l - 1], H[l - 1], Vown + poff[l - 1]);
            free(O);
        }
        if (l > 0 && p->illumination) {
            /* illumination differences of this level, low-passed, box-prolongated */
            size_t N = (size_t)w * h;
            double* r = (double*)malloc(sizeof(double) * 2 * N);
            double* R = (double*)malloc(sizeof(double) * 2 * N);
            sfo_illum_residual(w, h, s, nx, ny, planes, base, r);
            sfo_gauss_blur(w, h, r, p->illum_sigma, R);
            sfo_gauss_blur(w, h, r + N, p->illum_sigma, R + N);
            sfo_illum_upsample(w, h, R, W[l - 1], H[l - 1], Lmap + 2 * poff[l - 1]);
            free(r);
            free(R);
        }
        free(T);
        free(wf);
        free(A);
        free(b);
        free(x);
        free(trial);
        free(Wm);
        free(planes);
    }
    for (int l = 0; l < L; ++l) free(lvl_imgs[l]);
    free(Vown);
    free(Lmap);
    return 0;
}
