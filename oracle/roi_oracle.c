/*
 * roi_oracle.c -- FP64 CPU oracle for local ROI tomographic reconstruction.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it; the library itself never
 * does.  It shares no code, header or table with the CUDA path.
 *
 * Source: Pelt & Batenburg, "A method for locally approximating regularized
 * iterative tomographic reconstruction methods" (arXiv 1604.02292).
 *
 *   Sec. 2.1   parallel-beam geometry, W and W^T, masks M_L / M_F and the local
 *              and outer operators (Eq. locouter: W = W_L + W_F).
 *   Sec. 2.2   FBP(p, h) = W^T C_h p (Eq. fbp) with a Ram-Lak filter;
 *              SIRT x <- x + alpha W^T (p - W x) (Eq. sirtit).
 *   Sec. 2.3   regularized objective ||p - W x||^2 + lambda g(x) over x in D
 *              (Eq. priorsys); box-constrained SIRT (Eq. sirtbox); TV g = ||grad x||_1;
 *              Chambolle-Pock named as a solver.
 *   Sec. 3.1   alpha = 1 / (N_theta N_d).
 *   Sec. 1     the exterior-subtraction ROI scheme: subtract the reprojection of a
 *              global reconstruction outside the ROI, then reconstruct the ROI
 *              algebraically.
 *   Sec. 3     the paper's own local method: filters approximating SIRT (Alg. filtcalc,
 *              Eq. filtcalc, Eq. sirtapp), the local recursion with a prior term
 *              (Alg. method, Eq. localmethod), its FISTA form with a TV prox computed
 *              by FGP (Alg. methodfista), Haar-wavelet ISTA (Eq. sirtista) as its prior
 *              term, and the disc subtraction (Sec. 3.3).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - W is Joseph's method: one ray per bin centre; when |cos| >= |sin| (ties,
 *     within 1e-12, go this way) the ray is sampled once per image row and
 *     linearly interpolated between the two nearest columns, weight 1/|cos|;
 *     otherwise once per column, interpolated between rows, weight 1/|sin|.
 *     Pixels off the grid contribute zero.  Row/column samples are summed in
 *     ascending index order.
 *   - W^T is its exact transpose, evaluated per pixel: at angle theta, bin d
 *     receives weight (1 - |t_d - t_ij| / w) / w when |t_d - t_ij| < w, where
 *     t_ij = x_j cos + y_i sin and w = max(|cos|, |sin|) of the branch taken.
 *   - FBP uses the spatial Ram-Lak filter h[0] = 1/4, h[odd k] = -1/(pi^2 k^2),
 *     h[even k != 0] = 0, applied as a linear zero-padded convolution of length
 *     2 N_d - 1, scaled by pi / N_theta.
 *   - The exterior step reprojects the global reconstruction only inside its field of
 *     view: the pixels whose centre lies within min(N, N_d)/2 of the rotation axis (for
 *     N_d >= N the disc of diameter N that Sec. 3.3 takes as the object's support).
 *     Outside it the detector misses the pixel at some angles, the FBP value there is
 *     not determined by the data, and its reprojection would make p' inconsistent
 *     (Sec. 1 warns that a poor global reconstruction causes artifacts in the ROI).
 *   - TV is isotropic, forward differences with a zero last difference (Neumann).
 *   - Chambolle-Pock uses the diagonal preconditioning of Pock & Chambolle (2011,
 *     alpha = 1) or scalar steps 0.99/||K|| from a power iteration.
 *   - The data term keeps the paper's form ||p - Wx||^2 without a factor 1/2.
 *   - Alg. filtcalc: the impulse sits on the rotation axis (shared by the four central
 *     pixels when N is even); u_k = alpha W q_k is read at the integer offsets of a
 *     linear convolution from a detector with the acquisition's bin phase (see
 *     orc_filtcalc).  The approximation of SIRT it gives is checked loosely (it is an
 *     approximation); the algorithm's steps are pinned exactly.
 *
 * Coordinates: pixel (i, j) -- row from the top, column -- has its centre at
 * (x_j, y_i) = (j - (N-1)/2, (N-1)/2 - i); bin d has centre t_d = d - (N_d-1)/2.
 * A rectangle (x0, y0, w, h) covers columns [x0, x0+w) and rows [y0, y0+h).
 * Images are row-major [h][w]; sinograms are row-major [n_angles][n_det].
 *
 * Parity: pinned by the CPU tests (explicit 16x16 system matrix, theta = 0 and
 * pi/2 column/row sums, closed-form line integrals, the adjoint identity,
 * Eq. locouter, the closed form Eq. sirtfull2, least-squares limits, a reference
 * TV solver).  The local-versus-global difference inside the ROI is reported,
 * not pinned.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* Branch rule: sample per row when |cos| >= |sin| (ties within 1e-12 go to rows). */
static int row_branch(double c, double s) { return fabs(c) >= fabs(s) - 1e-12; }

typedef struct {
    int x0, y0, w, h;
} rect_t;

static int in_rect(const rect_t* r, int i, int j) {
    return r->w > 0 && j >= r->x0 && j < r->x0 + r->w && i >= r->y0 && i < r->y0 + r->h;
}

/* value of pixel (i, j) of an image that covers `sup` and is zero elsewhere and inside `hole` */
static double pix(const double* img, const rect_t* sup, const rect_t* hole, int i, int j) {
    if (!in_rect(sup, i, j)) return 0.0;
    if (hole && in_rect(hole, i, j)) return 0.0;
    return img[(size_t)(i - sup->y0) * sup->w + (j - sup->x0)];
}

/* A ray can only reach pixels whose centre projection t_ij lies within max(|c|,|s|) <= 1
 * of its offset t; rays farther than that from every pixel of `sup` are skipped. */
static int ray_misses(int N, const rect_t* sup, double c, double s, double t) {
    double xc = (sup->x0 + 0.5 * (sup->w - 1)) - 0.5 * (N - 1);
    double yc = 0.5 * (N - 1) - (sup->y0 + 0.5 * (sup->h - 1));
    double half = 0.5 * (fabs(c) * (sup->w - 1) + fabs(s) * (sup->h - 1));
    return fabs(t - (xc * c + yc * s)) >= half + 1.0;
}

/* ---------------------------------------------------------------------------
 * Forward projection W (Sec. 2.1): sino[a][d] = sum of Joseph samples of the
 * image along ray (theta_a, t_d).  The image is given on rectangle `sup`
 * (zero outside it); pixels inside `hole` (if hole_w > 0) count as zero, which
 * realises W M_F when sup is the whole grid and hole is the local part.
 * ------------------------------------------------------------------------- */
void orc_forward(int N, int na, int nd, const double* ang,
                 int x0, int y0, int w, int h, const double* img,
                 int hx0, int hy0, int hw, int hh, double* sino) {
    rect_t sup = {x0, y0, w, h}, hole = {hx0, hy0, hw, hh};
    const rect_t* hp = hw > 0 ? &hole : NULL;
    const double half = 0.5 * (N - 1);
#pragma omp parallel for schedule(static)
    for (long r = 0; r < (long)na * nd; ++r) {
        int a = (int)(r / nd), d = (int)(r % nd);
        double c = cos(ang[a]), s = sin(ang[a]);
        double t = d - 0.5 * (nd - 1);
        double acc = 0.0;
        if (!ray_misses(N, &sup, c, s, t)) {
            if (row_branch(c, s)) {
                for (int i = y0; i < y0 + h; ++i) {          /* rows of the support, ascending */
                    double y = half - i;
                    double u = (t - y * s) / c + half;       /* fractional column index */
                    double fl = floor(u);
                    int j0 = (int)fl;
                    double f = u - fl;
                    acc += (1.0 - f) * pix(img, &sup, hp, i, j0) + f * pix(img, &sup, hp, i, j0 + 1);
                }
                acc /= fabs(c);
            } else {
                for (int j = x0; j < x0 + w; ++j) {          /* columns of the support, ascending */
                    double x = j - half;
                    double v = half - (t - x * c) / s;       /* fractional row index */
                    double fl = floor(v);
                    int i0 = (int)fl;
                    double f = v - fl;
                    acc += (1.0 - f) * pix(img, &sup, hp, i0, j) + f * pix(img, &sup, hp, i0 + 1, j);
                }
                acc /= fabs(s);
            }
        }
        sino[r] = acc;
    }
}

/* ---------------------------------------------------------------------------
 * Backprojection W^T (Sec. 2.1), the exact transpose of orc_forward, evaluated
 * per pixel of rectangle `sup` (pixels in `hole` are set to zero: M_F W^T or
 * M_L W^T by choice of sup/hole).  Angles are summed in ascending order.
 * ------------------------------------------------------------------------- */
void orc_back(int N, int na, int nd, const double* ang,
              int x0, int y0, int w, int h,
              int hx0, int hy0, int hw, int hh,
              const double* sino, double* img) {
    rect_t hole = {hx0, hy0, hw, hh};
    const double half = 0.5 * (N - 1), dhalf = 0.5 * (nd - 1);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < (long)w * h; ++q) {
        int i = y0 + (int)(q / w), j = x0 + (int)(q % w);
        double acc = 0.0;
        if (!(hw > 0 && in_rect(&hole, i, j))) {
            double xj = j - half, yi = half - i;
            for (int a = 0; a < na; ++a) {
                double c = cos(ang[a]), s = sin(ang[a]);
                double wd = row_branch(c, s) ? fabs(c) : fabs(s);
                double tij = xj * c + yi * s;
                double tau = tij + dhalf;                     /* continuous bin index */
                int dlo = (int)floor(tau - wd), dhi = (int)ceil(tau + wd);
                for (int d = dlo; d <= dhi; ++d) {
                    if (d < 0 || d >= nd) continue;
                    double dist = fabs((d - dhalf) - tij);
                    if (dist < wd) acc += (1.0 - dist / wd) / wd * sino[(size_t)a * nd + d];
                }
            }
        }
        img[q] = acc;
    }
}

/* ---------------------------------------------------------------------------
 * Ram-Lak row filter C_h (Sec. 2.2, Eq. fbp) with the FBP scale pi/N_theta:
 * q[a][d] = (pi/na) * sum_k h[d-k] p[a][k], linear convolution, zero padded.
 * ------------------------------------------------------------------------- */
static double ramlak(int k) {
    if (k == 0) return 0.25;
    if ((k & 1) == 0) return 0.0;
    return -1.0 / (ORC_PI * ORC_PI * (double)k * (double)k);
}

void orc_ramp(int na, int nd, const double* p, double* q) {
    const double scale = ORC_PI / na;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < (long)na * nd; ++r) {
        int a = (int)(r / nd), d = (int)(r % nd);
        double acc = 0.0;
        for (int k = 0; k < nd; ++k) acc += ramlak(d - k) * p[(size_t)a * nd + k];
        q[r] = scale * acc;
    }
}

/* FBP(p, h) = W^T C_h p on the whole N x N grid (Eq. fbp). */
void orc_fbp(int N, int na, int nd, const double* ang, const double* p, double* x) {
    double* q = (double*)malloc(sizeof(double) * (size_t)na * nd);
    orc_ramp(na, nd, p, q);
    orc_back(N, na, nd, ang, 0, 0, N, N, 0, 0, 0, 0, q, x);
    free(q);
}

/* Field of view of the global reconstruction: pixel (i, j) lies in it when its centre
 * is within D/2 of the rotation axis, D = min(N, N_d); in doubled coordinates
 * (2 x_j, 2 y_i) = (2j - (N-1), (N-1) - 2i) the test is exact in integers. */
static int in_fov(int N, int nd, int i, int j) {
    const long long X = 2LL * j - (N - 1), Y = (long long)(N - 1) - 2LL * i;
    const long long D = N < nd ? N : nd;
    return X * X + Y * Y <= D * D;
}

/* x (N x N) restricted to the field of view: pixels outside it set to 0. */
void orc_fov(int N, int nd, double* x) {
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            if (!in_fov(N, nd, i, j)) x[(size_t)i * N + j] = 0.0;
}

/* Exterior subtraction (Sec. 1): p' = p - W M_F M_V x_fbp, every bin of the sinogram,
 * M_V the field of view of the global reconstruction (orc_fov). */
void orc_exterior(int N, int na, int nd, const double* ang,
                  int bx0, int by0, int bw, int bh,
                  const double* p, const double* xfbp, double* pprime) {
    double* xv = (double*)malloc(sizeof(double) * (size_t)N * N);
    memcpy(xv, xfbp, sizeof(double) * (size_t)N * N);
    orc_fov(N, nd, xv);
    orc_forward(N, na, nd, ang, 0, 0, N, N, xv, bx0, by0, bw, bh, pprime);
    for (long r = 0; r < (long)na * nd; ++r) pprime[r] = p[r] - pprime[r];
    free(xv);
}

/* Row sums W_L 1 (per ray) and column sums W_L^T 1 (per box pixel). */
void orc_rowcol_sums(int N, int na, int nd, const double* ang,
                     int bx0, int by0, int bw, int bh, double* rows, double* cols) {
    size_t nb = (size_t)bw * bh, ns = (size_t)na * nd;
    double* one = (double*)malloc(sizeof(double) * (nb > ns ? nb : ns));
    for (size_t k = 0; k < nb; ++k) one[k] = 1.0;
    orc_forward(N, na, nd, ang, bx0, by0, bw, bh, one, 0, 0, 0, 0, rows);
    for (size_t k = 0; k < ns; ++k) one[k] = 1.0;
    orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, one, cols);
    free(one);
}

/* ---------------------------------------------------------------------------
 * SIRT on the local part (Eq. sirtit with W_L, Eq. sirtbox with l = 0, r = inf):
 *   x^0 = 0;  x <- P(x + alpha W_L^T (p' - W_L x))   (weighting = 0)
 *   x <- P(x + C W_L^T R (p' - W_L x))               (weighting = 1)
 * with R = 1/(W_L 1), C = 1/(W_L^T 1), zero where the sum is below 1e-3, and
 * P the projection onto x >= 0 when nonneg != 0 (identity otherwise).
 * x is the box image [bh][bw]; alpha is given by the caller (the paper uses
 * 1/(N_theta N_d), Sec. 3.1).
 * ------------------------------------------------------------------------- */
void orc_sirt(int N, int na, int nd, const double* ang,
              int bx0, int by0, int bw, int bh,
              const double* pprime, int iters, double alpha, int weighting, int nonneg,
              double* x) {
    size_t nb = (size_t)bw * bh, ns = (size_t)na * nd;
    double* r = (double*)malloc(sizeof(double) * ns);
    double* g = (double*)malloc(sizeof(double) * nb);
    double* R = NULL;
    double* C = NULL;
    if (weighting) {
        R = (double*)malloc(sizeof(double) * ns);
        C = (double*)malloc(sizeof(double) * nb);
        orc_rowcol_sums(N, na, nd, ang, bx0, by0, bw, bh, R, C);
        for (size_t k = 0; k < ns; ++k) R[k] = R[k] > 1e-3 ? 1.0 / R[k] : 0.0;
        for (size_t k = 0; k < nb; ++k) C[k] = C[k] > 1e-3 ? 1.0 / C[k] : 0.0;
    }
    for (size_t k = 0; k < nb; ++k) x[k] = 0.0;
    for (int it = 0; it < iters; ++it) {
        orc_forward(N, na, nd, ang, bx0, by0, bw, bh, x, 0, 0, 0, 0, r);
        for (size_t k = 0; k < ns; ++k) {
            r[k] = pprime[k] - r[k];
            if (weighting) r[k] *= R[k];
        }
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, r, g);
        for (size_t k = 0; k < nb; ++k) {
            double v = x[k] + (weighting ? C[k] : alpha) * g[k];
            x[k] = (nonneg && v < 0.0) ? 0.0 : v;
        }
    }
    free(r);
    free(g);
    free(R);
    free(C);
}

/* ---------------------------------------------------------------------------
 * Discrete gradient (forward differences, zero last difference) and its
 * negative adjoint, the divergence, on a [h][w] image.
 * gx[i][j] = x[i][j+1] - x[i][j] (j < w-1), gy[i][j] = x[i+1][j] - x[i][j] (i < h-1).
 * ------------------------------------------------------------------------- */
void orc_grad(int w, int h, const double* x, double* gx, double* gy) {
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            size_t k = (size_t)i * w + j;
            gx[k] = j < w - 1 ? x[k + 1] - x[k] : 0.0;
            gy[k] = i < h - 1 ? x[k + w] - x[k] : 0.0;
        }
}

/* div = -grad^T:  div(v)[i][j] = vx[i][j] - vx[i][j-1] + vy[i][j] - vy[i-1][j],
 * where terms that refer to a difference outside the grid, or to the zero last
 * difference, are left out. */
void orc_div(int w, int h, const double* vx, const double* vy, double* dv) {
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            size_t k = (size_t)i * w + j;
            double d = 0.0;
            if (j < w - 1) d += vx[k];
            if (j > 0) d -= vx[k - 1];
            if (i < h - 1) d += vy[k];
            if (i > 0) d -= vy[k - w];
            dv[k] = d;
        }
}

/* Objective of Eq. priorsys on the local part with isotropic TV:
 *   ||W_L x - p'||^2 over rays that reach the box (row sum > 1e-6)
 *   + lambda * sum_ij sqrt(gx^2 + gy^2). */
double orc_objective(int N, int na, int nd, const double* ang,
                     int bx0, int by0, int bw, int bh,
                     const double* pprime, const double* x, double lambda) {
    size_t nb = (size_t)bw * bh, ns = (size_t)na * nd;
    double* wx = (double*)malloc(sizeof(double) * ns);
    double* rows = (double*)malloc(sizeof(double) * ns);
    double* cols = (double*)malloc(sizeof(double) * nb);
    double* gx = (double*)malloc(sizeof(double) * nb);
    double* gy = (double*)malloc(sizeof(double) * nb);
    orc_rowcol_sums(N, na, nd, ang, bx0, by0, bw, bh, rows, cols);
    orc_forward(N, na, nd, ang, bx0, by0, bw, bh, x, 0, 0, 0, 0, wx);
    double data = 0.0, tv = 0.0;
    for (size_t k = 0; k < ns; ++k)
        if (rows[k] > 1e-6) data += (wx[k] - pprime[k]) * (wx[k] - pprime[k]);
    orc_grad(bw, bh, x, gx, gy);
    for (size_t k = 0; k < nb; ++k) tv += sqrt(gx[k] * gx[k] + gy[k] * gy[k]);
    free(wx);
    free(rows);
    free(cols);
    free(gx);
    free(gy);
    return data + lambda * tv;
}

/* ||K|| for K = [W_L; grad] by power iteration on K^T K from the all-ones image. */
double orc_power_norm(int N, int na, int nd, const double* ang,
                      int bx0, int by0, int bw, int bh, int iters) {
    size_t nb = (size_t)bw * bh, ns = (size_t)na * nd;
    double* x = (double*)malloc(sizeof(double) * nb);
    double* y = (double*)malloc(sizeof(double) * nb);
    double* s = (double*)malloc(sizeof(double) * ns);
    double* gx = (double*)malloc(sizeof(double) * nb);
    double* gy = (double*)malloc(sizeof(double) * nb);
    double* dv = (double*)malloc(sizeof(double) * nb);
    double nrm = 0.0, L2 = 0.0;
    for (size_t k = 0; k < nb; ++k) x[k] = 1.0;
    for (size_t k = 0; k < nb; ++k) nrm += x[k] * x[k];
    nrm = sqrt(nrm);
    for (size_t k = 0; k < nb; ++k) x[k] /= nrm;
    for (int it = 0; it < iters; ++it) {
        orc_forward(N, na, nd, ang, bx0, by0, bw, bh, x, 0, 0, 0, 0, s);
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, s, y);
        orc_grad(bw, bh, x, gx, gy);
        orc_div(bw, bh, gx, gy, dv);
        nrm = 0.0;
        for (size_t k = 0; k < nb; ++k) {
            y[k] -= dv[k];                 /* K^T K x = W^T W x + grad^T grad x */
            nrm += y[k] * y[k];
        }
        nrm = sqrt(nrm);
        L2 = nrm;                          /* ||K^T K x|| with ||x|| = 1 -> ||K||^2 */
        for (size_t k = 0; k < nb; ++k) x[k] = y[k] / nrm;
    }
    free(x);
    free(y);
    free(s);
    free(gx);
    free(gy);
    free(dv);
    return sqrt(L2);
}

/* ---------------------------------------------------------------------------
 * Chambolle-Pock for min_x ||W_L x - p'||^2 + lambda ||grad x||_{2,1}
 * (Eq. priorsys with g = TV, D = R^n), K = [W_L; grad].  x^0 = xbar^0 = 0,
 * duals u (rays) and v = (vx, vy) (pixels) start at 0.  Per iteration:
 *   u <- (u + sigma_u (W_L xbar - p')) / (1 + sigma_u / 2)   prox of f*, f = ||. - p'||^2
 *   v <- projection of v + sigma_v grad xbar onto {|v_ij|_2 <= lambda}
 *   x+ = x - tau (W_L^T u - div v);  xbar = 2 x+ - x.
 * precond = 1: sigma_u = 1 / (W_L 1) (0 where the row sum is <= 1e-6),
 *              sigma_v = 1/2, tau_j = 1 / ((W_L^T 1)_j + column sum of |grad|).
 * precond = 0: sigma = tau = 0.99 / L with L = ||K|| supplied by the caller.
 * x is the box image [bh][bw].
 * ------------------------------------------------------------------------- */
void orc_cp(int N, int na, int nd, const double* ang,
            int bx0, int by0, int bw, int bh,
            const double* pprime, int iters, double lambda, int precond, double L,
            double* x) {
    size_t nb = (size_t)bw * bh, ns = (size_t)na * nd;
    double* u = (double*)calloc(ns, sizeof(double));
    double* vx = (double*)calloc(nb, sizeof(double));
    double* vy = (double*)calloc(nb, sizeof(double));
    double* xb = (double*)calloc(nb, sizeof(double));
    double* wx = (double*)malloc(sizeof(double) * ns);
    double* wtu = (double*)malloc(sizeof(double) * nb);
    double* gx = (double*)malloc(sizeof(double) * nb);
    double* gy = (double*)malloc(sizeof(double) * nb);
    double* dv = (double*)malloc(sizeof(double) * nb);
    double* su = (double*)malloc(sizeof(double) * ns);
    double* tau = (double*)malloc(sizeof(double) * nb);
    double sv;
    if (precond) {
        orc_rowcol_sums(N, na, nd, ang, bx0, by0, bw, bh, su, tau);
        for (size_t k = 0; k < ns; ++k) su[k] = su[k] > 1e-6 ? 1.0 / su[k] : 0.0;
        for (int i = 0; i < bh; ++i)
            for (int j = 0; j < bw; ++j) {
                size_t k = (size_t)i * bw + j;
                int cnt = (j < bw - 1) + (j > 0) + (i < bh - 1) + (i > 0);
                tau[k] = 1.0 / (tau[k] + cnt);
            }
        sv = 0.5;
    } else {
        double st = 0.99 / L;
        for (size_t k = 0; k < ns; ++k) su[k] = st;
        for (size_t k = 0; k < nb; ++k) tau[k] = st;
        sv = st;
    }
    for (size_t k = 0; k < nb; ++k) x[k] = 0.0;
    for (int it = 0; it < iters; ++it) {
        orc_forward(N, na, nd, ang, bx0, by0, bw, bh, xb, 0, 0, 0, 0, wx);
        for (size_t k = 0; k < ns; ++k) u[k] = (u[k] + su[k] * (wx[k] - pprime[k])) / (1.0 + 0.5 * su[k]);
        orc_grad(bw, bh, xb, gx, gy);
        for (size_t k = 0; k < nb; ++k) {
            double ax = vx[k] + sv * gx[k], ay = vy[k] + sv * gy[k];
            double m = sqrt(ax * ax + ay * ay);
            double sc = m > lambda ? lambda / m : 1.0;
            vx[k] = ax * sc;
            vy[k] = ay * sc;
        }
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, u, wtu);
        orc_div(bw, bh, vx, vy, dv);
        for (size_t k = 0; k < nb; ++k) {
            double xn = x[k] - tau[k] * (wtu[k] - dv[k]);
            xb[k] = 2.0 * xn - x[k];
            x[k] = xn;
        }
    }
    free(u);
    free(vx);
    free(vy);
    free(xb);
    free(wx);
    free(wtu);
    free(gx);
    free(gy);
    free(dv);
    free(su);
    free(tau);
}

/* ===========================================================================
 * The paper's own local method (Sec. 3): SIRT approximated by filtered
 * backprojection with iteration-dependent filters, the prior applied only on
 * the local part.
 * ======================================================================== */

/* Unit impulse at the grid centre.  For even N the centre is the corner of four
 * pixels and the impulse is shared by them (1/4 each), so that it stays centred
 * on the rotation axis; for odd N it is the central pixel. */
static void centre_impulse(int N, double* c) {
    memset(c, 0, sizeof(double) * (size_t)N * N);
    if (N % 2) {
        c[(size_t)(N / 2) * N + N / 2] = 1.0;
    } else {
        int m = N / 2;
        c[(size_t)(m - 1) * N + m - 1] = 0.25;
        c[(size_t)(m - 1) * N + m] = 0.25;
        c[(size_t)m * N + m - 1] = 0.25;
        c[(size_t)m * N + m] = 0.25;
    }
}

/* ---------------------------------------------------------------------------
 * Alg. filtcalc (Sec. 3.1; Eq. filtcalc, Eq. sirtapp), one filter per iteration:
 *     q_0 = 0, c = impulse;  for k = 1..n:  q_k = q_{k-1} + c;  c = c - alpha W^T W c;
 *     u_k = alpha W q_k, sampled at the integer detector offsets a convolution uses.
 * W is the acquisition projector on the N x N grid (so q_k = sum_{j<k} A^j c with
 * A = I - alpha W^T W).  Reading of "u_k = alpha W q_k": the projection of q_k is taken
 * on a detector that extends the acquisition one (same bin phase relative to the
 * rotation axis) to the offsets -(N_d - 1) .. N_d - 1 around the axis, then read at
 * those integer offsets by linear interpolation: for odd N_d the bins lie on the
 * integers (2 N_d - 1 bins, read as they are); for even N_d they lie on the
 * half-integers (2 N_d bins) and tap m is the mean of the bins at m - 1/2 and m + 1/2.
 * u: [n][na][2 nd - 1], tap m of angle a of filter k at u[k-1][a][m + nd - 1].
 * ------------------------------------------------------------------------- */
void orc_filtcalc(int N, int na, int nd, const double* ang, int n, double alpha, double* u) {
    const int nd2 = 2 * nd - 1, ndp = (nd % 2) ? nd2 : 2 * nd;
    const size_t nn = (size_t)N * N, ns = (size_t)na * nd, nu = (size_t)na * nd2;
    double* c = (double*)malloc(sizeof(double) * nn);
    double* q = (double*)calloc(nn, sizeof(double));
    double* wc = (double*)malloc(sizeof(double) * ns);
    double* g = (double*)malloc(sizeof(double) * nn);
    double* h = (double*)malloc(sizeof(double) * (size_t)na * ndp);
    centre_impulse(N, c);
    for (int k = 1; k <= n; ++k) {
        for (size_t i = 0; i < nn; ++i) q[i] += c[i];
        double* uk = u + (size_t)(k - 1) * nu;
        orc_forward(N, na, ndp, ang, 0, 0, N, N, q, 0, 0, 0, 0, h);
        for (int a = 0; a < na; ++a)
            for (int m = 0; m < nd2; ++m) {
                const double* ha = h + (size_t)a * ndp;
                double v = (nd % 2) ? ha[m] : 0.5 * (ha[m] + ha[m + 1]);
                uk[(size_t)a * nd2 + m] = alpha * v;
            }
        orc_forward(N, na, nd, ang, 0, 0, N, N, c, 0, 0, 0, 0, wc);
        orc_back(N, na, nd, ang, 0, 0, N, N, 0, 0, 0, 0, wc, g);
        for (size_t i = 0; i < nn; ++i) c[i] -= alpha * g[i];
    }
    free(c);
    free(q);
    free(wc);
    free(g);
    free(h);
}

/* C_{u_k} p (Sec. 3.1, Eq. sirtapp): for every angle a linear, zero-padded
 * convolution of the row p[a] with the filter row uk[a]:
 *     out[a][d] = sum_{d'} uk[a][(d - d') + nd - 1] p[a][d'].   uk: [na][2 nd - 1]. */
void orc_filter_conv(int na, int nd, const double* uk, const double* p, double* out) {
    const int nd2 = 2 * nd - 1;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < (long)na * nd; ++r) {
        int a = (int)(r / nd), d = (int)(r % nd);
        double acc = 0.0;
        for (int e = 0; e < nd; ++e) acc += uk[(size_t)a * nd2 + (d - e) + nd - 1] * p[(size_t)a * nd + e];
        out[r] = acc;
    }
}

/* Disc subtraction (Sec. 3.3).  D = the disc of diameter N centred on the rotation
 * axis: the pixels whose centre lies within N/2 of it.  Its grey value g minimises
 * sum_a (sum_d (p - g W D)[a][d])^2, the squared l2 norm of the zero-frequency
 * components of all projections:  g = sum_a P_a T_a / sum_a T_a^2,
 * P_a = sum_d p[a][d], T_a = sum_d (W D)[a][d].  Writes pd = p - g W D, returns g.
 * disc (optional): receives D [N][N]. */
double orc_disc(int N, int na, int nd, const double* ang, const double* p, double* pd, double* disc) {
    const size_t nn = (size_t)N * N, ns = (size_t)na * nd;
    double* D = (double*)malloc(sizeof(double) * nn);
    double* wd = (double*)malloc(sizeof(double) * ns);
    const double half = 0.5 * (N - 1), r2 = 0.25 * (double)N * N;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double x = j - half, y = half - i;
            D[(size_t)i * N + j] = (x * x + y * y <= r2) ? 1.0 : 0.0;
        }
    orc_forward(N, na, nd, ang, 0, 0, N, N, D, 0, 0, 0, 0, wd);
    double num = 0.0, den = 0.0;
    for (int a = 0; a < na; ++a) {
        double P = 0.0, T = 0.0;
        for (int d = 0; d < nd; ++d) {
            P += p[(size_t)a * nd + d];
            T += wd[(size_t)a * nd + d];
        }
        num += P * T;
        den += T * T;
    }
    double g = den > 0.0 ? num / den : 0.0;
    for (size_t r = 0; r < ns; ++r) pd[r] = p[r] - g * wd[r];
    if (disc) memcpy(disc, D, sizeof(double) * nn);
    free(D);
    free(wd);
    return g;
}

/* ---------------------------------------------------------------------------
 * Alg. method (Sec. 3.2, Eq. localmethod) on the local part L = the box, with the
 * box constraint of Eq. sirtbox as the prior term d:
 *     y^0 = 0;  for k = 1..n:
 *         x_s^k = FBP_L(p, u_k) = W_L^T C_{u_k} p
 *         s     = x_s^k + y^{k-1} - alpha W_L^T W_L y^{k-1}      (= S(x^{k-1}) on L)
 *         x^k   = clamp(s + shift, lo, hi) - shift              (d^k = x^k - s)
 *         y^k   = x^k - x_s^k
 *     result x^n + shift.
 * shift (optional, box [bh][bw]) is an image that is added back after the
 * reconstruction (the disc of Sec. 3.3, restricted to the box), so the constraint
 * applies to the final image; lo = -inf / hi = +inf switch a side off.
 * W_L and W_L^T use every bin of the detector (bins whose rays miss the box add 0).
 * p: [na][nd] (disc-subtracted data), u: [n][na][2 nd - 1], x: box [bh][bw].
 * ------------------------------------------------------------------------- */
void orc_filter_method(int N, int na, int nd, const double* ang,
                       int bx0, int by0, int bw, int bh,
                       const double* p, int n, double alpha, const double* u,
                       const double* shift, double lo, double hi, double* x) {
    const size_t nb = (size_t)bw * bh, ns = (size_t)na * nd, nu = (size_t)na * (2 * nd - 1);
    double* cp = (double*)malloc(sizeof(double) * ns);
    double* xs = (double*)malloc(sizeof(double) * nb);
    double* y = (double*)calloc(nb, sizeof(double));
    double* wy = (double*)malloc(sizeof(double) * ns);
    double* g = (double*)malloc(sizeof(double) * nb);
    for (size_t i = 0; i < nb; ++i) x[i] = 0.0;
    for (int k = 1; k <= n; ++k) {
        orc_filter_conv(na, nd, u + (size_t)(k - 1) * nu, p, cp);
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, cp, xs);
        orc_forward(N, na, nd, ang, bx0, by0, bw, bh, y, 0, 0, 0, 0, wy);
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, wy, g);
        for (size_t i = 0; i < nb; ++i) {
            double sh = shift ? shift[i] : 0.0;
            double s = xs[i] + y[i] - alpha * g[i];
            double v = s + sh;
            if (v < lo) v = lo;
            if (v > hi) v = hi;
            x[i] = v - sh;
        }
        for (size_t i = 0; i < nb; ++i) y[i] = x[i] - xs[i];
    }
    for (size_t i = 0; i < nb; ++i) x[i] += shift ? shift[i] : 0.0;
    free(cp);
    free(xs);
    free(y);
    free(wy);
    free(g);
}

/* ---------------------------------------------------------------------------
 * FGP (the fast gradient projection of Beck & Teboulle 2009, named in Sec. 3.2 for
 * Alg. methodfista): the TV denoising problem
 *     min_x ||x - z||^2 + 2 lam TV(x),  TV(x) = sum |grad x|_2 (isotropic, orc_grad),
 * solved through its dual: x(v) = z + lam div v, and projected gradient ascent on v with
 * |v_ij|_2 <= 1, step 1/(8 lam) (||div||^2 <= 8), accelerated by the FISTA sequence:
 *     v_0 = r_1 = 0, t_1 = 1;  for k = 1..iters:
 *         x   = z + lam div r_k
 *         v_k = P(r_k + grad x / (8 lam))          P: v_ij <- v_ij / max(1, |v_ij|)
 *         t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
 *         r_{k+1} = v_k + ((t_k - 1) / t_{k+1}) (v_k - v_{k-1})
 *     x = z + lam div v_iters.
 * lam = 0 returns z.  Image [h][w].
 * ------------------------------------------------------------------------- */
void orc_fgp(int w, int h, const double* z, double lam, int iters, double* x) {
    const size_t n = (size_t)w * h;
    if (lam <= 0.0 || iters <= 0) {
        memcpy(x, z, sizeof(double) * n);
        return;
    }
    double* vx = (double*)calloc(n, sizeof(double));
    double* vy = (double*)calloc(n, sizeof(double));
    double* rx = (double*)calloc(n, sizeof(double));
    double* ry = (double*)calloc(n, sizeof(double));
    double* gx = (double*)malloc(sizeof(double) * n);
    double* gy = (double*)malloc(sizeof(double) * n);
    double* dv = (double*)malloc(sizeof(double) * n);
    double t = 1.0;
    for (int k = 1; k <= iters; ++k) {
        orc_div(w, h, rx, ry, dv);
        for (size_t i = 0; i < n; ++i) x[i] = z[i] + lam * dv[i];
        orc_grad(w, h, x, gx, gy);
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double beta = (t - 1.0) / tn;
        for (size_t i = 0; i < n; ++i) {
            double ax = rx[i] + gx[i] / (8.0 * lam), ay = ry[i] + gy[i] / (8.0 * lam);
            double m = sqrt(ax * ax + ay * ay);
            if (m > 1.0) {
                ax /= m;
                ay /= m;
            }
            rx[i] = ax + beta * (ax - vx[i]);
            ry[i] = ay + beta * (ay - vy[i]);
            vx[i] = ax;
            vy[i] = ay;
        }
        t = tn;
    }
    orc_div(w, h, vx, vy, dv);
    for (size_t i = 0; i < n; ++i) x[i] = z[i] + lam * dv[i];
    free(vx);
    free(vy);
    free(rx);
    free(ry);
    free(gx);
    free(gy);
    free(dv);
}

/* ---------------------------------------------------------------------------
 * Alg. methodfista (Sec. 3.2): the paper's local method with FISTA minimising
 * ||p - W x||^2 + lambda TV(x) (Eq. priorsys with g = TV), the TV prox by FGP:
 *     t_0 = 1, x_L = 0, x^0 = 0;  for k = 1..n:
 *         x_s = FBP_L(p, u_k) = W_L^T C_{u_k} p
 *         q   = x_L - alpha W_L^T W_L x_L
 *         x^k = FGP(x_s + q + shift, lam_f, n_fgp) - shift
 *         t_k = (1 + sqrt(1 + 4 t_{k-1}^2)) / 2
 *         r   = x^k + ((t_{k-1} - 1) / t_k) (x^k - x^{k-1})
 *         x_L = r - x_s
 *     result x^n + shift.
 * Readings: the t and r lines of the printed algorithm are garbled; they are taken as
 * the standard FISTA updates above.  The SIRT step x + alpha W^T (p - W x) is a gradient
 * step of ||p - W x||^2 with step alpha / 2, so the prox of lambda TV at that step is the
 * FGP problem with lam_f = alpha lambda / 2.  The prox acts on the image with the disc of
 * Sec. 3.3 added back (shift), like the box constraint of orc_filter_method.
 * ------------------------------------------------------------------------- */
void orc_filter_fista(int N, int na, int nd, const double* ang,
                      int bx0, int by0, int bw, int bh,
                      const double* p, int n, double alpha, const double* u,
                      const double* shift, double lambda, int n_fgp, double* x) {
    const size_t nb = (size_t)bw * bh, ns = (size_t)na * nd, nu = (size_t)na * (2 * nd - 1);
    double* cp = (double*)malloc(sizeof(double) * ns);
    double* xs = (double*)malloc(sizeof(double) * nb);
    double* xl = (double*)calloc(nb, sizeof(double));
    double* xprev = (double*)calloc(nb, sizeof(double));
    double* z = (double*)malloc(sizeof(double) * nb);
    double* wy = (double*)malloc(sizeof(double) * ns);
    double* g = (double*)malloc(sizeof(double) * nb);
    const double lam_f = 0.5 * alpha * lambda;
    double t = 1.0;
    for (int k = 1; k <= n; ++k) {
        orc_filter_conv(na, nd, u + (size_t)(k - 1) * nu, p, cp);
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, cp, xs);
        orc_forward(N, na, nd, ang, bx0, by0, bw, bh, xl, 0, 0, 0, 0, wy);
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, wy, g);
        for (size_t i = 0; i < nb; ++i) z[i] = xs[i] + xl[i] - alpha * g[i] + (shift ? shift[i] : 0.0);
        orc_fgp(bw, bh, z, lam_f, n_fgp, x);
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double beta = (t - 1.0) / tn;
        for (size_t i = 0; i < nb; ++i) {
            double xk = x[i] - (shift ? shift[i] : 0.0);
            double r = xk + beta * (xk - xprev[i]);
            xl[i] = r - xs[i];
            xprev[i] = xk;
        }
        t = tn;
    }
    for (size_t i = 0; i < nb; ++i) x[i] = xprev[i] + (shift ? shift[i] : 0.0);
    free(cp);
    free(xs);
    free(xl);
    free(xprev);
    free(z);
    free(wy);
    free(g);
}

/* ---------------------------------------------------------------------------
 * Haar wavelet ISTA inside the paper's method (Eq. sirtista, d of Alg. method).
 * B is the orthonormal 2D Haar decomposition of a [h][w] box image:
 *   level 0 block = the whole image; at each level, while the block [hl][wl] has hl >= 2
 *   and wl >= 2 (and at most `levels` levels): every row of the block becomes
 *   [pair sums / sqrt(2) | pair differences / sqrt(2)] -- entries 2j, 2j+1 give sum j and
 *   difference ceil(wl/2) + j; an odd last entry is copied to sum position wl/2 -- then
 *   every column of the block the same way; the next block is [ceil(hl/2)][ceil(wl/2)].
 * Every step is orthogonal, so B^-1 = B^T (orc_haar_inv undoes the steps in reverse).
 * ------------------------------------------------------------------------- */
static void haar_split(const double* in, double* out, int L, int stride) {
    const int m = L / 2, c = (L + 1) / 2;
    const double s = 1.0 / sqrt(2.0);
    for (int j = 0; j < m; ++j) {
        double a = in[(size_t)(2 * j) * stride], b = in[(size_t)(2 * j + 1) * stride];
        out[(size_t)j * stride] = s * (a + b);
        out[(size_t)(c + j) * stride] = s * (a - b);
    }
    if (L % 2) out[(size_t)m * stride] = in[(size_t)(L - 1) * stride];
}

static void haar_merge(const double* in, double* out, int L, int stride) {
    const int m = L / 2, c = (L + 1) / 2;
    const double s = 1.0 / sqrt(2.0);
    for (int j = 0; j < m; ++j) {
        double u = in[(size_t)j * stride], v = in[(size_t)(c + j) * stride];
        out[(size_t)(2 * j) * stride] = s * (u + v);
        out[(size_t)(2 * j + 1) * stride] = s * (u - v);
    }
    if (L % 2) out[(size_t)(L - 1) * stride] = in[(size_t)m * stride];
}

static int haar_levels(int w, int h, int levels, int* hl, int* wl) {
    int n = 0;
    int H = h, Wd = w;
    while (n < levels && H >= 2 && Wd >= 2) {
        hl[n] = H;
        wl[n] = Wd;
        H = (H + 1) / 2;
        Wd = (Wd + 1) / 2;
        ++n;
    }
    return n;
}

void orc_haar(int w, int h, int levels, const double* x, double* c) {
    int hl[32], wl[32];
    const int n = haar_levels(w, h, levels > 32 ? 32 : levels, hl, wl);
    double* t = (double*)malloc(sizeof(double) * (size_t)w * h);
    memcpy(c, x, sizeof(double) * (size_t)w * h);
    for (int l = 0; l < n; ++l) {
        for (int i = 0; i < hl[l]; ++i) haar_split(c + (size_t)i * w, t + (size_t)i * w, wl[l], 1);
        for (int j = 0; j < wl[l]; ++j) haar_split(t + j, c + j, hl[l], w);
    }
    free(t);
}

void orc_haar_inv(int w, int h, int levels, const double* c, double* x) {
    int hl[32], wl[32];
    const int n = haar_levels(w, h, levels > 32 ? 32 : levels, hl, wl);
    double* t = (double*)malloc(sizeof(double) * (size_t)w * h);
    memcpy(x, c, sizeof(double) * (size_t)w * h);
    for (int l = n - 1; l >= 0; --l) {
        for (int j = 0; j < wl[l]; ++j) haar_merge(x + j, t + j, hl[l], w);
        for (int i = 0; i < hl[l]; ++i) haar_merge(t + (size_t)i * w, x + (size_t)i * w, wl[l], 1);
    }
    free(t);
}

/* Alg. method with the ISTA prior of Eq. sirtista (l1 norm of the Haar coefficients):
 *     s   = x_s^k + y^{k-1} - alpha W_L^T W_L y^{k-1}
 *     x^k = B^-1 P_tau(B (s + shift)) - shift,   tau = alpha lambda / 2
 *     y^k = x^k - x_s^k;  result x^n + shift.
 * P_tau is soft thresholding of every coefficient (sgn(c) max(|c| - tau, 0)); tau follows
 * from the SIRT step being a gradient step of ||p - W x||^2 with step alpha / 2, as for
 * orc_filter_fista. */
void orc_filter_ista(int N, int na, int nd, const double* ang,
                     int bx0, int by0, int bw, int bh,
                     const double* p, int n, double alpha, const double* u,
                     const double* shift, double lambda, int levels, double* x) {
    const size_t nb = (size_t)bw * bh, ns = (size_t)na * nd, nu = (size_t)na * (2 * nd - 1);
    double* cp = (double*)malloc(sizeof(double) * ns);
    double* xs = (double*)malloc(sizeof(double) * nb);
    double* y = (double*)calloc(nb, sizeof(double));
    double* wy = (double*)malloc(sizeof(double) * ns);
    double* g = (double*)malloc(sizeof(double) * nb);
    double* z = (double*)malloc(sizeof(double) * nb);
    double* cf = (double*)malloc(sizeof(double) * nb);
    const double tau = 0.5 * alpha * lambda;
    for (size_t i = 0; i < nb; ++i) x[i] = 0.0;
    for (int k = 1; k <= n; ++k) {
        orc_filter_conv(na, nd, u + (size_t)(k - 1) * nu, p, cp);
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, cp, xs);
        orc_forward(N, na, nd, ang, bx0, by0, bw, bh, y, 0, 0, 0, 0, wy);
        orc_back(N, na, nd, ang, bx0, by0, bw, bh, 0, 0, 0, 0, wy, g);
        for (size_t i = 0; i < nb; ++i) z[i] = xs[i] + y[i] - alpha * g[i] + (shift ? shift[i] : 0.0);
        orc_haar(bw, bh, levels, z, cf);
        for (size_t i = 0; i < nb; ++i) {
            double a = fabs(cf[i]) - tau;
            cf[i] = a > 0.0 ? (cf[i] > 0.0 ? a : -a) : 0.0;
        }
        orc_haar_inv(bw, bh, levels, cf, x);
        for (size_t i = 0; i < nb; ++i) {
            x[i] -= shift ? shift[i] : 0.0;
            y[i] = x[i] - xs[i];
        }
    }
    for (size_t i = 0; i < nb; ++i) x[i] += shift ? shift[i] : 0.0;
    free(cp);
    free(xs);
    free(y);
    free(wy);
    free(g);
    free(z);
    free(cf);
}
