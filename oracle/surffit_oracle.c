/*
 * surffit_oracle.c -- plain, slow, FP64 CPU oracle for dense RGBD plane fitting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, imports or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes, for every pixel p of a W x H depth image and a k x k
 * window centred on p (k odd, r = (k-1)/2), following
 * "Real-Time Surface Fitting to RGBD Sensor Data" (Papadakis & Willis):
 *
 *  1. V(p): pixels q of the window inside the image whose depth Z_q is finite
 *     and > 0; n = |V(p)|.  Pixels outside the image count as missing.
 *  2. p is valid when n >= min_valid and (if require_center) p itself is in V.
 *     Invalid pixels get NaN normal, offset and curvature.
 *  3. Direct window sums over V (no integral images, the "naive" structure of
 *     Section III.B):
 *       standard (Eq. 1, Eq. 6): P = Z*m, A = sum P P^T, g = sum P, s = n
 *       disparity (Eq. 10, Eq. 14): A = sum m m^T, g = sum (1/Z) m, s = sum 1/Z^2
 *     with the ray m = [(x+dx-cx)/fx, (y+dy-cy)/fy, 1] of Eq. 10.
 *     [[A, g], [g^T, s]] is the 4x4 scatter matrix M^T M of Eq. 6 / Eq. 14.
 *  4. Constraint |(a,b,c)| = 1 (the reading under which the fit is Euclidean
 *     invariant, Section I.C): the offset d is eliminated, leaving the Schur
 *     complement R = A - g g^T / s, whose smallest eigenvector is the unit
 *     normal (Eq. 4-5 restricted to the normal).  The literal constraint
 *     |(a,b,c,d)| = 1 of Eq. 4 is available as constraint mode 1: smallest
 *     eigenvector alpha of the 4x4 scatter, n = alpha[0:3]/|alpha[0:3]|,
 *     d = alpha[3]/|alpha[0:3]|.
 *  5. d = -n.g/s; if d < 0 flip n and d; if d == 0 make n_z < 0, and if n_z is
 *     0 too make the first nonzero component negative.
 *  6. curvature = lambda0 / (lambda0 + lambda1 + lambda2) of R (0 if the trace is 0).
 *
 * Explicit fits (Section I.D and II.B) are methods 2 and 3 (a window whose
 * valid pixels are collinear in the image has no explicit fit: NaN):
 *     explicit disparity (Eq. 15-16): minimise sum (a tx + b ty + c - 1/Z)^2,
 *         alpha = (M^T M)^-1 M^T b with M rows [tx, ty, 1], b = 1/Z.  The plane
 *         a tx + b ty + c - 1/Z = 0 is n.P + d = 0 with n ~ (a,b,c), d ~ -1.
 *     explicit standard (Eq. 7-9): minimise sum (aX + bY + c - Z)^2, the plane
 *         aX + bY - Z + c = 0, n ~ (a, b, -1), d ~ c.
 *     Their third output is the mean squared residual in the fit's own units.
 *
 * The eigen-solver is cyclic Jacobi in FP64, run until the off-diagonal mass
 * is below 1e-15 of the Frobenius norm.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { M_DISPARITY = 0, M_STANDARD = 1, M_EXPLICIT_DISPARITY = 2, M_EXPLICIT_STANDARD = 3 };

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi for a symmetric n x n matrix (n <= 4).                      */
/* On return a[] holds the eigenvalues on its diagonal; v (row-major, n x n) */
/* holds the eigenvectors in its COLUMNS.                                    */
/* ------------------------------------------------------------------------ */
static void jacobi_sym(int n, double a[4][4], double v[4][4]) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) v[i][j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) fro += a[i][j] * a[i][j];
    fro = sqrt(fro);
    if (fro == 0.0) return;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += a[i][j] * a[i][j];
        if (sqrt(off) <= 1e-15 * fro) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                if (a[p][q] == 0.0) continue;
                /* rotation angle that zeroes a[p][q] */
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* columns p, q */
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* rows p, q */
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - s * vkq;
                    v[k][q] = s * vkp + c * vkq;
                }
            }
        }
    }
}

/* Sorted eigen-decomposition: lam ascending, vec[k] = unit eigenvector k. */
static void eig_sorted(int n, const double m[4][4], double lam[4], double vec[4][4]) {
    double a[4][4], v[4][4];
    memcpy(a, m, sizeof(a));
    jacobi_sym(n, a, v);
    int idx[4] = {0, 1, 2, 3};
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (a[idx[j]][idx[j]] < a[idx[i]][idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int i = 0; i < n; ++i) {
        lam[i] = a[idx[i]][idx[i]];
        double nn = 0.0;
        for (int k = 0; k < n; ++k) nn += v[k][idx[i]] * v[k][idx[i]];
        nn = sqrt(nn);
        for (int k = 0; k < n; ++k) vec[i][k] = v[k][idx[i]] / nn;
    }
}

/* Orientation rule: d > 0; ties broken toward n_z < 0, then first nonzero < 0. */
static void orient(double nrm[3], double* d) {
    int flip = 0;
    if (*d < 0) flip = 1;
    else if (*d == 0.0) {
        if (nrm[2] > 0) flip = 1;
        else if (nrm[2] == 0.0) {
            for (int i = 0; i < 3; ++i) {
                if (nrm[i] != 0.0) { flip = nrm[i] > 0; break; }
            }
        }
    }
    if (flip) { nrm[0] = -nrm[0]; nrm[1] = -nrm[1]; nrm[2] = -nrm[2]; *d = -*d; }
}

static inline int valid_depth(double z) { return isfinite(z) && z > 0.0; }

/* Direct sums of the method's monomials over the valid pixels of the box
 * [xa, xb] x [ya, yb] (inclusive, clipped to the image).
 * A: 3x3, g: 3, s: scalar; also bb = sum b^2 (explicit fits only); pm: the
 * pixel offsets from the reference pixel (px, py), NULL allowed.
 * ddx, ddy: per-pixel adjustments [H][W] added to (dx, dy) in the rays of
 * Eq. 1 / Eq. 10, or NULL (constant dx, dy only). */
static int box_sums(const double* Z, int W, int H, const double* intr, const double* ddx, const double* ddy,
                    int method, int xa, int xb, int ya, int yb, int px, int py, double A[3][3], double g[3],
                    double* s, double* bb, int64_t pm[5]) {
    const double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3], dx = intr[4], dy = intr[5];
    memset(A, 0, 9 * sizeof(double));
    g[0] = g[1] = g[2] = 0.0;
    *s = 0.0; *bb = 0.0;
    int n = 0;
    if (pm) pm[0] = pm[1] = pm[2] = pm[3] = pm[4] = 0;
    for (int y = ya; y <= yb; ++y) {
        if (y < 0 || y >= H) continue;
        const double ty0 = (y + dy - cy) / fy;
        for (int x = xa; x <= xb; ++x) {
            if (x < 0 || x >= W) continue;
            const size_t q = (size_t)y * W + x;
            const double z = Z[q];
            if (!valid_depth(z)) continue;
            const double tx = ddx ? (x + dx + ddx[q] - cx) / fx : (x + dx - cx) / fx;
            const double ty = ddy ? (y + dy + ddy[q] - cy) / fy : ty0;
            double u[3];
            double wgt, b;
            if (method == M_DISPARITY || method == M_EXPLICIT_DISPARITY) {
                /* Eq. 14 / Eq. 16: monomials [tx, ty, 1] and 1/Z */
                u[0] = tx; u[1] = ty; u[2] = 1.0;
                wgt = 1.0 / z; b = wgt;
            } else if (method == M_STANDARD) {
                /* Eq. 6: monomials [X, Y, Z] and 1 */
                u[0] = z * tx; u[1] = z * ty; u[2] = z;
                wgt = 1.0; b = 1.0;
            } else {
                /* Eq. 9: monomials [X, Y, 1], target Z */
                u[0] = z * tx; u[1] = z * ty; u[2] = 1.0;
                wgt = z; b = z;
            }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) A[i][j] += u[i] * u[j];
            for (int i = 0; i < 3; ++i) g[i] += wgt * u[i];
            *s += wgt * wgt;
            *bb += b * b;
            ++n;
            if (pm) {  /* pixel offsets from the reference pixel: sum j, i, j^2, j i, i^2 */
                const int64_t j = x - px, i = y - py;
                pm[0] += j; pm[1] += i; pm[2] += j * j; pm[3] += j * i; pm[4] += i * i;
            }
        }
    }
    return n;
}

/* Direct window sums over V(p): the k x k box centred on p. */
static int window_sums(const double* Z, int W, int H, const double* intr, const double* ddx, const double* ddy,
                       int r, int method, int px, int py, double A[3][3], double g[3], double* s, double* bb,
                       int64_t pm[5]) {
    return box_sums(Z, W, H, intr, ddx, ddy, method, px - r, px + r, py - r, py + r, px, py, A, g, s, bb, pm);
}

/* Solve the 3x3 symmetric system A x = g in FP64 by Gaussian elimination with
 * partial pivoting.  Returns 0 when A is singular. */
static int solve3(const double A[3][3], const double g[3], double x[3]) {
    double m[3][4];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) m[i][j] = A[i][j];
        m[i][3] = g[i];
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int i = c + 1; i < 3; ++i)
            if (fabs(m[i][c]) > fabs(m[piv][c])) piv = i;
        if (m[piv][c] == 0.0) return 0;
        if (piv != c)
            for (int j = 0; j < 4; ++j) { double t = m[c][j]; m[c][j] = m[piv][j]; m[piv][j] = t; }
        for (int i = c + 1; i < 3; ++i) {
            double f = m[i][c] / m[c][c];
            for (int j = c; j < 4; ++j) m[i][j] -= f * m[c][j];
        }
    }
    for (int i = 2; i >= 0; --i) {
        double acc = m[i][3];
        for (int j = i + 1; j < 3; ++j) acc -= m[i][j] * x[j];
        x[i] = acc / m[i][i];
    }
    return 1;
}

/*
 * The fit of one set of sums (steps 2-6 of the header), shared by the
 * per-pixel windows and the rectangles of the quadtree.
 *   n, pm    valid count and pixel-offset moments (explicit rank rule)
 *   outputs  nrm[3], d, third (curvature, or the mean squared residual of an
 *            explicit fit), l[3] eigenvalues of R ascending (NaN for explicit
 *            fits), lam0 (the minimised residual: lambda0 of R, or the
 *            residual sum of an explicit fit)
 * Returns 1 when the fit is defined, 0 when it is not (then nothing is set).
 */
static int fit_sums(int method, int unit4, double A[3][3], const double g[3], double s, double bb, int n,
                    const int64_t pm[5], double nrm[3], double* d_out, double* third_out, double l_out[3],
                    double* lam0_out) {
    if (method <= M_STANDARD && s <= 0.0) return 0;
    if (method >= M_EXPLICIT_DISPARITY) {
        /* An explicit fit needs a design matrix of full rank: the valid
         * pixels must not be collinear in the image, decided exactly on
         * integer offsets, n^2 det cov(j, i) != 0. */
        const int64_t nn = n;
        const int64_t cjj = nn * pm[2] - pm[0] * pm[0], cii = nn * pm[4] - pm[1] * pm[1];
        const int64_t cji = nn * pm[3] - pm[0] * pm[1];
        if (cjj * cii - cji * cji == 0) return 0;
    }
    double d, third;
    if (method <= M_STANDARD) {
        double R[4][4] = {{0}}, l[4], vec[4][4];
        if (!unit4) {
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) R[i][j] = A[i][j] - g[i] * g[j] / s;
            eig_sorted(3, R, l, vec);
            for (int i = 0; i < 3; ++i) nrm[i] = vec[0][i];
            d = -(nrm[0] * g[0] + nrm[1] * g[1] + nrm[2] * g[2]) / s;
            double tr = l[0] + l[1] + l[2];
            third = tr != 0.0 ? l[0] / tr : 0.0;
        } else {
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) R[i][j] = A[i][j];
                R[i][3] = R[3][i] = g[i];
            }
            R[3][3] = s;
            eig_sorted(4, R, l, vec);
            double nn = sqrt(vec[0][0] * vec[0][0] + vec[0][1] * vec[0][1] + vec[0][2] * vec[0][2]);
            for (int i = 0; i < 3; ++i) nrm[i] = vec[0][i] / nn;
            d = vec[0][3] / nn;
            double tr = l[0] + l[1] + l[2] + l[3];
            third = tr != 0.0 ? l[0] / tr : 0.0;
        }
        l_out[0] = l[0]; l_out[1] = l[1]; l_out[2] = l[2];
        *lam0_out = l[0];
    } else {
        double x[3];
        if (!solve3(A, g, x)) return 0;
        /* residual sum b^T b - alpha^T M^T b (normal equations) */
        double res = bb - (x[0] * g[0] + x[1] * g[1] + x[2] * g[2]);
        third = res / n;
        double v[3];
        if (method == M_EXPLICIT_DISPARITY) { v[0] = x[0]; v[1] = x[1]; v[2] = x[2]; d = -1.0; }
        else { v[0] = x[0]; v[1] = x[1]; v[2] = -1.0; d = x[2]; }
        double nn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int i = 0; i < 3; ++i) nrm[i] = v[i] / nn;
        d /= nn;
        l_out[0] = l_out[1] = l_out[2] = NAN;
        *lam0_out = res;
    }
    orient(nrm, &d);
    *d_out = d;
    *third_out = third;
    return 1;
}

/* Steps 1-6 of the header for the window of pixel (px, py); results go to output slot o. */
static void fit_pixel(const double* Z, int W, int H, const double* intr, const double* ddx, const double* ddy, int r,
                      int method, int unit4, int min_valid, int require_center, int px, int py, size_t o,
                      double* normals, double* offsets, double* curv, int32_t* counts, double* lam,
                      double* moments) {
    double A[3][3], g[3], s, bb;
    int64_t pm[5];
    int n = window_sums(Z, W, H, intr, ddx, ddy, r, method, px, py, A, g, &s, &bb, pm);
    if (counts) counts[o] = n;
    if (moments) {
        double* mo = moments + o * 10;
        mo[0] = A[0][0]; mo[1] = A[0][1]; mo[2] = A[0][2];
        mo[3] = A[1][1]; mo[4] = A[1][2]; mo[5] = A[2][2];
        mo[6] = g[0]; mo[7] = g[1]; mo[8] = g[2]; mo[9] = s;
    }
    int ok = n >= min_valid && n > 0;
    if (require_center && !valid_depth(Z[(size_t)py * W + px])) ok = 0;
    double nrm[3], d, third, l[3], lam0;
    if (ok) ok = fit_sums(method, unit4, A, g, s, bb, n, pm, nrm, &d, &third, l, &lam0);
    if (!ok) {
        normals[3 * o] = normals[3 * o + 1] = normals[3 * o + 2] = NAN;
        offsets[o] = NAN; curv[o] = NAN;
        if (lam) lam[3 * o] = lam[3 * o + 1] = lam[3 * o + 2] = NAN;
        return;
    }
    normals[3 * o] = nrm[0]; normals[3 * o + 1] = nrm[1]; normals[3 * o + 2] = nrm[2];
    offsets[o] = d;
    curv[o] = third;
    if (lam) { lam[3 * o] = l[0]; lam[3 * o + 1] = l[1]; lam[3 * o + 2] = l[2]; }
}

/*
 * sfo_fit: the whole forward oracle.
 *   Z        [H*W] depth (metres), non-finite or <= 0 means missing
 *   intr     fx, fy, cx, cy, dx, dy
 *   k        odd window size
 *   method   0 disparity (implicit), 1 standard (implicit), 2 explicit disparity, 3 explicit standard
 *   unit4    0: |(a,b,c)| = 1 (Schur complement); 1: |(a,b,c,d)| = 1 (literal Eq. 4)
 *   outputs  normals [H*W*3], offsets [H*W], curv [H*W], counts [H*W]
 *   lam      optional [H*W*3] eigenvalues of R, ascending (implicit methods)
 *   moments  optional [H*W*10]: A11 A12 A13 A22 A23 A33 g1 g2 g3 s
 * Returns 0 on success, -1 on bad arguments.
 */
int sfo_fit_delta(const double* Z, int W, int H, const double* intr, const double* ddx, const double* ddy, int k,
                  int method, int unit4, int min_valid, int require_center, double* normals, double* offsets,
                  double* curv, int32_t* counts, double* lam, double* moments, int nthreads);

int sfo_fit(const double* Z, int W, int H, const double* intr, int k, int method, int unit4,
            int min_valid, int require_center, double* normals, double* offsets, double* curv,
            int32_t* counts, double* lam, double* moments, int nthreads) {
    return sfo_fit_delta(Z, W, H, intr, NULL, NULL, k, method, unit4, min_valid, require_center, normals, offsets,
                         curv, counts, lam, moments, nthreads);
}

/* sfo_fit with per-pixel ray adjustments ddx, ddy [H*W] (pixels, added to
 * intr's dx, dy in Eq. 1 / Eq. 10), or NULL for none. */
int sfo_fit_delta(const double* Z, int W, int H, const double* intr, const double* ddx, const double* ddy, int k,
                  int method, int unit4, int min_valid, int require_center, double* normals, double* offsets,
                  double* curv, int32_t* counts, double* lam, double* moments, int nthreads) {
    if (!Z || W <= 0 || H <= 0 || !intr || k < 1 || (k & 1) == 0 || method < 0 || method > 3 || (!ddx != !ddy))
        return -1;
    const int r = (k - 1) / 2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 2)
#endif
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px)
            fit_pixel(Z, W, H, intr, ddx, ddy, r, method, unit4, min_valid, require_center, px, py,
                      (size_t)py * W + px, normals, offsets, curv, counts, lam, moments);
    return 0;
}

/*
 * sfo_fit_at: sfo_fit evaluated at npix pixels only, xy = [x0, y0, x1, y1, ...];
 * output slot i holds pixel i (same layouts as sfo_fit with H*W -> npix).
 * sfo_fit_at_delta: the same with per-pixel ray adjustments (as sfo_fit_delta).
 */
int sfo_fit_at_delta(const double* Z, int W, int H, const double* intr, const double* ddx, const double* ddy, int k,
                     int method, int unit4, int min_valid, int require_center, int npix, const int32_t* xy,
                     double* normals, double* offsets, double* curv, int32_t* counts, double* lam, double* moments,
                     int nthreads) {
    if (!Z || W <= 0 || H <= 0 || !intr || k < 1 || (k & 1) == 0 || method < 0 || method > 3 || npix < 0 || !xy ||
        (!ddx != !ddy))
        return -1;
    for (int i = 0; i < npix; ++i)
        if (xy[2 * i] < 0 || xy[2 * i] >= W || xy[2 * i + 1] < 0 || xy[2 * i + 1] >= H) return -1;
    const int r = (k - 1) / 2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int i = 0; i < npix; ++i)
        fit_pixel(Z, W, H, intr, ddx, ddy, r, method, unit4, min_valid, require_center, xy[2 * i], xy[2 * i + 1],
                  (size_t)i, normals, offsets, curv, counts, lam, moments);
    return 0;
}

int sfo_fit_at(const double* Z, int W, int H, const double* intr, int k, int method, int unit4, int min_valid,
               int require_center, int npix, const int32_t* xy, double* normals, double* offsets, double* curv,
               int32_t* counts, double* lam, double* moments, int nthreads) {
    return sfo_fit_at_delta(Z, W, H, intr, NULL, NULL, k, method, unit4, min_valid, require_center, npix, xy, normals,
                            offsets, curv, counts, lam, moments, nthreads);
}

/*
 * sfo_fit_rect: the fit of one rectangle of pixels, [x0, x0 + w) x [y0, y0 + h)
 * clipped to the image (the grid tiles of the planar segmentation, Section
 * III), with the same sums and solve as the per-pixel windows.  The pixel
 * offsets of the explicit rank rule are taken from (x0, y0).
 *   out[0..2] normal, out[3] offset, out[4] curvature (or mean squared
 *   residual), out[5..7] eigenvalues of R, out[8] the minimised residual
 *   (lambda0, or the explicit residual sum); *count = valid pixels.
 * A rectangle whose valid pixels are collinear in the image has no surface
 * fit with any method: its implicit fit would be the plane through the camera
 * centre that contains their rays (d = 0), for every depth (exact integer
 * test on the pixel offsets, as for the explicit fits).
 * Returns 1 when the fit is defined, 0 when it is not (n < min_valid, no
 * data, collinear pixels; out is then NaN), -1 on bad arguments.
 */
int sfo_fit_rect(const double* Z, int W, int H, const double* intr, int x0, int y0, int w, int h, int method,
                 int min_valid, double* out, int32_t* count) {
    if (!Z || W <= 0 || H <= 0 || !intr || w <= 0 || h <= 0 || method < 0 || method > 3 || !out || !count)
        return -1;
    double A[3][3], g[3], s, bb;
    int64_t pm[5];
    int n = box_sums(Z, W, H, intr, NULL, NULL, method, x0, x0 + w - 1, y0, y0 + h - 1, x0, y0, A, g, &s, &bb, pm);
    *count = n;
    for (int i = 0; i < 9; ++i) out[i] = NAN;
    if (n < min_valid || n <= 0) return 0;
    {
        const int64_t nn = n;
        const int64_t cjj = nn * pm[2] - pm[0] * pm[0], cii = nn * pm[4] - pm[1] * pm[1];
        const int64_t cji = nn * pm[3] - pm[0] * pm[1];
        if (cjj * cii - cji * cji == 0) return 0;
    }
    double nrm[3], d, third, l[3], lam0;
    if (!fit_sums(method, 0, A, g, s, bb, n, pm, nrm, &d, &third, l, &lam0)) return 0;
    out[0] = nrm[0]; out[1] = nrm[1]; out[2] = nrm[2];
    out[3] = d; out[4] = third;
    out[5] = l[0]; out[6] = l[1]; out[7] = l[2];
    out[8] = lam0;
    return 1;
}

/*
 * sfo_backward: analytic FP64 adjoint of the implicit fit (unit3 constraint)
 * with respect to the depth image.
 *
 * Per valid pixel p, with R = A - g g^T/s and eigenpairs (lambda_k, v_k):
 *   curvature kappa = lambda0 / tr(R):  dkappa = v0^T dR v0 / tr - lambda0 tr(dR) / tr^2
 *   normal n = sigma v0 (sigma = +-1 from the orientation rule, locally constant):
 *       dv0 = sum_{k != 0} v_k (v_k^T dR v0) / (lambda0 - lambda_k)
 *   offset d = -n.g/s.
 * The adjoint gives dL/dA (symmetric), dL/dg, dL/ds per window; then every
 * pixel q collects, from each window p containing it:
 *   disparity: dL/dw_q = gbar_p . m_q + 2 w_q sbar_p, dL/dZ_q = -dL/dw_q / Z_q^2
 *   standard:  dL/dP_q = 2 Abar_p P_q + gbar_p,       dL/dZ_q = dL/dP_q . m_q
 * (A depends only on the mask in the disparity form; Abar_p is symmetric.)
 * Invalid pixels p contribute nothing; missing pixels q get gradient 0.
 */
int sfo_backward(const double* Z, int W, int H, const double* intr, int k, int method,
                 int min_valid, int require_center, const double* g_normals, const double* g_offsets,
                 const double* g_curv, double* g_depth, int nthreads) {
    if (!Z || W <= 0 || H <= 0 || !intr || k < 1 || (k & 1) == 0 || method < 0 || method > 1)
        return -1;
    const int r = (k - 1) / 2;
    const size_t N = (size_t)W * H;
    /* per-window adjoints: Abar (6 unique, symmetric), gbar (3), sbar (1) */
    double* adj = (double*)calloc(N * 10, sizeof(double));
    if (!adj) return -2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 2)
#endif
    for (int py = 0; py < H; ++py) {
        for (int px = 0; px < W; ++px) {
            const size_t o = (size_t)py * W + px;
            double A[3][3], g[3], s, bb;
            int n = window_sums(Z, W, H, intr, NULL, NULL, r, method, px, py, A, g, &s, &bb, NULL);
            int ok = n >= min_valid && n > 0 && s > 0.0;
            if (require_center && !valid_depth(Z[o])) ok = 0;
            if (!ok) continue;
            double R[4][4] = {{0}}, l[4], vec[4][4];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) R[i][j] = A[i][j] - g[i] * g[j] / s;
            eig_sorted(3, R, l, vec);
            double v0[3] = {vec[0][0], vec[0][1], vec[0][2]};
            double d0 = -(v0[0] * g[0] + v0[1] * g[1] + v0[2] * g[2]) / s;
            double nrm[3] = {v0[0], v0[1], v0[2]}, d = d0;
            orient(nrm, &d);
            double sigma = (nrm[0] * v0[0] + nrm[1] * v0[1] + nrm[2] * v0[2]) >= 0 ? 1.0 : -1.0;
            const double gn[3] = {g_normals[3 * o], g_normals[3 * o + 1], g_normals[3 * o + 2]};
            const double gd = g_offsets[o], gk = g_curv[o];
            /* d = -n.g/s */
            double nbar[3], gbar[3], sbar;
            for (int i = 0; i < 3; ++i) nbar[i] = gn[i] - gd * g[i] / s;
            for (int i = 0; i < 3; ++i) gbar[i] = -gd * nrm[i] / s;
            sbar = gd * (nrm[0] * g[0] + nrm[1] * g[1] + nrm[2] * g[2]) / (s * s);
            /* n = sigma v0 */
            double vbar[3] = {sigma * nbar[0], sigma * nbar[1], sigma * nbar[2]};
            /* Rbar from the eigenvector: sum_k c_k v_k v0^T, c_k = (vbar.v_k)/(l0 - l_k) */
            double Rb[3][3] = {{0}};
            for (int kk = 1; kk < 3; ++kk) {
                double den = l[0] - l[kk];
                if (den == 0.0) continue;
                double ck = (vbar[0] * vec[kk][0] + vbar[1] * vec[kk][1] + vbar[2] * vec[kk][2]) / den;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Rb[i][j] += ck * vec[kk][i] * v0[j];
            }
            /* curvature */
            double tr = l[0] + l[1] + l[2];
            if (tr != 0.0) {
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        Rb[i][j] += gk * (v0[i] * v0[j] / tr - (i == j ? l[0] / (tr * tr) : 0.0));
            }
            /* symmetrise: R only enters through symmetric perturbations */
            double Rs[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Rs[i][j] = 0.5 * (Rb[i][j] + Rb[j][i]);
            /* R = A - g g^T / s */
            for (int i = 0; i < 3; ++i) {
                double acc = 0.0;
                for (int j = 0; j < 3; ++j) acc += Rs[i][j] * g[j];
                gbar[i] += -2.0 * acc / s;
            }
            double gRg = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) gRg += g[i] * Rs[i][j] * g[j];
            sbar += gRg / (s * s);
            double* a = adj + o * 10;
            a[0] = Rs[0][0]; a[1] = Rs[0][1]; a[2] = Rs[0][2];
            a[3] = Rs[1][1]; a[4] = Rs[1][2]; a[5] = Rs[2][2];
            a[6] = gbar[0]; a[7] = gbar[1]; a[8] = gbar[2]; a[9] = sbar;
        }
    }
    const double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3], dx = intr[4], dy = intr[5];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 2)
#endif
    for (int qy = 0; qy < H; ++qy) {
        for (int qx = 0; qx < W; ++qx) {
            const size_t o = (size_t)qy * W + qx;
            const double z = Z[o];
            if (!valid_depth(z)) { g_depth[o] = 0.0; continue; }
            const double m[3] = {(qx + dx - cx) / fx, (qy + dy - cy) / fy, 1.0};
            double acc = 0.0;
            for (int py = qy - r; py <= qy + r; ++py) {
                if (py < 0 || py >= H) continue;
                for (int px = qx - r; px <= qx + r; ++px) {
                    if (px < 0 || px >= W) continue;
                    const double* a = adj + ((size_t)py * W + px) * 10;
                    if (method == M_DISPARITY) {
                        const double w = 1.0 / z;
                        double gw = a[6] * m[0] + a[7] * m[1] + a[8] * m[2] + 2.0 * w * a[9];
                        acc += -gw / (z * z);
                    } else {
                        const double P[3] = {z * m[0], z * m[1], z * m[2]};
                        const double Ab[3][3] = {{a[0], a[1], a[2]}, {a[1], a[3], a[4]}, {a[2], a[4], a[5]}};
                        double gP[3];
                        for (int i = 0; i < 3; ++i)
                            gP[i] = 2.0 * (Ab[i][0] * P[0] + Ab[i][1] * P[1] + Ab[i][2] * P[2]) + a[6 + i];
                        acc += gP[0] * m[0] + gP[1] * m[1] + gP[2] * m[2];
                    }
                }
            }
            g_depth[o] = acc;
        }
    }
    free(adj);
    return 0;
}

/* Exposed for the pins: the Jacobi eigen-decomposition of one symmetric matrix. */
int sfo_eig_sym(int n, const double* m, double* lam, double* vecs) {
    if (n < 1 || n > 4) return -1;
    double a[4][4] = {{0}}, l[4], v[4][4];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) a[i][j] = m[i * n + j];
    eig_sorted(n, a, l, v);
    for (int i = 0; i < n; ++i) {
        lam[i] = l[i];
        for (int j = 0; j < n; ++j) vecs[i * n + j] = v[i][j];
    }
    return 0;
}

int sfo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
