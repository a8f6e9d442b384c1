/*
 * sf_oracle.c -- plain FP64 CPU oracle of the per-frame predictor-update loop
 * of "Real-time Structure Flow" (Adarve & Mahony, arXiv 2406.18031).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the CUDA library computes.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg load it; the product
 * library never links, loads or calls it, and the two share no source,
 * header, table or constant.
 *
 * Style: every stage is written per pixel, in the paper's order and notation,
 * in double precision, as full-array passes (no fusion, tiling or
 * reordering).  Build with -O2 -ffp-contract=off so no FMA contraction
 * changes the rounding of the written expressions.  Optional OpenMP over
 * rows does not change any result (each output pixel is computed by exactly
 * one thread from read-only inputs).
 *
 * Notation (Sec. 3, Sec. 4): pixel p = (i, j), i = row (beta_2 axis),
 * j = column (beta_1 axis); eta = unit ray, B = [b1 b2] tangent basis,
 * dmu = pixel spacing; w = structure flow (rad/frame inside the filter),
 * dw = lower-level flow increment, rho = inverse depth, Y = brightness.
 *
 * Readings of points where the paper is silent, ambiguous or garbled are
 * marked [Rn]; the list is kept with the design notes of this repository:
 *  R1  dominant flow picks the neighbour speed of LARGER magnitude (Eqs.
 *      55-56 literally pick the smaller one; SFO_DOMINANT_LITERAL runs the
 *      literal text).  Ties go to the j-1 / i-1 neighbour.
 *  R2  the row-pass rho update of Eq. 65 uses the row operator and v-hat.
 *  R3  the scheme output is w^N (N full sub-iterations = one frame).
 *  R4  lifts to tangent space are dmu * B * d_beta (Eqs. 31, 34 write B^T),
 *      and Eq. 54 is Phi = (1/dmu) B^T P w.
 *  R5  image model residual uses the offset q - p.
 *  R6  E_t at the top level is w^{k+1} - w^{k+} (Eq. 45 prints a plus).
 *  R7  lower-level rho is transported by w_h (Eq. 40 prints w_H).
 *  R9  w is kept in rad/frame; a change of dt rescales w and dw.
 *  R10 gamma3 at level h is gamma[2] * (2^(h-1)/fx)^2.
 *  R11 top level temporal terms use Y^k, rho^k; lower levels use the
 *      propagated Y^{k+}, rho^{k+}.
 *  R12 lower levels propagate the fitted Y-hat.
 *  R13 every stencil replicates the border pixel (clamp to edge).
 *  R14 pyramid: 2x2 mean of Y; mean of the valid children's inverse depth;
 *      up-sampling is bilinear x2 at pixel centres, no rescaling of w.
 *  R17 depth <= 0 or non-finite: no measurement (gamma2 = gamma4 = 0 there);
 *      a depth difference uses the valid side, else 0.
 *  R18 the first frame after reset only initialises (w = dw = 0).
 *  R22 Eqs. 59-66 put the whole source term -f<eta,w> into BOTH axis passes,
 *      which integrates it over two time units per frame, at odds with the
 *      single source of Eq. 53.  The default keeps the printed passes;
 *      SFO_SOURCE_SPLIT applies half of it in each pass (once per
 *      sub-iteration), which is consistent with Eq. 53.
 *  R23 the inertial source terms the paper drops by the assumption of Sec.
 *      4.4 (-Omega x w + a_w of the total-derivative equation of Sec. 3,
 *      a_w = rho a_c - Omega x (w + Omega x eta), so -2 Omega x w -
 *      Omega x (Omega x eta) + rho a_c in all) are integrated once per
 *      sub-iteration, after its two axis passes: one explicit Euler step
 *      with dt = 1/N evaluated at the state the passes left (SFO_IMU).
 *  R24 the acceleration enters as -rho a_c: with dv_c/dt = -Omega x v_c + a_c
 *      (the camera's equation of motion, Sec. 3) the derivative of
 *      rho (v_p - v_c) carries -rho a_c; the derivation prints +rho a_c.
 *  R25 lower levels: the transported w_h takes the full source; the
 *      increment dw takes its linear part -2 Omega x dw only (the coarser
 *      levels carry -Omega x (Omega x eta) and rho a_c; the remainder
 *      (rho_h - up rho_{h+1}) a_c is dropped).  Omega and a_c enter in frame
 *      units, Omega dt (rad/frame) and a_c dt^2 (m/frame^2), like w.
 *  R26 remapping camera data onto the grid (the paper maps its panoramic
 *      renders and camera frames onto the grid before filtering and counts
 *      that in its runtime, Sec. 6, without describing the resampling): each
 *      grid ray, rotated into the camera frame by R, is projected into the
 *      source image; brightness is bilinear between pixel centres with
 *      replicated edges, range is the nearest pixel's (no mixing of depths
 *      across an occlusion edge); a ray behind the camera or outside the
 *      source image gets brightness 0 and range 0 (no measurement).
 *  R27 panoramas are equirectangular: column u spans longitude
 *      phi = 2 pi (u / Ws) - pi, row v latitude theta = pi/2 - pi (v / Hs)
 *      (pixel k covers [k, k+1)); the ray (cos th sin phi, -sin th,
 *      cos th cos phi) in the camera frame (x right, y down, z forward);
 *      longitude wraps around.
 *  G1  grid: level h is a pinhole grid with intrinsics scaled by 2^(1-h);
 *      rays pass through pixel centres; the neighbour rays that define B
 *      and dmu exist analytically beyond the image edge.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SFO_DOMINANT_LITERAL 1
#define SFO_SOURCE_SPLIT 2
#define SFO_IMU 32

/* ------------------------------------------------------------------------ */
/* small helpers                                                              */
/* ------------------------------------------------------------------------ */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

int sfo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* P_eta v = (I - eta eta^T) v, the tangent projector of Eq. 2. */
static void project(const double* eta, const double* v, double* out)
{
    double P[3][3];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) P[r][c] = (r == c ? 1.0 : 0.0) - eta[r] * eta[c];
    for (int r = 0; r < 3; r++) out[r] = P[r][0] * v[0] + P[r][1] * v[1] + P[r][2] * v[2];
}

/* Solve the n x n system M x = r (n <= 3) by Gaussian elimination with
 * partial pivoting.  M and r are overwritten. */
static void gauss_solve(int n, double M[3][3], double r[3], double x[3])
{
    for (int k = 0; k < n; k++) {
        int piv = k;
        for (int q = k + 1; q < n; q++)
            if (fabs(M[q][k]) > fabs(M[piv][k])) piv = q;
        if (piv != k) {
            for (int c = 0; c < n; c++) { double t = M[k][c]; M[k][c] = M[piv][c]; M[piv][c] = t; }
            double t = r[k]; r[k] = r[piv]; r[piv] = t;
        }
        for (int q = k + 1; q < n; q++) {
            double f = M[q][k] / M[k][k];
            for (int c = k; c < n; c++) M[q][c] -= f * M[k][c];
            r[q] -= f * r[k];
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        double s = r[k];
        for (int c = k + 1; c < n; c++) s -= M[k][c] * x[c];
        x[k] = s / M[k][k];
    }
}

/* Solve the symmetric positive definite 3x3 system A x = b by Cholesky
 * factorisation A = L L^T. */
static void cholesky3_solve(const double A[3][3], const double b[3], double x[3])
{
    double L[3][3] = {{0}};
    for (int r = 0; r < 3; r++) {
        for (int c = 0; c <= r; c++) {
            double s = A[r][c];
            for (int k = 0; k < c; k++) s -= L[r][k] * L[c][k];
            if (r == c) L[r][c] = sqrt(s);
            else L[r][c] = s / L[c][c];
        }
    }
    double y[3];
    for (int r = 0; r < 3; r++) {
        double s = b[r];
        for (int k = 0; k < r; k++) s -= L[r][k] * y[k];
        y[r] = s / L[r][r];
    }
    for (int r = 2; r >= 0; r--) {
        double s = y[r];
        for (int k = r + 1; k < 3; k++) s -= L[k][r] * x[k];
        x[r] = s / L[r][r];
    }
}

/* ------------------------------------------------------------------------ */
/* Grid geometry (Sec. 4.1, Eqs. 27-29; pinhole substitute for Spherepix, G1) */
/* ------------------------------------------------------------------------ */

/* Unit ray through the centre of pixel (i, j) of a pinhole grid. */
static void pinhole_ray(double fx, double fy, double cx, double cy, double i, double j, double* e)
{
    double x = (j + 0.5 - cx) / fx;
    double y = (i + 0.5 - cy) / fy;
    double n = sqrt(x * x + y * y + 1.0);
    e[0] = x / n;
    e[1] = y / n;
    e[2] = 1.0 / n;
}

/*
 * Per pixel: eta_ij; B_ij = [b1 b2] with b1 the normalised projection of
 * eta_{i,j+1} onto the tangent space of eta_ij (Eq. 27) and b2 the
 * normalised projection of eta_{i+1,j} made orthogonal to b1 (Gram-Schmidt,
 * so B is orthonormal as Sec. 4.1 requires); dmu_ij = || P eta_{i,j+1} ||.
 * Layout: eta[p*3+c], B[p*6 + 0..2] = b1, B[p*6 + 3..5] = b2, dmu[p].
 */
void sfo_geometry(int H, int W, double fx, double fy, double cx, double cy,
                  double* eta, double* B, double* dmu)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; i++) {
        for (int j = 0; j < W; j++) {
            int p = i * W + j;
            double e[3], e1[3], e2[3], p1[3], p2[3];
            pinhole_ray(fx, fy, cx, cy, i, j, e);
            pinhole_ray(fx, fy, cx, cy, i, j + 1, e1);
            pinhole_ray(fx, fy, cx, cy, i + 1, j, e2);
            project(e, e1, p1);
            double d = sqrt(dot3(p1, p1));
            double b1[3] = {p1[0] / d, p1[1] / d, p1[2] / d};
            project(e, e2, p2);
            double c = dot3(b1, p2);
            double b2[3] = {p2[0] - c * b1[0], p2[1] - c * b1[1], p2[2] - c * b1[2]};
            double n2 = sqrt(dot3(b2, b2));
            for (int k = 0; k < 3; k++) {
                eta[p * 3 + k] = e[k];
                B[p * 6 + k] = b1[k];
                B[p * 6 + 3 + k] = b2[k] / n2;
            }
            dmu[p] = d;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Image model [I_Y] (Sec. 4.2, Eqs. 30-31)                                   */
/* ------------------------------------------------------------------------ */

static const double g5[5] = {1.0 / 16.0, 4.0 / 16.0, 6.0 / 16.0, 4.0 / 16.0, 1.0 / 16.0};

/*
 * Weighted least-squares fit of Y_q ~ Yhat_p + dbeta . (q - p) over the 5x5
 * window around p with weights G = g^T g (Eq. 30, offsets q - p [R5],
 * replicated border [R13]).  The 3x3 normal equations are formed and solved
 * per pixel.  dbeta[p*2+0] is the column (beta_1) slope, dbeta[p*2+1] the row
 * (beta_2) slope.  grad[p*3+c] = dmu * (b1 dbeta_1 + b2 dbeta_2) (Eq. 31 [R4]).
 * dbeta may be NULL.
 */
void sfo_image_model(int H, int W, const double* Y, const double* B, const double* dmu,
                     double* Yhat, double* dbeta, double* grad)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; i++) {
        for (int j = 0; j < W; j++) {
            int p = i * W + j;
            double M[3][3] = {{0}}, r[3] = {0}, x[3];
            for (int di = -2; di <= 2; di++) {
                for (int dj = -2; dj <= 2; dj++) {
                    double G = g5[di + 2] * g5[dj + 2];
                    int qi = clampi(i + di, 0, H - 1), qj = clampi(j + dj, 0, W - 1);
                    double phi[3] = {1.0, (double)dj, (double)di};
                    double yq = Y[qi * W + qj];
                    for (int a = 0; a < 3; a++) {
                        r[a] += G * phi[a] * yq;
                        for (int b = 0; b < 3; b++) M[a][b] += G * phi[a] * phi[b];
                    }
                }
            }
            gauss_solve(3, M, r, x);
            Yhat[p] = x[0];
            if (dbeta) { dbeta[p * 2] = x[1]; dbeta[p * 2 + 1] = x[2]; }
            const double* b1 = B + p * 6;
            const double* b2 = B + p * 6 + 3;
            for (int c = 0; c < 3; c++) grad[p * 3 + c] = dmu[p] * (b1[c] * x[1] + b2[c] * x[2]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Inverse-depth model [I_rho] (Sec. 4.3, Eqs. 32-34, Table 1)                */
/* ------------------------------------------------------------------------ */

/* Eqs. 32-33: the one-sided difference of smaller magnitude, forward on a
 * tie; a side whose neighbour has no measurement is not used [R17]; at the
 * image border the replicated neighbour gives a zero difference [R13]. */
static double min_abs_diff(const double* rho, const unsigned char* valid, int p, int pp, int pm)
{
    int hp = valid[pp], hm = valid[pm];
    double dplus = rho[pp] - rho[p];   /* forward difference, Table 1  */
    double dminus = rho[p] - rho[pm];  /* backward difference, Table 1 */
    if (hp && hm) return fabs(dplus) <= fabs(dminus) ? dplus : dminus;
    if (hp) return dplus;
    if (hm) return dminus;
    return 0.0;
}

/*
 * rhohat is the raw inverse depth (constant term, Sec. 4.3).  grad[p*3+c] is
 * the tangent-space gradient dmu * B * (d_beta1, d_beta2) (Eq. 34 [R4]); zero
 * where the pixel itself has no measurement.  dbeta may be NULL.
 */
void sfo_invdepth_model(int H, int W, const double* rho, const unsigned char* valid,
                        const double* B, const double* dmu, double* dbeta, double* grad)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; i++) {
        for (int j = 0; j < W; j++) {
            int p = i * W + j;
            double d1 = 0.0, d2 = 0.0;
            if (valid[p]) {
                d1 = min_abs_diff(rho, valid, p, i * W + clampi(j + 1, 0, W - 1), i * W + clampi(j - 1, 0, W - 1));
                d2 = min_abs_diff(rho, valid, p, clampi(i + 1, 0, H - 1) * W + j, clampi(i - 1, 0, H - 1) * W + j);
            }
            if (dbeta) { dbeta[p * 2] = d1; dbeta[p * 2 + 1] = d2; }
            const double* b1 = B + p * 6;
            const double* b2 = B + p * 6 + 3;
            for (int c = 0; c < 3; c++) grad[p * 3 + c] = dmu[p] * (b1[c] * d1 + b2[c] * d2);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Numerical prediction [P], [P_[]] (Sec. 4.4, Sec. 4.6, Eqs. 53-67)          */
/* ------------------------------------------------------------------------ */

/* Eqs. 55-56 with reading R1 (or the literal text under SFO_DOMINANT_LITERAL). */
static double dominant(double s_minus, double s_plus, int flags)
{
    double central = fabs(s_plus) - fabs(s_minus); /* central difference of |u| */
    if (flags & SFO_DOMINANT_LITERAL) return central > 0.0 ? s_minus : s_plus;
    return central > 0.0 ? s_plus : s_minus;
}

/* Upwind difference of Eqs. 57-58 with the Table 1 operators. */
static double upwind(double f_minus, double f, double f_plus, double speed)
{
    return speed > 0.0 ? f - f_minus : f_plus - f;
}

/* One explicit Euler step of one axis pass for a field f with a source
 * (Eqs. 59-61, 63-65): f - dt [speed D + f <eta,w>]  [R22 for the split]. */
static double advance(double f, double dt, double speed, double D, double src, int flags)
{
    if (flags & SFO_SOURCE_SPLIT) return f - (dt * (speed * D) + (0.5 * dt) * (f * src));
    return f - dt * (speed * D + f * src);
}

/*
 * One axis pass of the scheme (Eqs. 59-62 for axis 0 = columns, Eqs. 63-66
 * for axis 1 = rows) over all pixels, Jacobi style (all reads from the
 * input arrays).  w is the transporting structure flow; dw (may be NULL),
 * rho and Y (may be NULL) are transported by it.  Y has no source term.
 * Returns max dt*|speed hat| for the CFL check of Eq. 67.  margin (may be
 * NULL) receives the minimum relative gap ||s+| - |s-|| / max(|s+|,|s-|)
 * over passes at pixels whose two neighbour speeds have opposite signs
 * (the only place where the dominant-speed choice is discontinuous).
 */
static double axis_pass(int H, int W, int axis, double dt, int flags,
                        const double* eta, const double* B, const double* dmu,
                        const double* w, const double* dw, const double* rho, const double* Y,
                        double* w_o, double* dw_o, double* rho_o, double* Y_o,
                        double* speed, double* margin)
{
    /* Eq. 54 [R4]: Phi = (1/dmu) B^T P w; speed = its component on this axis. */
#pragma omp parallel for schedule(static)
    for (int p = 0; p < H * W; p++) {
        double Pw[3];
        project(eta + p * 3, w + p * 3, Pw);
        speed[p] = dot3(B + p * 6 + 3 * axis, Pw) / dmu[p];
    }
    double cfl = 0.0;
#pragma omp parallel for schedule(static) reduction(max : cfl)
    for (int i = 0; i < H; i++) {
        for (int j = 0; j < W; j++) {
            int p = i * W + j, pm, pp;
            if (axis == 0) { pm = i * W + clampi(j - 1, 0, W - 1); pp = i * W + clampi(j + 1, 0, W - 1); }
            else { pm = clampi(i - 1, 0, H - 1) * W + j; pp = clampi(i + 1, 0, H - 1) * W + j; }
            double sm = speed[pm], sp = speed[pp];
            double s = dominant(sm, sp, flags);
            if (dt * fabs(s) > cfl) cfl = dt * fabs(s);
            if (margin && sm * sp < 0.0) {
                double m = fabs(fabs(sp) - fabs(sm)) / fmax(fabs(sp), fabs(sm));
                if (m < margin[p]) margin[p] = m;
            }
            double src = dot3(eta + p * 3, w + p * 3); /* <eta, w> at this pixel */
            for (int c = 0; c < 3; c++) {
                double D = upwind(w[pm * 3 + c], w[p * 3 + c], w[pp * 3 + c], s);
                w_o[p * 3 + c] = advance(w[p * 3 + c], dt, s, D, src, flags);
                if (dw) {
                    double Dd = upwind(dw[pm * 3 + c], dw[p * 3 + c], dw[pp * 3 + c], s);
                    dw_o[p * 3 + c] = advance(dw[p * 3 + c], dt, s, Dd, src, flags);
                }
            }
            double Dr = upwind(rho[pm], rho[p], rho[pp], s);
            rho_o[p] = advance(rho[p], dt, s, Dr, src, flags);
            if (Y) {
                double Dy = upwind(Y[pm], Y[p], Y[pp], s);
                Y_o[p] = Y[p] - dt * s * Dy;
            }
        }
    }
    return cfl;
}

/*
 * N sub-iterations with dt = 1/N (Eq. 53); each is a column pass driven by
 * u-hat from w^n, then a row pass driven by v-hat from w* (Sec. 4.6).  The
 * fields are updated in place and hold w^N on return [R3].  Top level: dw and
 * Y are NULL (Eqs. 36-37); lower levels transport w, dw, rho and Y by w
 * (Eqs. 38-41 [R7]).  With SFO_IMU in flags and imu non-NULL, each
 * sub-iteration ends with the inertial source step [R23].  Returns the CFL
 * number dt * max |speed hat| (Eq. 67).
 */
static void cross3(const double* a, const double* b, double* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/*
 * The inertial source terms of one sub-iteration [R23-R25]: with Omega and a
 * in frame units (imu = (Omega_x, Omega_y, Omega_z, a_x, a_y, a_z)),
 *   w  <- w  + dt (-2 Omega x w - Omega x (Omega x eta) - rho a)
 *   dw <- dw + dt (-2 Omega x dw)                     (lower levels)
 * at every pixel, from the values the two axis passes left.
 */
void sfo_imu_step(int H, int W, double dt, const double* imu, const double* eta,
                  double* w, double* dw, const double* rho)
{
    const double* om = imu;
    const double* acc = imu + 3;
#pragma omp parallel for schedule(static)
    for (int p = 0; p < H * W; p++) {
        double ow[3], oe[3], ooe[3];
        cross3(om, w + p * 3, ow);
        cross3(om, eta + p * 3, oe);
        cross3(om, oe, ooe);
        double odw[3] = {0.0, 0.0, 0.0};
        if (dw) cross3(om, dw + p * 3, odw);
        for (int c = 0; c < 3; c++) {
            w[p * 3 + c] += dt * (-2.0 * ow[c] - ooe[c] - rho[p] * acc[c]);
            if (dw) dw[p * 3 + c] += dt * (-2.0 * odw[c]);
        }
    }
}

double sfo_propagate(int H, int W, int N, int flags,
                     const double* eta, const double* B, const double* dmu,
                     double* w, double* dw, double* rho, double* Y, double* margin, const double* imu)
{
    size_t n = (size_t)H * W;
    double* w1 = malloc(n * 3 * sizeof(double));
    double* dw1 = dw ? malloc(n * 3 * sizeof(double)) : NULL;
    double* r1 = malloc(n * sizeof(double));
    double* y1 = Y ? malloc(n * sizeof(double)) : NULL;
    double* speed = malloc(n * sizeof(double));
    double dt = 1.0 / N, cfl = 0.0;
    if (margin)
        for (size_t p = 0; p < n; p++) margin[p] = INFINITY;
    for (int it = 0; it < N; it++) {
        double c0 = axis_pass(H, W, 0, dt, flags, eta, B, dmu, w, dw, rho, Y, w1, dw1, r1, y1, speed, margin);
        double c1 = axis_pass(H, W, 1, dt, flags, eta, B, dmu, w1, dw1, r1, y1, w, dw, rho, Y, speed, margin);
        if (imu && (flags & SFO_IMU)) sfo_imu_step(H, W, dt, imu, eta, w, dw, rho);
        if (c0 > cfl) cfl = c0;
        if (c1 > cfl) cfl = c1;
    }
    free(w1); free(dw1); free(r1); free(y1); free(speed);
    return cfl;
}

/* ------------------------------------------------------------------------ */
/* Update [U], [Delta U] (Sec. 4.5, Eqs. 42-50)                               */
/* ------------------------------------------------------------------------ */

/*
 * Minimise g1 |E_Y|^2 + g2 |E_rho|^2 + g3 |E_t|^2 over the unknown x per pixel:
 *   E_Y   = gradY^T P x + dmu^2 (Yhat - Yref)                    (Eqs. 43, 48)
 *   E_rho = gradR^T P x + dmu^2 ((rhohat - rhoref) + rhohat <eta, x>)  (44, 49)
 *   E_t   = x - prior                                          (Eqs. 45 [R6], 50)
 * i.e. the normal equations A x = b of Eq. 46, solved by Cholesky.
 * Top level: x = w^{k+1}, Yref = Y^k, rhoref = rho^k, prior = w^{k+} [R11];
 * lower levels: x = dw^{k+1}, Yref = Y^{k+}, rhoref = rho^{k+}, prior = dw^{k+}.
 * A pixel without a depth measurement has g2 = 0 [R17].
 */
void sfo_update(int H, int W, double g1, double g2, double g3,
                const double* eta, const double* dmu,
                const double* Yhat, const double* gradY,
                const double* rhohat, const double* gradR, const unsigned char* valid,
                const double* Yref, const double* rhoref, const double* prior, double* x_out)
{
#pragma omp parallel for schedule(static)
    for (int p = 0; p < H * W; p++) {
        const double* e = eta + p * 3;
        double d2 = dmu[p] * dmu[p];
        double rY[3], rR[3];
        project(e, gradY + p * 3, rY);     /* (gradY^T P)^T = P gradY, P symmetric */
        project(e, gradR + p * 3, rR);
        for (int c = 0; c < 3; c++) rR[c] += d2 * rhohat[p] * e[c];
        double cY = d2 * (Yhat[p] - Yref[p]);
        double cR = d2 * (rhohat[p] - rhoref[p]);
        double gr = valid[p] ? g2 : 0.0;
        double A[3][3], b[3];
        for (int r = 0; r < 3; r++) {
            for (int c = 0; c < 3; c++) A[r][c] = g1 * rY[r] * rY[c] + gr * rR[r] * rR[c] + (r == c ? g3 : 0.0);
            b[r] = -g1 * rY[r] * cY - gr * rR[r] * cR + g3 * prior[p * 3 + r];
        }
        cholesky3_solve(A, b, x_out + p * 3);
    }
}

/* Eqs. 51-52: rho^{k+1} = (g4 rhohat + g5 rho^{k+}) / (g4 + g5); g4 = 0 where
 * there is no measurement. */
void sfo_blend(int n, double g4, double g5, const double* rhohat, const unsigned char* valid,
               const double* rho_pred, double* rho_out)
{
    for (int p = 0; p < n; p++) {
        double a = valid[p] ? g4 : 0.0;
        rho_out[p] = (a * rhohat[p] + g5 * rho_pred[p]) / (a + g5);
    }
}

/* Sec. 4.5: S passes of a 5x5 average filter on a 3-channel field [R13]. */
void sfo_smooth(int H, int W, int S, double* f)
{
    size_t n = (size_t)H * W * 3;
    double* t = malloc(n * sizeof(double));
    for (int s = 0; s < S; s++) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < H; i++) {
            for (int j = 0; j < W; j++) {
                for (int c = 0; c < 3; c++) {
                    double acc = 0.0;
                    for (int di = -2; di <= 2; di++)
                        for (int dj = -2; dj <= 2; dj++)
                            acc += f[(clampi(i + di, 0, H - 1) * W + clampi(j + dj, 0, W - 1)) * 3 + c];
                    t[(i * W + j) * 3 + c] = acc / 25.0;
                }
            }
        }
        memcpy(f, t, n * sizeof(double));
    }
    free(t);
}

/* ------------------------------------------------------------------------ */
/* Pyramid (Sec. 4, Eq. 26 [R14])                                             */
/* ------------------------------------------------------------------------ */

/* Level h+1 from level h: 2x2 mean of Y; mean of the valid children's
 * inverse depth, no measurement if none is valid. */
void sfo_downsample(int H, int W, const double* Y, const double* rho, const unsigned char* valid,
                    double* Y2, double* rho2, unsigned char* valid2)
{
    int H2 = H / 2, W2 = W / 2;
    for (int i = 0; i < H2; i++) {
        for (int j = 0; j < W2; j++) {
            double ys = 0.0, rs = 0.0;
            int nv = 0;
            for (int a = 0; a < 2; a++) {
                for (int b = 0; b < 2; b++) {
                    int q = (2 * i + a) * W + (2 * j + b);
                    ys += Y[q];
                    if (valid[q]) { rs += rho[q]; nv++; }
                }
            }
            Y2[i * W2 + j] = ys / 4.0;
            rho2[i * W2 + j] = nv ? rs / nv : 0.0;
            valid2[i * W2 + j] = nv > 0;
        }
    }
}

/* Eq. 26: w_h = up(w_{h+1}) + dw_h; up() is bilinear x2 at pixel centres with
 * replicated border, no scaling (w is angular) [R14]. */
void sfo_upsample_add(int Hc, int Wc, const double* wc, int H, int W, const double* dw, double* w_out)
{
    for (int i = 0; i < H; i++) {
        double y = (i + 0.5) / 2.0 - 0.5;
        int i0 = (int)floor(y);
        double fy = y - i0;
        int ia = clampi(i0, 0, Hc - 1), ib = clampi(i0 + 1, 0, Hc - 1);
        for (int j = 0; j < W; j++) {
            double x = (j + 0.5) / 2.0 - 0.5;
            int j0 = (int)floor(x);
            double fx = x - j0;
            int ja = clampi(j0, 0, Wc - 1), jb = clampi(j0 + 1, 0, Wc - 1);
            for (int c = 0; c < 3; c++) {
                double up = (1 - fy) * ((1 - fx) * wc[(ia * Wc + ja) * 3 + c] + fx * wc[(ia * Wc + jb) * 3 + c])
                          + fy * ((1 - fx) * wc[(ib * Wc + ja) * 3 + c] + fx * wc[(ib * Wc + jb) * 3 + c]);
                w_out[(i * W + j) * 3 + c] = up + (dw ? dw[(i * W + j) * 3 + c] : 0.0);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Whole filter (Sec. 4, Fig. 3)                                              */
/* ------------------------------------------------------------------------ */

#define SFO_MAX_LEVELS 8

typedef struct {
    int H, W;
    double *eta, *B, *dmu;          /* geometry                              */
    double *w, *dw, *rho, *Yhat;    /* state: w (top: w_H, lower: w_h), dw,  */
                                    /* rho, Y-hat of the last frame          */
    double *Y, *rhohat;             /* this frame's data at this level       */
    unsigned char* valid;
} sfo_level;

typedef struct {
    int H, W, L, flags, initialised;
    double fx, fy, cx, cy, lambda_ref, dt_prev;
    int iters[SFO_MAX_LEVELS], smooth[SFO_MAX_LEVELS];
    double gamma[5];
    double last_cfl;
    double omega[3], accel[3];      /* camera angular velocity (rad/s) and    */
                                    /* linear acceleration (m/s^2) over the   */
                                    /* next frame interval, camera frame [R23] */
    sfo_level lv[SFO_MAX_LEVELS];
} sfo_ctx;

sfo_ctx* sfo_create(int H, int W, int L, double fx, double fy, double cx, double cy,
                    const int* iters, const int* smooth, const double* gamma,
                    double lambda_ref, int flags)
{
    if (L < 1 || L > SFO_MAX_LEVELS) return NULL;
    if (H % (1 << (L - 1)) || W % (1 << (L - 1))) return NULL;
    sfo_ctx* c = calloc(1, sizeof(sfo_ctx));
    c->H = H; c->W = W; c->L = L; c->flags = flags;
    c->fx = fx; c->fy = fy; c->cx = cx; c->cy = cy; c->lambda_ref = lambda_ref;
    for (int k = 0; k < 5; k++) c->gamma[k] = gamma[k];
    for (int h = 0; h < L; h++) {
        c->iters[h] = iters[h];
        c->smooth[h] = smooth[h];
        sfo_level* l = &c->lv[h];
        double s = (double)(1 << h);
        l->H = H >> h; l->W = W >> h;
        size_t n = (size_t)l->H * l->W;
        l->eta = malloc(n * 3 * sizeof(double));
        l->B = malloc(n * 6 * sizeof(double));
        l->dmu = malloc(n * sizeof(double));
        sfo_geometry(l->H, l->W, fx / s, fy / s, cx / s, cy / s, l->eta, l->B, l->dmu);
        l->w = calloc(n * 3, sizeof(double));
        l->dw = calloc(n * 3, sizeof(double));
        l->rho = calloc(n, sizeof(double));
        l->Yhat = calloc(n, sizeof(double));
        l->Y = calloc(n, sizeof(double));
        l->rhohat = calloc(n, sizeof(double));
        l->valid = calloc(n, 1);
    }
    return c;
}

/* Camera angular velocity (rad/s) and linear acceleration (m/s^2), camera
 * frame, used by the following frames' predictions under SFO_IMU [R23]. */
void sfo_set_motion(sfo_ctx* c, const double* omega, const double* accel)
{
    for (int k = 0; k < 3; k++) {
        c->omega[k] = omega ? omega[k] : 0.0;
        c->accel[k] = accel ? accel[k] : 0.0;
    }
}

void sfo_destroy(sfo_ctx* c)
{
    if (!c) return;
    for (int h = 0; h < c->L; h++) {
        sfo_level* l = &c->lv[h];
        free(l->eta); free(l->B); free(l->dmu); free(l->w); free(l->dw);
        free(l->rho); free(l->Yhat); free(l->Y); free(l->rhohat); free(l->valid);
    }
    free(c);
}

void sfo_reset(sfo_ctx* c) { c->initialised = 0; }

/* Level data: level 1 from the input (rho = lambda_ref / lambda, Eq. 8), then
 * the pyramid [R14]. */
static void build_pyramid(sfo_ctx* c, const double* image, const double* range)
{
    sfo_level* l0 = &c->lv[0];
    for (int p = 0; p < l0->H * l0->W; p++) {
        l0->Y[p] = image[p];
        double lam = range[p];
        int ok = isfinite(lam) && lam > 0.0;
        l0->valid[p] = ok;
        l0->rhohat[p] = ok ? c->lambda_ref / lam : 0.0;
    }
    for (int h = 1; h < c->L; h++) {
        sfo_level* a = &c->lv[h - 1];
        sfo_level* b = &c->lv[h];
        sfo_downsample(a->H, a->W, a->Y, a->rhohat, a->valid, b->Y, b->rhohat, b->valid);
    }
}

/*
 * One frame k -> k+1 (Fig. 3).  image and range are H x W row-major; flow_out
 * (3 x H x W planar, rad/s) and invdepth_out (H x W) may be NULL.  Returns the
 * largest CFL number seen in the prediction (Eq. 67).
 */
double sfo_step(sfo_ctx* c, const double* image, const double* range, double dt,
                double* flow_out, double* invdepth_out)
{
    int L = c->L;
    build_pyramid(c, image, range);
    double cfl = 0.0;
    if (!c->initialised) {
        /* R18: initial condition w = dw = 0, rho = rhohat, Y-hat from the model. */
        for (int h = 0; h < L; h++) {
            sfo_level* l = &c->lv[h];
            size_t n = (size_t)l->H * l->W;
            double* grad = malloc(n * 3 * sizeof(double));
            sfo_image_model(l->H, l->W, l->Y, l->B, l->dmu, l->Yhat, NULL, grad);
            free(grad);
            for (size_t p = 0; p < n; p++) l->rho[p] = l->valid[p] ? l->rhohat[p] : 0.0;
            memset(l->w, 0, n * 3 * sizeof(double));
            memset(l->dw, 0, n * 3 * sizeof(double));
        }
        c->initialised = 1;
    } else {
        /* R9: the state holds rad/frame at the previous frame's dt. */
        if (dt != c->dt_prev) {
            double k = dt / c->dt_prev;
            for (int h = 0; h < L; h++) {
                sfo_level* l = &c->lv[h];
                for (int q = 0; q < l->H * l->W * 3; q++) { l->w[q] *= k; l->dw[q] *= k; }
            }
        }
        for (int h = L - 1; h >= 0; h--) {
            sfo_level* l = &c->lv[h];
            int top = (h == L - 1);
            size_t n = (size_t)l->H * l->W;
            double* rho_k = malloc(n * sizeof(double));
            double* Y_k = malloc(n * sizeof(double));
            double* Ynew = malloc(n * sizeof(double));
            double* gY = malloc(n * 3 * sizeof(double));
            double* gR = malloc(n * 3 * sizeof(double));
            double* x = malloc(n * 3 * sizeof(double));
            memcpy(rho_k, l->rho, n * sizeof(double));
            memcpy(Y_k, l->Yhat, n * sizeof(double));
            /* prediction k -> k+ (Sec. 4.4, 4.6) */
            /* R25: Omega dt and a_c dt^2, the frame units of w */
            double imu[6] = {c->omega[0] * dt, c->omega[1] * dt, c->omega[2] * dt,
                             c->accel[0] * dt * dt, c->accel[1] * dt * dt, c->accel[2] * dt * dt};
            double cf = sfo_propagate(l->H, l->W, c->iters[h], c->flags, l->eta, l->B, l->dmu,
                                      l->w, top ? NULL : l->dw, l->rho, top ? NULL : l->Yhat, NULL, imu);
            if (cf > cfl) cfl = cf;
            /* measurement models at k+1 (Sec. 4.2, 4.3) */
            sfo_image_model(l->H, l->W, l->Y, l->B, l->dmu, Ynew, NULL, gY);
            sfo_invdepth_model(l->H, l->W, l->rhohat, l->valid, l->B, l->dmu, NULL, gR);
            /* update k+ -> k+1 (Sec. 4.5) */
            double s = (double)(1 << h);
            double g3 = c->gamma[2] * (s / c->fx) * (s / c->fx); /* R10 */
            if (top)
                sfo_update(l->H, l->W, c->gamma[0], c->gamma[1], g3, l->eta, l->dmu, Ynew, gY,
                           l->rhohat, gR, l->valid, Y_k, rho_k, l->w, x);
            else
                sfo_update(l->H, l->W, c->gamma[0], c->gamma[1], g3, l->eta, l->dmu, Ynew, gY,
                           l->rhohat, gR, l->valid, l->Yhat, l->rho, l->dw, x);
            sfo_blend((int)n, c->gamma[3], c->gamma[4], l->rhohat, l->valid, l->rho, l->rho);
            sfo_smooth(l->H, l->W, c->smooth[h], x);
            memcpy(top ? l->w : l->dw, x, n * 3 * sizeof(double));
            memcpy(l->Yhat, Ynew, n * sizeof(double));
            if (!top) {
                sfo_level* u = &c->lv[h + 1];
                sfo_upsample_add(u->H, u->W, u->w, l->H, l->W, l->dw, l->w);
            }
            free(rho_k); free(Y_k); free(Ynew); free(gY); free(gR); free(x);
        }
    }
    c->dt_prev = dt;
    c->last_cfl = cfl;
    sfo_level* l0 = &c->lv[0];
    size_t n0 = (size_t)l0->H * l0->W;
    if (flow_out)
        for (size_t p = 0; p < n0; p++)
            for (int k = 0; k < 3; k++) flow_out[k * n0 + p] = l0->w[p * 3 + k] / dt;
    if (invdepth_out)
        for (size_t p = 0; p < n0; p++) invdepth_out[p] = l0->rho[p];
    return cfl;
}

/* State access for tests: copies level h's arrays (any pointer may be NULL). */
void sfo_get_state(const sfo_ctx* c, int h, double* w, double* dw, double* rho, double* Yhat)
{
    const sfo_level* l = &c->lv[h];
    size_t n = (size_t)l->H * l->W;
    if (w) memcpy(w, l->w, n * 3 * sizeof(double));
    if (dw) memcpy(dw, l->dw, n * 3 * sizeof(double));
    if (rho) memcpy(rho, l->rho, n * sizeof(double));
    if (Yhat) memcpy(Yhat, l->Yhat, n * sizeof(double));
}

void sfo_set_state(sfo_ctx* c, int h, const double* w, const double* dw, const double* rho,
                   const double* Yhat, double dt_prev)
{
    sfo_level* l = &c->lv[h];
    size_t n = (size_t)l->H * l->W;
    if (w) memcpy(l->w, w, n * 3 * sizeof(double));
    if (dw) memcpy(l->dw, dw, n * 3 * sizeof(double));
    if (rho) memcpy(l->rho, rho, n * sizeof(double));
    if (Yhat) memcpy(l->Yhat, Yhat, n * sizeof(double));
    c->dt_prev = dt_prev;
    c->initialised = 1;
}

void sfo_get_geometry(const sfo_ctx* c, int h, double* eta, double* B, double* dmu)
{
    const sfo_level* l = &c->lv[h];
    size_t n = (size_t)l->H * l->W;
    if (eta) memcpy(eta, l->eta, n * 3 * sizeof(double));
    if (B) memcpy(B, l->B, n * 6 * sizeof(double));
    if (dmu) memcpy(dmu, l->dmu, n * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* Remapping camera data onto the grid [R26, R27]                             */
/* ------------------------------------------------------------------------ */

/* Source sampling at continuous pixel coordinates (u, v) of an Hs x Ws image
 * whose pixel k covers [k, k+1): bilinear brightness between pixel centres
 * with replicated edges (columns wrap when `wrap`), nearest-pixel range. */
static void sample_source(int Hs, int Ws, const double* img, const double* rng, double u, double v, int wrap,
                          double* Y, double* lam)
{
    double p = u - 0.5, q = v - 0.5;
    double j0f = floor(p), i0f = floor(q);
    double fx = p - j0f, fy = q - i0f;
    int j0 = (int)j0f, i0 = (int)i0f, j1 = j0 + 1, i1 = i0 + 1;
    if (wrap) { j0 = ((j0 % Ws) + Ws) % Ws; j1 = ((j1 % Ws) + Ws) % Ws; }
    else { j0 = clampi(j0, 0, Ws - 1); j1 = clampi(j1, 0, Ws - 1); }
    i0 = clampi(i0, 0, Hs - 1); i1 = clampi(i1, 0, Hs - 1);
    *Y = (1.0 - fy) * ((1.0 - fx) * img[i0 * Ws + j0] + fx * img[i0 * Ws + j1]) +
         fy * ((1.0 - fx) * img[i1 * Ws + j0] + fx * img[i1 * Ws + j1]);
    if (rng) {
        int jn = (int)floor(u), in = clampi((int)floor(v), 0, Hs - 1);
        jn = wrap ? ((jn % Ws) + Ws) % Ws : clampi(jn, 0, Ws - 1);
        *lam = rng[in * Ws + jn];
    }
}

/* the grid ray of pixel (i, j) (not normalised) rotated into the camera frame */
static void grid_ray_in_camera(double gfx, double gfy, double gcx, double gcy, const double* R, int i, int j,
                               double* d)
{
    double m[3] = {(j + 0.5 - gcx) / gfx, (i + 0.5 - gcy) / gfy, 1.0};
    for (int r = 0; r < 3; r++) d[r] = R[3 * r] * m[0] + R[3 * r + 1] * m[1] + R[3 * r + 2] * m[2];
}

/* A pinhole camera frame (intrinsics cam = fx, fy, cx, cy of an Hs x Ws image)
 * onto the H x W grid with intrinsics (gfx, gfy, gcx, gcy); R = camera <- grid
 * rotation, row-major.  rng / out_rng may be NULL. */
void sfo_remap_pinhole(int H, int W, double gfx, double gfy, double gcx, double gcy, const double* R, int Hs,
                       int Ws, const double* cam, const double* img, const double* rng, double* out_img,
                       double* out_rng)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; i++) {
        for (int j = 0; j < W; j++) {
            double d[3], Y = 0.0, lam = 0.0;
            grid_ray_in_camera(gfx, gfy, gcx, gcy, R, i, j, d);
            if (d[2] > 0.0) {
                double u = cam[0] * d[0] / d[2] + cam[2];
                double v = cam[1] * d[1] / d[2] + cam[3];
                if (u >= 0.0 && u <= Ws && v >= 0.0 && v <= Hs) sample_source(Hs, Ws, img, rng, u, v, 0, &Y, &lam);
            }
            out_img[i * W + j] = Y;
            if (out_rng) out_rng[i * W + j] = lam;
        }
    }
}

/* An equirectangular panorama (Hs x Ws) onto the grid [R27]. */
void sfo_remap_equirect(int H, int W, double gfx, double gfy, double gcx, double gcy, const double* R, int Hs,
                        int Ws, const double* img, const double* rng, double* out_img, double* out_rng)
{
    const double pi = 3.14159265358979323846;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; i++) {
        for (int j = 0; j < W; j++) {
            double d[3], Y = 0.0, lam = 0.0;
            grid_ray_in_camera(gfx, gfy, gcx, gcy, R, i, j, d);
            double n = sqrt(dot3(d, d));
            double phi = atan2(d[0], d[2]);
            double theta = asin(-d[1] / n);
            double u = (phi + pi) / (2.0 * pi) * Ws;
            double v = (pi / 2.0 - theta) / pi * Hs;
            sample_source(Hs, Ws, img, rng, u, v, 1, &Y, &lam);
            out_img[i * W + j] = Y;
            if (out_rng) out_rng[i * W + j] = lam;
        }
    }
}
