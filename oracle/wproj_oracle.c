/*
 * FP64 CPU oracle for Hankel-accelerated w-projection
 * (Lucas, Skipper & Scaife, "Fast W-Projection for Wide-field Imaging", MNRAS 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA
 * path is checked against.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Every routine is written straight from its definition in the paper (section /
 * equation cited at each function), in double precision, with no blocking, fusion
 * or reordering beyond what the definition states.  Where the paper is silent the
 * reading used is stated in the comment ("Reading: ...").
 *
 * Complex arrays are interleaved (re, im) pairs of doubles.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC -o liboracle.so
 * (-ffp-contract=off keeps a*b+c as two rounded operations on every host CPU, so the
 * FP64 integer decisions of the binning step are the same on x86-64 and aarch64.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* Bessel function of the first kind, order 0.                                */
/* ------------------------------------------------------------------------- */
/*
 * J0(x) = (1/pi) * integral_0^pi cos(x sin(theta)) dtheta   (Abramowitz & Stegun 9.1.18).
 * The integrand is analytic and pi-periodic in theta, so the composite trapezoid rule
 * converges geometrically; its error is 2*J_{2n}(x) for n panels, which is below
 * 1e-16 once 2n exceeds x by ~120.  n = ceil(x/2) + 64 panels.
 */
double or_j0(double x)
{
    x = fabs(x);
    int n = (int)ceil(0.5 * x) + 64;
    double s = 1.0; /* (f(0) + f(pi)) / 2 = (1 + 1) / 2 */
    for (int m = 1; m < n; ++m) {
        double th = M_PI * (double)m / (double)n;
        s += cos(x * sin(th));
    }
    return s / (double)n;
}

void or_j0_array(int64_t n, const double *x, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = or_j0(x[i]);
}

/* ------------------------------------------------------------------------- */
/* Order-0 Hankel transform (Section 4.3, Eq. 12 with k = 2*pi*rho).          */
/* ------------------------------------------------------------------------- */
/*
 * F(rho) = 2*pi * integral_0^{r_max} f(r) J0(2*pi*rho*r) r dr, which equals the 2D
 * Fourier transform of the radially symmetric function f (Section 4.3).
 * Reading: the 2*pi factor makes the order-0 transform of Eq. 12 (kernel J0(kr),
 * k = 2*pi*rho) equal to the 2D Fourier transform; the integral runs over the disc
 * of radius r_max (the circular region whose diameter is the image size, Section 6)
 * and is discretised by the midpoint rule r_i = (i + 1/2) dr, dr = r_max / R, with
 * weight 2*pi*r_i*dr.  The discrete transform is a matrix times a vector
 * (Section 4.3): out[k] = sum_i H[k][i] f[i], H[k][i] = 2*pi*r_i*dr*J0(2*pi*rho_k*r_i).
 */
void or_hankel_matrix(int R, double r_max, int K, const double *rho, double *H /* [K][R] */)
{
    double dr = r_max / (double)R;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        for (int i = 0; i < R; ++i) {
            double r = ((double)i + 0.5) * dr;
            H[(int64_t)k * R + i] = 2.0 * M_PI * r * dr * or_j0(2.0 * M_PI * rho[k] * r);
        }
    }
}

/* out[k] (complex) = sum_i H[k][i] * f[i] (complex) -- the matrix-vector product. */
void or_hankel_apply(int R, int K, const double *H, const double *f, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < K; ++k) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < R; ++i) {
            double h = H[(int64_t)k * R + i];
            re += h * f[2 * i];
            im += h * f[2 * i + 1];
        }
        out[2 * k] = re;
        out[2 * k + 1] = im;
    }
}

/* Direct transform at arbitrary radii (no matrix kept): same sum, J0 evaluated per term. */
void or_hankel_direct(int R, double r_max, const double *f, int K, const double *rho, double *out)
{
    double dr = r_max / (double)R;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < R; ++i) {
            double r = ((double)i + 0.5) * dr;
            double h = 2.0 * M_PI * r * dr * or_j0(2.0 * M_PI * rho[k] * r);
            re += h * f[2 * i];
            im += h * f[2 * i + 1];
        }
        out[2 * k] = re;
        out[2 * k + 1] = im;
    }
}

/* ------------------------------------------------------------------------- */
/* Image-domain convolution function on the radial line (Alg. 2, w-kernel     */
/* times AA-kernel; w-kernel G of Eq. 9).                                     */
/* ------------------------------------------------------------------------- */
/*
 * f[i] = t(r_i) * exp(+2*pi*j*w*(sqrt(1 - r_i^2) - 1)), r_i = (i + 1/2) r_max / R.
 * Reading: Eq. 9 gives G = exp(-2*pi*j*w*(n - 1)) for the prediction direction; the
 * gridding kernel is its adjoint, so the screen carries the + sign here, and the
 * kernel for -w is the complex conjugate of the kernel for |w| (Section 4.1).
 * taper[i] = t(r_i) is the radial anti-aliasing function sampled at the same nodes.
 */
void or_screen(int R, double r_max, const double *taper, double w, double *f)
{
    double dr = r_max / (double)R;
    for (int i = 0; i < R; ++i) {
        double r = ((double)i + 0.5) * dr;
        double n = sqrt(1.0 - r * r);
        double ph = 2.0 * M_PI * w * (n - 1.0);
        f[2 * i] = taper[i] * cos(ph);
        f[2 * i + 1] = taper[i] * sin(ph);
    }
}

/* ------------------------------------------------------------------------- */
/* Kernel truncation (Section 3.1, Alg. 1 / Alg. 2 truncation step).          */
/* ------------------------------------------------------------------------- */
/*
 * The kernel is cut where its magnitude falls below tau times its maximum.
 * Reading: on the radial line C[k] at rho_k = k*du/os, take the LAST k whose
 * |C[k]| >= tau * max_k |C[k]|; the support (half-width, in uv cells) is
 * ceil(k_last / os), clamped to [s_min, s_max].
 */
int or_support(int K, const double *C, double tau, int os, int s_min, int s_max)
{
    double mx = 0.0;
    for (int k = 0; k < K; ++k) {
        double a = hypot(C[2 * k], C[2 * k + 1]);
        if (a > mx) mx = a;
    }
    int k_last = 0;
    for (int k = 0; k < K; ++k) {
        if (hypot(C[2 * k], C[2 * k + 1]) >= tau * mx) k_last = k;
    }
    int s = (k_last + os - 1) / os;
    if (s < s_min) s = s_min;
    if (s > s_max) s = s_max;
    return s;
}

/* ------------------------------------------------------------------------- */
/* Cubic spline on the radial line (Section 4.3.2).                           */
/* ------------------------------------------------------------------------- */
/*
 * Second derivatives m[k] of the interpolating cubic spline through (k*h, y[k]),
 * k = 0..K-1 (complex y: real and imaginary parts are splined independently, which
 * is the same linear system).  Reading: the kernel is even in rho, so the spline is
 * clamped with zero slope at rho = 0; at the far end it is natural (m = 0).
 *   k = 0      : 2 m0 + m1              = 6 (y1 - y0) / h^2
 *   0 < k < K-1: m_{k-1} + 4 m_k + m_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}) / h^2
 *   k = K-1    : m_{K-1}                = 0
 * Solved with the Thomas algorithm.
 */
void or_spline_m(int K, const double *y, double h, double *m)
{
    double *cp = (double *)malloc(sizeof(double) * K);
    double *dp = (double *)malloc(sizeof(double) * 2 * K);
    double ih2 = 6.0 / (h * h);
    /* row 0: b=2, c=1 */
    cp[0] = 1.0 / 2.0;
    dp[0] = ih2 * (y[2] - y[0]) / 2.0;
    dp[1] = ih2 * (y[3] - y[1]) / 2.0;
    for (int k = 1; k < K - 1; ++k) {
        double den = 4.0 - cp[k - 1];
        cp[k] = 1.0 / den;
        for (int c = 0; c < 2; ++c) {
            double rhs = ih2 * (y[2 * (k + 1) + c] - 2.0 * y[2 * k + c] + y[2 * (k - 1) + c]);
            dp[2 * k + c] = (rhs - dp[2 * (k - 1) + c]) / den;
        }
    }
    /* last row: m_{K-1} = 0 */
    m[2 * (K - 1)] = 0.0;
    m[2 * (K - 1) + 1] = 0.0;
    for (int k = K - 2; k >= 0; --k) {
        for (int c = 0; c < 2; ++c) m[2 * k + c] = dp[2 * k + c] - cp[k] * m[2 * (k + 1) + c];
    }
    free(cp);
    free(dp);
}

/*
 * Value at x (in units of the node spacing, 0 <= x <= K-1) of the cubic spline
 * (interp = 0) or of the linear interpolant (interp = 1) -- Section 4.3.2.
 */
static void spline_eval(int K, const double *y, const double *m, double h, int interp, double x,
                        double *re, double *im)
{
    int k = (int)floor(x);
    if (k > K - 2) k = K - 2;
    if (k < 0) k = 0;
    double a = x - (double)k;
    double b = 1.0 - a;
    double vr = b * y[2 * k] + a * y[2 * (k + 1)];
    double vi = b * y[2 * k + 1] + a * y[2 * (k + 1) + 1];
    if (interp == 0) {
        double cb = (b * b * b - b) * h * h / 6.0;
        double ca = (a * a * a - a) * h * h / 6.0;
        vr += cb * m[2 * k] + ca * m[2 * (k + 1)];
        vi += cb * m[2 * k + 1] + ca * m[2 * (k + 1) + 1];
    }
    *re = vr;
    *im = vi;
}

void or_spline_eval_array(int K, const double *y, const double *m, double h, int interp,
                          int64_t n, const double *x, double *out)
{
    for (int64_t i = 0; i < n; ++i) spline_eval(K, y, m, h, interp, x[i], &out[2 * i], &out[2 * i + 1]);
}

/* ------------------------------------------------------------------------- */
/* 2D kernel from the radial line + oversampled kernel cache                  */
/* (Section 4.3.2 and the cache-building step of Alg. 2).                     */
/* ------------------------------------------------------------------------- */
/*
 * cache[fv][fu][jy][jx], fu, fv in [0, os), jx, jy in [0, 2S], W = 2S + 1.
 * The tap (jx, jy) of sub-kernel (fu, fv) sits at uv offset
 *   (jx - S - fu/os, jy - S - fv/os) cells from the visibility, i.e. at radius
 *   x = sqrt((os*(jx - S) - fu)^2 + (os*(jy - S) - fv)^2) radial samples (spacing du/os).
 * Reading: the truncated radial line is rotated about rho = 0, so taps beyond the
 * support radius (x > os*S) are zero (circular support; the paper's circular image
 * region is the image-domain face of the same fact).
 * y, m: radial values and spline second derivatives, K samples at spacing h = 1/os cells.
 */
void or_resample(int K, const double *y, const double *m, int os, int S, int interp, double *cache)
{
    int W = 2 * S + 1;
    double h = 1.0; /* x and the node spacing are both in radial-sample units */
    int64_t lim = (int64_t)os * S;
    lim = lim * lim;
    /* the os^2 sub-kernels are independent: one per OpenMP iteration, same arithmetic */
    #pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int fv = 0; fv < os; ++fv)
        for (int fu = 0; fu < os; ++fu)
            for (int jy = 0; jy < W; ++jy)
                for (int jx = 0; jx < W; ++jx) {
                    int64_t dx = (int64_t)os * (jx - S) - fu;
                    int64_t dy = (int64_t)os * (jy - S) - fv;
                    int64_t q = dx * dx + dy * dy;
                    int64_t idx = ((((int64_t)fv * os + fu) * W + jy) * W + jx) * 2;
                    if (q > lim) {
                        cache[idx] = 0.0;
                        cache[idx + 1] = 0.0;
                    } else {
                        spline_eval(K, y, m, h, interp, sqrt((double)q), &cache[idx], &cache[idx + 1]);
                    }
                }
}

/* ------------------------------------------------------------------------- */
/* Visibility binning (Alg. 1 steps 1-3, Alg. 2 steps 1-3, Section 4.1).      */
/* ------------------------------------------------------------------------- */
/*
 * For each visibility (u, v, w in wavelengths, given as float32 values):
 *   plane  = index of the |w|-plane nearest to |w| (ties -> lower index);
 *   conj   = 1 if w < 0 (kernel of -w is the conjugate of the kernel of |w|);
 *   uc     = u / du + N/2 (continuous grid coordinate), t = rint(uc * os),
 *   iu     = floor(t / os), fu = t - iu*os in [0, os)   (same for v);
 *   drop   = 1 if any tap of the (2S+1)^2 footprint leaves [0, N)^2, or if u, v or w is
 *            not finite (no nearest plane or grid cell exists for it).
 * Reading: the paper assigns equal-count chunks of the |w|-sorted data to planes;
 * this routine takes any ascending list of plane values and the nearest one
 * (a chunk's members are nearest to its own mean except near chunk borders).
 * All decisions are taken in FP64 from the float32 inputs, as the paper's FP64 build.
 */
void or_bin(int64_t V, const float *uvw, int P, const double *w_planes, const int *support,
            int N, double du, int os,
            int *plane, int *conj, int *iu, int *iv, int *fu, int *fv, int *drop)
{
    for (int64_t k = 0; k < V; ++k) {
        double u = (double)uvw[3 * k], v = (double)uvw[3 * k + 1], w = (double)uvw[3 * k + 2];
        double aw = fabs(w);
        int best = 0;
        double bd = fabs(aw - w_planes[0]);
        for (int p = 1; p < P; ++p) {
            double d = fabs(aw - w_planes[p]);
            if (d < bd) { bd = d; best = p; }
        }
        plane[k] = best;
        conj[k] = (w < 0.0) ? 1 : 0;
        double uc = u / du + (double)(N / 2);
        double vc = v / du + (double)(N / 2);
        double tu = rint(uc * (double)os);
        double tv = rint(vc * (double)os);
        double giu = floor(tu / (double)os);
        double giv = floor(tv / (double)os);
        int S = support[best];
        int ok = isfinite(u) && isfinite(v) && isfinite(w) &&
                 (giu - S >= 0.0) && (giu + S <= (double)(N - 1)) && (giv - S >= 0.0) && (giv + S <= (double)(N - 1));
        drop[k] = ok ? 0 : 1;
        if (ok) {
            iu[k] = (int)giu;
            iv[k] = (int)giv;
            fu[k] = (int)(tu - giu * (double)os);
            fv[k] = (int)(tv - giv * (double)os);
        } else {
            iu[k] = iv[k] = fu[k] = fv[k] = 0;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Convolutional gridding (Alg. 1 / Alg. 2 gridding step) and its adjoint.    */
/* ------------------------------------------------------------------------- */
/*
 * grid[iv - S + jy][iu - S + jx] += wt * V * K, where K is tap (jx, jy) of sub-kernel
 * (fu, fv) of the visibility's plane, conjugated when w < 0 (Section 4.1).
 * cache_off[p]: start (in complex elements) of plane p's [os][os][W][W] block.
 */
void or_grid(int64_t V, const int *plane, const int *conj, const int *iu, const int *iv,
             const int *fu, const int *fv, const int *drop, const float *vis, const float *wt,
             const int *support, const int64_t *cache_off, const double *cache, int os, int N,
             double *grid)
{
    for (int64_t k = 0; k < V; ++k) {
        if (drop[k]) continue;
        int p = plane[k], S = support[p], W = 2 * S + 1;
        double vr = (double)vis[2 * k], vi = (double)vis[2 * k + 1];
        double a = wt ? (double)wt[k] : 1.0;
        vr *= a;
        vi *= a;
        const double *sk = cache + 2 * (cache_off[p] + ((int64_t)fv[k] * os + fu[k]) * W * W);
        for (int jy = 0; jy < W; ++jy)
            for (int jx = 0; jx < W; ++jx) {
                double kr = sk[2 * (jy * W + jx)], ki = sk[2 * (jy * W + jx) + 1];
                if (conj[k]) ki = -ki;
                int64_t g = ((int64_t)(iv[k] - S + jy) * N + (iu[k] - S + jx)) * 2;
                grid[g] += vr * kr - vi * ki;
                grid[g + 1] += vr * ki + vi * kr;
            }
    }
}

/*
 * Degridding (prediction), the adjoint of or_grid without weights:
 *   V[k] = sum_taps conj(K) * grid[...], K conjugated for w < 0 as in gridding.
 * Dropped visibilities get 0.
 */
void or_degrid(int64_t V, const int *plane, const int *conj, const int *iu, const int *iv,
               const int *fu, const int *fv, const int *drop, const int *support,
               const int64_t *cache_off, const double *cache, int os, int N, const double *grid,
               double *vis_out)
{
    for (int64_t k = 0; k < V; ++k) {
        vis_out[2 * k] = 0.0;
        vis_out[2 * k + 1] = 0.0;
        if (drop[k]) continue;
        int p = plane[k], S = support[p], W = 2 * S + 1;
        const double *sk = cache + 2 * (cache_off[p] + ((int64_t)fv[k] * os + fu[k]) * W * W);
        double sr = 0.0, si = 0.0;
        for (int jy = 0; jy < W; ++jy)
            for (int jx = 0; jx < W; ++jx) {
                double kr = sk[2 * (jy * W + jx)], ki = sk[2 * (jy * W + jx) + 1];
                if (conj[k]) ki = -ki;
                int64_t g = ((int64_t)(iv[k] - S + jy) * N + (iu[k] - S + jx)) * 2;
                double gr = grid[g], gi = grid[g + 1];
                /* conj(K) * g */
                sr += kr * gr + ki * gi;
                si += kr * gi - ki * gr;
            }
        vis_out[2 * k] = sr;
        vis_out[2 * k + 1] = si;
    }
}

/* ------------------------------------------------------------------------- */
/* Brute-force imaging: adjoint of the non-coplanar visibility equation (Eq. 2)*/
/* ------------------------------------------------------------------------- */
/*
 * I_D(l, m) = (1 / sum wt) * sum_k wt_k * Re[V_k exp(+2*pi*j*(u_k l + v_k m + w_k (n - 1)))],
 * n = sqrt(1 - l^2 - m^2), on pixel centres l = (il - N/2) dl, m = (im - N/2) dl.
 * Reading: the 1/n factor of Eq. 2 is absorbed in the apparent flux of each source.
 */
void or_dft_image(int64_t V, const float *uvw, const float *vis, const float *wt, int N, double dl,
                  int npix, const int *pix_l, const int *pix_m, double *out)
{
    double wsum = 0.0;
    for (int64_t k = 0; k < V; ++k) wsum += wt ? (double)wt[k] : 1.0;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int q = 0; q < npix; ++q) {
        double l = (double)(pix_l[q] - N / 2) * dl;
        double m = (double)(pix_m[q] - N / 2) * dl;
        double n = sqrt(1.0 - l * l - m * m);
        double s = 0.0;
        for (int64_t k = 0; k < V; ++k) {
            double ph = 2.0 * M_PI * ((double)uvw[3 * k] * l + (double)uvw[3 * k + 1] * m +
                                      (double)uvw[3 * k + 2] * (n - 1.0));
            double a = wt ? (double)wt[k] : 1.0;
            s += a * ((double)vis[2 * k] * cos(ph) - (double)vis[2 * k + 1] * sin(ph));
        }
        out[q] = s / wsum;
    }
}

/*
 * Gridded value at selected cells only (the gridding sum of Alg. 1 / Alg. 2 evaluated cell by
 * cell, for checks at sizes where the full oracle grid is too slow):
 *   out[c] = sum over visibilities k whose footprint covers cell c of wt_k V_k K_k(cell),
 * with the tap K evaluated directly from plane p's radial line (spline or linear, as
 * or_resample: zero beyond the support radius, conjugated for w < 0).
 *   radial, spline_m: [P][K] complex lines; cells: (cu[c], cv[c]) grid column / row.
 */
void or_grid_cells(int64_t V, const int *plane, const int *conj, const int *iu, const int *iv,
                   const int *fu, const int *fv, const int *drop, const float *vis, const float *wt,
                   const int *support, int K, const double *radial, const double *spline_m, int interp,
                   int os, int ncells, const int *cu, const int *cv, double *out)
{
    for (int c = 0; c < ncells; ++c) out[2 * c] = out[2 * c + 1] = 0.0;
    for (int64_t k = 0; k < V; ++k) {
        if (drop[k]) continue;
        int p = plane[k], S = support[p];
        int64_t lim = (int64_t)os * S;
        lim = lim * lim;
        double a = wt ? (double)wt[k] : 1.0;
        double vr = a * (double)vis[2 * k], vi = a * (double)vis[2 * k + 1];
        for (int c = 0; c < ncells; ++c) {
            int jx = cu[c] - (iu[k] - S), jy = cv[c] - (iv[k] - S);
            if (jx < 0 || jx > 2 * S || jy < 0 || jy > 2 * S) continue;
            int64_t dx = (int64_t)os * (jx - S) - fu[k];
            int64_t dy = (int64_t)os * (jy - S) - fv[k];
            int64_t q = dx * dx + dy * dy;
            if (q > lim) continue;
            double kr, ki;
            spline_eval(K, radial + (int64_t)2 * p * K, spline_m + (int64_t)2 * p * K, 1.0, interp,
                        sqrt((double)q), &kr, &ki);
            if (conj[k]) ki = -ki;
            out[2 * c] += vr * kr - vi * ki;
            out[2 * c + 1] += vr * ki + vi * kr;
        }
    }
}
