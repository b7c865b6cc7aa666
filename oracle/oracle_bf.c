/*
 * CPU checker (test infrastructure only): plain, slow FP64 implementations of
 * the bilateral filter and of its Gaussian-polynomial approximation (GPA),
 * written from Chaudhury & Dabhade, "Fast and Provably Accurate Bilateral
 * Filtering" (arXiv 1603.08109).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use this file; the GPU library shares no code,
 * header or table with it.
 *
 * Conventions (readings of the paper, each listed in the design notes):
 *  - images are row-major H x W arrays of doubles, values in [0, 2T];
 *  - the spatial kernel w lives on Omega = [-r, r]^2, stored as
 *    w[(dy + r) * (2r + 1) + (dx + r)], normalised to sum 1 (eq. normal);
 *  - the image domain I is finite (Sec. I): sums over j in Omega only take
 *    neighbours i - j that lie inside I (no padding, no renormalisation;
 *    w cancels in every ratio);
 *  - the range kernel is centred: both arguments are h = f - T (eq. shift,
 *    Prop. centering), and T is added back to the output;
 *  - "order N" means N Taylor terms, n = 0 .. N-1 (eq. approx), so
 *    Algorithm 2 performs N + 1 spatial filterings.
 *
 * Every function returns 0 on success, a negative code on bad arguments and
 * 1 if a non-finite value appeared.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_BAD_ARG (-1)
#define ORC_NONFINITE 1

#define IDX(y, x, W) ((long)(y) * (long)(W) + (long)(x))

/* eqs. spatial_kernel1 (Gaussian) and spatial_kernel2 (box) on
 * Omega = [-r, r]^2, normalised to unit sum (eq. normal). kind 0 = box,
 * kind 1 = Gaussian. */
int orc_spatial_kernel(int kind, int r, double sigma_s, double *w)
{
    if (r < 0 || !w) return ORC_BAD_ARG;
    if (kind == 1 && !(sigma_s > 0.0)) return ORC_BAD_ARG;
    int S = 2 * r + 1;
    double total = 0.0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            double v;
            if (kind == 0) {
                v = 1.0;
            } else if (kind == 1) {
                double d2 = (double)dx * dx + (double)dy * dy;
                v = exp(-d2 / (2.0 * sigma_s * sigma_s));
            } else {
                return ORC_BAD_ARG;
            }
            w[(dy + r) * S + (dx + r)] = v;
            total += v;
        }
    for (int k = 0; k < S * S; ++k) w[k] /= total;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Range kernels and their partial derivatives.                              */
/*   kind 0: g_{sigma_r}(t - tau) = exp(-(t - tau)^2 / (2 sigma_r^2))        */
/*           (eq. range_kernel inside eq. BF);                               */
/*   kind 1: phi_{N,sigma_r}(t, tau) = exp(-(t^2 + tau^2) / (2 sigma_r^2))   */
/*           * sum_{n=0}^{N-1} (tau t / sigma_r^2)^n / n!  (eq. GaussPolynomial). */
/*   kind 2: the same N terms of phi_N taken in absolute value,              */
/*           exp(-(t^2 + tau^2) / (2 sigma_r^2)) * sum_n |tau t / sigma_r^2|^n / n!, */
/*           the magnitude of the sum a finite-precision evaluation of       */
/*           eq. GPA accumulates (value only; d[1..3] are not set).          */
/* d[0] = value, d[1] = d/dt, d[2] = d/dtau, d[3] = d/dsigma_r.              */
/* ------------------------------------------------------------------------ */

/* Truncated exponential series sum_{n=0}^{m-1} x^n / n!, term by term. */
static double trunc_exp(double x, int m)
{
    double s = 0.0, term = 1.0;
    for (int n = 0; n < m; ++n) {
        s += term;
        term *= x / (double)(n + 1);
    }
    return s;
}

static void range_kernel(int kind, double t, double tau, double sr, int N, double d[4])
{
    double s2 = sr * sr;
    if (kind == 0) {
        double u = t - tau;
        double g = exp(-u * u / (2.0 * s2));
        d[0] = g;
        d[1] = -u / s2 * g;
        d[2] = u / s2 * g;
        d[3] = u * u / (s2 * sr) * g;
    } else if (kind == 2) {
        d[0] = exp(-(t * t + tau * tau) / (2.0 * s2)) * trunc_exp(fabs(t * tau / s2), N);
        d[1] = d[2] = d[3] = 0.0;
    } else {
        double gauss = exp(-(t * t + tau * tau) / (2.0 * s2));
        double x = t * tau / s2;
        double SN = trunc_exp(x, N);       /* value of the polynomial factor */
        double SN1 = trunc_exp(x, N - 1);  /* its derivative in x            */
        double phi = gauss * SN;
        d[0] = phi;
        d[1] = -t / s2 * phi + gauss * SN1 * tau / s2;
        d[2] = -tau / s2 * phi + gauss * SN1 * t / s2;
        /* d/dsigma_r: gaussian factor gives (t^2+tau^2)/sigma_r^3, x gives -2x/sigma_r */
        d[3] = (t * t + tau * tau) / (s2 * sr) * phi + gauss * SN1 * (-2.0 * x / sr);
    }
}

/* Ratio of eq. BF (kind 0) or eq. GPA (kind 1) at pixel (y, x), on centred
 * values h: num = sum_j w(j) k(h(i-j), h(i)) h(i-j), den = sum_j w(j) k(...).
 * kind 2 sums the term magnitudes: num = sum_j w(j) k_2(...) |h(i-j)|. */
static void ratio_at(int kind, const double *h, int H, int W, const double *w, int r,
                     double sr, int N, int y, int x, double *num, double *den)
{
    int S = 2 * r + 1;
    double tau = h[IDX(y, x, W)];
    double nsum = 0.0, dsum = 0.0, d[4];
    for (int dy = -r; dy <= r; ++dy) {
        int yy = y - dy;
        if (yy < 0 || yy >= H) continue;
        for (int dx = -r; dx <= r; ++dx) {
            int xx = x - dx;
            if (xx < 0 || xx >= W) continue;
            double t = h[IDX(yy, xx, W)];
            range_kernel(kind, t, tau, sr, N, d);
            double wk = w[(dy + r) * S + (dx + r)];
            nsum += wk * d[0] * (kind == 2 ? fabs(t) : t);
            dsum += wk * d[0];
        }
    }
    *num = nsum;
    *den = dsum;
}

static double *centred_copy(const double *f, long n, double T)
{
    double *h = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!h) return NULL;
    for (long k = 0; k < n; ++k) h[k] = f[k] - T;
    return h;
}

/* eq. BF (kind 0) or eq. GPA written out with phi_N (kind 1), brute force;
 * kind 2 gives the term magnitudes of eq. GPA in num/den (out is then not a
 * filter output).  If iy == NULL every pixel is computed and out/num/den hold H*W values;
 * otherwise nsamp pixels (iy[k], ix[k]) are computed.  num/den may be NULL. */
int orc_range_filter(int kind, const double *f, int H, int W, const double *w, int r,
                     double sr, int N, double T, const int *iy, const int *ix, long nsamp,
                     double *out, double *num, double *den)
{
    if (!f || !w || !out || H < 1 || W < 1 || r < 0 || !(sr > 0.0)) return ORC_BAD_ARG;
    if (kind != 0 && kind != 1 && kind != 2) return ORC_BAD_ARG;
    if (kind != 0 && N < 1) return ORC_BAD_ARG;
    long npix = (long)H * W;
    double *h = centred_copy(f, npix, T);
    if (!h) return ORC_BAD_ARG;
    long count = iy ? nsamp : npix;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long k = 0; k < count; ++k) {
        int y, x;
        if (iy) {
            y = iy[k];
            x = ix[k];
        } else {
            y = (int)(k / W);
            x = (int)(k % W);
        }
        if (y < 0 || y >= H || x < 0 || x >= W) {
            bad |= 2;
            continue;
        }
        double nsum, dsum;
        ratio_at(kind, h, H, W, w, r, sr, N, y, x, &nsum, &dsum);
        double o = T + nsum / dsum; /* Prop. centering: add the centre back */
        out[k] = o;
        if (num) num[k] = nsum;
        if (den) den[k] = dsum;
        if (!isfinite(o)) bad |= 1;
    }
    free(h);
    if (bad & 2) return ORC_BAD_ARG;
    return bad ? ORC_NONFINITE : ORC_OK;
}

/* Cross (joint) bilateral filter, the extension named in Sec. I and Sec. V:
 * the range kernel compares guide values e while the data f is averaged,
 *   out(i) = T + sum_j w(j) k(e(i-j)-T, e(i)-T) (f(i-j)-T) / sum_j w(j) k(...),
 * with k the exact Gaussian range kernel (kind 0) or phi_N (kind 1, the
 * Gaussian-polynomial approximation of eq. GaussPolynomial).  Same sample
 * conventions as orc_range_filter; num/den may be NULL. */
int orc_joint_filter(int kind, const double *f, const double *e, int H, int W, const double *w,
                     int r, double sr, int N, double T, const int *iy, const int *ix, long nsamp,
                     double *out, double *num, double *den)
{
    if (!f || !e || !w || !out || H < 1 || W < 1 || r < 0 || !(sr > 0.0)) return ORC_BAD_ARG;
    if (kind != 0 && kind != 1) return ORC_BAD_ARG;
    if (kind == 1 && N < 1) return ORC_BAD_ARG;
    int S = 2 * r + 1;
    long npix = (long)H * W;
    long count = iy ? nsamp : npix;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long k = 0; k < count; ++k) {
        int y, x;
        if (iy) {
            y = iy[k];
            x = ix[k];
        } else {
            y = (int)(k / W);
            x = (int)(k % W);
        }
        if (y < 0 || y >= H || x < 0 || x >= W) {
            bad |= 2;
            continue;
        }
        double tau = e[IDX(y, x, W)] - T, nsum = 0.0, dsum = 0.0, d[4];
        for (int dy = -r; dy <= r; ++dy) {
            int yy = y - dy;
            if (yy < 0 || yy >= H) continue;
            for (int dx = -r; dx <= r; ++dx) {
                int xx = x - dx;
                if (xx < 0 || xx >= W) continue;
                range_kernel(kind, e[IDX(yy, xx, W)] - T, tau, sr, N, d);
                double wk = w[(dy + r) * S + (dx + r)];
                nsum += wk * d[0] * (f[IDX(yy, xx, W)] - T);
                dsum += wk * d[0];
            }
        }
        double o = T + nsum / dsum;
        out[k] = o;
        if (num) num[k] = nsum;
        if (den) den[k] = dsum;
        if (!isfinite(o)) bad |= 1;
    }
    if (bad & 2) return ORC_BAD_ARG;
    return bad ? ORC_NONFINITE : ORC_OK;
}

/* Gradient of the same ratio with respect to the input image and sigma_r,
 * for a loss with d(loss)/d(out) = gout.  Exact partial derivatives of the
 * definition (chain rule on the ratio), evaluated brute force:
 *   u_i = num_i / den_i,
 *   d u_i / d t_ij   = w_j [k + (t_ij - u_i) k_t] / den_i      (neighbour i-j),
 *   d u_i / d tau_i  = sum_j w_j (t_ij - u_i) k_tau / den_i    (centre),
 *   d u_i / d sigma  = sum_j w_j (t_ij - u_i) k_sigma / den_i.
 * gin: H*W values (all pixels) or nsamp values at (iy, ix).  gsigma (may be
 * NULL) receives the full sum over all pixels. */
int orc_range_filter_grad(int kind, const double *f, int H, int W, const double *w, int r,
                          double sr, int N, double T, const double *gout,
                          const int *iy, const int *ix, long nsamp,
                          double *gin, double *gsigma)
{
    if (!f || !w || !gout || H < 1 || W < 1 || r < 0 || !(sr > 0.0)) return ORC_BAD_ARG;
    if (kind != 0 && kind != 1) return ORC_BAD_ARG;
    if (kind == 1 && N < 1) return ORC_BAD_ARG;
    long npix = (long)H * W;
    int S = 2 * r + 1;
    double *h = centred_copy(f, npix, T);
    double *den = (double *)malloc(sizeof(double) * (size_t)npix);
    double *u = (double *)malloc(sizeof(double) * (size_t)npix);
    double *self = (double *)malloc(sizeof(double) * (size_t)npix);
    if (!h || !den || !u || !self) {
        free(h); free(den); free(u); free(self);
        return ORC_BAD_ARG;
    }
    int bad = 0;
    double gs_total = 0.0;
    /* Per-pixel ratio, its centre derivative and its sigma_r derivative. */
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : gs_total) reduction(| : bad)
    for (long i = 0; i < npix; ++i) {
        int y = (int)(i / W), x = (int)(i % W);
        double nsum, dsum, d[4];
        ratio_at(kind, h, H, W, w, r, sr, N, y, x, &nsum, &dsum);
        double ui = nsum / dsum;
        double tau = h[i];
        double ctau = 0.0, csig = 0.0;
        for (int dy = -r; dy <= r; ++dy) {
            int yy = y - dy;
            if (yy < 0 || yy >= H) continue;
            for (int dx = -r; dx <= r; ++dx) {
                int xx = x - dx;
                if (xx < 0 || xx >= W) continue;
                double t = h[IDX(yy, xx, W)];
                range_kernel(kind, t, tau, sr, N, d);
                double wk = w[(dy + r) * S + (dx + r)];
                ctau += wk * (t - ui) * d[2];
                csig += wk * (t - ui) * d[3];
            }
        }
        den[i] = dsum;
        u[i] = ui;
        self[i] = gout[i] * ctau / dsum;
        gs_total += gout[i] * csig / dsum;
        if (!isfinite(ui)) bad = 1;
    }
    /* Gather: pixel k feeds output i = k + j as the neighbour t_ij. */
    long count = iy ? nsamp : npix;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long q = 0; q < count; ++q) {
        int y, x;
        if (iy) {
            y = iy[q];
            x = ix[q];
        } else {
            y = (int)(q / W);
            x = (int)(q % W);
        }
        if (y < 0 || y >= H || x < 0 || x >= W) {
            bad |= 2;
            continue;
        }
        long k = IDX(y, x, W);
        double t = h[k], acc = self[k], d[4];
        for (int dy = -r; dy <= r; ++dy) {
            int yi = y + dy;
            if (yi < 0 || yi >= H) continue;
            for (int dx = -r; dx <= r; ++dx) {
                int xi = x + dx;
                if (xi < 0 || xi >= W) continue;
                long i = IDX(yi, xi, W);
                range_kernel(kind, t, h[i], sr, N, d);
                double wk = w[(dy + r) * S + (dx + r)];
                acc += gout[i] * wk * (d[0] + (t - u[i]) * d[1]) / den[i];
            }
        }
        gin[q] = acc;
        if (!isfinite(acc)) bad |= 1;
    }
    if (gsigma) *gsigma = gs_total;
    free(h); free(den); free(u); free(self);
    if (bad & 2) return ORC_BAD_ARG;
    return bad ? ORC_NONFINITE : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 (GPA), step by step on whole images, FP64.                    */
/* The six working images of the paper: F, G, P, Q, H (named Hs here) and   */
/* Fbar. The spatial filtering Fbar = F * w is eq. spatialFiltering:         */
/* Fbar(i) = sum_{j in Omega, i-j in I} w(j) F(i - j).                       */
/* ------------------------------------------------------------------------ */
static void filter2d(const double *F, int H, int W, const double *w, int r, double *Fbar)
{
    int S = 2 * r + 1;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int dy = -r; dy <= r; ++dy) {
                int yy = y - dy;
                if (yy < 0 || yy >= H) continue;
                for (int dx = -r; dx <= r; ++dx) {
                    int xx = x - dx;
                    if (xx < 0 || xx >= W) continue;
                    acc += w[(dy + r) * S + (dx + r)] * F[IDX(yy, xx, W)];
                }
            }
            Fbar[IDX(y, x, W)] = acc;
        }
}

/* Algorithm 2 over the whole image. P and Q (may be NULL) receive the
 * algorithm's P and Q images (P includes the factor sigma_r of the final
 * step, i.e. out = P / Q + T).  Fbar_planes (may be NULL) receives the N + 1
 * filtered images Fbar_n = F_n * w, n = 0..N, as consecutive H x W planes. */
int orc_gpa_alg2(const double *f, int H, int W, const double *w, int r, double sr, int N,
                 double T, double *out, double *Pout, double *Qout, double *Fbar_planes)
{
    if (!f || !w || !out || H < 1 || W < 1 || r < 0 || !(sr > 0.0) || N < 1) return ORC_BAD_ARG;
    long npix = (long)H * W;
    size_t bytes = sizeof(double) * (size_t)npix;
    double *F = malloc(bytes), *G = malloc(bytes), *P = malloc(bytes), *Q = malloc(bytes);
    double *Hs = malloc(bytes), *Fbar = malloc(bytes);
    if (!F || !G || !P || !Q || !Hs || !Fbar) {
        free(F); free(G); free(P); free(Q); free(Hs); free(Fbar);
        return ORC_BAD_ARG;
    }
    /* initialisation loop over i in I */
    for (long i = 0; i < npix; ++i) {
        double h = f[i] - T;
        F[i] = exp(-h * h / (2.0 * sr * sr)); /* the one transcendental */
        G[i] = 1.0;
        P[i] = 0.0;
        Q[i] = 0.0;
        Hs[i] = h / sr;
    }
    filter2d(F, H, W, w, r, Fbar);
    if (Fbar_planes) memcpy(Fbar_planes, Fbar, bytes);
    for (int n = 1; n <= N; ++n) {
        for (long i = 0; i < npix; ++i) {
            Q[i] = Q[i] + G[i] * Fbar[i];
            F[i] = Hs[i] * F[i];
        }
        filter2d(F, H, W, w, r, Fbar);
        if (Fbar_planes) memcpy(Fbar_planes + (long)n * npix, Fbar, bytes);
        for (long i = 0; i < npix; ++i) {
            P[i] = P[i] + G[i] * Fbar[i];
            G[i] = Hs[i] * G[i] / (double)n;
        }
    }
    int bad = 0;
    for (long i = 0; i < npix; ++i) {
        out[i] = sr * (P[i] / Q[i]) + T;
        if (Pout) Pout[i] = sr * P[i];
        if (Qout) Qout[i] = Q[i];
        if (!isfinite(out[i])) bad = 1;
    }
    free(F); free(G); free(P); free(Q); free(Hs); free(Fbar);
    return bad ? ORC_NONFINITE : ORC_OK;
}

/* Algorithm 2 evaluated at selected pixels only.  The filtering step at
 * pixel i reads F on i - Omega alone, so each sample keeps its own copy of F
 * on that neighbourhood and runs the same recursions (same arithmetic, same
 * summation order as orc_gpa_alg2). */
int orc_gpa_alg2_at(const double *f, int H, int W, const double *w, int r, double sr, int N,
                    double T, const int *iy, const int *ix, long nsamp,
                    double *out, double *Pout, double *Qout)
{
    if (!f || !w || !out || !iy || !ix || H < 1 || W < 1 || r < 0 || !(sr > 0.0) || N < 1)
        return ORC_BAD_ARG;
    int S = 2 * r + 1;
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        double *Floc = (double *)malloc(sizeof(double) * (size_t)S * S);
        double *Hloc = (double *)malloc(sizeof(double) * (size_t)S * S);
        unsigned char *in = (unsigned char *)malloc((size_t)S * S);
        if (!Floc || !Hloc || !in) bad |= 2;
#pragma omp for schedule(dynamic, 4)
        for (long k = 0; k < nsamp; ++k) {
            if (bad & 2) continue;
            int y = iy[k], x = ix[k];
            if (y < 0 || y >= H || x < 0 || x >= W) {
                bad |= 2;
                continue;
            }
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    int yy = y - dy, xx = x - dx, q = (dy + r) * S + (dx + r);
                    in[q] = (yy >= 0 && yy < H && xx >= 0 && xx < W);
                    if (in[q]) {
                        double h = f[IDX(yy, xx, W)] - T;
                        Floc[q] = exp(-h * h / (2.0 * sr * sr));
                        Hloc[q] = h / sr;
                    }
                }
            double hc = f[IDX(y, x, W)] - T;
            double G = 1.0, P = 0.0, Q = 0.0, Hc = hc / sr;
            double Fbar = 0.0;
            for (int q = 0; q < S * S; ++q)
                if (in[q]) Fbar += w[q] * Floc[q];
            for (int n = 1; n <= N; ++n) {
                Q = Q + G * Fbar;
                Fbar = 0.0;
                for (int q = 0; q < S * S; ++q)
                    if (in[q]) {
                        Floc[q] = Hloc[q] * Floc[q];
                        Fbar += w[q] * Floc[q];
                    }
                P = P + G * Fbar;
                G = Hc * G / (double)n;
            }
            out[k] = sr * (P / Q) + T;
            if (Pout) Pout[k] = sr * P;
            if (Qout) Qout[k] = Q;
            if (!isfinite(out[k])) bad |= 1;
        }
        free(Floc);
        free(Hloc);
        free(in);
    }
    if (bad & 2) return ORC_BAD_ARG;
    return bad ? ORC_NONFINITE : ORC_OK;
}
