/*
 * FP64 CPU oracle for the Domain Transform Solver (Bapat & Frahm, "The Domain
 * Transform Solver", ECCV 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library: every formula below is
 * written out again from the paper (and from the Gastal & Oliveira recursive
 * filter that the paper cites in §2 "The domain transform" and §3.2).
 *
 * Everything is double precision, round to nearest, no FMA contraction (the
 * build passes -ffp-contract=off).  Layout: row-major planes, H rows of W
 * values, no padding; a C-channel guide is C such planes back to back.
 * OpenMP is used only across independent lines inside one directional pass.
 *
 * Functions and the passage each follows:
 *   orc_schedule        per-pass sigma_i and feedback a_i of the recursive
 *                       filter (G&O, cited in §2/§3.2; not printed in the paper)
 *   orc_distances       domain-transform distances, Eq. 8-9 (§3.2), L1 or L2
 *   orc_causal/anticausal  the first-order recurrence J[n] = (1-w)x[n] + w J[n-1]
 *                       with w = a^d (G&O recursive filter, §2 and §3.2)
 *   orc_row_pass / orc_col_pass   one horizontal / vertical pass (§3.2, last
 *                       paragraph: alternating X and Y passes)
 *   orc_filter          edge-aware mean z_bar = A z, Eq. 10 with the RF kernel
 *   orc_support         sum_j W_ij support used to weight the confidence (§3.1,
 *                       discussion after Eq. 6)
 *   orc_box_filter      the edge-aware mean with the box kernel Eq. 10 prints,
 *                       W_ij = 1 if |DT_i - DT_j| <= r (normalized convolution in
 *                       the transformed domain, G&O), r_i = sigma_i sqrt(3) per pass
 *   orc_solve_cg        conjugate gradients on the objective of Eq. 2 itself,
 *                       F(z) = lambda/2 |z - A z|^2 + sum_i c_i (z_i - t_i)^2, whose
 *                       minimiser solves (lambda (I-A)^T (I-A) + 2C) z = 2 C t
 *                       (§3.1 notes that Eq. 3's update drops the factor 2 and
 *                       treats z_bar as constant; this is the true gradient)
 *   orc_confidence      confidence from the edge-aware variance of the target,
 *                       Eq. 7 (§3.1): c = exp(-V / (2 sigma_c^2)),
 *                       V = DT(t^2) - DT(t)^2 with DT the edge-aware mean
 *   orc_solve           gradient-descent iterations on Eq. 3 (step 0.99, §4)
 *                       or the fixed-point update of Eq. 4; with eps > 0 the
 *                       Charbonnier loss rho(r) = sqrt(r^2 + eps^2) on the target
 *                       term instead of the square (§4, the stereo loss of Eq. 11:
 *                       eps = 0.001): the gradient step takes c rho'(z - t), the
 *                       fixed point the loss's weight at the current iterate
 *   orc_solve_backward  hand-written reverse mode of orc_solve (the paper has
 *                       no backward; derived from the forward steps above)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NORM_L1 0
#define ORC_NORM_L2 1
#define ORC_UPDATE_GD 0
#define ORC_UPDATE_JACOBI 1
#define ORC_CONF_PLAIN 0
#define ORC_CONF_SUPPORT 1

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Per-pass schedule of the 2-D recursive filter (Gastal & Oliveira, the
 * filter the paper uses in §2 and §3.2).  Pass i = 1..N uses
 *   sigma_i = sigma_s * sqrt(3) * 2^(N-i) / sqrt(4^N - 1)
 * so that the N passes compose to a kernel of total variance sigma_s^2, and
 * the feedback coefficient a_i = exp(-sqrt(2) / sigma_i). */
void orc_schedule(double sigma_s, int N, double* sigma, double* a) {
    for (int i = 1; i <= N; ++i) {
        double s = sigma_s * sqrt(3.0) * pow(2.0, (double)(N - i)) / sqrt(pow(4.0, (double)N) - 1.0);
        sigma[i - 1] = s;
        a[i - 1] = exp(-sqrt(2.0) / s);
    }
}

/* Domain-transform distances between neighbouring pixels (§3.2, Eq. 8-9).
 * dX[y][x] is the distance between (y, x-1) and (y, x); dY[y][x] between
 * (y-1, x) and (y, x).  With k = sigma_s / sigma_r:
 *   L1 (the form the solver uses by default):  1 + k * sum_c |I_c(p) - I_c(q)|
 *   L2 (the norm §3.2 derives):                sqrt(1 + k^2 * sum_c (I_c(p) - I_c(q))^2)
 * The first column of dX and the first row of dY have no left / upper
 * neighbour; they are set to 1 (zero colour difference) and are never read by
 * the passes. */
void orc_distances(int C, int H, int W, const double* I, double sigma_s, double sigma_r, int norm,
                   double* dX, double* dY) {
    double k = sigma_s / sigma_r;
    long plane = (long)H * W;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            if (x == 0) {
                dX[p] = 1.0;
            } else {
                double s = 0.0;
                for (int c = 0; c < C; ++c) {
                    double diff = I[c * plane + p] - I[c * plane + p - 1];
                    s += (norm == ORC_NORM_L2) ? diff * diff : fabs(diff);
                }
                dX[p] = (norm == ORC_NORM_L2) ? sqrt(1.0 + k * k * s) : 1.0 + k * s;
            }
            if (y == 0) {
                dY[p] = 1.0;
            } else {
                double s = 0.0;
                for (int c = 0; c < C; ++c) {
                    double diff = I[c * plane + p] - I[c * plane + p - W];
                    s += (norm == ORC_NORM_L2) ? diff * diff : fabs(diff);
                }
                dY[p] = (norm == ORC_NORM_L2) ? sqrt(1.0 + k * k * s) : 1.0 + k * s;
            }
        }
    }
}

/* Causal recurrence along one line of n values (stride su), in place:
 *   J[0] = x[0];  J[j] = (1 - w_j) x[j] + w_j J[j-1],  w_j = a^d[j],  j = 1..n-1
 * d[j] is the distance between positions j-1 and j. */
void orc_causal(int n, double* u, long su, const double* d, long sd, double a) {
    for (int j = 1; j < n; ++j) {
        double w = pow(a, d[j * sd]);
        u[j * su] = (1.0 - w) * u[j * su] + w * u[(j - 1) * su];
    }
}

/* Anti-causal recurrence, in place, right to left:
 *   K[n-1] = x[n-1];  K[j] = (1 - w'_j) x[j] + w'_j K[j+1],  w'_j = a^d[j+1]
 * (d[j+1] is the distance between j and j+1). */
void orc_anticausal(int n, double* u, long su, const double* d, long sd, double a) {
    for (int j = n - 2; j >= 0; --j) {
        double w = pow(a, d[(j + 1) * sd]);
        u[j * su] = (1.0 - w) * u[j * su] + w * u[(j + 1) * su];
    }
}

/* One horizontal pass: causal then anti-causal along every row. */
void orc_row_pass(int H, int W, double* u, const double* dX, double a) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        orc_causal(W, u + (long)y * W, 1, dX + (long)y * W, 1, a);
        orc_anticausal(W, u + (long)y * W, 1, dX + (long)y * W, 1, a);
    }
}

/* One vertical pass: causal (top to bottom) then anti-causal along every column. */
void orc_col_pass(int H, int W, double* u, const double* dY, double a) {
#pragma omp parallel for schedule(static)
    for (int x = 0; x < W; ++x) {
        orc_causal(H, u + x, W, dY + x, W, a);
        orc_anticausal(H, u + x, W, dY + x, W, a);
    }
}

/* Edge-aware mean z_bar = A src (Eq. 10 with the recursive-filter kernel):
 * A = V(a_N) H(a_N) ... V(a_1) H(a_1); the first pass applied is horizontal. */
void orc_filter(int H, int W, const double* dX, const double* dY, int N, const double* a,
                const double* src, double* dst) {
    memcpy(dst, src, sizeof(double) * (size_t)H * W);
    for (int i = 0; i < N; ++i) {
        orc_row_pass(H, W, dst, dX, a[i]);
        orc_col_pass(H, W, dst, dY, a[i]);
    }
}

/* Box-kernel edge-aware mean along one line (Eq. 10 with the kernel it prints,
 * W_ij = 1 if |DT_i - DT_j| <= r): the domain coordinate is ct[0] = 0, ct[n] = ct[n-1] + d[n]
 * (d[n] the distance between n-1 and n), and out[n] is the plain average of x[m] over every m
 * with |ct[m] - ct[n]| <= r.  Written from the definition: for each n, every m is tested.
 * The distances are taken as given; coordinates are summed in double precision. */
static void box_line(int n, double* x, long sx, const double* d, long sd, double r, double* ct, double* tmp) {
    ct[0] = 0.0;
    for (int j = 1; j < n; ++j) ct[j] = ct[j - 1] + d[j * sd];
    for (int i = 0; i < n; ++i) {
        double sum = 0.0;
        int cnt = 0;
        for (int m = 0; m < n; ++m) {
            if (fabs(ct[m] - ct[i]) <= r) {
                sum += x[m * sx];
                ++cnt;
            }
        }
        tmp[i] = sum / cnt;  /* m = i is always in the window */
    }
    for (int i = 0; i < n; ++i) x[i * sx] = tmp[i];
}

/* The box-kernel filter: N passes, each a horizontal then a vertical box average with radius
 * r_i = sigma_i sqrt(3) (a box of half-width r has variance r^2 / 3, the sigma_i^2 of the
 * recursive filter's pass i; schedule of orc_schedule), the first pass horizontal. */
void orc_box_filter(int H, int W, const double* dX, const double* dY, int N, const double* sigma,
                    const double* src, double* dst) {
    memcpy(dst, src, sizeof(double) * (size_t)H * W);
    const int n = H > W ? H : W;
    for (int i = 0; i < N; ++i) {
        const double r = sigma[i] * sqrt(3.0);
#pragma omp parallel
        {
            double* ct = (double*)malloc(sizeof(double) * n);
            double* tmp = (double*)malloc(sizeof(double) * n);
#pragma omp for schedule(static)
            for (int y = 0; y < H; ++y) box_line(W, dst + (long)y * W, 1, dX + (long)y * W, 1, r, ct, tmp);
#pragma omp for schedule(static)
            for (int x = 0; x < W; ++x) box_line(H, dst + x, W, dY + x, W, r, ct, tmp);
            free(ct);
            free(tmp);
        }
    }
}

/* Confidence of Eq. 7 (§3.1): the edge-aware mean DT (Eq. 10, orc_filter) of the target and of
 * its square give the local variance V = DT(t^2) - DT(t)^2, and c = exp(-V / (2 sigma_c^2)).
 * V is never negative in exact arithmetic (DT is a non-negative, row-stochastic average); a
 * negative value from rounding is taken as 0. */
void orc_confidence(int H, int W, const double* dX, const double* dY, int N, const double* a,
                    const double* t, double sigma_c, double* c) {
    const size_t n = (size_t)H * W;
    double* t2 = (double*)malloc(sizeof(double) * n);
    double* m1 = (double*)malloc(sizeof(double) * n);
    double* m2 = (double*)malloc(sizeof(double) * n);
    for (size_t i = 0; i < n; ++i) t2[i] = t[i] * t[i];
    orc_filter(H, W, dX, dY, N, a, t, m1);
    orc_filter(H, W, dX, dY, N, a, t2, m2);
    for (size_t i = 0; i < n; ++i) {
        double v = m2[i] - m1[i] * m1[i];
        if (v < 0.0) v = 0.0;
        c[i] = exp(-v / (2.0 * sigma_c * sigma_c));
    }
    free(t2);
    free(m1);
    free(m2);
}

/* Support S_i = sum_j W_ij of the (unnormalised) separable recursive-filter
 * kernel, W_ij = a^(domain-transform distance between i and j) along a row
 * then along a column, with a = exp(-sqrt(2) / sigma_s).  Along one line:
 *   P[j] = x[j] + w_j P[j-1]      (all j' <= j)
 *   Q[j] = x[j] + w_{j+1} Q[j+1]  (all j' >= j)
 *   out  = P + Q - x              (j itself counted once)
 * Rows run on x = 1, columns on the row result.  For a flat guide and an
 * unbounded image S = ((1 + a) / (1 - a))^2, which is returned as *s_flat.
 * Used to weight the confidence by the support (§3.1, after Eq. 6). */
static void support_line(int n, const double* x, long sx, double* out, long so, const double* d, long sd,
                         double a, double* P, double* Q) {
    P[0] = x[0];
    for (int j = 1; j < n; ++j) P[j] = x[j * sx] + pow(a, d[j * sd]) * P[j - 1];
    Q[n - 1] = x[(n - 1) * sx];
    for (int j = n - 2; j >= 0; --j) Q[j] = x[j * sx] + pow(a, d[(j + 1) * sd]) * Q[j + 1];
    for (int j = 0; j < n; ++j) out[j * so] = P[j] + Q[j] - x[j * sx];
}

void orc_support(int H, int W, const double* dX, const double* dY, double sigma_s, double* S, double* s_flat) {
    double a = exp(-sqrt(2.0) / sigma_s);
    double* s = (double*)malloc(sizeof(double) * (size_t)H * W);
    double* ones = (double*)malloc(sizeof(double) * (size_t)W);
    for (int x = 0; x < W; ++x) ones[x] = 1.0;
#pragma omp parallel
    {
        int n = H > W ? H : W;
        double* P = (double*)malloc(sizeof(double) * (size_t)n);
        double* Q = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
        for (int y = 0; y < H; ++y)
            support_line(W, ones, 1, s + (long)y * W, 1, dX + (long)y * W, 1, a, P, Q);
#pragma omp for schedule(static)
        for (int x = 0; x < W; ++x)
            support_line(H, s + x, W, S + x, W, dY + x, W, a, P, Q);
        free(P);
        free(Q);
    }
    free(s);
    free(ones);
    if (s_flat) *s_flat = ((1.0 + a) / (1.0 - a)) * ((1.0 + a) / (1.0 - a));
}

/* Confidence actually used by the update: c itself (PLAIN) or c * S_flat / S
 * (SUPPORT: less weight on the target where the edge-aware support is large). */
static void effective_confidence(int H, int W, const double* dX, const double* dY, const double* c,
                                 double sigma_s, int conf_mode, double* chat) {
    long n = (long)H * W;
    if (conf_mode == ORC_CONF_SUPPORT) {
        double sf;
        orc_support(H, W, dX, dY, sigma_s, chat, &sf);
        for (long p = 0; p < n; ++p) chat[p] = c[p] * sf / chat[p];
    } else {
        memcpy(chat, c, sizeof(double) * (size_t)n);
    }
}

/* Derivative of the target term's loss per unit confidence at r = z - t: the square's r
 * (Eq. 3 writes c (z - t), without the factor 2 of Eq. 2), or for eps > 0 the Charbonnier
 * loss rho(r) = sqrt(r^2 + eps^2) of §4, rho'(r) = r / sqrt(r^2 + eps^2). */
static double target_slope(double r, double eps) { return eps > 0.0 ? r / sqrt(r * r + eps * eps) : r; }

/* One data-term update given z_k, z_bar = A z_k and the effective confidence.
 *   GD (Eq. 3, step eta; §4 uses eta = 0.99):
 *       z_{k+1} = z_k - eta * (lambda (z_k - z_bar) + c rho'(z_k - t))
 *     with rho'(r) = r for the square, r / sqrt(r^2 + eps^2) for the Charbonnier loss
 *     In SUPPORT mode the step is limited to eta_i = min(eta, 1 / (lambda + c_i))
 *     so that the iteration stays stable where c_i is large.
 *   Jacobi (the fixed point of Eq. 4):
 *       z_{k+1} = (lambda z_bar + c t) / (lambda + c);  z_k is kept where lambda + c = 0.
 *     With the Charbonnier loss (eps > 0) Eq. 4 is taken with the loss's weight at the current
 *     iterate, c~ = c / sqrt((z_k - t)^2 + eps^2) in place of c (the loss written as
 *     c~ (z - t)^2 / 2 plus a constant around z_k): a fixed point of the iteration satisfies
 *     lambda (z - z_bar) + c rho'(z - t) = 0, the stationarity the gradient step aims at. */
static void update(long n, const double* zk, const double* zbar, const double* t, const double* chat, double lambda,
                   double eta, int update_mode, double eps, int clamp_step, double* out) {
    for (long p = 0; p < n; ++p) {
        if (update_mode == ORC_UPDATE_JACOBI) {
            double cw = chat[p];
            if (eps > 0.0) {
                const double r = zk[p] - t[p];
                cw = chat[p] / sqrt(r * r + eps * eps);
            }
            double den = lambda + cw;
            out[p] = (den != 0.0) ? (lambda * zbar[p] + cw * t[p]) / den : zk[p];
        } else {
            double e = eta;
            if (clamp_step && lambda + chat[p] > 0.0 && 1.0 / (lambda + chat[p]) < e) e = 1.0 / (lambda + chat[p]);
            out[p] = zk[p] - e * (lambda * (zk[p] - zbar[p]) + chat[p] * target_slope(zk[p] - t[p], eps));
        }
    }
}

/* The solver: K iterations of  z_bar = A z_k;  z_{k+1} = update(z_k, z_bar)
 * starting from z_0 = z0 (the target t when z0 is NULL).  When ckpt is not
 * NULL it receives z_0 .. z_{K-1} (K planes).  Returns 0. */
/* The solve with either kernel of the edge-aware mean: kernel 0 the recursive filter
 * (orc_filter), kernel 1 the box kernel Eq. 10 prints (orc_box_filter); the iterations and the
 * update are the same. */
int orc_solve_kernel(int H, int W, const double* dX, const double* dY, const double* t, const double* c,
                     const double* z0, double lambda, double sigma_s, double eta, int K, int N, int update_mode,
                     double eps, int conf_mode, int kernel, double* z_out, double* ckpt);

int orc_solve(int H, int W, const double* dX, const double* dY, const double* t, const double* c, const double* z0,
              double lambda, double sigma_s, double eta, int K, int N, int update_mode, int conf_mode,
              double* z_out, double* ckpt) {
    return orc_solve_kernel(H, W, dX, dY, t, c, z0, lambda, sigma_s, eta, K, N, update_mode, 0.0, conf_mode, 0,
                            z_out, ckpt);
}

int orc_solve_kernel(int H, int W, const double* dX, const double* dY, const double* t, const double* c,
                     const double* z0, double lambda, double sigma_s, double eta, int K, int N, int update_mode,
                     double eps, int conf_mode, int kernel, double* z_out, double* ckpt) {
    long n = (long)H * W;
    double* sig = (double*)malloc(sizeof(double) * (size_t)N);
    double* a = (double*)malloc(sizeof(double) * (size_t)N);
    double* chat = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* zbar = (double*)malloc(sizeof(double) * (size_t)n);
    orc_schedule(sigma_s, N, sig, a);
    effective_confidence(H, W, dX, dY, c, sigma_s, conf_mode, chat);
    memcpy(z, z0 ? z0 : t, sizeof(double) * (size_t)n);
    for (int k = 0; k < K; ++k) {
        if (ckpt) memcpy(ckpt + (long)k * n, z, sizeof(double) * (size_t)n);
        if (kernel == 1) orc_box_filter(H, W, dX, dY, N, sig, z, zbar);
        else orc_filter(H, W, dX, dY, N, a, z, zbar);
        update(n, z, zbar, t, chat, lambda, eta, update_mode, eps, conf_mode == ORC_CONF_SUPPORT, z);
    }
    memcpy(z_out, z, sizeof(double) * (size_t)n);
    free(sig);
    free(a);
    free(chat);
    free(z);
    free(zbar);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Reverse mode.  The paper has no backward pass; the adjoints below follow
 * from the forward recurrences by the chain rule.
 *
 * Causal recurrence J[j] = (1 - w_j) x[j] + w_j J[j-1] (J[0] = x[0]).  Given
 * Jbar (the gradient arriving at every J[j]):
 *   g[n-1] = Jbar[n-1];  g[j] = Jbar[j] + w_{j+1} g[j+1]      (total gradient of J[j])
 *   xbar[j] = (1 - w_j) g[j] (j >= 1),  xbar[0] = g[0]
 *   wbar_j += g[j] (J[j-1] - x[j])                              (j >= 1)
 * Anti-causal K[j] = (1 - w_{j+1}) J[j] + w_{j+1} K[j+1] (K[n-1] = J[n-1]):
 *   h[0] = Kbar[0];  h[j] = Kbar[j] + w_j h[j-1]
 *   Jbar[j] = (1 - w_{j+1}) h[j] (j <= n-2),  Jbar[n-1] = h[n-1]
 *   wbar_{j+1} += h[j] (K[j+1] - J[j])                          (j <= n-2)
 * and dbar_j += wbar_j * w_j * ln(a) since w_j = a^d_j.
 * ------------------------------------------------------------------------- */
static void pass_line_adjoint(int n, const double* x, long sx, const double* d, long sd, double a,
                              const double* gout, long sg, double* gin, long si, double* dbar, long sb,
                              double* w, double* J, double* Kv, double* h, double* wbar) {
    /* recompute the forward sweep values of this line */
    w[0] = 0.0;
    for (int j = 1; j < n; ++j) w[j] = pow(a, d[j * sd]);
    J[0] = x[0];
    for (int j = 1; j < n; ++j) J[j] = (1.0 - w[j]) * x[j * sx] + w[j] * J[j - 1];
    Kv[n - 1] = J[n - 1];
    for (int j = n - 2; j >= 0; --j) Kv[j] = (1.0 - w[j + 1]) * J[j] + w[j + 1] * Kv[j + 1];
    for (int j = 0; j < n; ++j) wbar[j] = 0.0;
    /* anti-causal adjoint */
    h[0] = gout[0];
    for (int j = 1; j < n; ++j) h[j] = gout[j * sg] + w[j] * h[j - 1];
    /* h now holds the total gradient of K; turn it into Jbar in place */
    for (int j = 0; j <= n - 2; ++j) wbar[j + 1] += h[j] * (Kv[j + 1] - J[j]);
    for (int j = 0; j <= n - 2; ++j) h[j] = (1.0 - w[j + 1]) * h[j];
    /* causal adjoint: h is Jbar */
    double g = h[n - 1];
    double* gJ = Kv; /* reuse storage: Kv no longer needed */
    gJ[n - 1] = g;
    for (int j = n - 2; j >= 0; --j) gJ[j] = h[j] + w[j + 1] * gJ[j + 1];
    for (int j = 1; j < n; ++j) wbar[j] += gJ[j] * (J[j - 1] - x[j * sx]);
    gin[0] = gJ[0];
    for (int j = 1; j < n; ++j) gin[j * si] = (1.0 - w[j]) * gJ[j];
    double la = log(a);
    for (int j = 1; j < n; ++j) dbar[j * sb] += wbar[j] * w[j] * la;
}

static void row_pass_adjoint(int H, int W, const double* x, const double* dX, double a, const double* gout,
                             double* gin, double* dXbar) {
#pragma omp parallel
    {
        double* buf = (double*)malloc(sizeof(double) * 5 * (size_t)W);
#pragma omp for schedule(static)
        for (int y = 0; y < H; ++y) {
            long o = (long)y * W;
            pass_line_adjoint(W, x + o, 1, dX + o, 1, a, gout + o, 1, gin + o, 1, dXbar + o, 1, buf, buf + W,
                              buf + 2 * W, buf + 3 * W, buf + 4 * W);
        }
        free(buf);
    }
}

static void col_pass_adjoint(int H, int W, const double* x, const double* dY, double a, const double* gout,
                             double* gin, double* dYbar) {
#pragma omp parallel
    {
        double* buf = (double*)malloc(sizeof(double) * 5 * (size_t)H);
#pragma omp for schedule(static)
        for (int xx = 0; xx < W; ++xx) {
            pass_line_adjoint(H, x + xx, W, dY + xx, W, a, gout + xx, W, gin + xx, W, dYbar + xx, W, buf, buf + H,
                              buf + 2 * H, buf + 3 * H, buf + 4 * H);
        }
        free(buf);
    }
}

/* Adjoint of the edge-aware mean: gsrc = A^T gdst, accumulating into dXbar,
 * dYbar the gradient with respect to the distances.  The 2N pass inputs are
 * recomputed from src. */
void orc_filter_adjoint(int H, int W, const double* dX, const double* dY, int N, const double* a, const double* src,
                        const double* gdst, double* gsrc, double* dXbar, double* dYbar) {
    long n = (long)H * W;
    double* U = (double*)malloc(sizeof(double) * (size_t)(2 * N) * n);
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    double* g2 = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(U, src, sizeof(double) * (size_t)n);
    for (int p = 0; p < 2 * N - 1; ++p) {
        memcpy(U + (long)(p + 1) * n, U + (long)p * n, sizeof(double) * (size_t)n);
        if (p % 2 == 0)
            orc_row_pass(H, W, U + (long)(p + 1) * n, dX, a[p / 2]);
        else
            orc_col_pass(H, W, U + (long)(p + 1) * n, dY, a[p / 2]);
    }
    memcpy(g, gdst, sizeof(double) * (size_t)n);
    for (int p = 2 * N - 1; p >= 0; --p) {
        if (p % 2 == 0)
            row_pass_adjoint(H, W, U + (long)p * n, dX, a[p / 2], g, g2, dXbar);
        else
            col_pass_adjoint(H, W, U + (long)p * n, dY, a[p / 2], g, g2, dYbar);
        double* tmp = g;
        g = g2;
        g2 = tmp;
    }
    memcpy(gsrc, g, sizeof(double) * (size_t)n);
    free(U);
    free(g);
    free(g2);
}

/* Conjugate gradients on F(z) = lambda/2 |z - A z|^2 + sum_i c_i (z_i - t_i)^2 (Eq. 2 with the
 * recursive-filter mean): M = lambda (I - A)^T (I - A) + 2C is symmetric positive definite when
 * some c_i > 0 (A keeps constants, so I - A vanishes only on them), and the minimiser solves
 * M z = 2 C t.  K steps of textbook CG from z_0 (z_init, or t): r = b - M z, p = r; per step
 * q = M p, alpha = r.r / p.q, z += alpha p, r -= alpha q, beta = r'.r' / r.r, p = r' + beta p.
 * A^T comes from orc_filter_adjoint (its distance gradients are not needed here). */
static void cg_apply_M(int H, int W, const double* dX, const double* dY, int N, const double* a, const double* c,
                       double lambda, const double* p, double* q, double* t1, double* t2, double* junk) {
    const long n = (long)H * W;
    orc_filter(H, W, dX, dY, N, a, p, t1);
    for (long i = 0; i < n; ++i) t1[i] = p[i] - t1[i];  /* (I - A) p */
    memset(junk, 0, sizeof(double) * (size_t)(2 * n));
    orc_filter_adjoint(H, W, dX, dY, N, a, t1, t1, t2, junk, junk + n);  /* A^T (I - A) p */
    for (long i = 0; i < n; ++i) q[i] = lambda * (t1[i] - t2[i]) + 2.0 * c[i] * p[i];
}

int orc_solve_cg(int H, int W, const double* dX, const double* dY, const double* t, const double* c,
                 const double* z0, double lambda, double sigma_s, int K, int N, double* z_out) {
    const long n = (long)H * W;
    double* sig = (double*)malloc(sizeof(double) * (size_t)N);
    double* a = (double*)malloc(sizeof(double) * (size_t)N);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    double* t1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* t2 = (double*)malloc(sizeof(double) * (size_t)n);
    double* junk = (double*)malloc(sizeof(double) * (size_t)(2 * n));
    orc_schedule(sigma_s, N, sig, a);
    memcpy(z, z0 ? z0 : t, sizeof(double) * (size_t)n);
    cg_apply_M(H, W, dX, dY, N, a, c, lambda, z, q, t1, t2, junk);
    double rr = 0.0;
    for (long i = 0; i < n; ++i) {
        r[i] = 2.0 * c[i] * t[i] - q[i];
        p[i] = r[i];
        rr += r[i] * r[i];
    }
    for (int k = 0; k < K && rr > 0.0; ++k) {
        cg_apply_M(H, W, dX, dY, N, a, c, lambda, p, q, t1, t2, junk);
        double pq = 0.0;
        for (long i = 0; i < n; ++i) pq += p[i] * q[i];
        const double alpha = rr / pq;
        double rr_new = 0.0;
        for (long i = 0; i < n; ++i) {
            z[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            rr_new += r[i] * r[i];
        }
        const double beta = rr_new / rr;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
    memcpy(z_out, z, sizeof(double) * (size_t)n);
    free(sig);
    free(a);
    free(z);
    free(r);
    free(p);
    free(q);
    free(t1);
    free(t2);
    free(junk);
    return 0;
}

/* Gradient of the distances with respect to the guide (Eq. 8-9 forms above).
 * L1 uses the subgradient sign(0) = 0. */
void orc_distances_adjoint(int C, int H, int W, const double* I, double sigma_s, double sigma_r, int norm,
                           const double* dX, const double* dY, const double* dXbar, const double* dYbar,
                           double* Ibar) {
    double k = sigma_s / sigma_r;
    long plane = (long)H * W;
    memset(Ibar, 0, sizeof(double) * (size_t)C * plane);
    for (int c = 0; c < C; ++c) {
        const double* Ic = I + c * plane;
        double* Gc = Ibar + c * plane;
        for (int y = 0; y < H; ++y) {
            for (int x = 0; x < W; ++x) {
                long p = (long)y * W + x;
                if (x > 0) {
                    double diff = Ic[p] - Ic[p - 1];
                    double g = (norm == ORC_NORM_L2) ? dXbar[p] * k * k * diff / dX[p]
                                                     : dXbar[p] * k * ((diff > 0) - (diff < 0));
                    Gc[p] += g;
                    Gc[p - 1] -= g;
                }
                if (y > 0) {
                    double diff = Ic[p] - Ic[p - W];
                    double g = (norm == ORC_NORM_L2) ? dYbar[p] * k * k * diff / dY[p]
                                                     : dYbar[p] * k * ((diff > 0) - (diff < 0));
                    Gc[p] += g;
                    Gc[p - W] -= g;
                }
            }
        }
    }
}

/* Reverse mode of orc_solve (PLAIN confidence only; returns -1 for SUPPORT).
 * Inputs as for orc_solve plus the guide I (C planes) and gz = dL/dz_K.
 * Outputs (each may be NULL): gt = dL/dt (including the z_0 = t path when z0
 * is NULL), gc = dL/dc, gI = dL/dI (C planes), gz0 = dL/dz0 (only when z0 is
 * given).  The iterates are recomputed by a forward solve. */
int orc_solve_backward(int C, int H, int W, const double* I, double sigma_s, double sigma_r, int norm,
                       const double* t, const double* c, const double* z0, double lambda, double eta, int K, int N,
                       int update_mode, double eps, int conf_mode, const double* gz, double* gt, double* gc,
                       double* gI, double* gz0) {
    if (conf_mode != ORC_CONF_PLAIN) return -1;
    long n = (long)H * W;
    double* dX = (double*)malloc(sizeof(double) * (size_t)n);
    double* dY = (double*)malloc(sizeof(double) * (size_t)n);
    double* sig = (double*)malloc(sizeof(double) * (size_t)N);
    double* a = (double*)malloc(sizeof(double) * (size_t)N);
    double* Z = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1) * n);
    double* zlast = (double*)malloc(sizeof(double) * (size_t)n);
    double* zbar = (double*)malloc(sizeof(double) * (size_t)n);
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    double* gbar = (double*)malloc(sizeof(double) * (size_t)n);
    double* gprev = (double*)malloc(sizeof(double) * (size_t)n);
    double* dXbar = (double*)calloc((size_t)n, sizeof(double));
    double* dYbar = (double*)calloc((size_t)n, sizeof(double));
    double* tb = (double*)calloc((size_t)n, sizeof(double));
    double* cb = (double*)calloc((size_t)n, sizeof(double));

    orc_distances(C, H, W, I, sigma_s, sigma_r, norm, dX, dY);
    orc_schedule(sigma_s, N, sig, a);
    orc_solve_kernel(H, W, dX, dY, t, c, z0, lambda, sigma_s, eta, K, N, update_mode, eps, conf_mode, 0, zlast, Z);
    memcpy(g, gz, sizeof(double) * (size_t)n);

    for (int k = K - 1; k >= 0; --k) {
        const double* zk = Z + (long)k * n;
        orc_filter(H, W, dX, dY, N, a, zk, zbar);
        for (long p = 0; p < n; ++p) {
            if (update_mode == ORC_UPDATE_JACOBI) {
                /* the weight of the Charbonnier loss at z_k: w = 1 / sqrt(r^2 + eps^2), r = z_k - t
                 * (w = 1 for the square); c~ = c w enters like c, and reaches z_k and t through r,
                 * dc~/dr = -c r w^3 */
                const double r = zk[p] - t[p];
                const double w = eps > 0.0 ? 1.0 / sqrt(r * r + eps * eps) : 1.0;
                const double cw = c[p] * w;
                double den = lambda + cw;
                if (den != 0.0) {
                    const double gcw = lambda * (t[p] - zbar[p]) / (den * den) * g[p];
                    const double gr = eps > 0.0 ? -c[p] * r * w * w * w * gcw : 0.0;
                    tb[p] += cw / den * g[p] - gr;
                    cb[p] += w * gcw;
                    gbar[p] = lambda / den * g[p];
                    gprev[p] = gr;
                } else {
                    gbar[p] = 0.0;
                    gprev[p] = g[p];
                }
            } else {
                /* rho'(r) and rho''(r) at r = z_k - t: r and 1 for the square, r / s and
                 * eps^2 / s^3 (s = sqrt(r^2 + eps^2)) for the Charbonnier loss */
                const double r = zk[p] - t[p];
                const double s = sqrt(r * r + eps * eps);
                const double d1 = target_slope(r, eps);
                const double d2 = eps > 0.0 ? eps * eps / (s * s * s) : 1.0;
                tb[p] += eta * c[p] * d2 * g[p];
                cb[p] -= eta * d1 * g[p];
                gbar[p] = eta * lambda * g[p];
                gprev[p] = (1.0 - eta * lambda - eta * c[p] * d2) * g[p];
            }
        }
        /* g <- A^T gbar, accumulate distance gradients */
        orc_filter_adjoint(H, W, dX, dY, N, a, zk, gbar, g, dXbar, dYbar);
        for (long p = 0; p < n; ++p) g[p] += gprev[p];
    }
    if (z0 == NULL) {
        for (long p = 0; p < n; ++p) tb[p] += g[p];
    } else if (gz0) {
        memcpy(gz0, g, sizeof(double) * (size_t)n);
    }
    if (gt) memcpy(gt, tb, sizeof(double) * (size_t)n);
    if (gc) memcpy(gc, cb, sizeof(double) * (size_t)n);
    if (gI) orc_distances_adjoint(C, H, W, I, sigma_s, sigma_r, norm, dX, dY, dXbar, dYbar, gI);

    free(dX); free(dY); free(sig); free(a); free(Z); free(zlast); free(zbar); free(g);
    free(gbar); free(gprev); free(dXbar); free(dYbar); free(tb); free(cb);
    return 0;
}
