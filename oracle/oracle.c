/*
 * oracle.c -- plain FP64 CPU oracle for Kalman-MPC (Vaziri & Fang,
 * "Optimal Inferential Control of Convolutional Neural Networks",
 * arXiv 2410.09663).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library; it is written from the paper's equations, step by step, in
 * double precision, with no blocking, fusion or reordering beyond what the
 * equations state.  Random numbers the method draws (W, V) are inputs.
 *
 * Functions and the passages they follow:
 *   oracle_conv3x3        one 3x3 "same" convolution layer of CNN_theta, Eq. (1)
 *   oracle_cnn_step       X_{k+1} = CNN_theta(X_k, U_k), Eq. (1), surrogate
 *                         structure [X; B U] -> hidden tanh layers -> 1 channel,
 *                         residual X + s * out
 *   oracle_moments        ensemble means and covariances,
 *                         Eq. (mathcalX-prediction-sample-mean) and
 *                         Eq. (Ybar-sample-mean-cov) with lambda = 1
 *   oracle_cholesky       textbook Cholesky factorisation (Appendix,
 *                         conditioning formula needs Sigma_Y^{-1})
 *   oracle_gain           K = Sigma^{XY} (Sigma^{Y})^{-1}, Eq. (ensemble-based-
 *                         Kalman-update-samplewise)
 *   oracle_enks_analysis  member-wise update X^i += K (Ybar_t - Y^i),
 *                         Eq. (Ybar-samples) .. (ensemble-based-Kalman-update)
 *   oracle_enks_solve     one receding-horizon solve, Algorithm 1 inner loop,
 *                         with the full smoothed history script-X kept exactly as
 *                         Eq. (prediction-concatenate) writes it
 *   oracle_run            the receding-horizon loop of Algorithm 1 with the
 *                         plant taken to be CNN_theta itself
 *   oracle_control_expand U = u T, and
 *   oracle_control_reduce u = U T^T (T T^T)^{-1}: the right transformation for
 *                         controls with fewer columns than the state (the
 *                         paragraph on narrow controls after Table I)
 *   oracle_row_cov        lambda/N sum_i (X^i - Xhat)(X^i - Xhat)^T, the
 *                         ensemble row covariance of Eq. (ensemble-based-
 *                         Kalman-update-cov) and Eq. (prediction-cov); and
 *   oracle_enks_solve_cov the solve with Algorithm 1's optional covariance
 *                         steps executed: Sigma^X_{t|t-1} (whose last block
 *                         row and column are Eq. (prediction-cov) and Eq.
 *                         (prediction-cross-cov), concatenated as in Eq.
 *                         (prediction-cov-concatenate)) after each prediction
 *                         and Sigma^X_{t|t} after each update
 *   oracle_softplus_barrier phi(x) = ln(1 + e^{beta x}) / alpha, and
 *   oracle_constraint_obs z = phi(g(X, U)) + eps: the virtual observation of
 *                         a constraint g(X, U) <= 0 with reference 0 (the
 *                         paragraph on state/input constraints after
 *                         Table I); oracle_enks_solve_c and oracle_run_c
 *                         append its rows to the pseudo-observation
 *
 * Readings where the paper is silent or garbled (all fixed here):
 *   - means use 1/N (Eq. (mathcalX-prediction-sample-mean)); the sums printed
 *     without 1/N in Eq. (Ybar-sample-mean-cov) and Eq. (prediction-mean) are
 *     read as means;
 *   - lambda = 1 / tr(Psi) and the 1/N factor cancel inside K (the remark after
 *     Eq. (ensemble-based-Kalman-update)); lambda = 1 is used;
 *   - f_CNN on the augmented state [X; U; dU] is
 *     [CNN(X, U); U; 0] + [0; W; W] (Eq. (virtual-system) rows 1-3);
 *   - ensemble initialisation at step k: X^i = X_k, U^i = U_{k-1} + W0^i,
 *     dU^i = W0^i;
 *   - updates happen at t = k+1 .. k+H (Algorithm 1); the applied control is the
 *     smoothed mean of the U block at time k after the last update;
 *   - constraints: the paper's scalar g is evaluated column by column, so a
 *     constraint is one row of m values and c of them stack into a c x m
 *     virtual observation; the family is affine per column,
 *     g = Gx X_t + Gu U_t - h 1^T, taken at the predicted X_t and U_t of each
 *     assimilation time t = k+1 .. k+H, observed with noise eps ~ N(0, s_z^2)
 *     and reference 0; the rows are observations only, never state.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_LAYERS 8

typedef struct {
    int n, m, l;                              /* X is n x m, U is l x m         */
    int n_layers;                             /* conv layers                    */
    int channels[ORACLE_MAX_LAYERS + 1];      /* channels[0] = 2, last = 1      */
    const double *w;                          /* per layer [Cout][Cin][3][3]    */
    const double *b;                          /* per layer [Cout]               */
    const double *B;                          /* n x l input matrix             */
    double residual_scale;                    /* X_{k+1} = X_k + s * out        */
} oracle_net;

/* c virtual constraint observations (c = 0: none). */
typedef struct {
    int c;
    const double *Gx;                         /* c x n                          */
    const double *Gu;                         /* c x l                          */
    const double *h;                          /* c                              */
    double alpha, beta;                       /* softplus barrier parameters    */
} oracle_cons;

/* ------------------------------------------------------------------------ */
/* Eq. (1): one 3x3 convolution layer, stride 1, zero padding ("same"),
 * cross-correlation convention:
 *   out[o][y][x] = b[o] + sum_c sum_{dy,dx in {0,1,2}}
 *                  w[o][c][dy][dx] * in[c][y+dy-1][x+dx-1]
 * followed by tanh when apply_tanh is set.  in is [Cin][n][m], out [Cout][n][m]. */
void oracle_conv3x3(int Cin, int Cout, int n, int m, const double *in,
                    const double *w, const double *b, int apply_tanh, double *out)
{
    /* Same sum as written above, accumulated term by term in (c, dy, dx)
     * order for every output pixel; the pixel loops are innermost and skip
     * the taps that fall on the zero padding. */
    for (int o = 0; o < Cout; ++o) {
        double *po = out + (size_t)o * n * m;
        for (int i = 0; i < n * m; ++i) po[i] = b[o];
        for (int c = 0; c < Cin; ++c)
            for (int dy = 0; dy < 3; ++dy)
                for (int dx = 0; dx < 3; ++dx) {
                    const double wv = w[((o * Cin + c) * 3 + dy) * 3 + dx];
                    const double *pi = in + (size_t)c * n * m;
                    int y0 = dy == 0 ? 1 : 0, y1 = dy == 2 ? n - 1 : n;
                    int x0 = dx == 0 ? 1 : 0, x1 = dx == 2 ? m - 1 : m;
                    for (int y = y0; y < y1; ++y) {
                        const double *src = pi + (size_t)(y + dy - 1) * m + (dx - 1);
                        double *dst = po + (size_t)y * m;
                        for (int x = x0; x < x1; ++x) dst[x] += wv * src[x];
                    }
                }
        if (apply_tanh)
            for (int i = 0; i < n * m; ++i) po[i] = tanh(po[i]);
    }
}

/* Eq. (1): X_next = CNN_theta(X, U).  Input channels are X and B U (n x m);
 * hidden layers apply tanh, the last layer is linear with one output channel;
 * X_next = X + residual_scale * out.  Returns 0 on success. */
int oracle_cnn_step(const oracle_net *net, const double *X, const double *U, double *X_next)
{
    const int n = net->n, m = net->m, l = net->l;
    int cmax = 2;
    for (int k = 0; k <= net->n_layers; ++k)
        if (net->channels[k] > cmax) cmax = net->channels[k];
    double *a = malloc(sizeof(double) * (size_t)cmax * n * m);
    double *z = malloc(sizeof(double) * (size_t)cmax * n * m);
    if (!a || !z) { free(a); free(z); return 1; }
    /* channel 0: X; channel 1: B U */
    memcpy(a, X, sizeof(double) * (size_t)n * m);
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < m; ++x) {
            double s = 0.0;
            for (int c = 0; c < l; ++c) s += net->B[y * l + c] * U[c * m + x];
            a[(size_t)n * m + y * m + x] = s;
        }
    const double *w = net->w, *b = net->b;
    for (int k = 0; k < net->n_layers; ++k) {
        int cin = net->channels[k], cout = net->channels[k + 1];
        int last = (k == net->n_layers - 1);
        oracle_conv3x3(cin, cout, n, m, a, w, b, !last, z);
        w += (size_t)cout * cin * 9;
        b += cout;
        double *t = a; a = z; z = t;
    }
    for (int i = 0; i < n * m; ++i) X_next[i] = X[i] + net->residual_scale * a[i];
    free(a); free(z);
    return 0;
}

/* Batched form of oracle_cnn_step over `batch` independent (X, U) pairs;
 * each pair is the same computation, run in parallel over pairs. */
int oracle_cnn_step_batch(const oracle_net *net, int batch, const double *X,
                          const double *U, double *X_next)
{
    const size_t nx = (size_t)net->n * net->m, nu = (size_t)net->l * net->m;
    int err = 0;
#pragma omp parallel for schedule(dynamic) reduction(|:err)
    for (int i = 0; i < batch; ++i)
        err |= oracle_cnn_step(net, X + i * nx, U + i * nu, X_next + i * nx);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Eq. (mathcalX-prediction-sample-mean) and Eq. (Ybar-sample-mean-cov), with
 * lambda = 1:
 *   xmean = (1/N) sum_i X^i                    (R x m)
 *   ymean = (1/N) sum_i Y^i                    (p x m)
 *   Cxy   = (1/N) sum_i (X^i - xmean)(Y^i - ymean)^T      (R x p)
 *   Cyy   = (1/N) sum_i (Y^i - ymean)(Y^i - ymean)^T      (p x p)
 * X^i lives at X + i*xs (row-major R x m), Y^i at Y + i*p*m. */
void oracle_moments(int N, int R, int p, int m, const double *X, long xs,
                    const double *Y, double *xmean, double *ymean,
                    double *Cxy, double *Cyy)
{
    memset(xmean, 0, sizeof(double) * (size_t)R * m);
    memset(ymean, 0, sizeof(double) * (size_t)p * m);
    for (int i = 0; i < N; ++i) {
        for (int r = 0; r < R * m; ++r) xmean[r] += X[i * xs + r];
        for (int r = 0; r < p * m; ++r) ymean[r] += Y[(size_t)i * p * m + r];
    }
    for (int r = 0; r < R * m; ++r) xmean[r] /= N;
    for (int r = 0; r < p * m; ++r) ymean[r] /= N;

    /* Each (r, c) entry sums over members i = 0..N-1 in order, and over
     * columns j inside each member; rows are independent. */
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < R; ++r)
        for (int c = 0; c < p; ++c) {
            double acc = 0.0;
            for (int i = 0; i < N; ++i) {
                const double *Xi = X + i * xs, *Yi = Y + (size_t)i * p * m;
                double s = 0.0;
                for (int j = 0; j < m; ++j)
                    s += (Xi[r * m + j] - xmean[r * m + j]) * (Yi[c * m + j] - ymean[c * m + j]);
                acc += s;
            }
            Cxy[r * p + c] = acc / N;
        }
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < p; ++r)
        for (int c = 0; c < p; ++c) {
            double acc = 0.0;
            for (int i = 0; i < N; ++i) {
                const double *Yi = Y + (size_t)i * p * m;
                double s = 0.0;
                for (int j = 0; j < m; ++j)
                    s += (Yi[r * m + j] - ymean[r * m + j]) * (Yi[c * m + j] - ymean[c * m + j]);
                acc += s;
            }
            Cyy[r * p + c] = acc / N;
        }
}

/* Textbook Cholesky A = L L^T of a symmetric p x p matrix (row-major); L is
 * written lower-triangular with zeros above the diagonal.  Returns 0, or
 * j+1 when the j-th pivot is not positive (A not positive definite). */
int oracle_cholesky(int p, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)p * p);
    for (int j = 0; j < p; ++j) {
        double d = A[j * p + j];
        for (int k = 0; k < j; ++k) d -= L[j * p + k] * L[j * p + k];
        if (!(d > 0.0)) return j + 1;
        double ljj = sqrt(d);
        L[j * p + j] = ljj;
        for (int i = j + 1; i < p; ++i) {
            double s = A[i * p + j];
            for (int k = 0; k < j; ++k) s -= L[i * p + k] * L[j * p + k];
            L[i * p + j] = s / ljj;
        }
    }
    return 0;
}

/* Eq. (ensemble-based-Kalman-update-samplewise): K = Cxy Cyy^{-1}, R x p.
 * Each row k of K solves Cyy k^T = cxy^T (Cyy symmetric) by forward and back
 * substitution with the Cholesky factor.  Returns the Cholesky status. */
int oracle_gain(int R, int p, const double *Cxy, const double *Cyy, double *K)
{
    double *L = malloc(sizeof(double) * (size_t)p * p);
    double *z = malloc(sizeof(double) * (size_t)p);
    if (!L || !z) { free(L); free(z); return -1; }
    int st = oracle_cholesky(p, Cyy, L);
    if (st == 0) {
        for (int r = 0; r < R; ++r) {
            const double *c = Cxy + (size_t)r * p;
            double *k = K + (size_t)r * p;
            for (int i = 0; i < p; ++i) {           /* L z = c      */
                double s = c[i];
                for (int j = 0; j < i; ++j) s -= L[i * p + j] * z[j];
                z[i] = s / L[i * p + i];
            }
            for (int i = p - 1; i >= 0; --i) {      /* L^T k = z    */
                double s = z[i];
                for (int j = i + 1; j < p; ++j) s -= L[j * p + i] * k[j];
                k[i] = s / L[i * p + i];
            }
        }
    }
    free(L); free(z);
    return st;
}

/* Eq. (Ybar-samples) .. Eq. (ensemble-based-Kalman-update): given the prior
 * ensemble X^i (R x m at X + i*xs) and the perturbed predicted observations
 * Y^i = H X^i + V^i (p x m, contiguous per member), update in place
 *   X^i <- X^i + K (Ybar - Y^i),   K = Cxy Cyy^{-1}.
 * Returns the Cholesky status (0 on success; nothing is updated otherwise). */
int oracle_enks_analysis(int N, int R, int p, int m, double *X, long xs,
                         const double *Y, const double *Ybar)
{
    double *xmean = malloc(sizeof(double) * (size_t)R * m);
    double *ymean = malloc(sizeof(double) * (size_t)p * m);
    double *Cxy = malloc(sizeof(double) * (size_t)R * p);
    double *Cyy = malloc(sizeof(double) * (size_t)p * p);
    double *K = malloc(sizeof(double) * (size_t)R * p);
    if (!xmean || !ymean || !Cxy || !Cyy || !K) {
        free(xmean); free(ymean); free(Cxy); free(Cyy); free(K);
        return -1;
    }
    oracle_moments(N, R, p, m, X, xs, Y, xmean, ymean, Cxy, Cyy);
    int st = oracle_gain(R, p, Cxy, Cyy, K);
    if (st == 0) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < N; ++i) {
            double *Xi = X + i * xs;
            const double *Yi = Y + (size_t)i * p * m;
            for (int r = 0; r < R; ++r)
                for (int j = 0; j < m; ++j) {
                    double s = 0.0;
                    for (int c = 0; c < p; ++c)
                        s += K[r * p + c] * (Ybar[c * m + j] - Yi[c * m + j]);
                    Xi[r * m + j] += s;
                }
        }
    }
    free(xmean); free(ymean); free(Cxy); free(Cyy); free(K);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Eq. (ensemble-based-Kalman-update-cov) / Eq. (prediction-cov): the row
 * covariance of an ensemble of R x m matrices X^i (at X + i*xs),
 *   S = (lambda / N) sum_i (X^i - Xhat)(X^i - Xhat)^T,  Xhat = (1/N) sum_i X^i,
 * pooled over the m columns as the matrix-normal moments are (R x R). */
int oracle_row_cov(int N, int R, int m, const double *X, long xs, double lambda, double *S)
{
    double *mean = calloc((size_t)R * m, sizeof(double));
    if (!mean) return -1;
    for (int i = 0; i < N; ++i)
        for (size_t e = 0; e < (size_t)R * m; ++e) mean[e] += X[i * xs + e];
    for (size_t e = 0; e < (size_t)R * m; ++e) mean[e] /= N;
#pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) {
            double t = 0.0;
            for (int i = 0; i < N; ++i) {
                const double *xi = X + i * xs;
                for (int j = 0; j < m; ++j)
                    t += (xi[a * m + j] - mean[a * m + j]) * (xi[b * m + j] - mean[b * m + j]);
            }
            S[(size_t)a * R + b] = lambda / N * t;
        }
    free(mean);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Constraint rows (the paragraph on state/input constraints after Table I).
 * phi is evaluated as max(y, 0) + log1p(e^{-|y|}) with y = beta x, which is
 * ln(1 + e^{y}) rewritten so that e^{y} cannot overflow. */
double oracle_softplus_barrier(double x, double alpha, double beta)
{
    const double y = beta * x;
    return ((y > 0.0 ? y : 0.0) + log1p(exp(-fabs(y)))) / alpha;
}

/* z[r][j] = phi( sum_a Gx[r][a] X[a][j] + sum_b Gu[r][b] U[b][j] - h[r] )
 *           + eps[r][j]                       (X: n x m, U: l x m, z: c x m) */
void oracle_constraint_obs(const oracle_cons *cs, int n, int l, int m, const double *X,
                           const double *U, const double *eps, double *z)
{
    for (int r = 0; r < cs->c; ++r)
        for (int j = 0; j < m; ++j) {
            double g = -cs->h[r];
            for (int a = 0; a < n; ++a) g += cs->Gx[r * n + a] * X[a * m + j];
            for (int b = 0; b < l; ++b) g += cs->Gu[r * l + b] * U[b * m + j];
            z[r * m + j] = oracle_softplus_barrier(g, cs->alpha, cs->beta) + eps[r * m + j];
        }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 for one control step k (initialise, predict and update over the
   horizon, smoothed means).
 *
 * Augmented state X̄ = [X; U; dU] has q = n + 2l rows; the pseudo-observation
 * Ȳ = [X^ref; U^ref] has p = n + l rows and H = [I 0 0; 0 I 0].
 *
 * Inputs (all row-major, doubles):
 *   X_k    n x m          current field
 *   U_prev l x m          control applied at k-1
 *   X_ref  (H+1) x n x m  references for times k .. k+H
 *   U_ref  l x m
 *   noise  W0 [N][l][m], then W [H][N][l][m], VX [H][N][n][m], VU [H][N][l][m],
 *          then, with c > 0 constraint rows, VZ [H][N][c][m] (eps of z)
 *   cs     constraint rows (oracle_enks_solve_c only; NULL or c = 0: none);
 *          they extend Ȳ to p = n + l + c rows [X^ref; U^ref; 0]
 * Output:
 *   Xbar_hat (H+1) x q x m: smoothed means of blocks k .. k+H after the update
 *            at t = k+H (Eq. (ensemble-based-Kalman-update-mean)).
 * Returns 0, or the first nonzero Cholesky status. */
/* The solve above (cs: constraint rows, may be NULL) with Algorithm 1's
 * optional covariance steps executed: for
 * s = 1..H, slot s-1 of Sigma_pred / Sigma_post ((H+1) q x (H+1) q doubles
 * each) holds, compact row-major, the (s+1) q x (s+1) q row covariance of the
 * history blocks 0..s after the prediction to t = k+s (Sigma^X_{t|t-1}) and
 * after the update at t (Sigma^X_{t|t}), with factor lambda / N.  Either
 * output may be NULL. */
int oracle_enks_solve_cov(const oracle_net *net, int N, int H, const double *X_k,
                          const double *U_prev, const double *X_ref, const double *U_ref,
                          const double *noise, const oracle_cons *cs, double lambda,
                          double *Sigma_pred, double *Sigma_post, double *Xbar_hat)
{
    const int n = net->n, m = net->m, l = net->l;
    const int nc = cs ? cs->c : 0;
    const int q = n + 2 * l, p = n + l + nc;
    const size_t bq = (size_t)q * m;                   /* one block        */
    const long xs = (long)(H + 1) * (long)bq;          /* member stride    */
    const double *W0 = noise;
    const double *W = W0 + (size_t)N * l * m;
    const double *VX = W + (size_t)H * N * l * m;
    const double *VU = VX + (size_t)H * N * n * m;
    const double *VZ = VU + (size_t)H * N * l * m;     /* [H][N][c][m] */

    double *hist = calloc((size_t)N * xs, sizeof(double));
    double *Y = malloc(sizeof(double) * (size_t)N * p * m);
    double *Ybar = malloc(sizeof(double) * (size_t)p * m);
    if (!hist || !Y || !Ybar) { free(hist); free(Y); free(Ybar); return -1; }

    /* Algorithm 1's initialisation of X̄^i_{k|k} */
    for (int i = 0; i < N; ++i) {
        double *blk = hist + i * xs;
        const double *w0 = W0 + (size_t)i * l * m;
        memcpy(blk, X_k, sizeof(double) * (size_t)n * m);
        for (int r = 0; r < l * m; ++r) {
            blk[(size_t)n * m + r] = U_prev[r] + w0[r];          /* U  */
            blk[(size_t)(n + l) * m + r] = w0[r];                /* dU */
        }
    }

    int status = 0;
    for (int s = 1; s <= H; ++s) {                    /* t = k + s        */
        /* prediction, Eq. (prediction-samplewise):
         * X̄^i_{t|t-1} = f_CNN(X̄^i_{t-1|t-1}) + W̄^i_{t-1}               */
        const double *Ws = W + (size_t)(s - 1) * N * l * m;
        int err = 0;
#pragma omp parallel for schedule(dynamic) reduction(|:err)
        for (int i = 0; i < N; ++i) {
            const double *prev = hist + i * xs + (size_t)(s - 1) * bq;
            double *cur = hist + i * xs + (size_t)s * bq;
            const double *w = Ws + (size_t)i * l * m;
            err |= oracle_cnn_step(net, prev, prev + (size_t)n * m, cur);
            for (int r = 0; r < l * m; ++r) {
                cur[(size_t)n * m + r] = prev[(size_t)n * m + r] + w[r];   /* U  */
                cur[(size_t)(n + l) * m + r] = w[r];                       /* dU */
            }
        }
        if (err) { status = -1; break; }
        /* Eq. (prediction-concatenate): script-X^i = blocks 0..s,
         * which is the contiguous prefix of hist for member i.              */

        /* Eq. (Ybar-samples): Y^i = H X̄^i_t + V̄^i_t                       */
        const double *VXs = VX + (size_t)(s - 1) * N * n * m;
        const double *VUs = VU + (size_t)(s - 1) * N * l * m;
        for (int i = 0; i < N; ++i) {
            const double *cur = hist + i * xs + (size_t)s * bq;
            double *Yi = Y + (size_t)i * p * m;
            for (int r = 0; r < n * m; ++r) Yi[r] = cur[r] + VXs[(size_t)i * n * m + r];
            for (int r = 0; r < l * m; ++r)
                Yi[(size_t)n * m + r] = cur[(size_t)n * m + r] + VUs[(size_t)i * l * m + r];
            /* constraint rows z^i_t = phi(g(X^i_t, U^i_t)) + eps^i_t */
            if (nc > 0)
                oracle_constraint_obs(cs, n, l, m, cur, cur + (size_t)n * m,
                                      VZ + ((size_t)(s - 1) * N + i) * nc * m,
                                      Yi + (size_t)(n + l) * m);
        }
        /* Ȳ_t = [X^ref_t; U^ref; 0] */
        memcpy(Ybar, X_ref + (size_t)s * n * m, sizeof(double) * (size_t)n * m);
        memcpy(Ybar + (size_t)n * m, U_ref, sizeof(double) * (size_t)l * m);
        memset(Ybar + (size_t)(n + l) * m, 0, sizeof(double) * (size_t)nc * m);

        /* Eq. (Ybar-sample-mean-cov), Eq. (ensemble-based-
         * Kalman-update): update every block 0..s of every member.          */
        const int Rs = (s + 1) * q;
        const size_t slot = (size_t)(H + 1) * q * (size_t)(H + 1) * q;
        if (Sigma_pred && oracle_row_cov(N, Rs, m, hist, xs, lambda, Sigma_pred + (s - 1) * slot)) {
            status = -1;
            break;
        }
        int st = oracle_enks_analysis(N, Rs, p, m, hist, xs, Y, Ybar);
        if (st != 0) { status = st; break; }
        if (Sigma_post && oracle_row_cov(N, Rs, m, hist, xs, lambda, Sigma_post + (s - 1) * slot)) {
            status = -1;
            break;
        }
    }

    /* Algorithm 1's output: smoothed means of all blocks */
    if (status == 0) {
        memset(Xbar_hat, 0, sizeof(double) * (size_t)(H + 1) * bq);
        for (int i = 0; i < N; ++i)
            for (size_t r = 0; r < (size_t)(H + 1) * bq; ++r) Xbar_hat[r] += hist[i * xs + r];
        for (size_t r = 0; r < (size_t)(H + 1) * bq; ++r) Xbar_hat[r] /= N;
    }
    free(hist); free(Y); free(Ybar);
    return status;
}

int oracle_enks_solve_c(const oracle_net *net, int N, int H, const double *X_k,
                        const double *U_prev, const double *X_ref, const double *U_ref,
                        const double *noise, const oracle_cons *cs, double *Xbar_hat)
{
    return oracle_enks_solve_cov(net, N, H, X_k, U_prev, X_ref, U_ref, noise, cs, 1.0, NULL, NULL,
                                 Xbar_hat);
}

int oracle_enks_solve(const oracle_net *net, int N, int H, const double *X_k,
                      const double *U_prev, const double *X_ref, const double *U_ref,
                      const double *noise, double *Xbar_hat)
{
    return oracle_enks_solve_c(net, N, H, X_k, U_prev, X_ref, U_ref, noise, NULL, Xbar_hat);
}

/* Algorithm 1's receding-horizon loop for S control steps with the plant taken to be
 * CNN_theta itself (no model mismatch, no plant noise):
 *   solve at k -> U_k = smoothed U block at time k -> X_{k+1} = CNN(X_k, U_k).
 * Inputs: X_0 (n x m), U_init (U_{-1}, l x m), X_ref_all ((S+H) + 1 blocks of
 * n x m for absolute times 0 .. S+H-1 .. ), U_ref (l x m), noise_all (S blocks,
 * each laid out as oracle_enks_solve's noise).
 * Outputs: X_traj (S+1) x n x m (X_0 .. X_S), U_traj S x l x m (applied
 * controls), U_hat_all S x (H+1) x l x m (the smoothed U blocks of each solve;
 * may be NULL).  Returns 0 or the first failing status. */
int oracle_run_c(const oracle_net *net, int N, int H, int S, const double *X_0,
                 const double *U_init, const double *X_ref_all, const double *U_ref,
                 const double *noise_all, const oracle_cons *cs, double *X_traj, double *U_traj,
                 double *U_hat_all)
{
    const int n = net->n, m = net->m, l = net->l;
    const int q = n + 2 * l;
    const size_t nx = (size_t)n * m, nu = (size_t)l * m;
    const size_t nz = (size_t)(cs ? cs->c : 0) * m;
    const size_t noise_per = (size_t)N * nu + (size_t)H * N * (nu + nx + nu + nz);
    double *xhat = malloc(sizeof(double) * (size_t)(H + 1) * q * m);
    double *uprev = malloc(sizeof(double) * nu);
    if (!xhat || !uprev) { free(xhat); free(uprev); return -1; }
    memcpy(X_traj, X_0, sizeof(double) * nx);
    memcpy(uprev, U_init, sizeof(double) * nu);
    int status = 0;
    for (int k = 0; k < S; ++k) {
        status = oracle_enks_solve_c(net, N, H, X_traj + k * nx, uprev, X_ref_all + k * nx,
                                     U_ref, noise_all + k * noise_per, cs, xhat);
        if (status != 0) break;
        double *Uk = U_traj + k * nu;
        memcpy(Uk, xhat + nx, sizeof(double) * nu);        /* block 0, U rows */
        if (U_hat_all)
            for (int s = 0; s <= H; ++s)
                memcpy(U_hat_all + ((size_t)k * (H + 1) + s) * nu,
                       xhat + (size_t)s * q * m + nx, sizeof(double) * nu);
        status = oracle_cnn_step(net, X_traj + k * nx, Uk, X_traj + (k + 1) * nx);
        if (status != 0) break;
        memcpy(uprev, Uk, sizeof(double) * nu);
    }
    free(xhat); free(uprev);
    return status;
}

int oracle_run(const oracle_net *net, int N, int H, int S, const double *X_0,
               const double *U_init, const double *X_ref_all, const double *U_ref,
               const double *noise_all, double *X_traj, double *U_traj, double *U_hat_all)
{
    return oracle_run_c(net, N, H, S, X_0, U_init, X_ref_all, U_ref, noise_all, NULL, X_traj,
                        U_traj, U_hat_all);
}

/* Narrow controls (the paragraph after Table I): a control u with mu < m
 * columns is widened to U = u T (l x m) with a right-transformation matrix T
 * (mu x m, T T^T > 0), and a smoothed U is mapped back by
 * u = U T^T (T T^T)^{-1}.  Row-major throughout. */
void oracle_control_expand(int l, int mu, int m, const double *u, const double *T, double *U)
{
    for (int r = 0; r < l; ++r)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int c = 0; c < mu; ++c) s += u[r * mu + c] * T[c * m + j];
            U[r * m + j] = s;
        }
}

/* u = U T^T (T T^T)^{-1}: with G = T T^T (symmetric) each row of u solves
 * G u_r^T = (U T^T)_r^T, by the Cholesky factor of G and two substitutions.
 * Returns the Cholesky status (0, or the pivot + 1 where T T^T is not
 * positive definite), -1 if memory runs out. */
int oracle_control_reduce(int l, int m, int mu, const double *U, const double *T, double *u)
{
    double *G = malloc(sizeof(double) * (size_t)mu * mu);
    double *L = malloc(sizeof(double) * (size_t)mu * mu);
    double *w = malloc(sizeof(double) * (size_t)mu);
    double *z = malloc(sizeof(double) * (size_t)mu);
    if (!G || !L || !w || !z) { free(G); free(L); free(w); free(z); return -1; }
    for (int a = 0; a < mu; ++a)
        for (int b = 0; b < mu; ++b) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += T[a * m + j] * T[b * m + j];
            G[a * mu + b] = s;
        }
    int st = oracle_cholesky(mu, G, L);
    if (st == 0) {
        for (int r = 0; r < l; ++r) {
            for (int a = 0; a < mu; ++a) {          /* w = (U T^T)_r */
                double s = 0.0;
                for (int j = 0; j < m; ++j) s += U[r * m + j] * T[a * m + j];
                w[a] = s;
            }
            for (int i = 0; i < mu; ++i) {          /* L z = w */
                double s = w[i];
                for (int j = 0; j < i; ++j) s -= L[i * mu + j] * z[j];
                z[i] = s / L[i * mu + i];
            }
            for (int i = mu - 1; i >= 0; --i) {     /* L^T u_r = z */
                double s = z[i];
                for (int j = i + 1; j < mu; ++j) s -= L[j * mu + i] * u[r * mu + j];
                u[r * mu + i] = s / L[i * mu + i];
            }
        }
    }
    free(G); free(L); free(w); free(z);
    return st;
}
