/*
 * FP64 CPU oracle for the Generalized Tensor Transform (GTT).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Notation (Sec. 2.1): W is b x b, W[i][j] is row i, column j, 0-based.  An
 * index k < N = b^n has base-b digits k = sum_j k_j b^j; digit 0 is the least
 * significant.  Complex arrays are interleaved (re, im) doubles; inside the
 * file they are viewed as C99 `double complex`.
 *
 * Routes to G_N x (every one is a separate statement of the paper):
 *   O1 dense      G_N(p,q) = prod_j W[p_j][q_j]          (Sec. 2.6, element form)
 *   O2 basis      G_N(p,q) = f_q(x_p), x_p = (2p+1)/(2N) (Eq. defGNOne with the
 *                 recursion Eq. gtt_recursive_general_b_main, Sec. 2.2)
 *   O3 alg1       the recursive FastGTT of Sec. 3 / Algorithm 1: reshape to
 *                 (N/b) x b, Y = X W^T, recurse on each column, flatten rows
 *   O4 modes      one mode pass per digit k = 0..n-1, W applied to every
 *                 stride-b^k fibre (the cost structure of Sec. 3.1: n levels
 *                 of O(N b) each)
 *   O5 adjoint    O4 with W^H (the "inverse" G_N^dagger of Sec. 4)
 *   O6 gradient   reverse-mode derivative of y = G_N x for a real loss
 *                 (not in the paper; PyTorch's conjugate convention:
 *                 dx = (W^H)^{(x)n} dy, dW = sum_k sum_fibres g_{k+1} a_k^H)
 * Integer case: the same mode loop and dense product in uint32_t arithmetic,
 * which wraps modulo 2^32 (used for the unnormalised +-1 Hadamard base matrix).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- helpers */

static long long ipow(int b, int n) {
    long long r = 1;
    for (int i = 0; i < n; ++i) r *= b;
    return r;
}

/* digit j of k in base b */
static int digit(long long k, int b, int j) {
    for (int i = 0; i < j; ++i) k /= b;
    return (int)(k % b);
}

/* ------------------------------------------------------------ O1: dense */

/* y[p] = sum_q (prod_j W[p_j][q_j]) x[q].  O(N^2 n); intended for N <= 4096. */
int oracle_dense_c(int b, int n, const double *Wd, const double *xd, double *yd) {
    const cplx *W = (const cplx *)Wd;
    const cplx *x = (const cplx *)xd;
    cplx *y = (cplx *)yd;
    long long N = ipow(b, n);
    for (long long p = 0; p < N; ++p) {
        cplx acc = 0;
        for (long long q = 0; q < N; ++q) {
            cplx g = 1;
            for (int j = 0; j < n; ++j) g *= W[digit(p, b, j) * b + digit(q, b, j)];
            acc += g * x[q];
        }
        y[p] = acc;
    }
    return 0;
}

/* The dense matrix itself, G[p*N + q] = prod_j W[p_j][q_j]. */
int oracle_dense_matrix_c(int b, int n, const double *Wd, double *Gd) {
    const cplx *W = (const cplx *)Wd;
    cplx *G = (cplx *)Gd;
    long long N = ipow(b, n);
    for (long long p = 0; p < N; ++p)
        for (long long q = 0; q < N; ++q) {
            cplx g = 1;
            for (int j = 0; j < n; ++j) g *= W[digit(p, b, j) * b + digit(q, b, j)];
            G[p * N + q] = g;
        }
    return 0;
}

/* uint32 wrap-around version of O1. */
int oracle_dense_u32(int b, int n, const uint32_t *W, const uint32_t *x, uint32_t *y) {
    long long N = ipow(b, n);
    for (long long p = 0; p < N; ++p) {
        uint32_t acc = 0;
        for (long long q = 0; q < N; ++q) {
            uint32_t g = 1;
            for (int j = 0; j < n; ++j) g *= W[digit(p, b, j) * b + digit(q, b, j)];
            acc += g * x[q];
        }
        y[p] = acc;
    }
    return 0;
}

/* ------------------------------------------------------ O2: basis route */

/*
 * f_j^{(b^m)}(x) at x = num/den with 0 <= num < den, following
 * Eq. gtt_recursive_general_b_main:
 *   f_j^{(b^m)}(x) = W[floor(b x)][floor(j / b^{m-1})] * f_{j mod b^{m-1}}^{(b^{m-1})}({b x}),
 *   f_0^{(1)}(x) = 1 on [0, 1).
 * x is kept as an exact fraction so that floor(b x) and {b x} are integer
 * operations: floor(b x) = (b num) div den, {b x} = ((b num) mod den) / den.
 */
static cplx basis_f(const cplx *W, int b, int m, long long j, long long num, long long den) {
    if (m == 0) return (num >= 0 && num < den) ? 1.0 : 0.0;
    long long bm1 = ipow(b, m - 1);
    long long row = (b * num) / den;
    long long col = j / bm1;
    return W[row * b + col] * basis_f(W, b, m - 1, j % bm1, (b * num) % den, den);
}

/* G[p*N + q] = f_q^{(N)}((2p+1)/(2N))  (Eq. defGNOne). */
int oracle_basis_matrix_c(int b, int n, const double *Wd, double *Gd) {
    const cplx *W = (const cplx *)Wd;
    cplx *G = (cplx *)Gd;
    long long N = ipow(b, n);
    for (long long p = 0; p < N; ++p)
        for (long long q = 0; q < N; ++q) G[p * N + q] = basis_f(W, b, n, q, 2 * p + 1, 2 * N);
    return 0;
}

/* ------------------------------------------------------- O3: Algorithm 1 */

/*
 * FastGTT(x, W, n) of Sec. 3 written as stated there:
 *   n = 1: return W x.
 *   otherwise: X[p][q] = x[p b + q] (N/b rows, b columns); Y = X W^T;
 *   Z[:, j] = FastGTT(Y[:, j], W, n-1) for each column j; y = rows of Z
 *   concatenated.
 */
static void fast_gtt(const cplx *W, int b, int n, const cplx *x, cplx *y) {
    if (n == 1) {
        for (int i = 0; i < b; ++i) {
            cplx acc = 0;
            for (int j = 0; j < b; ++j) acc += W[i * b + j] * x[j];
            y[i] = acc;
        }
        return;
    }
    long long Ncur = ipow(b, n), Nprev = Ncur / b;
    cplx *Y = malloc(sizeof(cplx) * Ncur);   /* Y[p*b + j] */
    cplx *col = malloc(sizeof(cplx) * Nprev);
    cplx *zcol = malloc(sizeof(cplx) * Nprev);
    /* Y = X W^T : Y[p][j] = sum_q X[p][q] W^T[q][j] = sum_q x[p b + q] W[j][q] */
    for (long long p = 0; p < Nprev; ++p)
        for (int j = 0; j < b; ++j) {
            cplx acc = 0;
            for (int q = 0; q < b; ++q) acc += x[p * b + q] * W[j * b + q];
            Y[p * b + j] = acc;
        }
    /* recurse on each column, writing Z's column j straight into y[p b + j]
       (the row-by-row flattening of Z) */
    for (int j = 0; j < b; ++j) {
        for (long long p = 0; p < Nprev; ++p) col[p] = Y[p * b + j];
        fast_gtt(W, b, n - 1, col, zcol);
        for (long long p = 0; p < Nprev; ++p) y[p * b + j] = zcol[p];
    }
    free(Y);
    free(col);
    free(zcol);
}

int oracle_alg1_c(int b, int n, const double *Wd, const double *xd, double *yd) {
    if (n < 1) return -1;
    fast_gtt((const cplx *)Wd, b, n, (const cplx *)xd, (cplx *)yd);
    return 0;
}

/* ---------------------------------------------------- O4/O5: mode loop */

/*
 * One mode-k pass on a length-N vector: view it as [N/b^{k+1}][b][b^k] and
 *   out[h][i][l] = sum_j W[i][j] in[h][j][l].
 * Work is split across threads by fibre: fibre f = h * b^k + l.
 */
enum { KIND_C = 0, KIND_R = 1, KIND_U = 2 };

typedef struct {
    int kind, b;
    const void *W;
    const void *in;
    void *out;
    long long L;          /* b^k */
    long long f0, f1;     /* fibre range */
} pass_job;

static void pass_range(const pass_job *J) {
    const int b = J->b;
    const long long L = J->L, bL = (long long)b * L;
    for (long long f = J->f0; f < J->f1; ++f) {
        long long h = f / L, l = f % L, base = h * bL + l;
        if (J->kind == KIND_C) {
            const cplx *W = J->W, *in = J->in;
            cplx *out = J->out;
            for (int i = 0; i < b; ++i) {
                cplx acc = 0;
                for (int j = 0; j < b; ++j) acc += W[i * b + j] * in[base + j * L];
                out[base + i * L] = acc;
            }
        } else if (J->kind == KIND_R) {
            const double *W = J->W, *in = J->in;
            double *out = J->out;
            for (int i = 0; i < b; ++i) {
                double acc = 0;
                for (int j = 0; j < b; ++j) acc += W[i * b + j] * in[base + j * L];
                out[base + i * L] = acc;
            }
        } else {
            const uint32_t *W = J->W, *in = J->in;
            uint32_t *out = J->out;
            for (int i = 0; i < b; ++i) {
                uint32_t acc = 0;
                for (int j = 0; j < b; ++j) acc += W[i * b + j] * in[base + j * L];
                out[base + i * L] = acc;
            }
        }
    }
}

static void *pass_thread(void *arg) {
    pass_range((const pass_job *)arg);
    return NULL;
}

static size_t elem_size(int kind) {
    return kind == KIND_C ? sizeof(cplx) : kind == KIND_R ? sizeof(double) : sizeof(uint32_t);
}

/* Apply mode k to one vector, in -> out (distinct buffers), on `threads` threads. */
static void mode_pass(int kind, int b, const void *W, long long N, int k, const void *in,
                      void *out, int threads) {
    long long L = ipow(b, k);
    long long F = N / b;
    if (threads < 1) threads = 1;
    if ((long long)threads > F) threads = (int)F;
    if (threads == 1) {
        pass_job J = {kind, b, W, in, out, L, 0, F};
        pass_range(&J);
        return;
    }
    pthread_t *tid = malloc(sizeof(pthread_t) * threads);
    pass_job *jobs = malloc(sizeof(pass_job) * threads);
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (pass_job){kind, b, W, in, out, L, F * t / threads, F * (t + 1) / threads};
        pthread_create(&tid[t], NULL, pass_thread, &jobs[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    free(tid);
    free(jobs);
}

/* y[v] = G_N x[v] for each of `batch` vectors, applying modes 0..n-1 in order. */
static int modes_generic(int kind, int b, int n, const void *W, long long batch, const void *x,
                         void *y, int threads) {
    long long N = ipow(b, n);
    size_t es = elem_size(kind);
    char *tmp = malloc(es * N);
    if (!tmp) return -2;
    for (long long v = 0; v < batch; ++v) {
        const char *src = (const char *)x + es * N * v;
        char *dst = (char *)y + es * N * v;
        /* ping-pong between tmp and dst so that mode n-1 lands in dst */
        char *bufs[2] = {dst, tmp};
        int cur = (n % 2 == 1) ? 0 : 1; /* buffer receiving mode 0 */
        const void *in = src;
        for (int k = 0; k < n; ++k) {
            mode_pass(kind, b, W, N, k, in, bufs[cur], threads);
            in = bufs[cur];
            cur ^= 1;
        }
    }
    free(tmp);
    return 0;
}

int oracle_modes_c(int b, int n, const double *W, long long batch, const double *x, double *y,
                   int threads) {
    return modes_generic(KIND_C, b, n, W, batch, x, y, threads);
}

int oracle_modes_r(int b, int n, const double *W, long long batch, const double *x, double *y,
                   int threads) {
    return modes_generic(KIND_R, b, n, W, batch, x, y, threads);
}

int oracle_modes_u32(int b, int n, const uint32_t *W, long long batch, const uint32_t *x,
                     uint32_t *y, int threads) {
    return modes_generic(KIND_U, b, n, W, batch, x, y, threads);
}

/* One mode-k pass (complex) of one length-N vector, in -> out (distinct). */
int oracle_mode_pass_c(int b, int n, const double *W, int k, const double *x, double *y,
                       int threads) {
    if (k < 0 || k >= n) return -1;
    mode_pass(KIND_C, b, W, ipow(b, n), k, x, y, threads);
    return 0;
}

/* W^H (conjugate transpose) of a complex b x b matrix. */
static void adjoint_of(int b, const cplx *W, cplx *WH) {
    for (int i = 0; i < b; ++i)
        for (int j = 0; j < b; ++j) WH[i * b + j] = conj(W[j * b + i]);
}

/* O5: x = (W^H)^{(x)n} y  -- G_N^dagger applied to each vector. */
int oracle_adjoint_c(int b, int n, const double *Wd, long long batch, const double *y, double *x,
                     int threads) {
    cplx WH[256];
    if (b > 16) return -1;
    adjoint_of(b, (const cplx *)Wd, WH);
    return modes_generic(KIND_C, b, n, WH, batch, y, x, threads);
}

int oracle_adjoint_r(int b, int n, const double *W, long long batch, const double *y, double *x,
                     int threads) {
    double WT[256];
    if (b > 16) return -1;
    for (int i = 0; i < b; ++i)
        for (int j = 0; j < b; ++j) WT[i * b + j] = W[j * b + i];
    return modes_generic(KIND_R, b, n, WT, batch, y, x, threads);
}

/* -------------------------------------------------------- O6: gradient */

/*
 * For each vector: a_0 = x, a_{k+1} = P_k a_k (mode-k pass with W), y = a_n.
 * Given g_n = dL/dy:  for k = n-1 .. 0:
 *     dW[i][j] += sum over mode-k fibres of g_{k+1}[.., i, ..] * conj(a_k[.., j, ..])
 *     g_k       = mode-k pass of g_{k+1} with W^H
 * and dx = g_0.  dW is accumulated over all vectors of the batch; dx may be
 * NULL.  The real version is the same with conj() the identity.
 */
static int grad_generic(int kind, int b, int n, const void *W, long long batch, const void *x,
                        const void *dy, void *dx, void *dW, int threads) {
    long long N = ipow(b, n);
    size_t es = elem_size(kind);
    char *acts = malloc(es * N * (size_t)(n + 1));
    char *g = malloc(es * N), *g2 = malloc(es * N);
    if (!acts || !g || !g2) {
        free(acts), free(g), free(g2);
        return -2;
    }
    cplx WHc[256];
    double WTr[256];
    const void *Wadj;
    if (kind == KIND_C) {
        adjoint_of(b, (const cplx *)W, WHc);
        Wadj = WHc;
        memset(dW, 0, sizeof(cplx) * b * b);
    } else {
        const double *Wr = W;
        for (int i = 0; i < b; ++i)
            for (int j = 0; j < b; ++j) WTr[i * b + j] = Wr[j * b + i];
        Wadj = WTr;
        memset(dW, 0, sizeof(double) * b * b);
    }
    for (long long v = 0; v < batch; ++v) {
        memcpy(acts, (const char *)x + es * N * v, es * N);
        for (int k = 0; k < n; ++k)
            mode_pass(kind, b, W, N, k, acts + es * N * k, acts + es * N * (k + 1), threads);
        memcpy(g, (const char *)dy + es * N * v, es * N);
        for (int k = n - 1; k >= 0; --k) {
            long long L = ipow(b, k), bL = (long long)b * L;
            const char *ak = acts + es * N * k;
            for (long long h = 0; h < N / bL; ++h)
                for (long long l = 0; l < L; ++l) {
                    long long base = h * bL + l;
                    for (int i = 0; i < b; ++i)
                        for (int j = 0; j < b; ++j) {
                            if (kind == KIND_C) {
                                const cplx *gg = (const cplx *)g, *aa = (const cplx *)ak;
                                ((cplx *)dW)[i * b + j] += gg[base + i * L] * conj(aa[base + j * L]);
                            } else {
                                const double *gg = (const double *)g, *aa = (const double *)ak;
                                ((double *)dW)[i * b + j] += gg[base + i * L] * aa[base + j * L];
                            }
                        }
                }
            mode_pass(kind, b, Wadj, N, k, g, g2, threads);
            char *t = g;
            g = g2;
            g2 = t;
        }
        if (dx) memcpy((char *)dx + es * N * v, g, es * N);
    }
    free(acts), free(g), free(g2);
    return 0;
}

int oracle_grad_c(int b, int n, const double *W, long long batch, const double *x, const double *dy,
                  double *dx, double *dW, int threads) {
    if (b > 16) return -1;
    return grad_generic(KIND_C, b, n, W, batch, x, dy, dx, dW, threads);
}

int oracle_grad_r(int b, int n, const double *W, long long batch, const double *x, const double *dy,
                  double *dx, double *dW, int threads) {
    if (b > 16) return -1;
    return grad_generic(KIND_R, b, n, W, batch, x, dy, dx, dW, threads);
}
