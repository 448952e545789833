/*
 * FP64 CPU oracle for multi-level foreground estimation
 * (Germer, Uelwer, Conrad, Harmeling, "Fast Multi-Level Foreground Estimation").
 *
 * TEST INFRASTRUCTURE. This file is the plain, slow, obviously-correct statement of what
 * the GPU library computes. Only the tests, the smoke check and the benchmark's CPU
 * baseline may build, load or call it; the product path never does. It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Layout of every image: row-major, y outer, x inner, channels interleaved; an RGB image
 * of width w and height h is double[h][w][3], an alpha matte double[h][w].
 *
 * Readings of the paper taken here (each one is also listed in the design notes):
 *  - n_l = max(1, ceil(log2(max(w_hat, h_hat)))) (Algorithm 1; the max(1, .) keeps a
 *    1x1 input from producing zero levels).
 *  - round(x) = floor(x + 0.5) on the double result of pow(w_hat, l / n_l).
 *  - resize() is nearest neighbour with centre-aligned integer source index
 *    src = floor((2*dst + 1) * S / (2 * D)); I and alpha are always resized from the
 *    full-resolution input, F and B from the previous level (Algorithm 1).
 *  - "low resolution" (Section III-D) means w_l <= 32 and h_l <= 32.
 *  - N_i is the 4-neighbourhood; a neighbour outside the image is clamped onto the
 *    image (Algorithm 1), so at a border the pixel itself acts as that neighbour.
 *  - "while not converged" is the fixed per-level iteration count of Section III-D.
 *  - The default update order is Jacobi (every pixel of sweep t+1 reads sweep t);
 *    the paper's in-place raster order and a red-black order are also provided.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORACLE_JACOBI = 0, ORACLE_REDBLACK = 1, ORACLE_RASTER_GS = 2 };

typedef struct {
    double eps_r;      /* regularisation epsilon_r (paper: 5e-3) */
    double omega;      /* alpha-gradient weight omega (paper: 0.1) */
    int small_size;    /* "low resolution" threshold (paper: 32) */
    int small_iters;   /* iterations at low resolution (paper: 10) */
    int big_iters;     /* iterations otherwise (paper: 2) */
    int order;         /* ORACLE_JACOBI, ORACLE_REDBLACK or ORACLE_RASTER_GS */
    int clamp;         /* 1: clamp F, B to [0, 1] after each solve (Algorithm 1) */
    double init;       /* value of the 1x1 starting F and B (Algorithm 1 uses 0) */
} oracle_params;

/* ---------------------------------------------------------------- threads */

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------- level schedule */

/* ceil(log2(m)) for m >= 1, written as "smallest n with 2^n >= m". Algorithm 1. */
static int ceil_log2(long m)
{
    int n = 0;
    while ((1L << n) < m) n++;
    return n;
}

/* Number of levels n_l (Algorithm 1), with the max(1, .) reading for 1x1 input. */
int oracle_num_levels(int w_hat, int h_hat)
{
    long m = w_hat > h_hat ? w_hat : h_hat;
    int n = ceil_log2(m);
    return n < 1 ? 1 : n;
}

/* round(side^(l/n)) of Algorithm 1, with round(x) = floor(x + 0.5). */
int oracle_level_side(int side, int l, int n)
{
    double v = pow((double)side, (double)l / (double)n);
    return (int)floor(v + 0.5);
}

/* Iterations at a level of size w x h (Section III-D): small_iters if the level is at
 * most small_size x small_size, big_iters otherwise. */
int oracle_level_iters(int w, int h, const oracle_params *p)
{
    return (w <= p->small_size && h <= p->small_size) ? p->small_iters : p->big_iters;
}

/* Fills ws/hs/ks for levels 1..n (stored at index l-1); returns n, or -1 if cap < n. */
int oracle_schedule(int w_hat, int h_hat, const oracle_params *p,
                    int *ws, int *hs, int *ks, int cap)
{
    int n = oracle_num_levels(w_hat, h_hat);
    if (n > cap) return -1;
    for (int l = 1; l <= n; l++) {
        ws[l - 1] = oracle_level_side(w_hat, l, n);
        hs[l - 1] = oracle_level_side(h_hat, l, n);
        ks[l - 1] = oracle_level_iters(ws[l - 1], hs[l - 1], p);
    }
    return n;
}

/* ------------------------------------------------------------------ resize */

/* Nearest-neighbour resize of a [sh][sw][ch] image to [dh][dw][ch]:
 * dst(x, y) = src(floor((2x+1) sw / (2 dw)), floor((2y+1) sh / (2 dh))). */
void oracle_resize_nearest(const double *src, int sw, int sh, int ch,
                           double *dst, int dw, int dh)
{
    for (int y = 0; y < dh; y++) {
        long sy = ((2L * y + 1) * sh) / (2L * dh);
        for (int x = 0; x < dw; x++) {
            long sx = ((2L * x + 1) * sw) / (2L * dw);
            for (int c = 0; c < ch; c++)
                dst[((long)y * dw + x) * ch + c] = src[(sy * sw + sx) * ch + c];
        }
    }
}

/* ------------------------------------------------------- per-pixel update */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/*
 * One update of pixel (x, y), Algorithm 1 inner loop; the 2x2 solve is the closed form
 * g = (U U^T + R^T V R)^{-1} (I U + R^T V h) of Section III-C.
 * Reads alpha, I and the neighbours' F, B from (Fin, Bin); writes pixel i of (Fout, Bout).
 * Fin may equal Fout (in-place orders); the pixel's own old value is read before writing.
 */
static void update_pixel(const double *I, const double *a,
                         const double *Fin, const double *Bin,
                         double *Fout, double *Bout,
                         int w, int h, int x, int y, const oracle_params *p)
{
    static const int dx[4] = {-1, 1, 0, 0};
    static const int dy[4] = {0, 0, -1, 1};
    long i = (long)y * w + x;
    double ai = a[i];
    double u0 = ai, u1 = 1.0 - ai;             /* U = [alpha_i, 1 - alpha_i]^T */
    double A00 = u0 * u0, A01 = u0 * u1, A11 = u1 * u1;   /* A = U U^T */
    double b0[3], b1[3];                       /* b = U I_i^T (2 x 3) */
    for (int c = 0; c < 3; c++) {
        b0[c] = u0 * I[3 * i + c];
        b1[c] = u1 * I[3 * i + c];
    }
    for (int n = 0; n < 4; n++) {
        int xj = clampi(x + dx[n], 0, w - 1);
        int yj = clampi(y + dy[n], 0, h - 1);
        long j = (long)yj * w + xj;
        double d = p->eps_r + p->omega * fabs(ai - a[j]);
        A00 += d;
        A11 += d;
        for (int c = 0; c < 3; c++) {
            b0[c] += d * Fin[3 * j + c];
            b1[c] += d * Bin[3 * j + c];
        }
    }
    /* g = A^{-1} b with A^{-1} = adj(A) / det(A); A is symmetric. */
    double det = A00 * A11 - A01 * A01;
    for (int c = 0; c < 3; c++) {
        double gF = (A11 * b0[c] - A01 * b1[c]) / det;
        double gB = (A00 * b1[c] - A01 * b0[c]) / det;
        if (p->clamp) {
            gF = fmax(0.0, fmin(1.0, gF));
            gB = fmax(0.0, fmin(1.0, gB));
        }
        Fout[3 * i + c] = gF;
        Bout[3 * i + c] = gB;
    }
}

/* -------------------------------------------------------------- sweeps */

/* `iters` sweeps at one level, in place on F and B ([h][w][3] each). */
int oracle_level_iterate(const double *I, const double *a, int w, int h,
                         double *F, double *B, int iters, const oracle_params *p)
{
    long n3 = (long)w * h * 3;
    if (p->order == ORACLE_JACOBI) {
        double *F2 = (double *)malloc(sizeof(double) * n3);
        double *B2 = (double *)malloc(sizeof(double) * n3);
        if (!F2 || !B2) { free(F2); free(B2); return -1; }
        for (int t = 0; t < iters; t++) {
            /* every pixel reads sweep t and writes sweep t+1 */
            #pragma omp parallel for schedule(static)
            for (int y = 0; y < h; y++)
                for (int x = 0; x < w; x++)
                    update_pixel(I, a, F, B, F2, B2, w, h, x, y, p);
            memcpy(F, F2, sizeof(double) * n3);
            memcpy(B, B2, sizeof(double) * n3);
        }
        free(F2);
        free(B2);
    } else if (p->order == ORACLE_REDBLACK) {
        for (int t = 0; t < iters; t++) {
            for (int colour = 0; colour < 2; colour++) {
                /* pixels of one colour only read pixels of the other colour (or
                 * themselves at a clamped border), so in-place update is exact */
                #pragma omp parallel for schedule(static)
                for (int y = 0; y < h; y++)
                    for (int x = (y + colour) & 1; x < w; x += 2)
                        update_pixel(I, a, F, B, F, B, w, h, x, y, p);
            }
        }
    } else if (p->order == ORACLE_RASTER_GS) {
        /* the loop exactly as Algorithm 1 writes it: in place, row by row */
        for (int t = 0; t < iters; t++)
            for (int y = 0; y < h; y++)
                for (int x = 0; x < w; x++)
                    update_pixel(I, a, F, B, F, B, w, h, x, y, p);
    } else {
        return -2;
    }
    return 0;
}

/* ------------------------------------------------------------ Algorithm 1 */

/*
 * ML(I_hat, alpha_hat): the multi-level method of Algorithm 1.
 * I_hat: [H][W][3], a_hat: [H][W]; F_out, B_out: [H][W][3].
 * Returns 0 on success, negative on bad arguments or allocation failure.
 */
int oracle_ml(const double *I_hat, const double *a_hat, int W, int H,
              const oracle_params *p, double *F_out, double *B_out)
{
    if (W < 1 || H < 1) return -1;
    int n = oracle_num_levels(W, H);
    long N = (long)W * H;
    double *I = (double *)malloc(sizeof(double) * N * 3);
    double *a = (double *)malloc(sizeof(double) * N);
    double *F = (double *)malloc(sizeof(double) * N * 3);
    double *B = (double *)malloc(sizeof(double) * N * 3);
    double *Fp = (double *)malloc(sizeof(double) * N * 3);
    double *Bp = (double *)malloc(sizeof(double) * N * 3);
    int rc = 0;
    if (!I || !a || !F || !B || !Fp || !Bp) { rc = -3; goto done; }

    /* F <- 0_{1,1}, B <- 0_{1,1} (the starting value is a parameter, default 0) */
    int fw = 1, fh = 1;
    for (int c = 0; c < 3; c++) { F[c] = p->init; B[c] = p->init; }

    for (int l = 1; l <= n; l++) {
        int w = oracle_level_side(W, l, n);
        int h = oracle_level_side(H, l, n);
        /* I, alpha from the full-resolution input; F, B from the previous level */
        oracle_resize_nearest(I_hat, W, H, 3, I, w, h);
        oracle_resize_nearest(a_hat, W, H, 1, a, w, h);
        memcpy(Fp, F, sizeof(double) * (long)fw * fh * 3);
        memcpy(Bp, B, sizeof(double) * (long)fw * fh * 3);
        oracle_resize_nearest(Fp, fw, fh, 3, F, w, h);
        oracle_resize_nearest(Bp, fw, fh, 3, B, w, h);
        int k = oracle_level_iters(w, h, p);
        if (oracle_level_iterate(I, a, w, h, F, B, k, p) != 0) { rc = -3; goto done; }
        fw = w;
        fh = h;
    }
    /* the last level has the input's size: round(W^1) = W */
    memcpy(F_out, F, sizeof(double) * N * 3);
    memcpy(B_out, B, sizeof(double) * N * 3);
done:
    free(I); free(a); free(F); free(B); free(Fp); free(Bp);
    return rc;
}
