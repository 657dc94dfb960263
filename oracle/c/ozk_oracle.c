/*
 * Plain C oracle for the Ozaki-I emulated ZGEMM and the KKR tau_00 solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline legs of
 * the benchmark load this library.  It shares no code with the CUDA path; it restates
 * the same definitions as oracle/ozaki.py and oracle/kkr.py (which pin it) in plain,
 * unblocked C so that larger cases run in seconds.
 *
 * Conventions: matrices are complex binary64 stored as interleaved (re, im) doubles in
 * row-major order, in the mathematical orientation C = A B (A is m x k, B is k x n).
 *
 * Method (paper Sec. 2.2: slices by significant bits with exponent alignment, pairwise
 * low-precision products, higher-precision accumulation; Sec. 3.2/4: precision knob in
 * mantissa bits, read as B = 8S - 1):
 *   e_i  = frexp exponent of max_l max(|Re a_il|, |Im a_il|)     (0 for a zero row)
 *   X    = trunc(x 2^(B - e))
 *   X    = sum_t d_t 256^(S-t), balanced digits from the least significant one
 *   G_g  = sum_{s+t=g} A_s B_t^T  (4M stacked complex form, exact integers)
 *   Z    = RN( 2^(e_i + f_j - 2B) sum_g G_g 256^(2S-g) )      (one rounding)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

#define OZ_OK 0
#define OZ_ERR_ARG 1
#define OZ_ERR_NONFINITE 2
#define OZ_ERR_SINGULAR 3
#define OZ_ERR_RANGE 4

static int bits_for(int S) { return 8 * S - 1; }

/* ---------------------------------------------------------------- exponent scan */

/* e[r] for each row r of a complex R x K matrix with row stride ldx (in complex units). */
int oz_row_exponents(const double* X, int R, int K, long ldx, int* e) {
    for (int r = 0; r < R; r++) {
        double mu = 0.0;
        for (int l = 0; l < K; l++) {
            double a = X[2 * (r * ldx + l)], b = X[2 * (r * ldx + l) + 1];
            if (!isfinite(a) || !isfinite(b)) return OZ_ERR_NONFINITE;
            a = fabs(a); b = fabs(b);
            if (a > mu) mu = a;
            if (b > mu) mu = b;
        }
        int ex = 0;
        if (mu != 0.0) frexp(mu, &ex);
        e[r] = ex;
    }
    return OZ_OK;
}

/* ---------------------------------------------------------------- integer image, digits */

/* X = trunc(x 2^(B - e)) computed exactly from the binary64 fields of x. */
static i128 integer_image(double x, int e, int B) {
    if (x == 0.0) return 0;
    int ex;
    double m = frexp(fabs(x), &ex);            /* |x| = m 2^ex, m in [0.5, 1) */
    int64_t M53 = (int64_t)ldexp(m, 53);        /* exact 53-bit integer */
    int shift = ex - 53 + B - e;
    u128 mag;
    if (shift >= 0) mag = ((u128)M53) << shift;
    else if (shift > -64) mag = (u128)(M53 >> (-shift));
    else mag = 0;
    i128 X = (i128)mag;
    return x < 0 ? -X : X;
}

/* balanced base-256 digits of X, most significant first (d[0] = d_1). */
static void balanced_digits(i128 X, int S, int16_t* d, long stride) {
    i128 r = X;
    for (int t = S - 1; t >= 1; t--) {
        int dd = (int)((r + 128) & 255) - 128;
        d[(long)t * stride] = (int16_t)dd;
        r = (r - dd) >> 8;
    }
    d[0] = (int16_t)r;
}

/* Left operand A (m x k): e (m), D (S x m x 2k) = [Re digits | Im digits]. */
int oz_split_left(const double* A, int m, int k, int S, int* e, int16_t* D) {
    int st = oz_row_exponents(A, m, k, k, e);
    if (st) return st;
    const int B = bits_for(S);
    const long plane = (long)m * 2 * k;
    for (int i = 0; i < m; i++)
        for (int l = 0; l < k; l++) {
            i128 Xr = integer_image(A[2 * ((long)i * k + l)], e[i], B);
            i128 Xi = integer_image(A[2 * ((long)i * k + l) + 1], e[i], B);
            balanced_digits(Xr, S, D + (long)i * 2 * k + l, plane);
            balanced_digits(Xi, S, D + (long)i * 2 * k + k + l, plane);
        }
    return OZ_OK;
}

/* Right operand B (k x n): f (n), D (S x 2n x 2k); row 2j = [Re | -Im], 2j+1 = [Im | Re]. */
int oz_split_right(const double* Bm, int k, int n, int S, int* f, int16_t* D) {
    double* Bt = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1) * (size_t)(k > 0 ? k : 1));
    for (int j = 0; j < n; j++)
        for (int l = 0; l < k; l++) {
            Bt[2 * ((long)j * k + l)] = Bm[2 * ((long)l * n + j)];
            Bt[2 * ((long)j * k + l) + 1] = Bm[2 * ((long)l * n + j) + 1];
        }
    int st = oz_row_exponents(Bt, n, k, k, f);
    if (st) { free(Bt); return st; }
    const int B = bits_for(S);
    const long plane = (long)2 * n * 2 * k;
    int16_t* tmp = (int16_t*)malloc(sizeof(int16_t) * (size_t)S);
    for (int j = 0; j < n; j++)
        for (int l = 0; l < k; l++) {
            i128 Xr = integer_image(Bt[2 * ((long)j * k + l)], f[j], B);
            i128 Xi = integer_image(Bt[2 * ((long)j * k + l) + 1], f[j], B);
            int16_t* r0 = D + (long)(2 * j) * 2 * k;
            int16_t* r1 = D + (long)(2 * j + 1) * 2 * k;
            balanced_digits(Xr, S, r0 + l, plane);
            balanced_digits(Xr, S, r1 + k + l, plane);
            balanced_digits(Xi, S, r1 + l, plane);
            balanced_digits(Xi, S, tmp, 1);
            for (int s = 0; s < S; s++) r0[(long)s * plane + k + l] = (int16_t)(-tmp[s]);
        }
    free(tmp);
    free(Bt);
    return OZ_OK;
}

/* ---------------------------------------------------------------- pairs and groups */

static int pair_in_set(int s, int t, int S, int full) { return full ? 1 : (s + t <= S + 1); }

/* G[(g - 2)][i][j] = sum over pairs (s, t) (1-based) with s + t = g of DA_s[i] . DB_t[j].
 * Groups g = 2 .. gmax, gmax = S + 1 (triangular) or 2S (full). */
void oz_group_sums(const int16_t* DA, const int16_t* DB, int S, int rowsA, int rowsB, int Kp,
                   int full, int64_t* G) {
    const int gmax = full ? 2 * S : S + 1;
    const long pa = (long)rowsA * Kp, pb = (long)rowsB * Kp;
    memset(G, 0, sizeof(int64_t) * (size_t)(gmax - 1) * rowsA * rowsB);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < rowsA; i++)
        for (int s = 1; s <= S; s++)
            for (int t = 1; t <= S; t++) {
                if (!pair_in_set(s, t, S, full)) continue;
                const int16_t* a = DA + (s - 1) * pa + (long)i * Kp;
                int64_t* Gr = G + ((long)(s + t - 2) * rowsA + i) * rowsB;
                for (int j = 0; j < rowsB; j++) {
                    const int16_t* bb = DB + (t - 1) * pb + (long)j * Kp;
                    int64_t acc = 0;
                    for (int l = 0; l < Kp; l++) acc += (int32_t)a[l] * (int32_t)bb[l];
                    Gr[j] += acc;
                }
            }
}

/* ---------------------------------------------------------------- rounding */

static int clz128(u128 x) {
    uint64_t hi = (uint64_t)(x >> 64), lo = (uint64_t)x;
    if (hi) return __builtin_clzll(hi);
    if (lo) return 64 + __builtin_clzll(lo);
    return 128;
}

/* RN-even of T 2^E as binary64 (single rounding, subnormals and overflow included). */
double oz_round_scaled(i128 T, int E) {
    if (T == 0) return 0.0;
    int neg = T < 0;
    u128 mag = neg ? (u128)(-T) : (u128)T;
    int nbits = 128 - clz128(mag);
    /* exponent of the unit in the last place of the result */
    long q = (long)nbits - 53 + E;
    if (q < -1074) q = -1074;
    long shift = q - E;
    double r;
    if (shift <= 0) {
        r = ldexp((double)(uint64_t)mag, E);          /* mag < 2^53: exact */
    } else {
        u128 keep = shift >= 128 ? 0 : (mag >> shift);
        u128 rem = shift >= 128 ? mag : (mag & ((((u128)1) << shift) - 1));
        u128 half = shift > 128 ? (u128)0 : (((u128)1) << (shift - 1));
        int up = 0;
        if (shift <= 128) {
            if (rem > half) up = 1;
            else if (rem == half && (keep & 1)) up = 1;
        }
        keep += up;
        r = ldexp((double)(uint64_t)keep, (int)q);   /* keep <= 2^53: exact; may overflow to inf */
    }
    return neg ? -r : r;
}

/* test hook: T given as (hi, lo) 64-bit halves of a two's-complement 128-bit integer */
double oz_round_scaled_hl(int64_t hi, uint64_t lo, int E) {
    i128 T = (i128)(((u128)(uint64_t)hi << 64) | (u128)lo);
    return oz_round_scaled(T, E);
}

/* ---------------------------------------------------------------- emulated ZGEMM */

/* C (m x n) = emulated A B (mode 0: store) or C - emulated A B (mode 1: LU update). */
int oz_zgemm(const double* A, const double* Bm, int m, int n, int k, int S, int full, int lu,
             double* C) {
    if (m < 0 || n < 0 || k < 0 || S < 1 || S > 16) return OZ_ERR_ARG;
    if (m == 0 || n == 0) return OZ_OK;
    if (k == 0) {
        if (!lu) memset(C, 0, sizeof(double) * 2 * (size_t)m * n);
        return OZ_OK;
    }
    const int gmax = full ? 2 * S : S + 1;
    const int Kp = 2 * k;
    /* the exact sum must fit a signed 128-bit integer */
    int need = 8 * (gmax - 2) + 14 + 1 + (int)ceil(log2((double)Kp * S + 1.0)) + 1;
    if (need > 126) return OZ_ERR_RANGE;
    int* e = (int*)malloc(sizeof(int) * (size_t)m);
    int* f = (int*)malloc(sizeof(int) * (size_t)n);
    int16_t* DA = (int16_t*)malloc(sizeof(int16_t) * (size_t)S * m * Kp);
    int16_t* DB = (int16_t*)malloc(sizeof(int16_t) * (size_t)S * 2 * n * Kp);
    int64_t* G = (int64_t*)malloc(sizeof(int64_t) * (size_t)(gmax - 1) * m * 2 * n);
    int st = oz_split_left(A, m, k, S, e, DA);
    if (!st) st = oz_split_right(Bm, k, n, S, f, DB);
    if (!st) {
        oz_group_sums(DA, DB, S, m, 2 * n, Kp, full, G);
        const int B = bits_for(S);
        const int base = -2 * B + 8 * (2 * S - gmax);
        const long plane = (long)m * 2 * n;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < m; i++)
            for (int j2 = 0; j2 < 2 * n; j2++) {
                i128 T = 0;
                for (int g = 2; g <= gmax; g++) {
                    i128 w = ((i128)1) << (8 * (gmax - g));
                    T += (i128)G[(long)(g - 2) * plane + (long)i * 2 * n + j2] * w;
                }
                double z = oz_round_scaled(T, e[i] + f[j2 / 2] + base);
                long o = 2 * ((long)i * n + j2 / 2) + (j2 & 1);
                C[o] = lu ? (C[o] - z) : z;
            }
    }
    free(e); free(f); free(DA); free(DB); free(G);
    return st;
}

/* Plain binary64 complex triple loop, k ascending: C = A B. */
void oz_zgemm_fp64(const double* A, const double* Bm, int m, int n, int k, double* C) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            double cr = 0.0, ci = 0.0;
            for (int l = 0; l < k; l++) {
                double ar = A[2 * ((long)i * k + l)], ai = A[2 * ((long)i * k + l) + 1];
                double br = Bm[2 * ((long)l * n + j)], bi = Bm[2 * ((long)l * n + j) + 1];
                cr += ar * br - ai * bi;
                ci += ar * bi + ai * br;
            }
            C[2 * ((long)i * n + j)] = cr;
            C[2 * ((long)i * n + j) + 1] = ci;
        }
}

/* ---------------------------------------------------------------- KKR tau_00 */

/* Gauss-Jordan inverse with partial pivoting (largest |.|^2), in place, n x n complex. */
int oz_gepp_inverse(double* M, int n) {
    const int w = 2 * n;
    double* A = (double*)calloc((size_t)2 * n * w, sizeof(double));
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            A[2 * ((long)i * w + j)] = M[2 * ((long)i * n + j)];
            A[2 * ((long)i * w + j) + 1] = M[2 * ((long)i * n + j) + 1];
        }
        A[2 * ((long)i * w + n + i)] = 1.0;
    }
    int st = OZ_OK;
    for (int p = 0; p < n && !st; p++) {
        int piv = p;
        double best = -1.0;
        for (int i = p; i < n; i++) {
            double re = A[2 * ((long)i * w + p)], im = A[2 * ((long)i * w + p) + 1];
            double a = re * re + im * im;
            if (a > best) { best = a; piv = i; }
        }
        if (best == 0.0) { st = OZ_ERR_SINGULAR; break; }
        if (piv != p)
            for (int j = 0; j < w; j++) {
                double tr = A[2 * ((long)p * w + j)], ti = A[2 * ((long)p * w + j) + 1];
                A[2 * ((long)p * w + j)] = A[2 * ((long)piv * w + j)];
                A[2 * ((long)p * w + j) + 1] = A[2 * ((long)piv * w + j) + 1];
                A[2 * ((long)piv * w + j)] = tr;
                A[2 * ((long)piv * w + j) + 1] = ti;
            }
        /* row p /= pivot */
        double pr = A[2 * ((long)p * w + p)], pi = A[2 * ((long)p * w + p) + 1];
        double den = pr * pr + pi * pi;
        double ir = pr / den, ii = -pi / den;
        for (int j = 0; j < w; j++) {
            double xr = A[2 * ((long)p * w + j)], xi = A[2 * ((long)p * w + j) + 1];
            A[2 * ((long)p * w + j)] = xr * ir - xi * ii;
            A[2 * ((long)p * w + j) + 1] = xr * ii + xi * ir;
        }
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) {
            if (i == p) continue;
            double fr = A[2 * ((long)i * w + p)], fi = A[2 * ((long)i * w + p) + 1];
            if (fr == 0.0 && fi == 0.0) continue;
            for (int j = 0; j < w; j++) {
                double xr = A[2 * ((long)p * w + j)], xi = A[2 * ((long)p * w + j) + 1];
                A[2 * ((long)i * w + j)] -= fr * xr - fi * xi;
                A[2 * ((long)i * w + j) + 1] -= fr * xi + fi * xr;
            }
        }
    }
    if (!st)
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                M[2 * ((long)i * n + j)] = A[2 * ((long)i * w + n + j)];
                M[2 * ((long)i * n + j) + 1] = A[2 * ((long)i * w + n + j) + 1];
            }
    free(A);
    return st;
}

static void copy_block(const double* src, int lds, int r0, int c0, int rows, int cols, double* dst) {
    for (int i = 0; i < rows; i++)
        memcpy(dst + 2 * (long)i * cols, src + 2 * ((long)(r0 + i) * lds + c0), sizeof(double) * 2 * (size_t)cols);
}

static void put_block(double* dst, int ldd, int r0, int c0, int rows, int cols, const double* src) {
    for (int i = 0; i < rows; i++)
        memcpy(dst + 2 * ((long)(r0 + i) * ldd + c0), src + 2 * (long)i * cols, sizeof(double) * 2 * (size_t)cols);
}

/* tau_00 = S00^-1 t0 by block LU: panels J = [p, q) are eliminated from the trailing end
 * of M towards the front, so the remainder is always the leading block R = [0, p) and the
 * centre block (site 0, rows/cols 0..b-1) is eliminated last.  leaf = 0: the whole panel is
 * one pivot block (L_RJ = M_RJ D^-1, M_RR -= L_RJ M_JR).  leaf = w > 0: the panel is factored
 * leaf by leaf from its last w-wide leaf [a, a+w) (the front leaf narrower when w does not
 * divide the panel width): L column M[0:a, a:a+w] D_a^-1, then the rank-w update of
 * [0, a) x [0, a) outside [0, p) x [0, p); after the panel, [0, p) x [0, p) gets the whole
 * panel's update M[0:p, p:q] M[p:q, 0:p] at once.
 * S = 0: binary64 GEMMs; S > 0: every GEMM is the emulated ZGEMM. */
static int gemm_into(const double* X, const double* Y, int m, int n, int k, int S, int full, int lu, double* C) {
    if (S > 0) return oz_zgemm(X, Y, m, n, k, S, full, lu, C);
    if (!lu) { oz_zgemm_fp64(X, Y, m, n, k, C); return OZ_OK; }
    double* P = (double*)malloc(sizeof(double) * 2 * (size_t)m * n);
    oz_zgemm_fp64(X, Y, m, n, k, P);
    for (long x = 0; x < 2L * m * n; x++) C[x] -= P[x];
    free(P);
    return OZ_OK;
}

int oz_tau00_block(const double* M, const double* t0, int n, int b, int nb, int leaf, int S, int full,
                   double* tau) {
    if (n <= 0 || b <= 0 || n % b || nb <= 0 || leaf < 0) return OZ_ERR_ARG;
    double* A = (double*)malloc(sizeof(double) * 2 * (size_t)n * n);
    memcpy(A, M, sizeof(double) * 2 * (size_t)n * n);
    int st = OZ_OK;
    for (int q = n; q > b && !st;) {
        int p = q - nb > b ? q - nb : b;
        int wl = leaf > 0 ? leaf : q - p;
        /* leaves [a, hi) from the end of the panel; the front one narrower when the panel width
           is not a multiple of the leaf width */
        for (int hi = q; hi > p && !st; hi -= wl) {
            const int a = hi - wl > p ? hi - wl : p, w = hi - a;
            double* D = (double*)malloc(sizeof(double) * 2 * (size_t)w * w);
            double* Lc = (double*)malloc(sizeof(double) * 2 * (size_t)(a > 0 ? a : 1) * w);
            double* T = (double*)malloc(sizeof(double) * 2 * (size_t)(a > 0 ? a : 1) * w);
            copy_block(A, n, a, a, w, w, D);
            st = oz_gepp_inverse(D, w);
            if (!st && a > 0) {
                copy_block(A, n, 0, a, a, w, Lc);
                st = gemm_into(Lc, D, a, w, w, S, full, 0, T);
                put_block(A, n, 0, a, a, w, T);
            }
            if (!st && a > p) {
                double* Ur = (double*)malloc(sizeof(double) * 2 * (size_t)w * a);
                double* Cr = (double*)malloc(sizeof(double) * 2 * (size_t)a * a);
                double* box = (double*)malloc(sizeof(double) * 2 * (size_t)p * p);
                copy_block(A, n, a, 0, w, a, Ur);
                copy_block(A, n, 0, 0, a, a, Cr);
                copy_block(A, n, 0, 0, p, p, box);
                st = gemm_into(T, Ur, a, a, w, S, full, 1, Cr);
                put_block(A, n, 0, 0, a, a, Cr);
                put_block(A, n, 0, 0, p, p, box);
                free(Ur); free(Cr); free(box);
            }
            free(D); free(Lc); free(T);
        }
        if (!st) {
            int wp = q - p;
            double* Lp = (double*)malloc(sizeof(double) * 2 * (size_t)p * wp);
            double* Up = (double*)malloc(sizeof(double) * 2 * (size_t)wp * p);
            double* Cr = (double*)malloc(sizeof(double) * 2 * (size_t)p * p);
            copy_block(A, n, 0, p, p, wp, Lp);
            copy_block(A, n, p, 0, wp, p, Up);
            copy_block(A, n, 0, 0, p, p, Cr);
            st = gemm_into(Lp, Up, p, p, wp, S, full, 1, Cr);
            put_block(A, n, 0, 0, p, p, Cr);
            free(Lp); free(Up); free(Cr);
        }
        q = p;
    }
    if (!st) {
        double* S00 = (double*)malloc(sizeof(double) * 2 * (size_t)b * b);
        copy_block(A, n, 0, 0, b, b, S00);
        st = oz_gepp_inverse(S00, b);
        if (!st) oz_zgemm_fp64(S00, t0, b, b, b, tau);
        free(S00);
    }
    free(A);
    return st;
}

/* tau_00 from the full Gauss-Jordan inverse of M. */
int oz_tau00_full(const double* M, const double* t0, int n, int b, double* tau) {
    double* Mi = (double*)malloc(sizeof(double) * 2 * (size_t)n * n);
    memcpy(Mi, M, sizeof(double) * 2 * (size_t)n * n);
    int st = oz_gepp_inverse(Mi, n);
    if (!st) {
        double* Z = (double*)malloc(sizeof(double) * 2 * (size_t)b * b);
        copy_block(Mi, n, 0, 0, b, b, Z);
        oz_zgemm_fp64(Z, t0, b, b, b, tau);
        free(Z);
    }
    free(Mi);
    return st;
}

int oz_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
