/*
 * FC2T2 reference oracle -- plain, slow, FP64, CPU only.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * What it computes: the multi-level uniform-grid Taylor transform of
 * Lange & Kutz, "FC^2T^2: The Fast Continuous Convolutional Taylor Transform"
 * (arXiv 2111.00110), Section 3, approximating Eq. 1
 *        y_m = sum_n phi(p_n, q_m) w_n,     phi(p, q) = psi(p - q),
 * by the truncated separation of Eq. 2, followed through the paper's steps:
 *   P2M  (Sec. 3, definition of script-M after Eq. 2)
 *   M2M  (Sec. 3, binomial re-centring of M-terms; the final sum over k <= n)
 *   M2L  (Sec. 3, definition of script-L after Eq. 2, applied per level with the
 *         parity-dependent 6^D window minus the 3^D hole; near field at the
 *         finest level is also taken from the series, caption of the data-flow
 *         figure in Sec. 3)
 *   L2L  (Sec. 3, re-centring of L-terms, sum over k >= n)
 *   L2P  (Sec. 3, "L2P" line: sum over |k| <= rho of L(k, d_q) * script-L(k, q'))
 * and, for Sec. 4.1 (Jacobian Vector Product), the gradient of the local series
 * with respect to the evaluation point.
 *
 * Everything is unscaled FP64 in the paper's own notation: M(n) = sum w d^n/n!,
 * L(k) = sum_n (-1)^|k| d^(n+k) psi(c) M(n), y = sum_k L(k) d_q^k / k!.
 *
 * Readings of the paper where it is silent or garbled (each listed in the design
 * notes of the repository):
 *   - truncation is by total degree |n| + |k| <= rho (P = C(rho+D, D) terms per
 *     cell, e.g. 35 for rho = 4 in 3D, Sec. 3.2), not the per-dimension box of
 *     the re-indexed sum in Eq. 2;
 *   - the target displacement enters as (-d_q), hence the (-1)^|k| factor;
 *   - the coarsest level has 4 cells per dimension, so levels = log2(n) - 1 and
 *     the finest grid has 2^(levels+1) cells per dimension (Sec. 3.2);
 *   - interaction list at level l:  parent(s) near parent(t) and s not near t,
 *     plus, at the finest level only, every s near t (self included); "near"
 *     means Chebyshev distance <= 1 in cell indices; at the coarsest level every
 *     parent pair counts as near;
 *   - the domain is [lo, hi)^D; the cell of a coordinate is decided in FP32:
 *     t = (float)(x - lo) * (float)(n / (hi - lo)), cell = clamp(floor(t), 0, n-1),
 *     every operation rounded to FP32 (no contraction), so the oracle and the
 *     GPU always agree on the cell;
 *   - multi-indices are in graded order: degree first, then exponent of the
 *     first coordinate descending, then of the second descending.
 *
 * Kernels: Gaussian psi(x) = exp(-|x|^2 / (2 sigma^2)) (even, separable), with
 * derivatives from the physicists' Hermite recurrence; or a general polynomial
 * psi(x) = sum_a c_a x^a given by coefficients in graded order (used for the
 * polynomial-exactness checks; odd polynomials are allowed for forward checks).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 3
#define ORC_MAXRHO 12

typedef struct {
    int dim;                 /* 2 or 3 */
    int grid;                /* finest cells per dimension, power of two >= 4 */
    int order;               /* rho */
    int kernel;              /* 0 = Gaussian, 1 = polynomial */
    double sigma;            /* Gaussian width */
    const double *poly_coef; /* polynomial coefficients in graded order */
    int n_poly;              /* number of polynomial coefficients */
    double lo, hi;           /* domain [lo, hi)^dim */
    int fit;                 /* 0: Taylor coefficients in M2L; 1: least-squares fitted ones */
} orc_desc;

/* deliberate-mistake switches, used only by the pin-sensitivity tests */
enum {
    ORC_FAULT_NONE = 0,
    ORC_FAULT_DROP_SIGN = 1,      /* forget (-1)^|k| */
    ORC_FAULT_DROP_TOP_TERM = 2,  /* truncate at |n|+|k| <= rho-1 in M2L */
    ORC_FAULT_PARITY = 3,         /* swap the even/odd windows */
    ORC_FAULT_NO_L2L = 4,         /* drop coarse-level locals */
    ORC_FAULT_M2M_SIGN = 5,       /* re-centre moments with the wrong sign */
    ORC_FAULT_NO_SELF = 6,        /* near field without the cell itself */
    ORC_FAULT_TRANSPOSE = 7       /* use the target-to-source offset */
};

/* ------------------------------------------------------------------ indices */

static long binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

int orc_num_coeffs(int dim, int order) { return (int)binom(order + dim, dim); }

/* exponents of the graded multi-indices, row-major [P][dim] */
int orc_multi_indices(int dim, int order, int *out) {
    int i = 0;
    for (int d = 0; d <= order; ++d) {
        if (dim == 2) {
            for (int a0 = d; a0 >= 0; --a0) {
                out[2 * i] = a0; out[2 * i + 1] = d - a0; ++i;
            }
        } else {
            for (int a0 = d; a0 >= 0; --a0)
                for (int a1 = d - a0; a1 >= 0; --a1) {
                    out[3 * i] = a0; out[3 * i + 1] = a1; out[3 * i + 2] = d - a0 - a1; ++i;
                }
        }
    }
    return i;
}

typedef struct {
    int dim, order, P;
    int *ex;       /* [P][dim] exponents */
    int *deg;      /* [P] total degree */
    int *lookup;   /* exponent tuple -> graded index, (order+1)^dim entries, -1 if |a|>order */
    double fact[2 * ORC_MAXRHO + 2];
} orc_index;

static int lut_pos(const orc_index *ix, const int *a) {
    int r = ix->order + 1, pos = 0;
    for (int i = ix->dim - 1; i >= 0; --i) pos = pos * r + a[i];
    return pos;
}

static int idx_of(const orc_index *ix, const int *a) {
    int s = 0;
    for (int i = 0; i < ix->dim; ++i) { if (a[i] < 0) return -1; s += a[i]; }
    if (s > ix->order) return -1;
    return ix->lookup[lut_pos(ix, a)];
}

static void index_init(orc_index *ix, int dim, int order) {
    ix->dim = dim; ix->order = order; ix->P = orc_num_coeffs(dim, order);
    ix->ex = (int *)malloc(sizeof(int) * ix->P * dim);
    ix->deg = (int *)malloc(sizeof(int) * ix->P);
    orc_multi_indices(dim, order, ix->ex);
    int nl = 1;
    for (int i = 0; i < dim; ++i) nl *= (order + 1);
    ix->lookup = (int *)malloc(sizeof(int) * nl);
    for (int i = 0; i < nl; ++i) ix->lookup[i] = -1;
    for (int k = 0; k < ix->P; ++k) {
        int s = 0;
        for (int i = 0; i < dim; ++i) s += ix->ex[k * dim + i];
        ix->deg[k] = s;
        ix->lookup[lut_pos(ix, ix->ex + k * dim)] = k;
    }
    ix->fact[0] = 1.0;
    for (int i = 1; i < 2 * ORC_MAXRHO + 2; ++i) ix->fact[i] = ix->fact[i - 1] * i;
}

static void index_free(orc_index *ix) { free(ix->ex); free(ix->deg); free(ix->lookup); }

/* out[e] = x^e / e! for e = 0..rho (plain repeated products) */
static void powers_over_fact(double x, int rho, double *out) {
    out[0] = 1.0;
    for (int e = 1; e <= rho; ++e) out[e] = out[e - 1] * x / e;
}

/* prod_k x_k^(a_k) / a_k! from per-dimension power tables */
static double mono(const orc_index *ix, int a, double pw[][ORC_MAXRHO + 1]) {
    double m = 1.0;
    for (int k = 0; k < ix->dim; ++k) m *= pw[k][ix->ex[a * ix->dim + k]];
    return m;
}

/* Coefficients of the re-centring x^a/a! -> sum_{b <= a} d^(a-b)/(a-b)! x^b/b!:
 * for every a, the list of (b, prod_k d_k^(a_k-b_k)/(a_k-b_k)!) with b <= a componentwise. */
typedef struct { int *start, *b; double *coef; } orc_shift;

static void shift_init(orc_shift *s, const orc_index *ix, const double *dd) {
    int D = ix->dim, P = ix->P;
    double pw[ORC_MAXD][ORC_MAXRHO + 1];
    for (int k = 0; k < D; ++k) powers_over_fact(dd[k], ix->order, pw[k]);
    s->start = (int *)malloc(sizeof(int) * (P + 1));
    int cnt = 0;
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            int ok = 1;
            for (int k = 0; k < D; ++k) if (ix->ex[b * D + k] > ix->ex[a * D + k]) ok = 0;
            cnt += ok;
        }
    s->b = (int *)malloc(sizeof(int) * cnt);
    s->coef = (double *)malloc(sizeof(double) * cnt);
    cnt = 0;
    for (int a = 0; a < P; ++a) {
        s->start[a] = cnt;
        for (int b = 0; b < P; ++b) {
            double t = 1.0;
            int ok = 1;
            for (int k = 0; k < D; ++k) {
                int e = ix->ex[a * D + k] - ix->ex[b * D + k];
                if (e < 0) { ok = 0; break; }
                t *= pw[k][e];
            }
            if (ok) { s->b[cnt] = b; s->coef[cnt] = t; ++cnt; }
        }
    }
    s->start[P] = cnt;
}

static void shift_free(orc_shift *s) { free(s->start); free(s->b); free(s->coef); }

/* ------------------------------------------------------ kernel derivatives */

/* g^(j)(t) for g(t) = exp(-t^2/(2 sigma^2)), j = 0..J:
 * g^(j)(t) = (-1/(sigma sqrt2))^j H_j(t/(sigma sqrt2)) g(t),
 * H_0 = 1, H_1(u) = 2u, H_{j+1}(u) = 2u H_j(u) - 2j H_{j-1}(u). */
static void gauss_1d(double sigma, double t, int J, double *out) {
    double s = 1.0 / (sigma * sqrt(2.0));
    double u = t * s, g = exp(-u * u);
    double hm1 = 0.0, h = 1.0, scale = 1.0;
    for (int j = 0; j <= J; ++j) {
        out[j] = scale * h * g;
        double hn = 2.0 * u * h - 2.0 * j * hm1;
        hm1 = h; h = hn; scale *= -s;
    }
}

/* d^m psi(c) for every graded multi-index m with |m| <= order */
static void kernel_derivs_ix(const orc_desc *d, const orc_index *ix, const double *c, double *out) {
    int D = ix->dim;
    if (d->kernel == 0) {
        double g[ORC_MAXD][2 * ORC_MAXRHO + 2];
        for (int i = 0; i < D; ++i) gauss_1d(d->sigma, c[i], ix->order, g[i]);
        for (int k = 0; k < ix->P; ++k) {
            double v = 1.0;
            for (int i = 0; i < D; ++i) v *= g[i][ix->ex[k * D + i]];
            out[k] = v;
        }
        return;
    }
    /* polynomial: psi = sum_a coef_a x^a; d^m x^a = a!/(a-m)! x^(a-m) */
    int pdeg = 0;
    while (orc_num_coeffs(D, pdeg) < d->n_poly) ++pdeg;
    int *pex = (int *)malloc(sizeof(int) * D * orc_num_coeffs(D, pdeg));
    orc_multi_indices(D, pdeg, pex);
    for (int k = 0; k < ix->P; ++k) {
        double acc = 0.0;
        for (int a = 0; a < d->n_poly; ++a) {
            double term = d->poly_coef[a];
            if (term == 0.0) continue;
            for (int i = 0; i < D && term != 0.0; ++i) {
                int ai = pex[a * D + i], mi = ix->ex[k * D + i];
                if (ai < mi) { term = 0.0; break; }
                term *= ix->fact[ai] / ix->fact[ai - mi] * pow(c[i], ai - mi);
            }
            acc += term;
        }
        out[k] = acc;
    }
    free(pex);
}

int orc_kernel_derivs(const orc_desc *d, const double *c, double *out) {
    orc_index ix;
    index_init(&ix, d->dim, d->order);
    kernel_derivs_ix(d, &ix, c, out);
    index_free(&ix);
    return ix.P;
}

static double kernel_value(const orc_desc *d, const double *x) {
    int D = d->dim;
    if (d->kernel == 0) {
        double r2 = 0.0;
        for (int i = 0; i < D; ++i) r2 += x[i] * x[i];
        return exp(-r2 / (2.0 * d->sigma * d->sigma));
    }
    int pdeg = 0;
    while (orc_num_coeffs(D, pdeg) < d->n_poly) ++pdeg;
    int *pex = (int *)malloc(sizeof(int) * D * orc_num_coeffs(D, pdeg));
    orc_multi_indices(D, pdeg, pex);
    double acc = 0.0;
    for (int a = 0; a < d->n_poly; ++a) {
        double term = d->poly_coef[a];
        for (int i = 0; i < D; ++i) term *= pow(x[i], pex[a * D + i]);
        acc += term;
    }
    free(pex);
    return acc;
}


/* Gradient of psi at x: for the Gaussian d/dx_i psi = -(x_i / sigma^2) psi(x); for the polynomial
 * sum_a c_a x^a the term-by-term derivative sum_a c_a a_i x^(a - e_i). */
static void kernel_grad(const orc_desc *d, const double *x, double *g) {
    int D = d->dim;
    if (d->kernel == 0) {
        double v = kernel_value(d, x), s2 = d->sigma * d->sigma;
        for (int i = 0; i < D; ++i) g[i] = -x[i] / s2 * v;
        return;
    }
    int pdeg = 0;
    while (orc_num_coeffs(D, pdeg) < d->n_poly) ++pdeg;
    int *pex = (int *)malloc(sizeof(int) * D * orc_num_coeffs(D, pdeg));
    orc_multi_indices(D, pdeg, pex);
    for (int i = 0; i < D; ++i) g[i] = 0.0;
    for (int a = 0; a < d->n_poly; ++a) {
        for (int i = 0; i < D; ++i) {
            int ai = pex[a * D + i];
            if (ai == 0) continue;
            double term = d->poly_coef[a] * ai;
            for (int k = 0; k < D; ++k) term *= pow(x[k], pex[a * D + k] - (k == i ? 1 : 0));
            g[i] += term;
        }
    }
    free(pex);
}


/* ------------------------------------------------------- fitted operators
 * Sec. 3.1 replaces the Taylor coefficients of the kernel about a cell-pair offset c by those of
 * a polynomial fitted to the kernel in the least-squares sense over the separations the pair can
 * have.  Reading taken here: with x = h xi, the separation of a source and a target in cells of
 * width h whose centres are c apart ranges over c + [-h, h]^D, and the coefficients b_m (|m| <= rho)
 * of sum_m b_m xi^m / m! minimise sum_j w_j (psi(c + h xi_j) - sum_m b_m xi_j^m / m!)^2 over the
 * tensor Gauss-Legendre grid of rho + 2 points per dimension on [-1, 1]^D (weights w_j).  The
 * derivative of order m is then replaced by a_m = b_m / h^|m|. */
typedef struct { int npts, P, D; double *xi, *w, *phi, *chol; } orc_lsq;

/* Gauss-Legendre points and weights of K nodes on [-1, 1]: Newton's method on the Legendre
 * three-term recurrence */
static void legendre_nodes(int K, double *x, double *w) {
    for (int i = 0; i < K; ++i) {
        double z = cos(3.14159265358979323846 * (i + 0.75) / (K + 0.5)), dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = z;
            for (int m = 2; m <= K; ++m) {
                const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
                p0 = p1;
                p1 = p2;
            }
            dp = K * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-15) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static void lsq_init(orc_lsq *f, const orc_index *ix, int D, int rho) {
    const int K = rho + 2, P = ix->P;
    double x[ORC_MAXRHO + 2], w[ORC_MAXRHO + 2];
    legendre_nodes(K, x, w);
    int npts = 1;
    for (int i = 0; i < D; ++i) npts *= K;
    f->npts = npts; f->P = P; f->D = D;
    f->xi = (double *)malloc(sizeof(double) * npts * D);
    f->w = (double *)malloc(sizeof(double) * npts);
    f->phi = (double *)malloc(sizeof(double) * npts * P);
    f->chol = (double *)calloc((size_t)P * P, sizeof(double));
    for (int j = 0; j < npts; ++j) {
        int r = j;
        double pw[ORC_MAXD][ORC_MAXRHO + 1];
        f->w[j] = 1.0;
        for (int i = 0; i < D; ++i) {
            const int k = r % K;
            r /= K;
            f->xi[j * D + i] = x[k];
            f->w[j] *= w[k];
            powers_over_fact(x[k], rho, pw[i]);
        }
        for (int m = 0; m < P; ++m) f->phi[(size_t)j * P + m] = mono(ix, m, pw);
    }
    /* Gram matrix G = sum_j w_j phi_j phi_j^T, then its Cholesky factor (lower, in place) */
    double *G = f->chol;
    for (int j = 0; j < npts; ++j)
        for (int m = 0; m < P; ++m)
            for (int n2 = 0; n2 <= m; ++n2) G[m * P + n2] += f->w[j] * f->phi[(size_t)j * P + m] * f->phi[(size_t)j * P + n2];
    for (int m = 0; m < P; ++m) {
        for (int n2 = 0; n2 < m; ++n2) {
            double acc = G[m * P + n2];
            for (int k = 0; k < n2; ++k) acc -= G[m * P + k] * G[n2 * P + k];
            G[m * P + n2] = acc / G[n2 * P + n2];
        }
        double acc = G[m * P + m];
        for (int k = 0; k < m; ++k) acc -= G[m * P + k] * G[m * P + k];
        G[m * P + m] = sqrt(acc);
    }
}

static void lsq_free(orc_lsq *f) { free(f->xi); free(f->w); free(f->phi); free(f->chol); }

/* the fitted coefficients a_m (in place of d^m psi(c)) for offset c and cell width h */
static void lsq_fit(const orc_lsq *f, const orc_desc *d, const orc_index *ix, const double *c, double h,
                    double *out) {
    const int P = f->P, D = f->D;
    double *b = (double *)calloc((size_t)P, sizeof(double));
    for (int j = 0; j < f->npts; ++j) {
        double xx[ORC_MAXD];
        for (int i = 0; i < D; ++i) xx[i] = c[i] + h * f->xi[j * D + i];
        const double v = f->w[j] * kernel_value(d, xx);
        for (int m = 0; m < P; ++m) b[m] += v * f->phi[(size_t)j * P + m];
    }
    const double *Lc = f->chol;
    for (int m = 0; m < P; ++m) {          /* forward substitution */
        double acc = b[m];
        for (int k = 0; k < m; ++k) acc -= Lc[m * P + k] * b[k];
        b[m] = acc / Lc[m * P + m];
    }
    for (int m = P - 1; m >= 0; --m) {     /* back substitution with the transpose */
        double acc = b[m];
        for (int k = m + 1; k < P; ++k) acc -= Lc[k * P + m] * b[k];
        b[m] = acc / Lc[m * P + m];
    }
    for (int m = 0; m < P; ++m) out[m] = b[m] / pow(h, ix->deg[m]);
    free(b);
}

/* exported for the tests: the fitted coefficients at offset c, cell width h */
int orc_fit_coeffs(const orc_desc *d, const double *c, double h, double *out) {
    orc_index ix;
    index_init(&ix, d->dim, d->order);
    orc_lsq f;
    lsq_init(&f, &ix, d->dim, d->order);
    lsq_fit(&f, d, &ix, c, h, out);
    lsq_free(&f);
    index_free(&ix);
    return ix.P;
}

/* ----------------------------------------------------------------- binning */

/* Cell of one coordinate at a level with nl cells per dimension, decided in FP32. */
static int cell_1d(const orc_desc *d, int nl, double x) {
    volatile float xf = (float)x;
    volatile float lof = (float)d->lo;
    volatile float scale = (float)((double)nl / (d->hi - d->lo));
    volatile float diff = xf - lof;
    volatile float t = diff * scale;
    float f = floorf(t);
    int c;
    if (!(f >= 0.0f)) c = 0;                 /* negative or NaN */
    else if (f >= (float)nl) c = nl - 1;
    else c = (int)f;
    if (c > nl - 1) c = nl - 1;
    return c;
}

/* linear cell index, first coordinate fastest: c0 + n (c1 + n c2) */
int orc_bin(const orc_desc *d, const double *x, int64_t n, int32_t *cell) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t lin = 0;
        for (int k = d->dim - 1; k >= 0; --k) lin = lin * d->grid + cell_1d(d, d->grid, x[i * d->dim + k]);
        cell[i] = (int32_t)lin;
    }
    return 0;
}

/* ----------------------------------------------------------- the transform */

static int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

static void unravel(int64_t lin, int nl, int D, int *c) {
    for (int i = 0; i < D; ++i) { c[i] = (int)(lin % nl); lin /= nl; }
}

static int64_t ravel(const int *c, int nl, int D) {
    int64_t lin = 0;
    for (int i = D - 1; i >= 0; --i) lin = lin * nl + c[i];
    return lin;
}

static double centre(const orc_desc *d, int nl, int ci) {
    double h = (d->hi - d->lo) / nl;
    return d->lo + (ci + 0.5) * h;
}


/* ------------------------------------------------------------------- rays
 * Rays x(t) = o + t r for t in [t0, t1] (Sec. 6, the integral-implicit layer: "Line Integral"
 * with line2poly of Sec. 5, "Line to polynomial", and "Line Integral JVP" with ray2M).  A ray is cut into segments at the faces of the finest cells (the part
 * outside the domain box is dropped); each segment lies in one cell, found from its midpoint by
 * the binning rule.  (3D only.) */
typedef struct { const double *o, *r, *t0, *t1, *wt; int64_t n; } orc_rayset;
typedef struct { int64_t cell; double ta, tb; } orc_seg;

static int cmp_double(const void *a, const void *b) {
    const double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* the segments of one ray (allocated in *out; returns their number) */
static int64_t ray_segments(const orc_desc *d, const double *o, const double *r, double t0, double t1,
                            orc_seg **out) {
    const int D = d->dim, n = d->grid;
    const double h = (d->hi - d->lo) / n;
    double ta = t0, tb = t1;
    *out = NULL;
    for (int k = 0; k < D; ++k) {          /* clip to the domain box (slabs) */
        if (r[k] == 0.0) {
            if (o[k] < d->lo || o[k] >= d->hi) return 0;
            continue;
        }
        double a = (d->lo - o[k]) / r[k], b = (d->hi - o[k]) / r[k];
        if (a > b) { double tmp = a; a = b; b = tmp; }
        if (a > ta) ta = a;
        if (b < tb) tb = b;
    }
    if (!(tb > ta)) return 0;
    double *cut = (double *)malloc(sizeof(double) * (2 + (size_t)D * (n + 1)));
    int64_t nc = 0;
    cut[nc++] = ta;
    for (int k = 0; k < D; ++k) {          /* crossings of the interior faces */
        if (r[k] == 0.0) continue;
        for (int j = 1; j < n; ++j) {
            const double t = (d->lo + j * h - o[k]) / r[k];
            if (t > ta && t < tb) cut[nc++] = t;
        }
    }
    cut[nc++] = tb;
    qsort(cut, (size_t)nc, sizeof(double), cmp_double);
    orc_seg *seg = (orc_seg *)malloc(sizeof(orc_seg) * (size_t)nc);
    int64_t ns = 0;
    for (int64_t i = 0; i + 1 < nc; ++i) {
        if (!(cut[i + 1] > cut[i])) continue;
        const double tm = 0.5 * (cut[i] + cut[i + 1]);
        int c[ORC_MAXD];
        for (int k = 0; k < D; ++k) c[k] = cell_1d(d, n, o[k] + tm * r[k]);
        seg[ns].cell = ravel(c, n, D);
        seg[ns].ta = cut[i];
        seg[ns].tb = cut[i + 1];
        ++ns;
    }
    free(cut);
    *out = seg;
    return ns;
}

/* c[k][i] = dd^(k-i) / (k-i)! * r^i / i!  for i <= k <= rho: the coefficient of tau^i in
 * (dd + r tau)^k / k!  (binomial theorem) */
static void line_binomials(double dd, double r, int rho, double c[][ORC_MAXRHO + 1]) {
    double pd[ORC_MAXRHO + 1], pr[ORC_MAXRHO + 1];
    powers_over_fact(dd, rho, pd);
    powers_over_fact(r, rho, pr);
    for (int k = 0; k <= rho; ++k)
        for (int i = 0; i <= rho; ++i) c[k][i] = i <= k ? pd[k - i] * pr[i] : 0.0;
}

/* line2taylor: the moments of a segment entering the cell at dd (relative to its centre) along r
 * for a length s of the parameter,  out(n) = int_0^s prod_k (dd_k + r_k tau)^(n_k) / n_k! dtau
 * = sum_{i <= n} prod_k [dd_k^(n_k-i_k)/(n_k-i_k)! r_k^(i_k)/i_k!] s^(|i|+1) / (|i|+1) */
static void line2taylor(const orc_index *ix, int rho, const double *dd, const double *r, double s, double *out) {
    double c[3][ORC_MAXRHO + 1][ORC_MAXRHO + 1];
    for (int k = 0; k < 3; ++k) line_binomials(dd[k], r[k], rho, c[k]);
    double sp[3 * ORC_MAXRHO + 2];
    sp[0] = 1.0;
    for (int m = 1; m < 3 * ORC_MAXRHO + 2; ++m) sp[m] = sp[m - 1] * s;
    for (int a = 0; a < ix->P; ++a) {
        const int n1 = ix->ex[a * 3], n2 = ix->ex[a * 3 + 1], n3 = ix->ex[a * 3 + 2];
        double acc = 0.0;
        for (int i = 0; i <= n1; ++i)
            for (int j = 0; j <= n2; ++j)
                for (int k = 0; k <= n3; ++k)
                    acc += c[0][n1][i] * c[1][n2][j] * c[2][n3][k] * sp[i + j + k + 1] / (i + j + k + 1);
        out[a] = acc;
    }
}

/* line2poly: the local series L of a cell restricted to the line dd + r x, as a polynomial
 * sum_m a_m x^m (m <= rho):  a_m = sum_n L(n) sum_{i + j + k = m} prod [dd^(n-i)/(n-i)! r^i/i!] */
static void line2poly(const orc_index *ix, int rho, const double *L, const double *dd, const double *r, double *a) {
    double c[3][ORC_MAXRHO + 1][ORC_MAXRHO + 1];
    for (int k = 0; k < 3; ++k) line_binomials(dd[k], r[k], rho, c[k]);
    for (int m = 0; m <= rho; ++m) a[m] = 0.0;
    for (int b = 0; b < ix->P; ++b) {
        const int n1 = ix->ex[b * 3], n2 = ix->ex[b * 3 + 1], n3 = ix->ex[b * 3 + 2];
        for (int i = 0; i <= n1; ++i)
            for (int j = 0; j <= n2; ++j)
                for (int k = 0; k <= n3; ++k) a[i + j + k] += L[b] * c[0][n1][i] * c[1][n2][j] * c[2][n3][k];
    }
}

static int near_idx(const int *a, const int *b, int D) {
    for (int i = 0; i < D; ++i) if (abs(a[i] - b[i]) > 1) return 0;
    return 1;
}

/* Is source cell s in the interaction list of target cell t at level l? */
static int in_list(const int *s, const int *t, int D, int level, int top, int fault) {
    int ps[ORC_MAXD], pt[ORC_MAXD];
    for (int i = 0; i < D; ++i) {
        if (fault == ORC_FAULT_PARITY) { ps[i] = (s[i] + 1) >> 1; pt[i] = (t[i] + 1) >> 1; }
        else { ps[i] = s[i] >> 1; pt[i] = t[i] >> 1; }
    }
    int parent_near = (level == top) ? 1 : near_idx(ps, pt, D);
    if (!parent_near) return 0;
    if (level == 0) {
        if (fault == ORC_FAULT_NO_SELF) {
            int same = 1;
            for (int i = 0; i < D; ++i) if (s[i] != t[i]) same = 0;
            if (same) return 0;
        }
        return 1;
    }
    return !near_idx(s, t, D);
}

/*
 * The transform.  Sources src[n_src][dim] with weights wt[n_src]; targets
 * tgt[n_tgt][dim].  If src_cell / tgt_cell are given they replace the binning
 * (finest-level linear cell index per point: used for finite differences with
 * the binning held fixed).  sel[n_sel] lists the target indices to evaluate
 * (n_sel < 0: all targets, in order).  val[j] receives the series value at
 * target sel[j]; grad (if not NULL) receives its gradient, [n_sel][dim]; hess (if not
 * NULL) its second partials d^2/dx_i dx_k for i <= k in row-major order, [n_sel][dim(dim+1)/2]
 * (the accessor's second partials, Sec. 3, "How to use the implementation?").
 * Returns 0 on success, negative on bad arguments.
 */
static int pipeline(const orc_desc *d,
                    const double *src, const double *wt, int64_t n_src, const int32_t *src_cell,
                    const orc_rayset *src_rays,
                    const double *tgt, int64_t n_tgt, const int32_t *tgt_cell,
                    const int64_t *sel, int64_t n_sel, const orc_rayset *tgt_rays,
                    double *val, double *grad, double *hess, double *ray_val, int fault) {
    int D = d->dim, n = d->grid, rho = d->order;
    if (D < 2 || D > 3 || n < 4 || (n & (n - 1)) || rho < 0 || rho > ORC_MAXRHO) return -1;
    if ((src_rays || tgt_rays) && D != 3) return -1;
    if (!(d->hi > d->lo)) return -1;
    orc_index ix;
    index_init(&ix, D, rho);
    int P = ix.P;
    int nlev = ilog2(n) - 1, top = nlev - 1;
    if (n_sel < 0) n_sel = n_tgt;

    /* per-level storage */
    int64_t G[32];
    double *Mx[32], *Lx[32];
    unsigned char *need[32];
    for (int l = 0; l < nlev; ++l) {
        int nl = n >> l;
        G[l] = 1;
        for (int i = 0; i < D; ++i) G[l] *= nl;
        Mx[l] = (double *)calloc((size_t)G[l] * P, sizeof(double));
        Lx[l] = (double *)calloc((size_t)G[l] * P, sizeof(double));
        need[l] = (unsigned char *)calloc((size_t)G[l], 1);
    }

    /* ---- P2M: script-M(n, p') = sum_{i in I(p')} w_i prod d^n_j / n_j! */
    for (int64_t i = 0; i < n_src; ++i) {
        int c[ORC_MAXD];
        int64_t lin;
        if (src_cell) { lin = src_cell[i]; unravel(lin, n, D, c); }
        else { for (int k = 0; k < D; ++k) c[k] = cell_1d(d, n, src[i * D + k]); lin = ravel(c, n, D); }
        double pw[ORC_MAXD][ORC_MAXRHO + 1];
        for (int k = 0; k < D; ++k) powers_over_fact(src[i * D + k] - centre(d, n, c[k]), rho, pw[k]);
        for (int b = 0; b < P; ++b) Mx[0][lin * P + b] += wt[i] * mono(&ix, b, pw);
    }

    /* ---- ray2M (Sec. 6, "Line Integral JVP"): every segment of a source ray adds its weight times line2taylor to the
     * moments of its cell, entry point taken relative to the cell centre */
    if (src_rays) {
        double *mt = (double *)malloc(sizeof(double) * P);
        for (int64_t q = 0; q < src_rays->n; ++q) {
            orc_seg *seg;
            const double *o = src_rays->o + 3 * q, *r = src_rays->r + 3 * q;
            const int64_t ns = ray_segments(d, o, r, src_rays->t0[q], src_rays->t1[q], &seg);
            for (int64_t g = 0; g < ns; ++g) {
                int c[ORC_MAXD];
                unravel(seg[g].cell, n, D, c);
                double dd[3];
                for (int k = 0; k < 3; ++k) dd[k] = o[k] + seg[g].ta * r[k] - centre(d, n, c[k]);
                line2taylor(&ix, rho, dd, r, seg[g].tb - seg[g].ta, mt);
                for (int b = 0; b < P; ++b) Mx[0][seg[g].cell * P + b] += src_rays->wt[q] * mt[b];
            }
            free(seg);
        }
        free(mt);
    }

    /* ---- M2M: script-M(n, p'') = sum_{p' in I(p'')} sum_{k <= n} d'^(n-k)/(n-k)! script-M(k, p') */
    for (int l = 0; l + 1 < nlev; ++l) {
        int nl = n >> l, np = nl >> 1;
        orc_shift sh[1 << ORC_MAXD];
        for (int ch = 0; ch < (1 << D); ++ch) {
            /* d' = centre(child) - centre(parent) = +-h_l / 2 per dimension */
            double dd[ORC_MAXD];
            for (int k = 0; k < D; ++k) {
                dd[k] = centre(d, nl, (ch >> k) & 1) - centre(d, np, 0);
                if (fault == ORC_FAULT_M2M_SIGN) dd[k] = -dd[k];
            }
            shift_init(&sh[ch], &ix, dd);
        }
        for (int64_t C = 0; C < G[l + 1]; ++C) {
            int cp[ORC_MAXD];
            unravel(C, np, D, cp);
            for (int ch = 0; ch < (1 << D); ++ch) {
                int cc[ORC_MAXD];
                for (int k = 0; k < D; ++k) cc[k] = 2 * cp[k] + ((ch >> k) & 1);
                const double *Mc = Mx[l] + ravel(cc, nl, D) * P;
                for (int a = 0; a < P; ++a) {
                    double acc = 0.0;
                    for (int e = sh[ch].start[a]; e < sh[ch].start[a + 1]; ++e)
                        acc += sh[ch].coef[e] * Mc[sh[ch].b[e]];
                    Mx[l + 1][C * P + a] += acc;
                }
            }
        }
        for (int ch = 0; ch < (1 << D); ++ch) shift_free(&sh[ch]);
    }

    /* ---- which target cells are needed (selected targets and their ancestors) */
    int32_t *tcell = (int32_t *)malloc(sizeof(int32_t) * (n_sel > 0 ? n_sel : 1));
    for (int64_t j = 0; j < n_sel; ++j) {
        int64_t ti = sel ? sel[j] : j;
        int c[ORC_MAXD];
        int64_t lin;
        if (tgt_cell) lin = tgt_cell[ti];
        else { for (int k = 0; k < D; ++k) c[k] = cell_1d(d, n, tgt[ti * D + k]); lin = ravel(c, n, D); }
        tcell[j] = (int32_t)lin;
        need[0][lin] = 1;
    }
    if (tgt_rays)
        for (int64_t q = 0; q < tgt_rays->n; ++q) {
            orc_seg *seg;
            const int64_t ns = ray_segments(d, tgt_rays->o + 3 * q, tgt_rays->r + 3 * q, tgt_rays->t0[q],
                                            tgt_rays->t1[q], &seg);
            for (int64_t g = 0; g < ns; ++g) need[0][seg[g].cell] = 1;
            free(seg);
        }
    for (int l = 0; l + 1 < nlev; ++l) {
        int nl = n >> l;
        for (int64_t c = 0; c < G[l]; ++c) if (need[l][c]) {
            int cc[ORC_MAXD];
            unravel(c, nl, D, cc);
            for (int k = 0; k < D; ++k) cc[k] >>= 1;
            need[l + 1][ravel(cc, nl >> 1, D)] = 1;
        }
    }

    /* ---- M2L: script-L(k, q') = sum_{p'} sum_{|n| <= rho-|k|} (-1)^|k| d^(n+k) psi(p'-q') script-M(n, p')
     * the derivative tables for every offset in {-3..3}^D are built once per level */
    int nb = 1;
    for (int i = 0; i < D; ++i) nb *= 7;
    double *dtab = (double *)malloc(sizeof(double) * nb * P);
    orc_lsq lsq;
    if (d->fit) lsq_init(&lsq, &ix, D, rho);
    /* for every k: the n with |n| <= rho - |k| and the graded index of n + k */
    int *pstart = (int *)malloc(sizeof(int) * (P + 1));
    int *pn = (int *)malloc(sizeof(int) * P * P), *pnk = (int *)malloc(sizeof(int) * P * P);
    {
        int cnt = 0;
        for (int kk = 0; kk < P; ++kk) {
            pstart[kk] = cnt;
            int budget = rho - ix.deg[kk] - (fault == ORC_FAULT_DROP_TOP_TERM ? 1 : 0);
            for (int b = 0; b < P; ++b) {
                if (ix.deg[b] > budget) continue;
                int m[ORC_MAXD];
                for (int k = 0; k < D; ++k) m[k] = ix.ex[b * D + k] + ix.ex[kk * D + k];
                pn[cnt] = b; pnk[cnt] = idx_of(&ix, m); ++cnt;
            }
        }
        pstart[P] = cnt;
    }
    for (int l = 0; l < nlev; ++l) {
        int nl = n >> l;
        double h = (d->hi - d->lo) / nl;
        for (int o = 0; o < nb; ++o) {
            int oo[ORC_MAXD];
            int r = o;
            double c[ORC_MAXD];
            for (int k = 0; k < D; ++k) { oo[k] = r % 7 - 3; r /= 7; c[k] = oo[k] * h; }
            if (fault == ORC_FAULT_TRANSPOSE) for (int k = 0; k < D; ++k) c[k] = -c[k];
            if (d->fit) lsq_fit(&lsq, d, &ix, c, h, dtab + (size_t)o * P);
            else kernel_derivs_ix(d, &ix, c, dtab + (size_t)o * P);
        }
        int64_t Gl = G[l];
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t t = 0; t < Gl; ++t) {
            if (!need[l][t]) continue;
            int tc[ORC_MAXD];
            unravel(t, nl, D, tc);
            double *Lt = Lx[l] + t * P;
            int lo3[ORC_MAXD], hi3[ORC_MAXD];
            for (int k = 0; k < D; ++k) {
                lo3[k] = tc[k] - 3 < 0 ? 0 : tc[k] - 3;
                hi3[k] = tc[k] + 3 > nl - 1 ? nl - 1 : tc[k] + 3;
            }
            int sc[ORC_MAXD] = {0, 0, 0};
            for (sc[2] = (D == 3 ? lo3[2] : 0); sc[2] <= (D == 3 ? hi3[2] : 0); ++sc[2])
            for (sc[1] = lo3[1]; sc[1] <= hi3[1]; ++sc[1])
            for (sc[0] = lo3[0]; sc[0] <= hi3[0]; ++sc[0]) {
                if (!in_list(sc, tc, D, l, top, fault)) continue;
                int o = 0;
                for (int k = D - 1; k >= 0; --k) o = o * 7 + (sc[k] - tc[k] + 3);
                const double *dps = dtab + (size_t)o * P;
                const double *Ms = Mx[l] + ravel(sc, nl, D) * P;
                for (int kk = 0; kk < P; ++kk) {
                    double sgn = (ix.deg[kk] & 1) && fault != ORC_FAULT_DROP_SIGN ? -1.0 : 1.0;
                    double acc = 0.0;
                    for (int e = pstart[kk]; e < pstart[kk + 1]; ++e) acc += dps[pnk[e]] * Ms[pn[e]];
                    Lt[kk] += sgn * acc;
                }
            }
        }
    }
    free(dtab); free(pstart); free(pn); free(pnk);
    if (d->fit) lsq_free(&lsq);

    /* ---- L2L: script-L(n, q') += sum_{k >= n} d'^(k-n)/(k-n)! script-L(k, q''), coarse to fine */
    if (fault != ORC_FAULT_NO_L2L) {
        for (int l = nlev - 2; l >= 0; --l) {
            int nl = n >> l, np = nl >> 1;
            orc_shift sh[1 << ORC_MAXD];
            for (int ch = 0; ch < (1 << D); ++ch) {
                double dd[ORC_MAXD];
                for (int k = 0; k < D; ++k) dd[k] = centre(d, nl, (ch >> k) & 1) - centre(d, np, 0);
                shift_init(&sh[ch], &ix, dd);
            }
            for (int64_t c = 0; c < G[l]; ++c) {
                if (!need[l][c]) continue;
                int cc[ORC_MAXD], cp[ORC_MAXD], ch = 0;
                unravel(c, nl, D, cc);
                for (int k = 0; k < D; ++k) { cp[k] = cc[k] >> 1; ch |= (cc[k] & 1) << k; }
                const double *Lp = Lx[l + 1] + ravel(cp, np, D) * P;
                /* sh[ch] lists, for each g, the a <= g with coefficient d'^(g-a)/(g-a)! */
                for (int g = 0; g < P; ++g)
                    for (int e = sh[ch].start[g]; e < sh[ch].start[g + 1]; ++e)
                        Lx[l][c * P + sh[ch].b[e]] += sh[ch].coef[e] * Lp[g];
            }
            for (int ch = 0; ch < (1 << D); ++ch) shift_free(&sh[ch]);
        }
    }

    /* ---- L2P (and its gradient): y = sum_{|k| <= rho} L(k) prod d_q^k / k! */
    for (int64_t j = 0; j < n_sel; ++j) {
        int64_t ti = sel ? sel[j] : j;
        int c[ORC_MAXD];
        unravel(tcell[j], n, D, c);
        double pw[ORC_MAXD][ORC_MAXRHO + 1];
        for (int k = 0; k < D; ++k) powers_over_fact(tgt[ti * D + k] - centre(d, n, c[k]), rho, pw[k]);
        const double *Lc = Lx[0] + (int64_t)tcell[j] * P;
        double v = 0.0;
        for (int a = 0; a < P; ++a) v += Lc[a] * mono(&ix, a, pw);
        val[j] = v;
        if (grad) {
            /* d/dx_i of prod_k d_k^(a_k)/a_k! = d_i^(a_i - 1)/(a_i - 1)! prod_{k != i} ... */
            for (int i = 0; i < D; ++i) {
                double g = 0.0;
                for (int a = 0; a < P; ++a) {
                    if (ix.ex[a * D + i] == 0) continue;
                    double m = 1.0;
                    for (int k = 0; k < D; ++k) m *= pw[k][ix.ex[a * D + k] - (k == i ? 1 : 0)];
                    g += Lc[a] * m;
                }
                grad[j * D + i] = g;
            }
        }
        if (hess) {
            /* second partials d^2/dx_i dx_k, i <= k (row-major upper triangle): both exponents
             * lowered by one (or the one exponent by two when i = k), terms that cannot be
             * lowered vanish */
            int pos = 0;
            for (int i = 0; i < D; ++i)
                for (int k2 = i; k2 < D; ++k2, ++pos) {
                    double hsum = 0.0;
                    for (int a = 0; a < P; ++a) {
                        int e[ORC_MAXD], ok = 1;
                        for (int k = 0; k < D; ++k) e[k] = ix.ex[a * D + k];
                        e[i] -= 1;
                        e[k2] -= 1;
                        for (int k = 0; k < D; ++k) ok &= e[k] >= 0;
                        if (!ok) continue;
                        double m = 1.0;
                        for (int k = 0; k < D; ++k) m *= pw[k][e[k]];
                        hsum += Lc[a] * m;
                    }
                    hess[j * (D * (D + 1) / 2) + pos] = hsum;
                }
        }
    }

    /* ---- ray integrals (Sec. 6, "Line Integral"): each segment's cell series restricted to the line (line2poly),
     * integrated over the segment: int_0^s sum_m a_m x^m dx = sum_m a_m s^(m+1) / (m+1) */
    if (tgt_rays)
        for (int64_t q = 0; q < tgt_rays->n; ++q) {
            orc_seg *seg;
            const double *o = tgt_rays->o + 3 * q, *r = tgt_rays->r + 3 * q;
            const int64_t ns = ray_segments(d, o, r, tgt_rays->t0[q], tgt_rays->t1[q], &seg);
            double acc = 0.0;
            for (int64_t g = 0; g < ns; ++g) {
                int c[ORC_MAXD];
                unravel(seg[g].cell, n, D, c);
                double dd[3], a[ORC_MAXRHO + 1];
                for (int k = 0; k < 3; ++k) dd[k] = o[k] + seg[g].ta * r[k] - centre(d, n, c[k]);
                line2poly(&ix, rho, Lx[0] + seg[g].cell * P, dd, r, a);
                const double s = seg[g].tb - seg[g].ta;
                double sp = s;
                for (int m = 0; m <= rho; ++m, sp *= s) acc += a[m] * sp / (m + 1);
            }
            ray_val[q] = acc;
            free(seg);
        }

    free(tcell);
    for (int l = 0; l < nlev; ++l) { free(Mx[l]); free(Lx[l]); free(need[l]); }
    index_free(&ix);
    return 0;
}

int orc_transform_h(const orc_desc *d,
                    const double *src, const double *wt, int64_t n_src, const int32_t *src_cell,
                    const double *tgt, int64_t n_tgt, const int32_t *tgt_cell,
                    const int64_t *sel, int64_t n_sel,
                    double *val, double *grad, double *hess, int fault) {
    return pipeline(d, src, wt, n_src, src_cell, NULL, tgt, n_tgt, tgt_cell, sel, n_sel, NULL, val, grad, hess, NULL,
                    fault);
}

int orc_transform(const orc_desc *d,
                  const double *src, const double *wt, int64_t n_src, const int32_t *src_cell,
                  const double *tgt, int64_t n_tgt, const int32_t *tgt_cell,
                  const int64_t *sel, int64_t n_sel,
                  double *val, double *grad, int fault) {
    return orc_transform_h(d, src, wt, n_src, src_cell, tgt, n_tgt, tgt_cell, sel, n_sel, val, grad, NULL, fault);
}

/* Ray integrals of the transform (Sec. 6, integral-implicit layer), rays given by origins o and
 * directions r [n_ray][3] and parameter ranges [t0, t1] (clipped to the domain box):
 *   forward:  y_q = int_{t0}^{t1} f(o_q + t r_q) dt,  f the series of (src, wt)  (line2poly);
 *   backward: value (and gradient) at the targets of the transform whose sources are the rays with
 *             weights ybar (ray2M with line2taylor), i.e. wbar_n = sum_q ybar_q int T(p_n, x_q(t)) dt
 *             and, times w_n, pbar_n. */
int orc_ray_forward(const orc_desc *d, const double *src, const double *wt, int64_t n_src,
                    const double *o, const double *r, const double *t0, const double *t1, int64_t n_ray,
                    double *y) {
    orc_rayset rs = {o, r, t0, t1, NULL, n_ray};
    return pipeline(d, src, wt, n_src, NULL, NULL, NULL, 0, NULL, NULL, 0, &rs, NULL, NULL, NULL, y, ORC_FAULT_NONE);
}

int orc_ray_backward(const orc_desc *d, const double *o, const double *r, const double *t0, const double *t1,
                     const double *ybar, int64_t n_ray, const double *tgt, int64_t n_tgt, const int32_t *tgt_cell,
                     double *val, double *grad) {
    orc_rayset rs = {o, r, t0, t1, ybar, n_ray};
    return pipeline(d, NULL, NULL, 0, NULL, &rs, tgt, n_tgt, tgt_cell, NULL, -1, NULL, val, grad, NULL, NULL,
                    ORC_FAULT_NONE);
}

/* Exact O(N M) sum of Eq. 1 at the selected targets (accuracy reference). */
int orc_direct(const orc_desc *d, const double *src, const double *wt, int64_t n_src,
               const double *tgt, int64_t n_tgt, const int64_t *sel, int64_t n_sel, double *val) {
    int D = d->dim;
    if (n_sel < 0) n_sel = n_tgt;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_sel; ++j) {
        int64_t ti = sel ? sel[j] : j;
        double acc = 0.0;
        for (int64_t i = 0; i < n_src; ++i) {
            double x[ORC_MAXD];
            for (int k = 0; k < D; ++k) x[k] = src[i * D + k] - tgt[ti * D + k];
            acc += kernel_value(d, x) * wt[i];
        }
        val[j] = acc;
    }
    return 0;
}

/* Exact gradients of <ybar, y> for the direct sum y_m = sum_n psi(p_n - q_m) w_n of Eq. 1 (the dense
 * form of Sec. 4.1's Jacobian vector product), at the selected sources n:
 *   wbar_n = sum_m ybar_m psi(p_n - q_m),      pbar_n = w_n sum_m ybar_m (grad psi)(p_n - q_m).
 * pbar may be NULL. */
int orc_direct_grad(const orc_desc *d, const double *src, const double *wt, int64_t n_src,
                    const double *tgt, const double *ybar, int64_t n_tgt, const int64_t *sel, int64_t n_sel,
                    double *wbar, double *pbar) {
    int D = d->dim;
    if (n_sel < 0) n_sel = n_src;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_sel; ++j) {
        int64_t si = sel ? sel[j] : j;
        double acc = 0.0, ga[ORC_MAXD] = {0.0, 0.0, 0.0};
        for (int64_t m = 0; m < n_tgt; ++m) {
            double x[ORC_MAXD], g[ORC_MAXD];
            for (int k = 0; k < D; ++k) x[k] = src[si * D + k] - tgt[m * D + k];
            acc += kernel_value(d, x) * ybar[m];
            if (pbar) {
                kernel_grad(d, x, g);
                for (int k = 0; k < D; ++k) ga[k] += g[k] * ybar[m];
            }
        }
        wbar[j] = acc;
        if (pbar)
            for (int k = 0; k < D; ++k) pbar[j * D + k] = wt[si] * ga[k];
    }
    (void)n_src;
    return 0;
}
