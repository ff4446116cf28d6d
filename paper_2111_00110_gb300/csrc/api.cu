// C ABI of the FC2T2 library: plan creation (operator tables, workspace) and the
// forward / backward pipelines (Sec. 3 and Sec. 4.1 of arXiv 2111.00110).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <memory>
#include <cstdio>
#include <cstring>
#include <functional>
#include <unordered_map>
#include <string>
#include <vector>

#include "fc2t2_internal.cuh"

namespace fc2t2 {

static thread_local fc2t2_status g_err_code = FC2T2_OK;
static thread_local std::string g_err_msg;

fc2t2_status set_error(fc2t2_status st, const std::string &msg) {
    g_err_code = st;
    g_err_msg = msg;
    return st;
}

fc2t2_status check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return FC2T2_OK;
    return set_error(FC2T2_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------ host operator tables

struct HostIndex {
    int D = 0, rho = 0, P = 0;
    std::vector<int> e;      // [P][3]
    std::vector<int> deg;    // [P]
    HostIndex(int D_, int rho_) : D(D_), rho(rho_), P(ncoef(D_, rho_)), e(3 * P, 0), deg(P, 0) {
        for (int k = 0; k < P; ++k) {
            // invert the graded index by search (tiny)
            for (int a0 = 0; a0 <= rho; ++a0)
                for (int a1 = 0; a0 + a1 <= rho; ++a1)
                    for (int a2 = 0; a0 + a1 + a2 <= rho; ++a2) {
                        if (D == 2 && a2 != 0) continue;
                        const int g = D == 2 ? gidx2(a0, a1) : gidx3(a0, a1, a2);
                        if (g == k) { e[3 * k] = a0; e[3 * k + 1] = a1; e[3 * k + 2] = a2; deg[k] = a0 + a1 + a2; }
                    }
        }
    }
    int index(int a0, int a1, int a2) const {
        if (a0 < 0 || a1 < 0 || a2 < 0 || a0 + a1 + a2 > rho) return -1;
        return D == 2 ? gidx2(a0, a1) : gidx3(a0, a1, a2);
    }
};

// h^j g^(j)(x) for g(x) = exp(-x^2 / (2 sigma^2)), j = 0..J, via the probabilists' Hermite
// polynomials: g^(j)(x) = (-1/sigma)^j He_j(x/sigma) g(x),  He_{j+1}(v) = v He_j - j He_{j-1}.
static void gaussian_scaled_derivs_1d(double sigma, double h, double x, int J, double *out) {
    const double v = x / sigma, g = std::exp(-0.5 * v * v), r = -h / sigma;
    double hem1 = 0.0, he = 1.0, f = 1.0;
    for (int j = 0; j <= J; ++j) {
        out[j] = f * he * g;
        const double hn = v * he - j * hem1;
        hem1 = he;
        he = hn;
        f *= r;
    }
}

// psi(x) on the host (Gaussian or polynomial)
static double kernel_value_host(const fc2t2_plan_s *pl, const double *x) {
    const int D = pl->D;
    if (pl->desc.kernel == FC2T2_KERNEL_GAUSSIAN) {
        double r2 = 0.0;
        for (int d = 0; d < D; ++d) r2 += x[d] * x[d];
        return std::exp(-r2 / (2.0 * pl->desc.sigma * pl->desc.sigma));
    }
    int pdeg = 0;
    while (ncoef(D, pdeg) < (int)pl->poly.size()) ++pdeg;
    HostIndex px(D, pdeg);
    double acc = 0.0;
    for (int a = 0; a < (int)pl->poly.size(); ++a) {
        double term = pl->poly[a];
        for (int d = 0; d < D && term != 0.0; ++d)
            for (int t = 0; t < px.e[3 * a + d]; ++t) term *= x[d];
        acc += term;
    }
    return acc;
}

// Least-squares operators (Sec. 3.1: the Taylor coefficients of the kernel about a cell-pair
// offset c replaced by those of a polynomial fitted to the kernel over the pair's separations).
// With x = h xi, the separations of a source and a target in cells of width h whose centres are c
// apart are c + [-h, h]^D; the scaled coefficients b_m (|m| <= rho) of sum_m b_m xi^m / m! minimise
// sum_j w_j (psi(c + h xi_j) - sum_m b_m xi_j^m / m!)^2 over the tensor Gauss-Legendre grid of
// rho + 2 points per dimension on [-1, 1]^D.  b_m takes the place of Dt[m] = h^|m| d^m psi(c).  The
// Gram matrix depends only on the grid: it is factored once (Cholesky) and each offset solves
// against its own right-hand side.
struct LsqFit {
    int D = 0, P = 0, npts = 0;
    std::vector<double> xi, w, phi, chol;   // points [npts][D], weights, basis [npts][P], factor [P][P]

    LsqFit(const fc2t2_plan_s *pl, const HostIndex &ix) : D(pl->D), P(ix.P) {
        const int K = pl->rho + 2;
        std::vector<double> x(K), wk(K);
        for (int i = 0; i < K; ++i) {   // Legendre P_K roots by Newton's method on the recurrence
            double z = std::cos(M_PI * (i + 0.75) / (K + 0.5)), dp = 1.0;
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
                if (std::fabs(dz) < 1e-15) break;
            }
            x[i] = z;
            wk[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
        npts = 1;
        for (int d = 0; d < D; ++d) npts *= K;
        xi.resize((size_t)npts * D);
        w.resize(npts);
        phi.resize((size_t)npts * P);
        for (int j = 0; j < npts; ++j) {
            int r = j;
            double pw[3][kMaxOrder + 1];
            w[j] = 1.0;
            for (int d = 0; d < D; ++d) {
                const int k = r % K;
                r /= K;
                xi[(size_t)j * D + d] = x[k];
                w[j] *= wk[k];
                pw[d][0] = 1.0;
                for (int t = 1; t <= pl->rho; ++t) pw[d][t] = pw[d][t - 1] * x[k] / t;
            }
            for (int m = 0; m < P; ++m) {
                double v = 1.0;
                for (int d = 0; d < D; ++d) v *= pw[d][ix.e[3 * m + d]];
                phi[(size_t)j * P + m] = v;
            }
        }
        chol.assign((size_t)P * P, 0.0);
        for (int j = 0; j < npts; ++j)
            for (int m = 0; m < P; ++m) {
                const double a = w[j] * phi[(size_t)j * P + m];
                for (int n = 0; n <= m; ++n) chol[(size_t)m * P + n] += a * phi[(size_t)j * P + n];
            }
        for (int m = 0; m < P; ++m) {
            for (int n = 0; n < m; ++n) {
                double acc = chol[(size_t)m * P + n];
                for (int k = 0; k < n; ++k) acc -= chol[(size_t)m * P + k] * chol[(size_t)n * P + k];
                chol[(size_t)m * P + n] = acc / chol[(size_t)n * P + n];
            }
            double acc = chol[(size_t)m * P + m];
            for (int k = 0; k < m; ++k) acc -= chol[(size_t)m * P + k] * chol[(size_t)m * P + k];
            chol[(size_t)m * P + m] = std::sqrt(acc);
        }
    }

    void scaled(const fc2t2_plan_s *pl, const double *c, double h, double *out) const {
        std::vector<double> b(P, 0.0);
        for (int j = 0; j < npts; ++j) {
            double x[3] = {0.0, 0.0, 0.0};
            for (int d = 0; d < D; ++d) x[d] = c[d] + h * xi[(size_t)j * D + d];
            const double v = w[j] * kernel_value_host(pl, x);
            for (int m = 0; m < P; ++m) b[m] += v * phi[(size_t)j * P + m];
        }
        for (int m = 0; m < P; ++m) {
            double acc = b[m];
            for (int k = 0; k < m; ++k) acc -= chol[(size_t)m * P + k] * b[k];
            b[m] = acc / chol[(size_t)m * P + m];
        }
        for (int m = P - 1; m >= 0; --m) {
            double acc = b[m];
            for (int k = m + 1; k < P; ++k) acc -= chol[(size_t)k * P + m] * b[k];
            b[m] = acc / chol[(size_t)m * P + m];
        }
        for (int m = 0; m < P; ++m) out[m] = b[m];
    }
};

// Dt[m] = h^|m| d^m psi(c) for every graded m.
static void scaled_derivs(const fc2t2_plan_s *pl, const HostIndex &ix, const double *c, double h,
                          double *out) {
    const int D = pl->D;
    if (pl->desc.kernel == FC2T2_KERNEL_GAUSSIAN) {
        double g[3][kMaxOrder + 1];
        for (int d = 0; d < D; ++d) gaussian_scaled_derivs_1d(pl->desc.sigma, h, c[d], ix.rho, g[d]);
        for (int k = 0; k < ix.P; ++k) {
            double v = 1.0;
            for (int d = 0; d < D; ++d) v *= g[d][ix.e[3 * k + d]];
            out[k] = v;
        }
        return;
    }
    // polynomial psi = sum_a coef_a x^a  (graded coefficients of some degree pdeg)
    int pdeg = 0;
    while (ncoef(D, pdeg) < (int)pl->poly.size()) ++pdeg;
    HostIndex px(D, pdeg);
    for (int k = 0; k < ix.P; ++k) {
        double acc = 0.0;
        for (int a = 0; a < (int)pl->poly.size(); ++a) {
            double term = pl->poly[a];
            if (term == 0.0) continue;
            for (int d = 0; d < D; ++d) {
                const int ad = px.e[3 * a + d], md = ix.e[3 * k + d];
                if (ad < md) { term = 0.0; break; }
                double fall = 1.0;   // ad! / (ad - md)!
                for (int t = ad - md + 1; t <= ad; ++t) fall *= t;
                double pw = 1.0;
                for (int t = 0; t < ad - md; ++t) pw *= c[d];
                term *= fall * pw;
            }
            acc += term;
        }
        double hp = 1.0;
        for (int t = 0; t < ix.deg[k]; ++t) hp *= h;
        out[k] = acc * hp;
    }
}

template <typename T>
static fc2t2_status dev_alloc(T **p, size_t count, const char *what) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(FC2T2_ERR_OOM, std::string("cudaMalloc failed for ") + what);
    }
    return FC2T2_OK;
}

template <typename T>
static fc2t2_status upload(T *dst, const std::vector<T> &src, const char *what) {
    if (src.empty()) return FC2T2_OK;
    return check_cuda(cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice), what);
}

static void free_sort(SortWork &w) {
    cudaFree(w.count); cudaFree(w.start); cudaFree(w.key); cudaFree(w.rank);
    cudaFree(w.perm); cudaFree(w.rec);
    w = SortWork();
}

static fc2t2_status alloc_sort(SortWork &w, int64_t cap, int64_t G0, int D) {
    w.cap = cap;
    fc2t2_status st;
    if ((st = dev_alloc(&w.count, G0, "cell counts")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&w.start, G0 + 1, "cell starts")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&w.key, cap, "keys")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&w.rank, cap, "ranks")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&w.perm, cap, "permutation")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&w.rec, cap, "sorted points")) != FC2T2_OK) return st;
    return FC2T2_OK;
}

static void destroy(fc2t2_plan_s *pl) {
    if (!pl) return;
    for (auto &pr : pl->pending) { cudaEventDestroy(pr.a); cudaEventDestroy(pr.b); }
    for (auto e : pl->event_pool) cudaEventDestroy(e);
    if (pl->side) cudaStreamDestroy(pl->side);
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    if (pl->ev_sorted) cudaEventDestroy(pl->ev_sorted);
    if (pl->run) cudaStreamDestroy(pl->run);
    if (pl->ev_run_fork) cudaEventDestroy(pl->ev_run_fork);
    if (pl->ev_run_done) cudaEventDestroy(pl->ev_run_done);
    cudaFree(pl->d_M); cudaFree(pl->d_L); cudaFree(pl->d_hold); cudaFree(pl->d_dtab);
    cudaFree(pl->d_scan_tmp); cudaFree(pl->d_flags); cudaFree(pl->d_over); cudaFree(pl->d_over_ctr);
    cudaFree(pl->d_mma_ops);
    for (int l = 0; l < kMaxLevels; ++l) cudaFree(pl->tc.packed[l]);
    cudaFree(pl->sep.d_t);
    cudaFree(pl->occ.act); cudaFree(pl->occ.list); cudaFree(pl->occ.cnt); cudaFree(pl->occ.chunk_off);
    cudaFree(pl->occ.next); cudaFree(pl->occ.d_inst);
    free_sort(pl->src);
    free_sort(pl->qry);
    delete pl;
}

// M2L over occupied cells: occupancy bytes, target lists, the work queue, and the plan's
// descriptor for the queue's kernel (device memory, written once)
static fc2t2_status build_occ(fc2t2_plan_s *pl) {
    auto &o = pl->occ;
    fc2t2_status st;
    if ((st = dev_alloc(&o.act, (size_t)pl->G_total, "occupancy")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&o.list, (size_t)pl->G_total, "occupied targets")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&o.cnt, (size_t)kOccBuckets, "occupied target counts")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&o.chunk_off, (size_t)kOccMaxInst * kOccBuckets + 1, "work queue")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&o.next, (size_t)1, "work counter")) != FC2T2_OK) return st;
    if ((st = dev_alloc(&o.d_inst, (size_t)1, "queue descriptor")) != FC2T2_OK) return st;
    OccInst h{};
    h.M = pl->d_M;
    h.L = pl->d_L;
    h.dtab = pl->d_dtab;
    h.act = o.act;
    h.list = o.list;
    h.cnt = o.cnt;
    h.nlev = pl->nlev;
    h.n0 = pl->n;
    for (int l = 0; l < pl->nlev; ++l) h.off[l] = pl->lev[l].off;
    if ((st = check_cuda(cudaMemcpy(o.d_inst, &h, sizeof(h), cudaMemcpyHostToDevice), "upload queue descriptor")) != FC2T2_OK)
        return st;
    // the series of cells without targets are never read; zero them once so that they are finite
    if ((st = check_cuda(cudaMemset(pl->d_L, 0, sizeof(float) * (size_t)pl->G_total * pl->Pp), "clear locals")) != FC2T2_OK)
        return st;
    o.enabled = 1;
    return FC2T2_OK;
}

static fc2t2_status build_tables(fc2t2_plan_s *pl) {
    const int D = pl->D, rho = pl->rho, P = pl->P, Pp = pl->Pp;
    HostIndex ix(D, rho);
    const int nofs = D == 3 ? 343 : 49;

    // scaled kernel derivatives per level and offset o in {-3..3}^D
    std::vector<float> dtab((size_t)pl->nlev * nofs * Pp, 0.0f);
    std::vector<double> dtab64((size_t)pl->nlev * nofs * P, 0.0);
    std::vector<double> tmp(P);
    std::unique_ptr<LsqFit> fit;
    if (pl->desc.fit) fit.reset(new LsqFit(pl, ix));
    for (int l = 0; l < pl->nlev; ++l) {
        const double h = pl->lev[l].h;
        for (int o = 0; o < nofs; ++o) {
            double c[3] = {0, 0, 0};
            int r = o;
            for (int d = 0; d < D; ++d) { c[d] = (double)(r % 7 - 3) * h; r /= 7; }
            if (fit) fit->scaled(pl, c, h, tmp.data());
            else scaled_derivs(pl, ix, c, h, tmp.data());
            for (int k = 0; k < P; ++k) {
                dtab[((size_t)l * nofs + o) * Pp + k] = (float)tmp[k];
                dtab64[((size_t)l * nofs + o) * P + k] = tmp[k];
            }
        }
    }
    fc2t2_status st;
    if ((st = dev_alloc(&pl->d_dtab, dtab.size(), "derivative tables")) != FC2T2_OK) return st;
    if ((st = upload(pl->d_dtab, dtab, "upload derivative tables")) != FC2T2_OK) return st;
    // tensor-core operator images (3D; other dimensions keep the CUDA-core M2L)
    if (pl->desc.m2l == FC2T2_M2L_SEPARABLE) return build_sep(pl, dtab64);
    if (pl->desc.m2l == FC2T2_M2L_OCCUPIED) return build_occ(pl);
    if (pl->desc.m2l != FC2T2_M2L_FP32 && D == 3)
        if ((st = build_tc_operators(pl, dtab64)) != FC2T2_OK) return st;
    return FC2T2_OK;
}

static fc2t2_status validate_desc(const fc2t2_plan_desc *d) {
    if (!d) return set_error(FC2T2_ERR_INVALID_ARG, "desc is NULL");
    if (d->dim != 2 && d->dim != 3) return set_error(FC2T2_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (d->grid < 4 || d->grid > 1024 || (d->grid & (d->grid - 1)))
        return set_error(FC2T2_ERR_INVALID_ARG, "grid must be a power of two in [4, 1024]");
    if (d->order < 1 || d->order > kMaxOrder)
        return set_error(FC2T2_ERR_INVALID_ARG, "order must be in [1, 8]");
    if (!(d->hi > d->lo) || !std::isfinite(d->lo) || !std::isfinite(d->hi))
        return set_error(FC2T2_ERR_INVALID_ARG, "domain must satisfy lo < hi, both finite");
    if (d->kernel == FC2T2_KERNEL_GAUSSIAN) {
        if (!(d->sigma > 0.0) || !std::isfinite(d->sigma))
            return set_error(FC2T2_ERR_INVALID_ARG, "sigma must be positive");
    } else if (d->kernel == FC2T2_KERNEL_POLY) {
        if (!d->poly_coef || d->n_poly < 1)
            return set_error(FC2T2_ERR_INVALID_ARG, "polynomial kernel needs coefficients");
        int deg = 0;
        while (ncoef(d->dim, deg) < d->n_poly && deg < 64) ++deg;
        if (ncoef(d->dim, deg) != d->n_poly)
            return set_error(FC2T2_ERR_INVALID_ARG, "n_poly must be C(deg + dim, dim)");
    } else {
        return set_error(FC2T2_ERR_INVALID_ARG, "unknown kernel");
    }
    if (d->channels < 1 || d->channels > 4096) return set_error(FC2T2_ERR_INVALID_ARG, "channels must be in [1, 4096]");
    if (d->m2l != FC2T2_M2L_FP32 && d->m2l != FC2T2_M2L_TF32 && d->m2l != FC2T2_M2L_BF16 &&
        d->m2l != FC2T2_M2L_TF32X3 && d->m2l != FC2T2_M2L_BF16X3 && d->m2l != FC2T2_M2L_SEPARABLE &&
        d->m2l != FC2T2_M2L_OCCUPIED)
        return set_error(FC2T2_ERR_UNSUPPORTED, "unknown M2L precision");
    if (d->m2l == FC2T2_M2L_SEPARABLE && (d->kernel != FC2T2_KERNEL_GAUSSIAN || d->dim != 3))
        return set_error(FC2T2_ERR_UNSUPPORTED, "the separable M2L needs the Gaussian kernel and dim = 3");
    if (d->fit != 0 && d->fit != 1) return set_error(FC2T2_ERR_INVALID_ARG, "fit must be 0 or 1");
    if (d->tile != 0 && d->tile != 16 && d->tile != 32 && d->tile != 64)
        return set_error(FC2T2_ERR_INVALID_ARG, "tile must be 0, 16, 32 or 64");
    if (d->fit && d->m2l == FC2T2_M2L_SEPARABLE)
        return set_error(FC2T2_ERR_UNSUPPORTED, "fitted operators do not factor per dimension (no separable M2L)");
    if (d->max_sources < 0 || d->max_queries < 0 || d->max_sources > (int64_t)INT32_MAX ||
        d->max_queries > (int64_t)INT32_MAX)
        return set_error(FC2T2_ERR_INVALID_ARG, "max_sources / max_queries out of range");
    int64_t G = 1;
    for (int i = 0; i < d->dim; ++i) G *= d->grid;
    if (G > (int64_t)1 << 30) return set_error(FC2T2_ERR_INVALID_ARG, "grid too large");
    return FC2T2_OK;
}

// flags[0]: domain (cleared by every call); flags[2]: a bounded device-side wait gave up (sticky
// until fc2t2_plan_check; bit 2048: the CUDA-core M2L's staging, 1024 / 512: P2M's / L2P's, the
// low bits: the tensor-core M2L's pipeline)
static fc2t2_status read_flags(fc2t2_plan_s *pl, cudaStream_t s, bool clear_sticky) {
    int flags[3] = {0, 0, 0};
    fc2t2_status st = check_cuda(cudaMemcpyAsync(flags, pl->d_flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, s),
                                 "read flags");
    if (st != FC2T2_OK) return st;
    if (clear_sticky &&
        (st = check_cuda(cudaMemsetAsync(pl->d_flags + 2, 0, sizeof(int), s), "clear flags")) != FC2T2_OK)
        return st;
    st = check_cuda(cudaStreamSynchronize(s), "synchronise");
    if (st != FC2T2_OK) return st;
    if (flags[2])
        return set_error(FC2T2_ERR_TIMEOUT, "a bounded device-side wait gave up (code " + std::to_string(flags[2]) + ")");
    if (pl->desc.check_domain && (flags[0] & 1)) return set_error(FC2T2_ERR_DOMAIN, "a point lies outside [lo, hi)^dim");
    return FC2T2_OK;
}

static fc2t2_status finish_flags(fc2t2_plan_s *pl, cudaStream_t s) {
    if (!pl->desc.check_domain) return FC2T2_OK;
    return read_flags(pl, s, false);
}

// ---------------------------------------------------------------- stage profiling

static cudaEvent_t take_event(fc2t2_plan_s *pl) {
    if (!pl->event_pool.empty()) {
        cudaEvent_t e = pl->event_pool.back();
        pl->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

// Records an event pair around a stage's launches on the call's stream while profiling.
struct StageScope {
    fc2t2_plan_s *pl;
    cudaStream_t s;
    int stage;
    cudaEvent_t a = nullptr;
    StageScope(fc2t2_plan_s *pl_, cudaStream_t s_, int stage_) : pl(pl_), s(s_), stage(stage_) {
        if (pl->profiling && (a = take_event(pl)) != nullptr) cudaEventRecord(a, s);
    }
    ~StageScope() {
        if (!a) return;
        cudaEvent_t b = take_event(pl);
        if (!b) { pl->event_pool.push_back(a); return; }
        cudaEventRecord(b, s);
        pl->pending.push_back({stage, a, b});
    }
};

// bin + sort points (weights optional) into a sort workspace
static fc2t2_status sort_points(fc2t2_plan_s *pl, cudaStream_t s, const float *x, const float *wt,
                                int64_t n, SortWork &w) {
    StageScope scope(pl, s, FC2T2_STAGE_SORT);
    fc2t2_status st;
    if ((st = check_cuda(launch_bin_count(pl, s, x, n, w), "bin")) != FC2T2_OK) return st;
    if ((st = check_cuda(launch_scan(pl, s, w.count, w.start, pl->lev[0].G, w.scan_tmp), "scan")) != FC2T2_OK) return st;
    w.held_x = nullptr;
    w.held_n = -1;
    if ((st = check_cuda(launch_scatter(pl, s, x, wt, n, w), "scatter")) != FC2T2_OK) return st;
    w.held_x = x;
    w.held_w = wt;
    w.held_n = n;
    return FC2T2_OK;
}

// Whether an expansion runs the levels above the finest on the plan's second stream (separable
// M2L; stage profiling keeps everything on the call's stream, in order)
static bool forks(const fc2t2_plan_s *pl) {
    return pl->sep.enabled && pl->side && !pl->profiling && pl->nlev > 1;
}

// Sort the targets of a transform.  When the expansion forks, the sort runs on the second stream
// (ahead of the levels above the finest): only L2P reads it, after the join.  wait_targets()
// makes the call's stream wait for it before L2P.
static fc2t2_status sort_targets(fc2t2_plan_s *pl, cudaStream_t s, const float *x, const float *wt, int64_t n,
                                 SortWork &w) {
    if (!forks(pl)) return sort_points(pl, s, x, wt, n, w);
    fc2t2_status st;
    if ((st = check_cuda(cudaEventRecord(pl->ev_fork, s), "fork")) != FC2T2_OK) return st;
    if ((st = check_cuda(cudaStreamWaitEvent(pl->side, pl->ev_fork, 0), "fork")) != FC2T2_OK) return st;
    if ((st = sort_points(pl, pl->side, x, wt, n, w)) != FC2T2_OK) return st;
    return check_cuda(cudaEventRecord(pl->ev_sorted, pl->side), "join");
}

static fc2t2_status wait_targets(fc2t2_plan_s *pl, cudaStream_t s) {
    return forks(pl) ? check_cuda(cudaStreamWaitEvent(s, pl->ev_sorted, 0), "join") : FC2T2_OK;
}

// the weights of channel `wt` gathered into an existing sort
static fc2t2_status reweight(fc2t2_plan_s *pl, cudaStream_t s, const float *wt, int64_t n, SortWork &w) {
    StageScope scope(pl, s, FC2T2_STAGE_SORT);
    return check_cuda(launch_reweight(pl, s, wt, n, w), "reweight");
}

static fc2t2_status clear_flags(fc2t2_plan_s *pl, cudaStream_t s) {
    pl->expansion_held = false;
    return check_cuda(cudaMemsetAsync(pl->d_flags, 0, 2 * sizeof(int), s), "clear flags");
}

// Whether a transform with `targets` evaluation points skips the finest level's L2L and
// evaluates the finest level's own M2L series plus level 1's local series at the points
// (launch_l2p_two; the same result up to rounding, as L2L is an exact re-centring).  That trades
// the L2L pass over every finest coefficient row for one more series per target: worth it up to
// several targets per finest cell (more at orders 7-8, whose L2L is slower per row).
static bool l2p_two_levels(const fc2t2_plan_s *pl, int64_t targets) {
    const int64_t per_cell = pl->rho >= 7 ? 32 : 8;
    return pl->nlev > 1 && targets <= per_cell * pl->lev[0].G;
}

// L2P (value and/or gradient times weight) of the sorted targets w after expand()
static fc2t2_status evaluate_targets(fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m, bool two,
                                     float *val, float *grad, bool accumulate) {
    StageScope scope(pl, s, FC2T2_STAGE_L2P);
    return check_cuda(two ? launch_l2p_two(pl, s, w, m, val, grad, accumulate)
                             : launch_l2p(pl, s, w, m, val, grad, accumulate),
                      "l2p");
}

// P2M .. M2L .. L2L: expansion of sorted sources into local coefficients: with l2l, the finest
// level's rows of d_L hold the whole local series; without, L2L stops at level 1 and the finest
// level's rows hold its own M2L only (for launch_l2p_two)
static fc2t2_status expand(fc2t2_plan_s *pl, cudaStream_t s, const SortWork *src, const SortWork *tgt,
                           bool l2l = true) {
    fc2t2_status st;
    if (src) {   // (NULL: the finest moments are already in place, e.g. from ray2M)
        StageScope scope(pl, s, FC2T2_STAGE_P2M);
        if ((st = check_cuda(launch_p2m(pl, s, *src, pl->d_M), "p2m")) != FC2T2_OK) return st;
    }
    if (pl->occ.enabled) {   // which cells hold sources / have targets below them (NULL: all)
        StageScope scope(pl, s, FC2T2_STAGE_M2L);
        if ((st = check_cuda(launch_occupancy(pl, s, src ? src->count : nullptr, tgt ? tgt->count : nullptr),
                             "occupancy")) != FC2T2_OK)
            return st;
    }
    if (forks(pl)) {
        // The finest level's M2L needs only the finest moments; everything above it (M2M, the
        // coarser levels' M2L, L2L down to level 1) is a chain of small launches.  The chain runs
        // on the plan's high-priority second stream beside the finest level's passes, joined
        // before the finest L2L / L2P.  (Stage profiling keeps the serial order below.)
        if ((st = check_cuda(cudaEventRecord(pl->ev_fork, s), "fork")) != FC2T2_OK) return st;
        if ((st = check_cuda(cudaStreamWaitEvent(pl->side, pl->ev_fork, 0), "fork")) != FC2T2_OK) return st;
        for (int l = 0; l + 1 < pl->nlev; ++l)
            if ((st = check_cuda(launch_m2m(pl, pl->side, l), "m2m")) != FC2T2_OK) return st;
        if ((st = check_cuda(launch_m2l_sep(pl, pl->side, 2), "m2l (separable, coarser levels)")) != FC2T2_OK)
            return st;
        for (int l = pl->nlev - 2; l >= 1; --l)
            if ((st = check_cuda(launch_l2l(pl, pl->side, l), "l2l")) != FC2T2_OK) return st;
        if ((st = check_cuda(cudaEventRecord(pl->ev_join, pl->side), "join")) != FC2T2_OK) return st;
        if ((st = check_cuda(launch_m2l_sep(pl, s, 1), "m2l (separable, finest level)")) != FC2T2_OK) return st;
        if ((st = check_cuda(cudaStreamWaitEvent(s, pl->ev_join, 0), "join")) != FC2T2_OK) return st;
        if (l2l && (st = check_cuda(launch_l2l(pl, s, 0), "l2l")) != FC2T2_OK) return st;
        return FC2T2_OK;
    }
    {
        StageScope scope(pl, s, FC2T2_STAGE_M2M);
        for (int l = 0; l + 1 < pl->nlev; ++l)
            if ((st = check_cuda(launch_m2m(pl, s, l), "m2m")) != FC2T2_OK) return st;
    }
    // M2L of every level (independent given the moments): the tensor-core levels in one launch,
    // the others on the CUDA cores; then L2L from the coarsest level down
    if (pl->tc.enabled) {
        StageScope scope(pl, s, FC2T2_STAGE_M2L_PACK);
        if ((st = check_cuda(launch_tc_pack(pl, s), "m2l operand pack")) != FC2T2_OK) return st;
    }
    {
        StageScope scope(pl, s, FC2T2_STAGE_M2L);
        if (pl->sep.enabled) {
            if ((st = check_cuda(launch_m2l_sep(pl, s), "m2l (separable)")) != FC2T2_OK) return st;
        } else if (pl->occ.enabled) {
            const fc2t2_plan_s *one = pl;
            if ((st = check_cuda(launch_m2l_occ(&one, 1, s), "m2l (occupied cells)")) != FC2T2_OK) return st;
        } else {
            if (pl->tc.enabled && (st = check_cuda(launch_m2l_tc_all(pl, s), "m2l (tensor cores)")) != FC2T2_OK)
                return st;
            for (int l = pl->nlev - 1; l >= 0; --l)
                if (!(pl->tc.enabled && pl->tc.level_ok[l]))
                    if ((st = check_cuda(launch_m2l(pl, s, l), "m2l")) != FC2T2_OK) return st;
        }
    }
    for (int l = pl->nlev - 2; l >= (l2l ? 0 : 1); --l) {
        StageScope scope(pl, s, FC2T2_STAGE_L2L);
        if ((st = check_cuda(launch_l2l(pl, s, l), "l2l")) != FC2T2_OK) return st;
    }
    return FC2T2_OK;
}

}  // namespace fc2t2

using namespace fc2t2;

extern "C" {

fc2t2_status fc2t2_plan_create(const fc2t2_plan_desc *desc, fc2t2_plan *out) {
    if (!out) return set_error(FC2T2_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    fc2t2_status st = validate_desc(desc);
    if (st != FC2T2_OK) return st;
    fc2t2_plan_s *pl = new (std::nothrow) fc2t2_plan_s();
    if (!pl) return set_error(FC2T2_ERR_OOM, "host allocation failed");
    pl->desc = *desc;
    if (desc->kernel == FC2T2_KERNEL_POLY) pl->poly.assign(desc->poly_coef, desc->poly_coef + desc->n_poly);
    pl->desc.poly_coef = nullptr;
    pl->D = desc->dim;
    pl->n = desc->grid;
    pl->rho = desc->order;
    pl->C = desc->channels;
    pl->P = ncoef(pl->D, pl->rho);
    pl->Pp = pad4(pl->P);
    int lg = 0;
    while ((1 << lg) < pl->n) ++lg;
    pl->nlev = lg - 1;
    int64_t off = 0;
    for (int l = 0; l < pl->nlev; ++l) {
        Level &lv = pl->lev[l];
        lv.n = pl->n >> l;
        lv.G = 1;
        for (int d = 0; d < pl->D; ++d) lv.G *= lv.n;
        lv.off = off;
        lv.h = (desc->hi - desc->lo) / lv.n;
        off += lv.G;
    }
    pl->G_total = off;
    pl->lo_f = (float)desc->lo;
    pl->hi_f = (float)desc->hi;
    pl->scale0_f = (float)((double)pl->n / (desc->hi - desc->lo));

    if ((st = dev_alloc(&pl->d_M, (size_t)pl->G_total * pl->Pp, "moments")) != FC2T2_OK) { destroy(pl); return st; }
    if ((st = dev_alloc(&pl->d_L, (size_t)pl->G_total * pl->Pp, "locals")) != FC2T2_OK) { destroy(pl); return st; }
    if (pl->C > 1 &&
        (st = dev_alloc(&pl->d_hold, (size_t)pl->C * pl->lev[0].G * pl->Pp, "channel expansions")) != FC2T2_OK) {
        destroy(pl);
        return st;
    }
    if ((st = dev_alloc(&pl->d_flags, 4, "flags")) != FC2T2_OK) { destroy(pl); return st; }
    const int64_t G0 = pl->lev[0].G;
    int64_t tiles = (G0 + 4095) / 4096, tmp = 16;
    while (tiles > 1) { tmp += 2 * tiles + 1; tiles = (tiles + 4095) / 4096; }
    pl->scan_tmp_len = tmp;
    if ((st = dev_alloc(&pl->d_scan_tmp, 2 * (size_t)tmp, "scan workspace")) != FC2T2_OK) { destroy(pl); return st; }
    if ((st = dev_alloc(&pl->d_over, (size_t)G0, "P2M overflow list")) != FC2T2_OK ||
        (st = dev_alloc(&pl->d_over_ctr, 2, "P2M overflow counters")) != FC2T2_OK ||
        (st = check_cuda(cudaMemset(pl->d_over_ctr, 0, 2 * sizeof(unsigned long long)), "clear counters")) != FC2T2_OK) {
        destroy(pl);
        return st;
    }
    if ((st = alloc_sort(pl->src, desc->max_sources, G0, pl->D)) != FC2T2_OK) { destroy(pl); return st; }
    if ((st = alloc_sort(pl->qry, desc->max_queries, G0, pl->D)) != FC2T2_OK) { destroy(pl); return st; }
    pl->src.scan_tmp = pl->d_scan_tmp;
    pl->qry.scan_tmp = pl->d_scan_tmp + tmp;
    if ((st = build_tables(pl)) != FC2T2_OK) { destroy(pl); return st; }
    if ((st = check_cuda(cudaStreamCreateWithFlags(&pl->run, cudaStreamNonBlocking), "stream")) != FC2T2_OK ||
        (st = check_cuda(cudaEventCreateWithFlags(&pl->ev_run_fork, cudaEventDisableTiming), "event")) != FC2T2_OK ||
        (st = check_cuda(cudaEventCreateWithFlags(&pl->ev_run_done, cudaEventDisableTiming), "event")) != FC2T2_OK) {
        destroy(pl);
        return st;
    }
    if (pl->sep.enabled) {
        int lo_prio = 0, hi_prio = 0;
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        if ((st = check_cuda(cudaStreamCreateWithPriority(&pl->side, cudaStreamNonBlocking, hi_prio), "stream")) != FC2T2_OK ||
            (st = check_cuda(cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming), "event")) != FC2T2_OK ||
            (st = check_cuda(cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming), "event")) != FC2T2_OK ||
            (st = check_cuda(cudaEventCreateWithFlags(&pl->ev_sorted, cudaEventDisableTiming), "event")) != FC2T2_OK) {
            destroy(pl);
            return st;
        }
    }
    if ((st = check_cuda(cudaMemset(pl->d_flags, 0, 4 * sizeof(int)), "clear flags")) != FC2T2_OK) { destroy(pl); return st; }
    if ((st = check_cuda(cudaDeviceSynchronize(), "plan build")) != FC2T2_OK) { destroy(pl); return st; }
    *out = pl;
    return FC2T2_OK;
}

fc2t2_status fc2t2_plan_destroy(fc2t2_plan plan) {
    destroy(plan);
    return FC2T2_OK;
}

fc2t2_status fc2t2_forward(fc2t2_plan pl, void *stream, const float *p, const float *w, int64_t N,
                           const float *q, int64_t M, float *y) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    if (N < 0 || M < 0 || N > pl->src.cap || M > pl->qry.cap)
        return set_error(FC2T2_ERR_INVALID_ARG, "N or M outside [0, max]");
    if (M == 0) return FC2T2_OK;
    if (!q || !y || (N > 0 && (!p || !w))) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    const int C = pl->C;
    fc2t2_status st;
    if ((st = clear_flags(pl, s)) != FC2T2_OK) return st;
    if (N == 0) {
        if ((st = check_cuda(cudaMemsetAsync(y, 0, sizeof(float) * M * C, s), "zero y")) != FC2T2_OK) return st;
        if ((st = sort_points(pl, s, q, nullptr, M, pl->qry)) != FC2T2_OK) return st;   // domain check
        return finish_flags(pl, s);
    }
    if ((st = sort_targets(pl, s, q, nullptr, M, pl->qry)) != FC2T2_OK) return st;
    if ((st = sort_points(pl, s, p, w, N, pl->src)) != FC2T2_OK) return st;
    // one expansion per channel on the shared sorts
    const bool two = l2p_two_levels(pl, M);
    for (int c = 0; c < C; ++c) {
        if (c > 0 && (st = reweight(pl, s, w + (int64_t)c * N, N, pl->src)) != FC2T2_OK) return st;
        if ((st = expand(pl, s, &pl->src, &pl->qry, !two)) != FC2T2_OK) return st;
        if (c == 0 && (st = wait_targets(pl, s)) != FC2T2_OK) return st;
        if ((st = evaluate_targets(pl, s, pl->qry, M, two, y + (int64_t)c * M, nullptr, false)) != FC2T2_OK)
            return st;
    }
    pl->src.held_w = w;   // the sort of (p, w); later channels re-gather their weights
    return finish_flags(pl, s);
}

fc2t2_status fc2t2_backward(fc2t2_plan pl, void *stream, const float *p, const float *w, int64_t N,
                            const float *q, int64_t M, const float *ybar, float *wbar, float *pbar) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    if (N < 0 || M < 0 || N > pl->src.cap || M > pl->qry.cap)
        return set_error(FC2T2_ERR_INVALID_ARG, "N or M outside [0, max]");
    if (N == 0 || (!wbar && !pbar)) return FC2T2_OK;
    if (!p || !w || (M > 0 && (!q || !ybar))) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    const int C = pl->C;
    fc2t2_status st;
    if ((st = clear_flags(pl, s)) != FC2T2_OK) return st;
    if (M == 0) {
        if (wbar && (st = check_cuda(cudaMemsetAsync(wbar, 0, sizeof(float) * N * C, s), "zero wbar")) != FC2T2_OK) return st;
        if (pbar && (st = check_cuda(cudaMemsetAsync(pbar, 0, sizeof(float) * N * pl->D, s), "zero pbar")) != FC2T2_OK) return st;
        if ((st = sort_points(pl, s, p, w, N, pl->src)) != FC2T2_OK) return st;
        return finish_flags(pl, s);
    }
    // the transposed transform: sources q with weights ybar, targets p (Sec. 4.1)
    if ((st = sort_targets(pl, s, p, w, N, pl->src)) != FC2T2_OK) return st;
    if ((st = sort_points(pl, s, q, ybar, M, pl->qry)) != FC2T2_OK) return st;
    const bool two = l2p_two_levels(pl, N);
    for (int c = 0; c < C; ++c) {
        if (c > 0) {
            if ((st = reweight(pl, s, ybar + (int64_t)c * M, M, pl->qry)) != FC2T2_OK) return st;
            if (pbar && (st = reweight(pl, s, w + (int64_t)c * N, N, pl->src)) != FC2T2_OK) return st;
        }
        if ((st = expand(pl, s, &pl->qry, &pl->src, !two)) != FC2T2_OK) return st;
        if (c == 0 && (st = wait_targets(pl, s)) != FC2T2_OK) return st;
        // pbar sums the channels' contributions w[c] * grad g_c
        if ((st = evaluate_targets(pl, s, pl->src, N, two, wbar ? wbar + (int64_t)c * N : nullptr, pbar, c > 0)) !=
            FC2T2_OK)
            return st;
    }
    pl->src.held_w = w;
    return finish_flags(pl, s);
}

fc2t2_status fc2t2_backward_reuse(fc2t2_plan pl, void *stream, const float *p, const float *w, int64_t N,
                                  const float *q, int64_t M, const float *ybar, float *wbar, float *pbar) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    // the plan's workspaces must hold the forward's sorts of exactly these arrays
    const bool reuse = N > 0 && M > 0 && (wbar || pbar) && p && w && q && ybar &&
                       pl->src.held_x == p && pl->src.held_w == w && pl->src.held_n == N &&
                       pl->qry.held_x == q && pl->qry.held_n == M;
    if (!reuse) return fc2t2_backward(pl, stream, p, w, N, q, M, ybar, wbar, pbar);
    cudaStream_t s = (cudaStream_t)stream;
    const int C = pl->C;
    fc2t2_status st;
    if ((st = clear_flags(pl, s)) != FC2T2_OK) return st;
    // the transposed transform on the existing sorts: q becomes the sources with weights ybar
    const bool two = l2p_two_levels(pl, N);
    for (int c = 0; c < C; ++c) {
        if ((st = reweight(pl, s, ybar + (int64_t)c * M, M, pl->qry)) != FC2T2_OK) return st;
        // (one channel: the sort of p still carries w)
        if (C > 1 && pbar && (st = reweight(pl, s, w + (int64_t)c * N, N, pl->src)) != FC2T2_OK) return st;
        if ((st = expand(pl, s, &pl->qry, &pl->src, !two)) != FC2T2_OK) return st;
        if ((st = evaluate_targets(pl, s, pl->src, N, two, wbar ? wbar + (int64_t)c * N : nullptr, pbar, c > 0)) !=
            FC2T2_OK)
            return st;
    }
    pl->src.held_w = w;
    return finish_flags(pl, s);
}

fc2t2_status fc2t2_backward_q(fc2t2_plan pl, void *stream, const float *p, const float *w, int64_t N,
                              const float *q, int64_t M, const float *ybar, float *qbar) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    if (N < 0 || M < 0 || N > pl->src.cap || M > pl->qry.cap)
        return set_error(FC2T2_ERR_INVALID_ARG, "N or M outside [0, max]");
    if (M == 0) return FC2T2_OK;
    if (!q || !ybar || !qbar || (N > 0 && (!p || !w))) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    const int C = pl->C;
    fc2t2_status st;
    if ((st = clear_flags(pl, s)) != FC2T2_OK) return st;
    if (N == 0) {
        if ((st = check_cuda(cudaMemsetAsync(qbar, 0, sizeof(float) * M * pl->D, s), "zero qbar")) != FC2T2_OK) return st;
        if ((st = sort_points(pl, s, q, nullptr, M, pl->qry)) != FC2T2_OK) return st;   // domain check
        return finish_flags(pl, s);
    }
    // the forward expansion of (p, w), its local series differentiated at q, times ybar
    if ((st = sort_targets(pl, s, q, ybar, M, pl->qry)) != FC2T2_OK) return st;
    if ((st = sort_points(pl, s, p, w, N, pl->src)) != FC2T2_OK) return st;
    const bool two = l2p_two_levels(pl, M);
    for (int c = 0; c < C; ++c) {
        if (c > 0) {
            if ((st = reweight(pl, s, w + (int64_t)c * N, N, pl->src)) != FC2T2_OK) return st;
            if ((st = reweight(pl, s, ybar + (int64_t)c * M, M, pl->qry)) != FC2T2_OK) return st;
        }
        if ((st = expand(pl, s, &pl->src, &pl->qry, !two)) != FC2T2_OK) return st;
        if (c == 0 && (st = wait_targets(pl, s)) != FC2T2_OK) return st;
        if ((st = evaluate_targets(pl, s, pl->qry, M, two, nullptr, qbar, c > 0)) != FC2T2_OK) return st;
    }
    pl->src.held_w = w;
    pl->qry.held_w = ybar;
    return finish_flags(pl, s);
}

fc2t2_status fc2t2_ray_forward(fc2t2_plan pl, void *stream, const float *p, const float *w, int64_t N,
                               const float *rays, int64_t R, float *y) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    if (pl->D != 3) return set_error(FC2T2_ERR_UNSUPPORTED, "ray integrals need dim = 3");
    if (N < 0 || N > pl->src.cap || R < 0) return set_error(FC2T2_ERR_INVALID_ARG, "N outside [0, max_sources] or R < 0");
    if (R == 0) return FC2T2_OK;
    if (!rays || !y || (N > 0 && (!p || !w))) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    const int C = pl->C;
    fc2t2_status st;
    if ((st = clear_flags(pl, s)) != FC2T2_OK) return st;
    if (N == 0) return check_cuda(cudaMemsetAsync(y, 0, sizeof(float) * R * C, s), "zero y");
    if ((st = sort_points(pl, s, p, w, N, pl->src)) != FC2T2_OK) return st;
    for (int c = 0; c < C; ++c) {
        if (c > 0 && (st = reweight(pl, s, w + (int64_t)c * N, N, pl->src)) != FC2T2_OK) return st;
        if ((st = expand(pl, s, &pl->src, nullptr, true)) != FC2T2_OK) return st;   // the finest series, complete
        StageScope scope(pl, s, FC2T2_STAGE_L2P);
        if ((st = check_cuda(launch_ray_forward(pl, s, rays, R, y + (int64_t)c * R), "ray integrals")) != FC2T2_OK)
            return st;
    }
    pl->src.held_w = w;
    return finish_flags(pl, s);
}

fc2t2_status fc2t2_ray_backward(fc2t2_plan pl, void *stream, const float *p, const float *w, int64_t N,
                                const float *rays, int64_t R, const float *ybar, float *wbar, float *pbar) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    if (pl->D != 3) return set_error(FC2T2_ERR_UNSUPPORTED, "ray integrals need dim = 3");
    if (N < 0 || N > pl->src.cap || R < 0) return set_error(FC2T2_ERR_INVALID_ARG, "N outside [0, max_sources] or R < 0");
    if (N == 0 || (!wbar && !pbar)) return FC2T2_OK;
    if (!p || !w || (R > 0 && (!rays || !ybar))) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    const int C = pl->C;
    fc2t2_status st;
    if ((st = clear_flags(pl, s)) != FC2T2_OK) return st;
    // the transposed transform: sources = the rays with weights ybar (ray2M), targets p
    if ((st = sort_targets(pl, s, p, w, N, pl->src)) != FC2T2_OK) return st;
    const bool two = l2p_two_levels(pl, N);
    const size_t mbytes = sizeof(float) * (size_t)pl->lev[0].G * pl->Pp;
    for (int c = 0; c < C; ++c) {
        if (c > 0 && pbar && (st = reweight(pl, s, w + (int64_t)c * N, N, pl->src)) != FC2T2_OK) return st;
        {
            StageScope scope(pl, s, FC2T2_STAGE_P2M);
            if ((st = check_cuda(cudaMemsetAsync(pl->d_M, 0, mbytes, s), "zero moments")) != FC2T2_OK) return st;
            if ((st = check_cuda(launch_ray2m(pl, s, rays, R, ybar + (int64_t)c * R, pl->d_M), "ray2M")) != FC2T2_OK)
                return st;
        }
        if ((st = expand(pl, s, nullptr, &pl->src, !two)) != FC2T2_OK) return st;
        if (c == 0 && (st = wait_targets(pl, s)) != FC2T2_OK) return st;
        if ((st = evaluate_targets(pl, s, pl->src, N, two, wbar ? wbar + (int64_t)c * N : nullptr, pbar, c > 0)) !=
            FC2T2_OK)
            return st;
    }
    pl->src.held_w = w;
    return finish_flags(pl, s);
}

fc2t2_status fc2t2_expand(fc2t2_plan pl, void *stream, const float *p, const float *w, int64_t N) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    if (N < 0 || N > pl->src.cap) return set_error(FC2T2_ERR_INVALID_ARG, "N outside [0, max_sources]");
    if (N > 0 && (!p || !w)) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    const int C = pl->C;
    const size_t row_floats = (size_t)pl->lev[0].G * pl->Pp;   // one channel's finest locals
    float *hold = C > 1 ? pl->d_hold : pl->d_L;
    fc2t2_status st;
    if ((st = clear_flags(pl, s)) != FC2T2_OK) return st;
    if (N == 0) {
        if ((st = check_cuda(cudaMemsetAsync(hold, 0, sizeof(float) * row_floats * C, s), "zero field")) != FC2T2_OK)
            return st;
        pl->expansion_held = true;
        return FC2T2_OK;
    }
    if ((st = sort_points(pl, s, p, w, N, pl->src)) != FC2T2_OK) return st;
    for (int c = 0; c < C; ++c) {
        if (c > 0 && (st = reweight(pl, s, w + (int64_t)c * N, N, pl->src)) != FC2T2_OK) return st;
        if ((st = expand(pl, s, &pl->src, nullptr)) != FC2T2_OK) return st;
        // (one channel: the finest level of d_L is the held expansion)
        if (C > 1 && (st = check_cuda(cudaMemcpyAsync(hold + (size_t)c * row_floats, pl->d_L, sizeof(float) * row_floats,
                                                      cudaMemcpyDeviceToDevice, s),
                                      "keep channel expansion")) != FC2T2_OK)
            return st;
    }
    pl->src.held_w = w;
    if ((st = finish_flags(pl, s)) != FC2T2_OK) return st;
    pl->expansion_held = true;
    return FC2T2_OK;
}

fc2t2_status fc2t2_evaluate(fc2t2_plan pl, void *stream, const float *q, int64_t M, fc2t2_eval what, float *out) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    if (what != FC2T2_EVAL_VALUE && what != FC2T2_EVAL_PARTIALS && what != FC2T2_EVAL_PARTIALS2)
        return set_error(FC2T2_ERR_INVALID_ARG, "unknown evaluation");
    if (!pl->expansion_held) return set_error(FC2T2_ERR_INVALID_ARG, "no expansion held (call fc2t2_expand first)");
    if (M < 0 || M > pl->qry.cap) return set_error(FC2T2_ERR_INVALID_ARG, "M outside [0, max_queries]");
    if (M == 0) return FC2T2_OK;
    if (!q || !out) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    fc2t2_status st;
    if ((st = check_cuda(cudaMemsetAsync(pl->d_flags, 0, 2 * sizeof(int), s), "clear flags")) != FC2T2_OK) return st;
    if ((st = sort_points(pl, s, q, nullptr, M, pl->qry)) != FC2T2_OK) return st;
    {
        StageScope scope(pl, s, FC2T2_STAGE_L2P);
        if ((st = check_cuda(launch_eval_sorted(pl, s, pl->qry, M, pl->C > 1 ? pl->d_hold : pl->d_L, pl->C, (int)what, out),
                             "evaluate")) != FC2T2_OK)
            return st;
    }
    return finish_flags(pl, s);
}

fc2t2_status fc2t2_evaluate_grid(fc2t2_plan pl, void *stream, const float *const *axis, const int64_t *count,
                                 fc2t2_eval what, float *out) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    if (what != FC2T2_EVAL_VALUE && what != FC2T2_EVAL_PARTIALS && what != FC2T2_EVAL_PARTIALS2)
        return set_error(FC2T2_ERR_INVALID_ARG, "unknown evaluation");
    if (!pl->expansion_held) return set_error(FC2T2_ERR_INVALID_ARG, "no expansion held (call fc2t2_expand first)");
    if (!axis || !count) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    int64_t total = 1;
    for (int d = 0; d < pl->D; ++d) {
        if (count[d] < 0) return set_error(FC2T2_ERR_INVALID_ARG, "negative axis length");
        if (count[d] > 0 && !axis[d]) return set_error(FC2T2_ERR_INVALID_ARG, "NULL axis");
        if (count[d] > 0 && total > ((int64_t)1 << 40) / count[d])
            return set_error(FC2T2_ERR_INVALID_ARG, "grid of more than 2^40 points");
        total *= count[d];
    }
    if (total == 0) return FC2T2_OK;
    if (!out) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    StageScope scope(pl, s, FC2T2_STAGE_L2P);
    return check_cuda(launch_eval_grid(pl, s, axis, count, pl->C > 1 ? pl->d_hold : pl->d_L, pl->C, (int)what, out),
                      "evaluate on a grid");
}

fc2t2_status fc2t2_plan_check(fc2t2_plan pl, void *stream) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    return read_flags(pl, static_cast<cudaStream_t>(stream), true);
}

fc2t2_status fc2t2_profile_enable(fc2t2_plan pl, int enable) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    pl->profiling = enable != 0;
    return FC2T2_OK;
}

fc2t2_status fc2t2_profile_read(fc2t2_plan pl, double *ms, int64_t *launches, int reset) {
    if (!pl) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    fc2t2_status st = FC2T2_OK;
    for (auto &pr : pl->pending) {
        float t = 0.0f;
        if (st == FC2T2_OK) st = check_cuda(cudaEventSynchronize(pr.b), "profile sync");
        if (st == FC2T2_OK) st = check_cuda(cudaEventElapsedTime(&t, pr.a, pr.b), "profile time");
        pl->stage_ms[pr.stage] += t;
        pl->event_pool.push_back(pr.a);
        pl->event_pool.push_back(pr.b);
    }
    pl->pending.clear();
    for (int i = 0; i < FC2T2_NUM_STAGES; ++i) {
        if (ms) ms[i] = pl->stage_ms[i];
        if (launches) launches[i] = pl->launches[i];
        if (reset) { pl->stage_ms[i] = 0.0; pl->launches[i] = 0; }
    }
    return st;
}

namespace {

// Fork the call's stream into the stream of every distinct plan of a batch (in order of first
// appearance), so instances of different plans run side by side; join them back at the end.
std::atomic<uint64_t> g_batch_counter{0};

fc2t2_status batch_fork(int n_inst, const fc2t2_plan *plans, cudaStream_t s, uint64_t mark) {
    for (int i = 0; i < n_inst; ++i) {
        fc2t2_plan_s *pl = plans[i];
        if (pl->batch_mark == mark) continue;
        pl->batch_mark = mark;
        fc2t2_status st;
        if ((st = check_cuda(cudaEventRecord(pl->ev_run_fork, s), "fork")) != FC2T2_OK) return st;
        if ((st = check_cuda(cudaStreamWaitEvent(pl->run, pl->ev_run_fork, 0), "fork")) != FC2T2_OK) return st;
    }
    return FC2T2_OK;
}

fc2t2_status batch_join(int n_inst, const fc2t2_plan *plans, cudaStream_t s, uint64_t mark) {
    fc2t2_status first = FC2T2_OK;
    for (int i = 0; i < n_inst; ++i) {   // (every forked stream rejoins, even after an error)
        fc2t2_plan_s *pl = plans[i];
        if (pl->batch_mark != mark) continue;
        pl->batch_mark = 0;
        fc2t2_status st = check_cuda(cudaEventRecord(pl->ev_run_done, pl->run), "join");
        if (st == FC2T2_OK) st = check_cuda(cudaStreamWaitEvent(s, pl->ev_run_done, 0), "join");
        if (first == FC2T2_OK) first = st;
    }
    return first;
}

}  // namespace

// Instances of a batched call whose M2L joins the batch's shared launch: occupied-cell plans with
// one channel and points on both sides (the others run their whole transform on their stream).
static bool occ_batched(const fc2t2_plan_s *pl, int64_t n_src, int64_t n_tgt) {
    return pl->occ.enabled && pl->C == 1 && n_src > 0 && n_tgt > 0 && !pl->profiling;
}

// Per instance, whether its plan serves another instance of the batch too: those instances run one
// after another on the plan's stream (one workspace), none of them in the shared M2L launch.
static std::vector<char> plans_repeated(int n_inst, const fc2t2_plan *plans) {
    std::unordered_map<const fc2t2_plan_s *, int> uses;
    for (int i = 0; i < n_inst; ++i) ++uses[plans[i]];
    std::vector<char> rep(n_inst);
    for (int i = 0; i < n_inst; ++i) rep[i] = uses[plans[i]] > 1;
    return rep;
}

// One instance of a batched transform up to its M2L: sorts of targets (tx, tw) and sources
// (sx, sw), P2M, occupancy, M2M.  `tgt` / `srt` are the plan's sort workspaces for them.
static fc2t2_status occ_prepare(fc2t2_plan_s *pl, cudaStream_t s, const float *sx, const float *sw, int64_t ns,
                                SortWork &srt, const float *tx, const float *tw, int64_t nt, SortWork &tgt,
                                bool sorted = false) {
    if (ns > srt.cap || nt > tgt.cap) return set_error(FC2T2_ERR_INVALID_ARG, "N or M outside [0, max]");
    fc2t2_status st;
    if ((st = clear_flags(pl, s)) != FC2T2_OK) return st;
    if (sorted) {   // both sorts hold these points: only the source weights change
        if ((st = reweight(pl, s, sw, ns, srt)) != FC2T2_OK) return st;
    } else {
        if ((st = sort_points(pl, s, tx, tw, nt, tgt)) != FC2T2_OK) return st;
        if ((st = sort_points(pl, s, sx, sw, ns, srt)) != FC2T2_OK) return st;
    }
    if ((st = check_cuda(launch_p2m(pl, s, srt, pl->d_M), "p2m")) != FC2T2_OK) return st;
    if ((st = check_cuda(launch_occupancy(pl, s, srt.count, tgt.count), "occupancy")) != FC2T2_OK) return st;
    for (int l = 0; l + 1 < pl->nlev; ++l)
        if ((st = check_cuda(launch_m2m(pl, s, l), "m2m")) != FC2T2_OK) return st;
    return FC2T2_OK;
}

// After the batch's M2L: L2L and L2P of one instance (value into val, gradient times weight into grad)
static fc2t2_status occ_finish(fc2t2_plan_s *pl, cudaStream_t s, const SortWork &tgt, int64_t nt, float *val,
                               float *grad) {
    const bool two = l2p_two_levels(pl, nt);
    fc2t2_status st;
    for (int l = pl->nlev - 2; l >= (two ? 1 : 0); --l)
        if ((st = check_cuda(launch_l2l(pl, s, l), "l2l")) != FC2T2_OK) return st;
    if ((st = evaluate_targets(pl, s, tgt, nt, two, val, grad, false)) != FC2T2_OK) return st;
    return finish_flags(pl, s);
}

// The M2L of every batched occupied-cell instance: one persistent launch per (dimension, order)
// and per kOccMaxInst instances, on the call's stream.
static fc2t2_status occ_batch_m2l(int n_inst, const fc2t2_plan *plans, const std::vector<char> &joins, cudaStream_t s) {
    std::vector<const fc2t2_plan_s *> todo;
    for (int i = 0; i < n_inst; ++i)
        if (joins[i]) todo.push_back(plans[i]);
    while (!todo.empty()) {
        std::vector<const fc2t2_plan_s *> group, rest;
        // the queue numbers its work chunks (of at least 32 targets) in 32-bit integers: a launch
        // takes plans while their largest possible chunk count stays below 2^30
        int64_t chunks = 0;
        for (auto *pl : todo) {
            const int64_t most = pl->G_total / 32 + kOccBuckets;
            if (pl->D == todo[0]->D && pl->rho == todo[0]->rho && (int)group.size() < kOccMaxInst &&
                (group.empty() || chunks + most < ((int64_t)1 << 30))) {
                group.push_back(pl);
                chunks += most;
            } else {
                rest.push_back(pl);
            }
        }
        fc2t2_status st = check_cuda(launch_m2l_occ(group.data(), (int)group.size(), s), "m2l (occupied cells, batched)");
        if (st != FC2T2_OK) return st;
        todo.swap(rest);
    }
    return FC2T2_OK;
}

// The batch after every instance's first part: the streams of the occupied-cell instances are
// joined into s (the other instances' streams, forked with `mark`, run on), their shared M2L is
// launched on s, and their streams are forked again for L2L and L2P (finish(i, plan)) and joined.
static fc2t2_status occ_batch_after(int n_inst, const fc2t2_plan *plans, const std::vector<char> &joins, cudaStream_t s,
                                    uint64_t mark, const std::function<fc2t2_status(int, fc2t2_plan_s *)> &finish) {
    std::vector<fc2t2_plan> sub;
    for (int i = 0; i < n_inst; ++i)
        if (joins[i]) sub.push_back(plans[i]);
    fc2t2_status st = batch_join((int)sub.size(), sub.data(), s, mark);
    if (st == FC2T2_OK) st = occ_batch_m2l(n_inst, plans, joins, s);
    if (st != FC2T2_OK) return st;
    const uint64_t mark2 = ++g_batch_counter;
    st = batch_fork((int)sub.size(), sub.data(), s, mark2);
    for (int i = 0; i < n_inst && st == FC2T2_OK; ++i)
        if (joins[i]) st = finish(i, plans[i]);
    const fc2t2_status sj = batch_join((int)sub.size(), sub.data(), s, mark2);
    return st != FC2T2_OK ? st : sj;
}

fc2t2_status fc2t2_forward_batched(int n_inst, const fc2t2_plan *plans, void *stream, const float *const *p,
                                   const float *const *w, const int64_t *N, const float *const *q, const int64_t *M,
                                   float *const *y) {
    if (n_inst < 0) return set_error(FC2T2_ERR_INVALID_ARG, "n_inst < 0");
    if (n_inst == 0) return FC2T2_OK;
    if (!plans || !p || !w || !N || !q || !M || !y) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    for (int i = 0; i < n_inst; ++i)
        if (!plans[i]) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    // occupied-cell instances: sorts .. M2M on their streams, one M2L launch for all, then L2L, L2P
    std::vector<char> joins(n_inst, 0);
    const std::vector<char> repeated = plans_repeated(n_inst, plans);
    bool any = false;
    for (int i = 0; i < n_inst; ++i) {
        if (!occ_batched(plans[i], N[i], M[i]) || repeated[i]) continue;
        if (!p[i] || !w[i] || !q[i] || !y[i]) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
        joins[i] = 1;
        any = true;
    }
    uint64_t mark = ++g_batch_counter;
    fc2t2_status st = batch_fork(n_inst, plans, s, mark);
    for (int i = 0; i < n_inst && st == FC2T2_OK; ++i) {
        fc2t2_plan_s *pl = plans[i];
        st = joins[i] ? occ_prepare(pl, pl->run, p[i], w[i], N[i], pl->src, q[i], nullptr, M[i], pl->qry)
                      : fc2t2_forward(pl, pl->run, p[i], w[i], N[i], q[i], M[i], y[i]);
    }
    if (st != FC2T2_OK || !any) {
        const fc2t2_status sj = batch_join(n_inst, plans, s, mark);
        return st != FC2T2_OK ? st : sj;
    }
    st = occ_batch_after(n_inst, plans, joins, s, mark, [&](int i, fc2t2_plan_s *pl) {
        const fc2t2_status r = occ_finish(pl, pl->run, pl->qry, M[i], y[i], nullptr);
        pl->src.held_w = w[i];
        return r;
    });
    const fc2t2_status sj = batch_join(n_inst, plans, s, mark);   // the other instances' streams
    return st != FC2T2_OK ? st : sj;
}

static fc2t2_status backward_batched(int n_inst, const fc2t2_plan *plans, void *stream, const float *const *p,
                                     const float *const *w, const int64_t *N, const float *const *q, const int64_t *M,
                                     const float *const *ybar, float *const *wbar, float *const *pbar, bool reuse) {
    if (n_inst < 0) return set_error(FC2T2_ERR_INVALID_ARG, "n_inst < 0");
    if (n_inst == 0) return FC2T2_OK;
    if (!plans || !p || !w || !N || !q || !M || !ybar || !wbar || !pbar)
        return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    for (int i = 0; i < n_inst; ++i)
        if (!plans[i]) return set_error(FC2T2_ERR_INVALID_ARG, "plan is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    // occupied-cell instances (the transposed transform: sources q with weights ybar, targets p):
    // sorts .. M2M on their streams, one M2L launch for all, then L2L, L2P value and gradient
    std::vector<char> joins(n_inst, 0);
    const std::vector<char> repeated = plans_repeated(n_inst, plans);
    bool any = false;
    for (int i = 0; i < n_inst; ++i) {
        if (!occ_batched(plans[i], M[i], N[i]) || (!wbar[i] && !pbar[i]) || repeated[i]) continue;
        if (!p[i] || !w[i] || !q[i] || !ybar[i]) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
        joins[i] = 1;
        any = true;
    }
    uint64_t mark = ++g_batch_counter;
    fc2t2_status st = batch_fork(n_inst, plans, s, mark);
    for (int i = 0; i < n_inst && st == FC2T2_OK; ++i) {
        fc2t2_plan_s *pl = plans[i];
        // (reuse: the forward's sorts of exactly these arrays, as fc2t2_backward_reuse checks)
        const bool sorted = reuse && pl->src.held_x == p[i] && pl->src.held_w == w[i] && pl->src.held_n == N[i] &&
                            pl->qry.held_x == q[i] && pl->qry.held_n == M[i];
        if (joins[i])
            st = occ_prepare(pl, pl->run, q[i], ybar[i], M[i], pl->qry, p[i], w[i], N[i], pl->src, sorted);
        else if (reuse)
            st = fc2t2_backward_reuse(pl, pl->run, p[i], w[i], N[i], q[i], M[i], ybar[i], wbar[i], pbar[i]);
        else
            st = fc2t2_backward(pl, pl->run, p[i], w[i], N[i], q[i], M[i], ybar[i], wbar[i], pbar[i]);
    }
    if (st != FC2T2_OK || !any) {
        const fc2t2_status sj = batch_join(n_inst, plans, s, mark);
        return st != FC2T2_OK ? st : sj;
    }
    st = occ_batch_after(n_inst, plans, joins, s, mark, [&](int i, fc2t2_plan_s *pl) {
        return occ_finish(pl, pl->run, pl->src, N[i], wbar[i], pbar[i]);
    });
    const fc2t2_status sj = batch_join(n_inst, plans, s, mark);   // the other instances' streams
    return st != FC2T2_OK ? st : sj;
}

fc2t2_status fc2t2_backward_batched(int n_inst, const fc2t2_plan *plans, void *stream, const float *const *p,
                                    const float *const *w, const int64_t *N, const float *const *q, const int64_t *M,
                                    const float *const *ybar, float *const *wbar, float *const *pbar) {
    return backward_batched(n_inst, plans, stream, p, w, N, q, M, ybar, wbar, pbar, false);
}

fc2t2_status fc2t2_backward_batched_reuse(int n_inst, const fc2t2_plan *plans, void *stream, const float *const *p,
                                          const float *const *w, const int64_t *N, const float *const *q,
                                          const int64_t *M, const float *const *ybar, float *const *wbar,
                                          float *const *pbar) {
    return backward_batched(n_inst, plans, stream, p, w, N, q, M, ybar, wbar, pbar, true);
}

fc2t2_status fc2t2_plan_query(fc2t2_plan pl, fc2t2_plan_info *info) {
    if (!pl || !info) return set_error(FC2T2_ERR_INVALID_ARG, "NULL argument");
    info->levels = pl->nlev;
    info->coefficients = pl->P;
    info->m2l_tensor_cores = (pl->tc.enabled && pl->tc.level_ok[0]) ? 1 : 0;
    // interacting cell pairs per level: per-dimension window sums factorise
    double pairs_total = 0.0, issued = 0.0;
    double q = 1.0;   // #{(k, b) : |k| + |b| <= rho} = C(rho + 2D, 2D)
    for (int i = 1; i <= 2 * pl->D; ++i) q = q * (pl->rho + i) / i;
    for (int l = 0; l < pl->nlev; ++l) {
        const int nl = pl->lev[l].n;
        double W = 0.0, H = 0.0;
        for (int t = 0; t < nl; ++t) {
            const int lo = (t & 1) ? -3 : -2;
            for (int o = lo; o < lo + 6; ++o) W += (t + o >= 0 && t + o < nl) ? 1.0 : 0.0;
            for (int o = -1; o <= 1; ++o) H += (t + o >= 0 && t + o < nl) ? 1.0 : 0.0;
        }
        const double pairs = std::pow(W, pl->D) - (l > 0 ? std::pow(H, pl->D) : 0.0);
        pairs_total += pairs;
        if (pl->sep.enabled) continue;
        if (pl->tc.enabled && pl->tc.level_ok[l]) issued += pl->tc.mma_flops_level[l];
        else issued += 2.0 * q * pairs;
    }
    info->m2l_cell_pairs = pairs_total;
    info->m2l_useful_flops = 2.0 * q * pairs_total;
    info->m2l_issued_flops = pl->sep.enabled ? pl->sep.flops : issued;
    int64_t bytes = 2 * pl->G_total * pl->Pp * (int64_t)sizeof(float);
    if (pl->C > 1) bytes += (int64_t)pl->C * pl->lev[0].G * pl->Pp * (int64_t)sizeof(float);
    bytes += (int64_t)pl->mma_ops_bytes + pl->tc.packed_bytes + (int64_t)pl->sep.t_bytes;
    bytes += (pl->src.cap + pl->qry.cap) * (int64_t)(5 * sizeof(int) + (pl->D + 1) * sizeof(float));
    info->device_bytes = bytes;
    info->m2l_classes_per_cta = pl->tc.enabled ? pl->tc.ncls : 0;
    return FC2T2_OK;
}

const char *fc2t2_status_string(fc2t2_status st) {
    switch (st) {
        case FC2T2_OK: return "ok";
        case FC2T2_ERR_INVALID_ARG: return "invalid argument";
        case FC2T2_ERR_UNSUPPORTED: return "unsupported";
        case FC2T2_ERR_OOM: return "out of device memory";
        case FC2T2_ERR_DOMAIN: return "point outside the domain";
        case FC2T2_ERR_CUDA: return "CUDA error";
        case FC2T2_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

fc2t2_status fc2t2_last_error(char *buf, size_t n) {
    if (buf && n > 0) {
        std::snprintf(buf, n, "%s", g_err_msg.c_str());
    }
    return g_err_code;
}

}  // extern "C"
