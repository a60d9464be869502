/* cpu_parallel.c -- the all-cores CPU baseline of the solve phase.
 *
 * TEST INFRASTRUCTURE, like everything under oracle/: only the tests,
 * the smoke check and the benchmark's CPU leg use it; it shares no code with
 * the CUDA library.  It is compiled together with sgp_oracle.c (whose
 * functions it calls) into its own shared object, so the oracle proper stays
 * plain sequential C.
 *
 * What it runs is the oracle's preconditioned conjugate gradients
 * (Section 1.1) with the two data-parallel parts spread over OpenMP threads:
 *   - the product y = Gamma v in the row form of Appendix B.2,
 *       y_i = gamma0 v_i + sum_{j ~ i} Upsilon_ij (v_i - v_j),
 *     over a row-wise copy of the contact list (each row owned by one
 *     thread, no write conflicts);
 *   - the vector updates and inner products.
 * The preconditioner is the oracle's own sequential tree solve
 * (Appendix B.1, orc_tree_solve): forward and backward substitution along a
 * tree are chains of dependent steps, which the paper runs on one core.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_tree_solve(int64_t n, const int32_t *order, const int32_t *parent, const double *L,
                   const double *Dinv, const double *b, double *x);

enum { OMP_OK = 0, OMP_ERR_OOM = 3, OMP_ERR_NOT_SPD = 5, OMP_ERR_NO_CONVERGENCE = 6 };

int orc_omp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Row-wise copy of the contact list: both directions of every edge. */
typedef struct {
    int64_t *ptr;   /* n + 1 */
    int32_t *col;   /* 2m neighbour */
    int32_t *edge;  /* 2m edge index (the block) */
} Rows;

static int rows_build(int64_t n, int64_t m, const int32_t *ij, Rows *R)
{
    R->ptr = calloc((size_t)n + 1, sizeof(int64_t));
    R->col = malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    R->edge = malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int64_t *fill = calloc((size_t)n + 1, sizeof(int64_t));
    if (!R->ptr || !R->col || !R->edge || !fill) {
        free(fill);
        return OMP_ERR_OOM;
    }
    for (int64_t e = 0; e < m; ++e) {
        R->ptr[ij[2 * e] + 1]++;
        R->ptr[ij[2 * e + 1] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) R->ptr[i + 1] += R->ptr[i];
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = ij[2 * e], j = ij[2 * e + 1];
        int64_t si = R->ptr[i] + fill[i]++, sj = R->ptr[j] + fill[j]++;
        R->col[si] = (int32_t)j; R->edge[si] = (int32_t)e;
        R->col[sj] = (int32_t)i; R->edge[sj] = (int32_t)e;
    }
    free(fill);
    return OMP_OK;
}

static void rows_free(Rows *R)
{
    free(R->ptr); free(R->col); free(R->edge);
}

static void matvec_rows(int64_t n, const Rows *R, const double *blocks, double gamma0, const double *v,
                        double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {gamma0 * v[3 * i], gamma0 * v[3 * i + 1], gamma0 * v[3 * i + 2]};
        for (int64_t s = R->ptr[i]; s < R->ptr[i + 1]; ++s) {
            const int64_t j = R->col[s];
            const double *B = blocks + 9 * (int64_t)R->edge[s];
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = v[3 * i + a] - v[3 * j + a];
            for (int a = 0; a < 3; ++a) acc[a] += B[3 * a] * d[0] + B[3 * a + 1] * d[1] + B[3 * a + 2] * d[2];
        }
        y[3 * i] = acc[0]; y[3 * i + 1] = acc[1]; y[3 * i + 2] = acc[2];
    }
}

static double dot(int64_t k, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int64_t i = 0; i < k; ++i) s += a[i] * b[i];
    return s;
}

/* PCG with the tree preconditioner, Section 1.1 in the oracle's order;
 * x holds the initial guess on entry.  Returns OMP_OK, OMP_ERR_NOT_SPD,
 * OMP_ERR_NO_CONVERGENCE or OMP_ERR_OOM. */
int orc_omp_pcg_tree(int64_t n, int64_t m, const int32_t *ij, const double *blocks, double gamma0,
                     const int32_t *order, const int32_t *parent, const double *L, const double *Dinv,
                     const double *F, double *x, double tol, int64_t maxit, int64_t *iters_out,
                     double *relres_out)
{
    const int64_t k3 = 3 * n;
    Rows R = {0, 0, 0};
    if (rows_build(n, m, ij, &R)) { rows_free(&R); return OMP_ERR_OOM; }
    size_t sz = sizeof(double) * (size_t)(k3 + 1);
    double *r = malloc(sz), *z = malloc(sz), *p = malloc(sz), *q = malloc(sz);
    if (!r || !z || !p || !q) {
        free(r); free(z); free(p); free(q); rows_free(&R);
        return OMP_ERR_OOM;
    }
    int rc = OMP_OK;
    int64_t it = 0;
    const double FF = dot(k3, F, F);
    double rr = 0.0;
    if (FF == 0.0) {
        for (int64_t i = 0; i < k3; ++i) x[i] = 0.0;
        goto done;
    }
    matvec_rows(n, &R, blocks, gamma0, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < k3; ++i) r[i] = F[i] - q[i];
    rr = dot(k3, r, r);
    const double stop2 = tol * tol * FF;
    if (rr <= stop2) goto done;
    orc_tree_solve(n, order, parent, L, Dinv, r, z);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < k3; ++i) p[i] = z[i];
    double rho = dot(k3, r, z);
    for (;;) {
        matvec_rows(n, &R, blocks, gamma0, p, q);
        const double pq = dot(k3, p, q);
        if (!(pq > 0.0)) { rc = OMP_ERR_NOT_SPD; break; }
        const double alpha = rho / pq;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < k3; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        ++it;
        rr = dot(k3, r, r);
        if (rr <= stop2) break;
        if (it >= maxit) { rc = OMP_ERR_NO_CONVERGENCE; break; }
        orc_tree_solve(n, order, parent, L, Dinv, r, z);
        const double rho2 = dot(k3, r, z);
        const double beta = rho2 / rho;
        rho = rho2;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < k3; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    *iters_out = it;
    *relres_out = FF > 0 ? sqrt(rr / FF) : 0.0;
    free(r); free(z); free(p); free(q);
    rows_free(&R);
    return rc;
}
