/*
 * sgp_oracle.c -- CPU oracle for the support-graph preconditioned CG path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The GPU library
 * shares no code with it.
 *
 * Plain, slow, sequential FP64.  Compile with -ffp-contract=off (no fused
 * multiply-add) so the contact test and the friction blocks are evaluated
 * exactly as written.  Every function cites the passage of arXiv 2410.04512
 * ("Support Graph Preconditioners for Off-Lattice Cell-Based Models") that it
 * follows.  3x3 blocks are stored row-major, 9 doubles each.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_OOM = 3, ORC_ERR_DEGENERATE = 4,
       ORC_ERR_NOT_SPD = 5, ORC_ERR_NO_CONVERGENCE = 6 };

/* ------------------------------------------------------------------------
 * Section 2, Steps 1-2: cells i and j interact when their spheres overlap,
 * i.e. when the contact area A_ij is nonzero: |r_j - r_i| < R_i + R_j.
 * The distance is evaluated as sqrt((dx*dx + dy*dy) + dz*dz), dx = x_j - x_i.
 * ------------------------------------------------------------------------ */
static int in_contact(const double *pos, const double *radii, int64_t i, int64_t j)
{
    double dx = pos[3 * j + 0] - pos[3 * i + 0];
    double dy = pos[3 * j + 1] - pos[3 * i + 1];
    double dz = pos[3 * j + 2] - pos[3 * i + 2];
    double s = dx * dx;
    s = s + dy * dy;
    s = s + dz * dz;
    double d = sqrt(s);
    double rr = radii[i] + radii[j];
    return d < rr;
}

/* Brute force over all pairs i < j (the definition of the collision graph,
 * Section 1.1 "we draw an edge e = (i, j) ... when A_ij is nonzero").
 * Pairs come out sorted by i, then j.  Writes at most `cap` pairs and
 * returns the total count. */
int64_t orc_contacts(int64_t n, const double *pos, const double *radii,
                     int32_t *ij, int64_t cap)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (in_contact(pos, radii, i, j)) {
                if (m < cap) { ij[2 * m] = (int32_t)i; ij[2 * m + 1] = (int32_t)j; }
                ++m;
            }
    return m;
}

/* The same brute force restricted to the rows i listed in `rows`
 * (ascending): every j > i in contact with i.  For sampled checks at sizes
 * where the full O(N^2) scan is too slow. */
int64_t orc_contacts_of_rows(int64_t n, const double *pos, const double *radii,
                             const int64_t *rows, int64_t nrows, int32_t *ij, int64_t cap)
{
    int64_t m = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        for (int64_t j = i + 1; j < n; ++j)
            if (in_contact(pos, radii, i, j)) {
                if (m < cap) { ij[2 * m] = (int32_t)i; ij[2 * m + 1] = (int32_t)j; }
                ++m;
            }
    }
    return m;
}

/* ------------------------------------------------------------------------
 * Section 2, Step 3, eq. (1):
 *   Gamma^cc_ij = A_ij (g_par u u^T + g_perp (I - u u^T)),
 *   u = (r_j - r_i) / |r_j - r_i|.
 * The contact area is folded into the coefficients (g = A_ij * gamma).
 * Also the spanning-tree weight of Section 3.1: the minimum eigenvalue of the
 * edge block, which by Lemma 2.1 is min(g_par, g_perp).
 * Returns ORC_ERR_DEGENERATE if two centres in contact coincide (u undefined).
 * ------------------------------------------------------------------------ */
int orc_friction_blocks(int64_t m, const int32_t *ij, const double *pos,
                        const double *g_par, const double *g_perp,
                        double *blocks, double *weight)
{
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = ij[2 * e], j = ij[2 * e + 1];
        double dx = pos[3 * j + 0] - pos[3 * i + 0];
        double dy = pos[3 * j + 1] - pos[3 * i + 1];
        double dz = pos[3 * j + 2] - pos[3 * i + 2];
        double s = dx * dx;
        s = s + dy * dy;
        s = s + dz * dz;
        double d = sqrt(s);
        if (!(d > 0.0)) return ORC_ERR_DEGENERATE;
        double u[3] = { dx / d, dy / d, dz / d };
        double *B = blocks + 9 * e;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double uu = u[a] * u[b];
                double id = (a == b) ? 1.0 : 0.0;
                double t1 = g_par[e] * uu;
                double t2 = g_perp[e] * (id - uu);
                B[3 * a + b] = t1 + t2;
            }
        weight[e] = g_par[e] < g_perp[e] ? g_par[e] : g_perp[e];
    }
    return ORC_OK;
}

/* Definition "Block Laplacian" (Section 2) of the collision graph with
 * self-loops w(i,i) = gamma0 I (the cell-substrate friction of Step 3):
 *   L_ij = -w(i,j) (i != j),  L_ii = w(i,i) + sum_k w(i,k).
 * Dense (3n x 3n, row-major) for small n only. */
void orc_dense_laplacian(int64_t n, int64_t m, const int32_t *ij, const double *blocks,
                         double gamma0, double *out)
{
    int64_t N = 3 * n;
    memset(out, 0, sizeof(double) * (size_t)(N * N));
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) out[(3 * i + a) * N + 3 * i + a] += gamma0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = ij[2 * e], j = ij[2 * e + 1];
        const double *B = blocks + 9 * e;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                out[(3 * i + a) * N + 3 * j + b] -= B[3 * a + b];
                out[(3 * j + a) * N + 3 * i + b] -= B[3 * a + b];
                out[(3 * i + a) * N + 3 * i + b] += B[3 * a + b];
                out[(3 * j + a) * N + 3 * j + b] += B[3 * a + b];
            }
    }
}

/* ------------------------------------------------------------------------
 * Appendix B.2, "Matrix-Vector Product of a graph":
 *   x_i = w(i,i) v_i, then for every edge (i,j):
 *   x_i += w(i,j)(v_i - v_j),  x_j += w(i,j)(v_j - v_i).
 * With w(i,i) = gamma0 I this is the row of eq. (2) (Step 4).
 * ------------------------------------------------------------------------ */
void orc_matvec(int64_t n, int64_t m, const int32_t *ij, const double *blocks,
                double gamma0, const double *v, double *x)
{
    for (int64_t i = 0; i < 3 * n; ++i) x[i] = gamma0 * v[i];
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = ij[2 * e], j = ij[2 * e + 1];
        const double *B = blocks + 9 * e;
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = v[3 * i + a] - v[3 * j + a];
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int b = 0; b < 3; ++b) s += B[3 * a + b] * d[b];
            x[3 * i + a] += s;
            x[3 * j + a] -= s;
        }
    }
}

/* ------------------------------------------------------------------------
 * Section 3.1: maximum spanning tree by Prim's algorithm.  Edges are
 * compared by the strict total order (weight descending, then edge index
 * ascending), so the maximum spanning forest is unique.  A disconnected
 * graph yields a forest: each component is grown from its smallest
 * unvisited vertex.  Outputs the tree edges and the vertex insertion order,
 * with each vertex's parent (the endpoint already in the tree when the
 * vertex was added; -1 for the start vertex of a component) and the edge to
 * that parent.  Returns the number of tree edges, or -1 on allocation
 * failure.
 * ------------------------------------------------------------------------ */
static const double *g_w;
static int edge_better(int32_t a, int32_t b)   /* a strictly before b */
{
    if (g_w[a] != g_w[b]) return g_w[a] > g_w[b];
    return a < b;
}
static void heap_push(int32_t *h, int64_t *len, int32_t e)
{
    int64_t k = (*len)++;
    h[k] = e;
    while (k > 0) {
        int64_t p = (k - 1) / 2;
        if (!edge_better(h[k], h[p])) break;
        int32_t t = h[k]; h[k] = h[p]; h[p] = t;
        k = p;
    }
}
static int32_t heap_pop(int32_t *h, int64_t *len)
{
    int32_t top = h[0];
    h[0] = h[--(*len)];
    int64_t k = 0;
    for (;;) {
        int64_t l = 2 * k + 1, r = l + 1, b = k;
        if (l < *len && edge_better(h[l], h[b])) b = l;
        if (r < *len && edge_better(h[r], h[b])) b = r;
        if (b == k) break;
        int32_t t = h[k]; h[k] = h[b]; h[b] = t;
        k = b;
    }
    return top;
}

int64_t orc_prim_msf(int64_t n, int64_t m, const int32_t *ij, const double *w,
                     int32_t *tree_edges, int32_t *order, int32_t *parent,
                     int32_t *parent_edge)
{
    int64_t *deg = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *adj = malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int64_t *fill = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *heap = malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    char *vis = calloc((size_t)n + 1, 1);
    if (!deg || !adj || !fill || !heap || !vis) {
        free(deg); free(adj); free(fill); free(heap); free(vis);
        return -1;
    }
    for (int64_t e = 0; e < m; ++e) { deg[ij[2 * e] + 1]++; deg[ij[2 * e + 1] + 1]++; }
    for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = ij[2 * e], j = ij[2 * e + 1];
        adj[deg[i] + fill[i]++] = (int32_t)e;
        adj[deg[j] + fill[j]++] = (int32_t)e;
    }
    g_w = w;
    int64_t nt = 0, no = 0, hl = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (vis[s]) continue;
        vis[s] = 1;
        order[no++] = (int32_t)s;
        parent[s] = -1;
        parent_edge[s] = -1;
        for (int64_t k = deg[s]; k < deg[s + 1]; ++k) heap_push(heap, &hl, adj[k]);
        while (hl > 0) {
            int32_t e = heap_pop(heap, &hl);
            int64_t a = ij[2 * e], b = ij[2 * e + 1];
            int64_t v, from;
            if (vis[a] && !vis[b]) { v = b; from = a; }
            else if (vis[b] && !vis[a]) { v = a; from = b; }
            else continue;                       /* both ends already in the tree */
            vis[v] = 1;
            order[no++] = (int32_t)v;
            parent[v] = (int32_t)from;
            parent_edge[v] = e;
            tree_edges[nt++] = e;
            for (int64_t k = deg[v]; k < deg[v + 1]; ++k) {
                int32_t f = adj[k];
                int64_t o = ij[2 * f] == v ? ij[2 * f + 1] : ij[2 * f];
                if (!vis[o]) heap_push(heap, &hl, f);
            }
        }
    }
    free(deg); free(adj); free(fill); free(heap); free(vis);
    return nt;
}

/* ------------------------------------------------------------------------
 * 3x3 helpers
 * ------------------------------------------------------------------------ */
/* Inverse by the adjugate (cofactor) formula; returns 0 if the determinant
 * is not positive or not finite (a symmetric positive definite block has a
 * positive determinant). */
static int inv3(const double *A, double *R)
{
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det > 0.0) || !isfinite(det)) return 0;
    double id = 1.0 / det;
    R[0] = c00 * id;
    R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    R[3] = c01 * id;
    R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    R[6] = c02 * id;
    R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return 1;
}
static void mm3(const double *A, const double *B, double *C)      /* C = A B */
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * a + k] * B[3 * k + b];
            C[3 * a + b] = s;
        }
}
static void mmt3(const double *A, const double *B, double *C)     /* C = A B^T */
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * a + k] * B[3 * b + k];
            C[3 * a + b] = s;
        }
}
static void mv3(const double *A, const double *x, double *y)     /* y = A x */
{
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += A[3 * a + k] * x[k];
        y[a] = s;
    }
}
static void mtv3(const double *A, const double *x, double *y)    /* y = A^T x */
{
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += A[3 * k + a] * x[k];
        y[a] = s;
    }
}

/* ------------------------------------------------------------------------
 * Section 3.3, Algorithm 2 (TreeLDLT) on the preconditioner of Section 3.1:
 * P = block Laplacian of the spanning forest with the self-loops gamma0 I
 * kept.  Vertices are taken children-before-parents, in the reverse of
 * Prim's insertion order (Lemma 3.1 and its corollary: no fill):
 *   D_c = P_cc - sum_{k child of c} L_ck D_k L_ck^T,
 *   L_{p(c),c} = P_{p(c),c} D_c^{-1},   P_{p(c),c} = -Upsilon_{edge(c)}.
 * (The printed algorithm drops the transpose on the second L; L D L^T is
 * the symmetric Schur complement update.)  L is stored at the child: L[c] is
 * the block linking c to its parent.  Also returns D^{-1}.
 * Returns ORC_ERR_NOT_SPD if a pivot block is not positive definite.
 * ------------------------------------------------------------------------ */
int orc_tree_ldlt(int64_t n, const int32_t *order, const int32_t *parent,
                  const int32_t *parent_edge, const double *blocks, double gamma0,
                  double *L, double *D, double *Dinv)
{
    double *A = calloc((size_t)(9 * n) + 1, sizeof(double));
    int64_t *cptr = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *cfill = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *child = malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!A || !cptr || !cfill || !child) {
        free(A); free(cptr); free(cfill); free(child);
        return ORC_ERR_OOM;
    }
    /* diagonal blocks of P: gamma0 I plus the tree edges at each vertex */
    for (int64_t c = 0; c < n; ++c)
        for (int a = 0; a < 3; ++a) A[9 * c + 4 * a] = gamma0;
    for (int64_t c = 0; c < n; ++c) {
        if (parent[c] < 0) continue;
        const double *U = blocks + 9 * (int64_t)parent_edge[c];
        int64_t p = parent[c];
        for (int k = 0; k < 9; ++k) { A[9 * c + k] += U[k]; A[9 * p + k] += U[k]; }
    }
    /* children lists */
    for (int64_t c = 0; c < n; ++c) if (parent[c] >= 0) cptr[parent[c] + 1]++;
    for (int64_t c = 0; c < n; ++c) cptr[c + 1] += cptr[c];
    for (int64_t c = 0; c < n; ++c)
        if (parent[c] >= 0) child[cptr[parent[c]] + cfill[parent[c]]++] = (int32_t)c;

    int rc = ORC_OK;
    for (int64_t t = n - 1; t >= 0; --t) {
        int64_t c = order[t];
        double X[9] = { 0 };
        for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q) {
            int64_t k = child[q];
            double LD[9], LDL[9];
            mm3(L + 9 * k, D + 9 * k, LD);
            mmt3(LD, L + 9 * k, LDL);
            for (int a = 0; a < 9; ++a) X[a] += LDL[a];
        }
        for (int a = 0; a < 9; ++a) D[9 * c + a] = A[9 * c + a] - X[a];
        if (!inv3(D + 9 * c, Dinv + 9 * c)) { rc = ORC_ERR_NOT_SPD; break; }
        if (parent[c] >= 0) {
            const double *U = blocks + 9 * (int64_t)parent_edge[c];
            double Pneg[9];
            for (int a = 0; a < 9; ++a) Pneg[a] = -U[a];
            mm3(Pneg, Dinv + 9 * c, L + 9 * c);
        } else {
            for (int a = 0; a < 9; ++a) L[9 * c + a] = 0.0;
        }
    }
    free(A); free(cptr); free(cfill); free(child);
    return rc;
}

/* ------------------------------------------------------------------------
 * Appendix B.1: solve P x = b with P = L D L^T from orc_tree_ldlt.
 *   ForwardSolve: children before parents, z_i = b_i - sum_{j child} L_j z_j;
 *   DiagSolve:    y_i = D_i^{-1} z_i;
 *   BackwardSolve: parents before children, x_i = y_i - L_i^T x_{parent(i)}.
 * ------------------------------------------------------------------------ */
int orc_tree_solve(int64_t n, const int32_t *order, const int32_t *parent,
                   const double *L, const double *Dinv, const double *b, double *x)
{
    double *z = malloc(sizeof(double) * (size_t)(3 * n + 1));
    if (!z) return ORC_ERR_OOM;
    for (int64_t i = 0; i < 3 * n; ++i) z[i] = b[i];
    /* forward: when child c is final, subtract its term from its parent */
    for (int64_t t = n - 1; t >= 0; --t) {
        int64_t c = order[t];
        if (parent[c] >= 0) {
            double s[3];
            mv3(L + 9 * c, z + 3 * c, s);
            int64_t p = parent[c];
            for (int a = 0; a < 3; ++a) z[3 * p + a] -= s[a];
        }
    }
    /* diagonal */
    for (int64_t c = 0; c < n; ++c) mv3(Dinv + 9 * c, z + 3 * c, x + 3 * c);
    /* backward */
    for (int64_t t = 0; t < n; ++t) {
        int64_t c = order[t];
        if (parent[c] >= 0) {
            double s[3];
            mtv3(L + 9 * c, x + 3 * (int64_t)parent[c], s);
            for (int a = 0; a < 3; ++a) x[3 * c + a] -= s[a];
        }
    }
    free(z);
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Block Jacobi preconditioner (Section 5, preconditioner (2)): the inverses
 * of the diagonal blocks Gamma_ii = gamma0 I + sum_{j ~ i} Upsilon_ij.
 * ------------------------------------------------------------------------ */
int orc_block_jacobi(int64_t n, int64_t m, const int32_t *ij, const double *blocks,
                     double gamma0, double *Dinv)
{
    double *A = calloc((size_t)(9 * n) + 1, sizeof(double));
    if (!A) return ORC_ERR_OOM;
    for (int64_t c = 0; c < n; ++c)
        for (int a = 0; a < 3; ++a) A[9 * c + 4 * a] = gamma0;
    for (int64_t e = 0; e < m; ++e)
        for (int k = 0; k < 9; ++k) {
            A[9 * (int64_t)ij[2 * e] + k] += blocks[9 * e + k];
            A[9 * (int64_t)ij[2 * e + 1] + k] += blocks[9 * e + k];
        }
    int rc = ORC_OK;
    for (int64_t c = 0; c < n; ++c)
        if (!inv3(A + 9 * c, Dinv + 9 * c)) { rc = ORC_ERR_NOT_SPD; break; }
    free(A);
    return rc;
}

/* ------------------------------------------------------------------------
 * Section 1.1: preconditioned conjugate gradients for Gamma v = F.
 *   r = F - Gamma x0, z = H r, p = z, rho = r^T z; then repeat
 *     q = Gamma p; alpha = rho / p^T q; x += alpha p; r -= alpha q; k += 1;
 *     stop if |r|_2 <= tol |F|_2 (or k == maxit);
 *     z = H r; rho' = r^T z; beta = rho' / rho; p = z + beta p.
 * H = P^{-1} (precond 1: tree factor), blockdiag(Gamma)^{-1} (precond 2) or
 * I (precond 0).  A zero right-hand side returns x = 0 after 0 iterations.
 * If fixed_iters > 0 the loop runs exactly that many iterations (no
 * tolerance test).  Reports the iteration count and the recursive relative
 * residual |r|/|F|.
 * ------------------------------------------------------------------------ */
static double dot3n(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) s += a[i] * b[i];
    return s;
}

static int apply_precond(int precond, int64_t n, const int32_t *order, const int32_t *parent,
                         const double *L, const double *Dinv, const double *r, double *z)
{
    if (precond == 1) return orc_tree_solve(n, order, parent, L, Dinv, r, z);
    if (precond == 2) {
        for (int64_t c = 0; c < n; ++c) mv3(Dinv + 9 * c, r + 3 * c, z + 3 * c);
        return ORC_OK;
    }
    for (int64_t i = 0; i < 3 * n; ++i) z[i] = r[i];
    return ORC_OK;
}

int orc_pcg(int64_t n, int64_t m, const int32_t *ij, const double *blocks, double gamma0,
            int precond, const int32_t *order, const int32_t *parent, const double *L,
            const double *Dinv, const double *F, double *x, double tol, int64_t maxit,
            int64_t fixed_iters, int64_t *iters_out, double *relres_out)
{
    size_t sz = sizeof(double) * (size_t)(3 * n + 1);
    double *r = malloc(sz), *z = malloc(sz), *p = malloc(sz), *q = malloc(sz);
    if (!r || !z || !p || !q) { free(r); free(z); free(p); free(q); return ORC_ERR_OOM; }
    int rc = ORC_OK;
    int64_t k = 0;
    double FF = dot3n(n, F, F);
    if (FF == 0.0) {
        for (int64_t i = 0; i < 3 * n; ++i) x[i] = 0.0;
        *iters_out = 0; *relres_out = 0.0;
        free(r); free(z); free(p); free(q);
        return ORC_OK;
    }
    orc_matvec(n, m, ij, blocks, gamma0, x, q);
    for (int64_t i = 0; i < 3 * n; ++i) r[i] = F[i] - q[i];
    double rr = dot3n(n, r, r);
    double stop2 = tol * tol * FF;
    if (fixed_iters <= 0 && rr <= stop2) goto done;
    rc = apply_precond(precond, n, order, parent, L, Dinv, r, z);
    if (rc) goto done;
    for (int64_t i = 0; i < 3 * n; ++i) p[i] = z[i];
    double rho = dot3n(n, r, z);
    for (;;) {
        orc_matvec(n, m, ij, blocks, gamma0, p, q);
        double pq = dot3n(n, p, q);
        if (!(pq > 0.0)) { rc = ORC_ERR_NOT_SPD; break; }
        double alpha = rho / pq;
        for (int64_t i = 0; i < 3 * n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        ++k;
        rr = dot3n(n, r, r);
        if (fixed_iters > 0) { if (k >= fixed_iters) break; }
        else {
            if (rr <= stop2) break;
            if (k >= maxit) { rc = ORC_ERR_NO_CONVERGENCE; break; }
        }
        rc = apply_precond(precond, n, order, parent, L, Dinv, r, z);
        if (rc) break;
        double rho2 = dot3n(n, r, z);
        double beta = rho2 / rho;
        rho = rho2;
        for (int64_t i = 0; i < 3 * n; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    *iters_out = k;
    *relres_out = sqrt(rr / FF);
    free(r); free(z); free(p); free(q);
    return rc;
}
