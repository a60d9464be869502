/*
 * sgp.h -- C ABI of the GB300 support-graph preconditioned CG library.
 *
 * Solves the overdamped equation of motion of an off-lattice cell model,
 * Gamma v = F (arXiv 2410.04512, Section 2, eq. (2)), by conjugate gradients
 * preconditioned with the block Laplacian of a maximum spanning forest of the
 * collision graph (Section 3.1).  Every step runs in CUDA kernels built for
 * sm_103a.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named *_dev are DEVICE pointers on the context's device; the
 *   caller owns them, keeps them alive for the duration of the call and the
 *   library never frees or retains them.  Vectors of cells are n x 3 float64
 *   arrays, row-major and contiguous (cell i at [3i, 3i+3)).
 * - Handles (sgp_graph, sgp_matrix, sgp_tree, sgp_factor) are opaque and own
 *   their device memory.  A call that produces a handle takes a pointer to a
 *   handle variable: if it holds NULL a new handle is created; if it holds a
 *   handle produced earlier by the same call kind, that handle's memory is
 *   reused (grown when needed).  Free handles with the matching *_destroy.
 * - All work is ordered on the context's CUDA stream.  Calls that return host
 *   values (sizes, solve statistics) synchronise that stream.
 * - Every call returns an sgp_status; on failure sgp_last_error(ctx) holds a
 *   one-line reason.  No call aborts the process.
 * - A context is used by one host thread at a time.  A handle may be read by
 *   calls on several contexts, but not while calls that write it, or that
 *   use its workspace (sgp_tree_apply uses the factor's), overlap on the GPU;
 *   the block-Jacobi inverses are written into the matrix by its first
 *   block-Jacobi solve or warm start.  The solvers' workspace belongs to the
 *   context.
 */
#ifndef SGP_H
#define SGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SGP_OK = 0,
    SGP_ERR_INVALID_ARG = 1,    /* bad size, NULL pointer, non-positive or non-finite input */
    SGP_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    SGP_ERR_OOM = 3,            /* device allocation failed */
    SGP_ERR_DEGENERATE = 4,     /* two cells in contact share a centre: u of eq. (1) undefined */
    SGP_ERR_NOT_SPD = 5,        /* a pivot block or p^T Gamma p was not positive */
    SGP_ERR_NO_CONVERGENCE = 6, /* maxit reached; v holds the last iterate */
    SGP_ERR_TIMEOUT = 7         /* a bounded device wait gave up */
} sgp_status;

typedef enum {
    SGP_PREC_F64 = 0,   /* everything in FP64 */
    SGP_PREC_MIXED = 1  /* FP32 blocks and inner PCG inside FP64 iterative refinement */
} sgp_precision;

typedef enum {
    SGP_PRECOND_TREE = 0,          /* spanning-forest preconditioner (Section 3.1) */
    SGP_PRECOND_BLOCK_JACOBI = 1,  /* inverses of Gamma's 3x3 diagonal blocks (Section 5) */
    SGP_PRECOND_NONE = 2           /* plain CG */
} sgp_precond;

typedef enum {
    SGP_STOP_RESIDUAL = 0,  /* |r|_2 <= tol |F|_2 on the recursive residual */
    SGP_STOP_ERROR = 1      /* Gauss-Radau bound on the Gamma-norm error <= tol (Sections 4-5) */
} sgp_stop;

typedef struct sgp_ctx sgp_ctx;
typedef struct sgp_graph sgp_graph;
typedef struct sgp_matrix sgp_matrix;
typedef struct sgp_tree sgp_tree;
typedef struct sgp_factor sgp_factor;

typedef struct {
    double tol;          /* stop when |F - Gamma v|_2 <= tol |F|_2 (recursive residual), or
                            with stop = SGP_STOP_ERROR when the error bound is <= tol */
    int64_t maxit;       /* iteration cap (inner iterations in total for MIXED) */
    int32_t precond;     /* sgp_precond */
    int32_t precision;   /* sgp_precision; MIXED needs a matrix assembled with MIXED */
    int32_t x0_given;    /* 0: start from v = 0; 1: v holds the initial guess on entry */
    int32_t max_outer;   /* MIXED: refinement steps cap (<= 0 means 30) */
    double inner_tol;    /* MIXED: relative residual target of each FP32 inner solve (<= 0: 1e-3);
                            sgp_fcg_solve: that of each inner PCG (0: 0.1) */
    int32_t stop;        /* sgp_stop (sgp_pcg_solve in FP64 only; 0 elsewhere) */
    double mu;           /* SGP_STOP_ERROR: a lower bound of lambda_min(H Gamma) for the
                            Gauss-Radau rule; <= 0 takes 1 for the tree preconditioner
                            (Section 4: lambda_min(Gamma, P) >= 1) and gamma0 for none
                            (Lemma 2.4); block Jacobi needs it given */
} sgp_solve_opts;

typedef struct {
    int64_t iterations;        /* PCG iterations (inner iterations summed for MIXED and
                                  for sgp_fcg_solve) */
    int32_t outer_iterations;  /* MIXED refinement steps, or sgp_fcg_solve's flexible
                                  steps; 0 otherwise */
    int32_t status;            /* sgp_status of the solve */
    double rel_residual;       /* final recursive |r|/|F| (FP64 outer residual for MIXED) */
    double true_rel_residual;  /* |F - Gamma v|/|F| recomputed in FP64 at exit */
    double err_bound;          /* FP64 sgp_pcg_solve: Gauss-Radau upper bound on
                                  |v* - v|_Gamma / |v - v0|_Gamma at the last preconditioned
                                  residual the solve computed (v* the exact solution);
                                  0 elsewhere */
} sgp_solve_info;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device` whose work is ordered on `stream`
 * (a cudaStream_t; NULL means the legacy default stream). */
sgp_status sgp_create(sgp_ctx **ctx, int device, void *stream);
void sgp_destroy(sgp_ctx *ctx);
/* Reason for the last failure on this context ("" if none); owned by ctx. */
const char *sgp_last_error(const sgp_ctx *ctx);
/* Library version string, e.g. "sgp 0.1 sm_103a". */
const char *sgp_version(void);
/* Stream-ordered copy of `bytes` between two device buffers (for reading
 * arrays owned by handles, e.g. the edge list, into caller memory). */
sgp_status sgp_copy(sgp_ctx *ctx, void *dst_dev, const void *src_dev, int64_t bytes);

/* ---- Section 2, Steps 1-2: collision graph --------------------------------
 * Cells i < j are in contact iff |r_j - r_i| < R_i + R_j, evaluated in FP64
 * as sqrt((dx*dx + dy*dy) + dz*dz) with dx = x_j - x_i, round-to-nearest and
 * no fused multiply-add (Section 1.1: an edge wherever the contact area is
 * nonzero).  The edge list is canonical: pairs (i, j) with i < j, sorted by i
 * then j, so the result is independent of how the search is scheduled.
 * pos_dev: n x 3 float64; radii_dev: n float64, each > 0 and finite.
 * INVALID_ARG for n < 0, NULL pointers with n > 0, non-finite input or a
 * non-positive radius.  Synchronises (to size the edge list). */
sgp_status sgp_collision_graph(sgp_ctx *ctx, int64_t n, const double *pos_dev,
                               const double *radii_dev, sgp_graph **graph);
/* The same for a batch of independent configurations stored one after the
 * other: instance s owns cells [offsets[s], offsets[s+1]) (offsets: host
 * array of n_instances + 1 values, offsets[0] = 0, non-decreasing).  Cells
 * of different instances are never in contact, whatever their positions:
 * each instance gets its own cell grid.  The result is one canonical edge
 * list over global cell indices; assembly, spanning forest and tree factor
 * then work on the whole batch at once (a block-diagonal system).
 * Synchronises. */
sgp_status sgp_collision_graph_batched(sgp_ctx *ctx, int64_t n_instances, const int64_t *offsets,
                                       const double *pos_dev, const double *radii_dev, sgp_graph **graph);
/* n, m and the device edge list (m x 2 int32, owned by the graph). */
sgp_status sgp_graph_info(const sgp_graph *graph, int64_t *n, int64_t *m,
                          const int32_t **ij_dev);
void sgp_graph_destroy(sgp_graph *graph);

/* ---- Section 2, Step 3, eq. (1): friction blocks --------------------------
 * Upsilon_e = g_par u u^T + g_perp (I - u u^T), u = (r_j - r_i)/|r_j - r_i|,
 * for every edge e = (i, j) of the graph, in edge order; gamma_par_dev and
 * gamma_perp_dev hold m positive coefficients each (the contact area A_ij of
 * eq. (1) folded in).  Gamma is the block Laplacian of the collision graph
 * with self-loops gamma0 I (Section 2, Definition "Block Laplacian"):
 *   Gamma_ij = -Upsilon_e,  Gamma_ii = gamma0 I + sum_j Upsilon_ij.
 * The matrix keeps the blocks per directed edge (block-sparse rows, both
 * directions) in FP64, plus FP32 copies when precision is MIXED, and the
 * spanning-tree weight of Section 3.1, min(g_par, g_perp) = lambda_min
 * (Lemma 2.1).  gamma0 > 0.  DEGENERATE if two cells in contact coincide.
 * pos_dev must be the positions the graph was built from.  The rows are kept
 * in the graph's internal cell order (the cells sorted by uniform-grid cell,
 * by index inside a cell), so that cells close in space are close in memory;
 * every call below takes and returns cell vectors in the caller's order and
 * permutes them on the device. */
sgp_status sgp_friction_assemble(sgp_ctx *ctx, const sgp_graph *graph, const double *pos_dev,
                                 const double *gamma_par_dev, const double *gamma_perp_dev,
                                 double gamma0, int32_t precision, sgp_matrix **matrix);
/* Appendix B.2 matrix-free product y = Gamma v in FP64:
 *   y_i = gamma0 v_i + sum_{j ~ i} Upsilon_ij (v_i - v_j).
 * v_dev, y_dev: n x 3 float64, distinct buffers. */
sgp_status sgp_spmv(sgp_ctx *ctx, const sgp_matrix *matrix, const double *v_dev, double *y_dev);
/* y = Gamma v (as sgp_spmv) and *dot_dev = v^T y, allocating nothing.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run -- code inside a CUDA stream
 * capture (allocation calls are not allowed there), applications whose
 * device memory belongs to their own pool, or loops that cannot afford the
 * synchronisation of cudaMalloc/cudaFree.  Its scratch (one partial sum per
 * thread block and a counter, 33024 bytes) is a fixed array inside the
 * library that every GPU which loads the library keeps until the process
 * exits; hence at most 1,048,576 cells (4096 blocks of 256 rows): larger
 * matrices get SGP_ERR_INVALID_ARG.  sgp_create looks up the array's
 * device address, so every call, the first included, may run inside a
 * stream capture.  All calls share the array, which keeps the
 * last call's contents; its counter is cleared at the start of each call.
 * Calls whose GPU work overlaps (other streams or host threads) race on the
 * array.  v_dev, y_dev: n x 3 float64, distinct; dot_dev: one float64
 * (device).  Asynchronous on the context stream. */
sgp_status sgp_spmv_dot_noalloc(sgp_ctx *ctx, const sgp_matrix *matrix, const double *v_dev,
                                double *y_dev, double *dot_dev);
/* Copy the FP64 block of edge e (row-major 3x3) for every edge into
 * blocks_dev (m x 9 float64) and the tree weights into w_dev (m float64);
 * either pointer may be NULL. */
sgp_status sgp_matrix_edge_blocks(sgp_ctx *ctx, const sgp_matrix *matrix, double *blocks_dev,
                                  double *w_dev);
void sgp_matrix_destroy(sgp_matrix *matrix);

/* ---- Section 3.1: maximum spanning forest ----------------------------------
 * Boruvka's algorithm on the weights min(g_par, g_perp) under the strict
 * order (weight descending, then edge index ascending); under that order the
 * maximum spanning forest is unique.  A disconnected graph gives a forest
 * (one tree per connected component; isolated cells are single-vertex trees).
 * Up to 11264 cells every round runs in one thread block (one launch);
 * beyond, one round of launches at a time.  The forest is the same.
 * Synchronises (the round count is data dependent). */
sgp_status sgp_max_spanning_tree(sgp_ctx *ctx, const sgp_matrix *matrix, sgp_tree **tree);
/* Number of tree edges (n - components), the number of components and the
 * tree's edge ids (ascending, device int32 array owned by the tree). */
sgp_status sgp_tree_info(const sgp_tree *tree, int64_t *n_edges, int64_t *n_components,
                         const int32_t **edge_ids_dev);
void sgp_tree_destroy(sgp_tree *tree);

/* ---- Section 6: the partitioned ("local") spanning-forest preconditioner -----
 * The cells are split into spatial leaves; each leaf keeps the maximum
 * spanning forest of its own contacts, contacts between leaves are dropped,
 * and P_loc = gamma0 I + the block Laplacian of the union is block diagonal
 * over the leaves (its leaves are solved independently).  The forest is a
 * subgraph of the collision graph, so lambda_min(Gamma, P_loc) >= 1 still
 * holds (Section 4) and SGP_STOP_ERROR's mu = 1 stays valid.
 *
 * Leaf of every cell in the uniform grid of side h (the leaves of an octree
 * at one depth): k = floor(x / h) per axis (FP64, correctly rounded
 * division), label = (kx & 1023) | (ky & 1023) << 10 | (kz & 1023) << 20.
 * Leaves 1024 h apart along an axis share a label (no contact joins them).
 * pos_dev: n x 3 float64; leaf_dev: n int32, written.  INVALID_ARG unless
 * h is positive and finite. */
sgp_status sgp_grid_leaves(sgp_ctx *ctx, int64_t n, const double *pos_dev, double h, int32_t *leaf_dev);
/* The union of the leaves' maximum spanning forests: Boruvka under the same
 * strict order as sgp_max_spanning_tree over the contacts whose two cells
 * have equal labels in leaf_dev (n int32, any labels, the matrix's cell
 * numbering).  The result is an sgp_tree like that call's (sgp_tree_info,
 * sgp_tree_factor, the tree preconditioner of the solvers). */
sgp_status sgp_local_spanning_forest(sgp_ctx *ctx, const sgp_matrix *matrix, const int32_t *leaf_dev,
                                     sgp_tree **tree);

/* ---- Section 3.3 (Algorithm 2) and Appendix B.1: tree factor ----------------
 * P = gamma0 I + block Laplacian of the spanning forest (the self-loops kept,
 * Section 3.1) is factored P = L D L^T by block elimination.  The elimination
 * order comes from rake/compress tree contraction: each round eliminates every
 * leaf, then an independent set of degree-2 vertices, so any tree takes
 * O(log n) rounds.  Pivots D and their inverses are computed in FP64; MIXED
 * matrices also get FP32 copies of L and D^-1 for the inner solves.
 * NOT_SPD if a pivot is not positive definite.  Synchronises (the round count
 * is data dependent). */
sgp_status sgp_tree_factor(sgp_ctx *ctx, const sgp_matrix *matrix, const sgp_tree *tree,
                           sgp_factor **factor);
/* x = P^{-1} b in FP64 (forward substitution, diagonal solve, backward
 * substitution, Appendix B.1).  b_dev, x_dev: n x 3 float64; may alias. */
sgp_status sgp_tree_apply(sgp_ctx *ctx, const sgp_factor *factor, const double *b_dev,
                          double *x_dev);
/* Shape of the factor: contraction levels (rounds == levels: each level
 * eliminates leaves and degree-2 vertices together), the number of L blocks
 * (one per eliminated vertex and current neighbour) and of receiver entries
 * (vertex, level) of the forward substitution.  Any pointer may be NULL. */
sgp_status sgp_factor_info(const sgp_factor *factor, int32_t *rounds, int32_t *levels,
                           int64_t *l_blocks, int64_t *receiver_entries);
/* Layout of the factor's binned solve: number of bins, vertices of the top
 * part (solved by one thread block), products sent from bins to the top
 * ("leaks"), the subtree bound, and whether the FP32 and FP64 applications
 * use it (1) or run one launch per contraction level (0: the layout is off
 * or does not fit in shared memory).  Any pointer may be NULL. */
sgp_status sgp_factor_layout(const sgp_factor *factor, int32_t *bins, int32_t *top, int32_t *leaks,
                             int32_t *bin_cap, int32_t *fp32, int32_t *fp64);
void sgp_factor_destroy(sgp_factor *factor);

/* ---- Section 1.1: preconditioned conjugate gradients ------------------------
 * Solves Gamma v = F.  r = F - Gamma v0, z = H r, p = z, rho = r^T z; each
 * iteration: q = Gamma p, alpha = rho / p^T q, v += alpha p, r -= alpha q,
 * stop when |r|_2 <= tol |F|_2, z = H r, beta = r^T z / rho, p = z + beta p.
 * SGP_STOP_ERROR (FP64 only; the paper monitors CG with Gauss-Radau error
 * estimates, Section 5): after each new rho the Gauss-Radau upper bound of
 * the Gamma-norm error, phi rho with phi_0 = 1/mu and
 * phi <- (phi - alpha) / (mu (phi - alpha) + beta), is compared with
 * tol^2 sum_j alpha_j rho_j (= |v - v0|_Gamma^2); the solve stops when the
 * bound is below it, so |v* - v|_Gamma <= tol |v - v0|_Gamma in exact
 * arithmetic.  Scalars only: no extra pass over memory.
 * H is P^{-1} from `factor` (required for SGP_PRECOND_TREE), the block-Jacobi
 * inverse (computed inside the call) or I.  MIXED runs FP64 iterative
 * refinement: r = F - Gamma v in FP64, an FP32 inner PCG on r/|r| to
 * inner_tol (FP64 dot products), v += |r| d, until |r| <= tol |F|.  A
 * MIXED tree-preconditioned solve of a small system (every contraction level
 * in the factor's one-block tail and its vectors within one block's shared
 * memory: about a thousand cells) runs the whole refinement in one launch
 * of one thread block; the results are those of the same algorithm
 * (dot products summed in FP32 within a warp, in FP64 across warps).
 * F_dev, v_dev: n x 3 float64.  A zero F returns v = 0 after 0 iterations.
 * On NO_CONVERGENCE v holds the last iterate and info is filled.
 * info (host, may be NULL) receives the statistics.  Synchronises. */
sgp_status sgp_pcg_solve(sgp_ctx *ctx, const sgp_matrix *matrix, const sgp_factor *factor,
                         const double *F_dev, double *v_dev, const sgp_solve_opts *opts,
                         sgp_solve_info *info);

/* Batched PCG: every instance s of a block-diagonal matrix (assembled from a
 * batched collision graph with the same offsets) is solved for its own
 * Gamma_ss v_s = F_s with its own scalars (alpha, beta, rho) and its own
 * stopping test |r_s| <= tol |F_s|; all instances share each kernel launch
 * and the tree factor of the whole batch.  Converged instances drop out of
 * the products and vector updates.  Iterations are replayed as CUDA graphs.
 * opts as for sgp_pcg_solve (maxit per instance).  infos (host, n_instances
 * entries, may be NULL) receives each instance's statistics.  Returns the
 * first failing status (NOT_SPD before NO_CONVERGENCE); INVALID_ARG if an
 * edge joins two instances or if the matrix's internal cell order mixes
 * instances (a matrix built on a graph from sgp_collision_graph over the
 * whole union instead of sgp_collision_graph_batched).  Synchronises. */
sgp_status sgp_pcg_solve_batched(sgp_ctx *ctx, const sgp_matrix *matrix, const sgp_factor *factor,
                                 int64_t n_instances, const int64_t *offsets, const double *F_dev,
                                 double *v_dev, const sgp_solve_opts *opts, sgp_solve_info *infos);

/* ---- Section 3.1 (Vaidya's second preconditioner), Sections 3.3 and 5 --------
 * Augmented spanning forest.  The forest of `tree` is cut into pieces: every
 * tree is rooted at its smallest cell id, a depth-first preorder visits
 * children in ascending id order and the trees in ascending order of their
 * roots, and with s = ceil(n/t) a piece is a maximal set of tree-connected
 * cells whose preorder numbers share one block [k s, (k+1) s) (connected
 * subtrees of at most s cells, at least t of them, numbered in preorder of
 * their top cell).  For every pair of pieces that the collision graph joins,
 * the heaviest edge between them (weight descending, then edge index
 * ascending) is added back; the augmented forest T' is the union with the
 * tree edges and P' = gamma0 I + block Laplacian of T'.  t = 0 takes
 * round(n^(1/4)) (the section's optimum).  *aug is created, or rebuilt in
 * place when non-NULL.  INVALID_ARG for t < 0 or a tree that does not belong
 * to the matrix.  Synchronises. */
typedef struct sgp_aug sgp_aug;
sgp_status sgp_augment_tree(sgp_ctx *ctx, const sgp_matrix *matrix, const sgp_tree *tree, int32_t t,
                            sgp_aug **aug);
/* t used, number of pieces, the piece bound s, edges of T' and how many of
 * them are not tree edges.  Any pointer may be NULL. */
sgp_status sgp_aug_info(const sgp_aug *aug, int32_t *t, int32_t *pieces, int32_t *piece_cap, int64_t *edges,
                        int64_t *added);
/* piece_dev (n int32, device): the piece of every cell.  Asynchronous. */
sgp_status sgp_aug_pieces(sgp_ctx *ctx, const sgp_aug *aug, int32_t *piece_dev);
/* edges_dev (edges int32, device): the edge ids of T', ascending.  Asynchronous. */
sgp_status sgp_aug_edges(sgp_ctx *ctx, const sgp_aug *aug, int32_t *edges_dev);
/* P' as a matrix handle (FP64) owned by `aug`: sgp_spmv gives P' v, and
 * sgp_pcg_solve with the plain forest factor solves P' z = r -- the inner
 * solve of sgp_fcg_solve.  NULL for a NULL aug. */
const sgp_matrix *sgp_aug_matrix(const sgp_aug *aug);
void sgp_aug_destroy(sgp_aug *aug);

/* Flexible CG (Section 5: "nested (flexible) conjugate gradient") on
 * Gamma v = F with the augmented preconditioner: each outer step applies
 * z = P'^-1 r approximately by an inner PCG on P' preconditioned by the plain
 * forest `factor` (from z = 0, to |r_in| <= inner_tol |r| with
 * opts->inner_tol, 0 = 0.1 as in the paper, or inner_maxit iterations), then
 * keeps one previous direction (Notay's flexible CG with truncation 1):
 *   p = z - (z^T q_prev / p_prev^T q_prev) p_prev, q = Gamma p,
 *   alpha = p^T r / p^T q, v += alpha p, r -= alpha q,
 * until |r|_2 <= opts->tol |F|_2 or opts->maxit outer steps.  FP64 only
 * (opts->precision F64, opts->precond TREE).  info->outer_iterations counts
 * the outer steps, info->iterations the inner PCG iterations of all of them.
 * INVALID_ARG if `aug` or `factor` was not built from this matrix.
 * Synchronises. */
sgp_status sgp_fcg_solve(sgp_ctx *ctx, const sgp_matrix *matrix, const sgp_aug *aug, const sgp_factor *factor,
                         const double *F_dev, double *v_dev, const sgp_solve_opts *opts, int64_t inner_maxit,
                         sgp_solve_info *info);

/* ---- learned warm start (no counterpart in the paper) -----------------------
 * A message-passing network over the collision graph predicts the initial
 * guess v0 of the PCG of Section 1.1; the solver's own iteration count
 * measures the prediction.  Width 64, three message-passing layers, BF16
 * weights (round-to-nearest-even copies of FP32 master weights), FP32
 * activations and accumulation:
 *   basis  b0 = D^-1 F (block Jacobi), b1 = P^-1 F (spanning-forest factor),
 *          b2 = v_prev (zero when NULL)
 *   x_i    = |b0|, |b1|, |b2| / s; b0.b1, b0.b2, b1.b2 / s^2 (s = mean |b1|),
 *            deg_i / 6, 1
 *   h0 = relu(W_in x + b_in); h_{l+1} = relu(W_l [h_l ; mean_{j~i} h_l,j] + c_l)
 *   c = W_out h3 + b_out; v0_i = sum_k c_ik b_i^(k)
 * Parameters (FP32, flat, SGP_MPNN_PARAMS values) in the order W_in (64x8),
 * b_in (64), then W_l (64x128), c_l (64) for l = 0, 1, 2, then W_out (3x64),
 * b_out (3); matrices row-major.  Training minimises, with Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8), either loss against the converged solution v*:
 *   SGP_MPNN_LOSS_L2:     |v0 - v*|^2 / |v*|^2
 *   SGP_MPNN_LOSS_ENERGY: (v0 - v*)^T Gamma (v0 - v*) / v*^T Gamma v*, the
 *                         error norm conjugate gradients minimises. */
typedef struct sgp_mpnn sgp_mpnn;
#define SGP_MPNN_PARAMS 25539
#define SGP_MPNN_LOSS_L2 0
#define SGP_MPNN_LOSS_ENERGY 1
#define SGP_WARM_MR_SCALE 1
/* Create a network from `count` (== SGP_MPNN_PARAMS) host FP32 parameters
 * (copied; the caller keeps ownership).  INVALID_ARG on a wrong count. */
sgp_status sgp_mpnn_create(sgp_ctx *ctx, const float *params_host, int64_t count, sgp_mpnn **net);
void sgp_mpnn_destroy(sgp_mpnn *net);
/* Copy the FP32 master parameters and/or the last gradient (each
 * SGP_MPNN_PARAMS floats, host) out; either pointer may be NULL.
 * Synchronises. */
sgp_status sgp_mpnn_params(sgp_ctx *ctx, const sgp_mpnn *net, float *params_host, float *grads_host);
/* Inference: v0_dev (n x 3 float64) from F_dev (n x 3), the matrix (for the
 * neighbours and the block-Jacobi inverse), the factor of the same matrix
 * and v_prev_dev (n x 3, or NULL).  Activations are kept in `net` for a
 * following sgp_mpnn_backward; `matrix` must outlive that call.
 * Asynchronous apart from building the block-Jacobi inverse once. */
sgp_status sgp_mpnn_forward(sgp_ctx *ctx, sgp_mpnn *net, const sgp_matrix *matrix,
                            const sgp_factor *factor, const double *F_dev, const double *v_prev_dev,
                            double *v0_dev);
/* Gradient of loss `loss_kind` (SGP_MPNN_LOSS_*) of the last forward pass
 * against the target v_target_dev (n x 3 float64, the converged solution),
 * kept in `net`; loss (host, may be NULL) receives the loss value
 * (synchronises then).  The energy loss uses the matrix of the forward pass.
 * The weight gradients are reduced in a fixed order: the same inputs give
 * the same bits.  INVALID_ARG for an unknown loss or before any forward. */
sgp_status sgp_mpnn_backward(sgp_ctx *ctx, sgp_mpnn *net, const double *v_target_dev, int32_t loss_kind,
                             double *loss);
/* One Adam step with learning rate lr > 0 on the last gradient; refreshes
 * the BF16 weights.  Asynchronous. */
sgp_status sgp_mpnn_step(sgp_ctx *ctx, sgp_mpnn *net, float lr);
/* sgp_mpnn_forward, then (flag SGP_WARM_MR_SCALE) the minimal-residual
 * rescaling v0 <- alpha v0, alpha = (Gamma v0)^T F / |Gamma v0|^2, then the
 * acceptance test: v0 is kept when |F - Gamma v0| <= |F| (FP64), else set to
 * 0 (the zero guess has the smaller residual).  After a finite positive-
 * denominator rescaling the test holds by construction (the minimal-residual
 * step cannot raise the residual) and is not evaluated; otherwise it costs
 * one more FP64 product.  used (host, may be NULL) receives 1 if v0 was
 * kept.  INVALID_ARG for unknown flags.  Synchronises. */
sgp_status sgp_warm_start(sgp_ctx *ctx, sgp_mpnn *net, const sgp_matrix *matrix,
                          const sgp_factor *factor, const double *F_dev, const double *v_prev_dev,
                          double *v0_dev, int32_t flags, int32_t *used);

/* ---- tuning (no counterpart in the paper) -----------------------------------
 * Launch-shape knobs of the solver, kept per context. */
typedef struct {
    int32_t spmv_lpr;    /* lanes per block row of the PCG product: 1, 2, 4 or 8;
                            0 = default (1 for FP64, 2 for FP32) */
    int32_t tail_cap;    /* the tree solve runs its last contraction levels in one
                            thread block once at most tail_cap vertices are left
                            (-1: as many as fit in shared memory; 0: no tail;
                            default 1024); read when a factor is built */
    int32_t batch_chunk; /* rows per work item of the batched solver: 0 (default
                            2048) or 256..65536 */
    int32_t spmv_ilp;    /* row groups each lane of the PCG product keeps in flight
                            at once: 0 (default, 1), 1 or 2 */
    int32_t bin_cap;     /* the tree solve's thread-block bins: contraction subtrees
                            of at most bin_cap vertices are solved by one thread
                            block each (three launches per application); 0 =
                            default (1024 for the FP32 solve of a MIXED factor;
                            FP64 solves run one launch per contraction level),
                            -1 = off in both precisions, 64..8192 = that cap in
                            both precisions; read when a factor is built */
    double ms_per_iteration; /* sgp_autotune: the winning objective (ms per PCG
                                iteration, or per factor build + solve); 0 from
                                sgp_get_tuning */
} sgp_tuning;
sgp_status sgp_get_tuning(const sgp_ctx *ctx, sgp_tuning *tuning);
/* INVALID_ARG for a value outside the ranges above (nothing is changed). */
sgp_status sgp_set_tuning(sgp_ctx *ctx, const sgp_tuning *tuning);
/* Pick the knobs by timing the caller's own system for each candidate, one
 * knob after the other: tail_cap in {0, 256, 512, 1024, 2048, 4096, -1} and
 * bin_cap in {0, -1, 512, 1024, 2048} (tree preconditioner only; *factor is
 * rebuilt from `tree` for each candidate and left built with the chosen
 * values), then
 * spmv_lpr in {1, 2, 4, 8} with spmv_ilp in {1, 2}, then, when n_instances > 0
 * (a batch with host `offsets`, as for sgp_pcg_solve_batched), batch_chunk in
 * {512, ..., 8192} with the batched solver timed throughout.  The objective
 * is the time of one PCG iteration when iterations > 0 (each timed solve
 * runs exactly that many iterations; opts->tol is ignored), or, when
 * iterations == 0, the time of a whole solve to opts->tol plus the factor
 * build of the candidate (the cost of one time step).  The choice is stored
 * in the context and copied to `out` (may be NULL; ms_per_iteration then
 * holds the winning objective).  F_dev is only read.  On failure the previous
 * tuning is restored.  Synchronises. */
sgp_status sgp_autotune(sgp_ctx *ctx, const sgp_matrix *matrix, const sgp_tree *tree, sgp_factor **factor,
                        int64_t n_instances, const int64_t *offsets, const double *F_dev,
                        const sgp_solve_opts *opts, int32_t iterations, sgp_tuning *out);

/* ---- kernel timing ----------------------------------------------------------
 * When enabled, the library brackets every launch of the named kernel class
 * with CUDA events on the context stream and accumulates the elapsed time,
 * read back at the next synchronising call.  For roofline reporting. */
typedef enum {
    SGP_KT_SPMV = 0,       /* Gamma p products inside PCG (FP64 or FP32) */
    SGP_KT_TREE_SOLVE = 1, /* one whole P^{-1} r application */
    SGP_KT_PCG_VECTOR = 2, /* PCG vector updates and reductions */
    SGP_KT_WARM_BASIS = 3, /* warm start: the three basis fields (block-Jacobi and
                              spanning-forest solves of F, v_prev) and the features */
    SGP_KT_WARM_LAYERS = 4, /* warm start: the network's dense layers, aggregations and
                               output mix */
    SGP_KT_WARM_CHECK = 5, /* warm start: minimal-residual scaling and acceptance test */
    SGP_KT_COUNT = 6
} sgp_kernel_class;
sgp_status sgp_set_kernel_timing(sgp_ctx *ctx, int32_t enable);
/* Total milliseconds and launch count since the last reset. */
sgp_status sgp_kernel_time(sgp_ctx *ctx, int32_t kernel_class, double *total_ms,
                           int64_t *launches, int32_t reset);
/* Number of kernels this context has launched (every kernel of every call,
 * counted on the host at launch); reset to 0 when `reset` is nonzero. */
sgp_status sgp_launch_count(sgp_ctx *ctx, int64_t *count, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* SGP_H */
