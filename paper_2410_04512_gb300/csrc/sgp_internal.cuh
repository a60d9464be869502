// sgp_internal.cuh -- shared declarations of the sm_103a library behind sgp.h.
//
// Block storage conventions:
//   sym6: a symmetric 3x3 block as {xx, xy, xz, yy, yz, zz}
//   full9: a general 3x3 block, row-major
// Vectors of cells are n x 3, row-major (AoS), in the caller's cell order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/sgp.h"

// ---------------------------------------------------------------------------
// host side: context, errors, launches, buffers
// ---------------------------------------------------------------------------
struct KtRec {
    int cls;
    cudaEvent_t a, b;
};

// A captured chunk of solver work, replayed with cudaGraphLaunch.
struct GraphEntry {
    uint64_t key[32];
    int nkey = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;          // kernel nodes per replay
    std::vector<KtRec> ev;        // timing events recorded by the graph
    uint64_t last_use = 0;
};

struct sgp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;
    // pinned staging for small device->host reads
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    // kernel timing
    int timing = 0;
    double kt_ms[SGP_KT_COUNT] = {};
    int64_t kt_n[SGP_KT_COUNT] = {};
    std::vector<cudaEvent_t> ev_free;
    std::vector<cudaEvent_t> ev_pending[SGP_KT_COUNT];  // start,end pairs
    // the no-allocation product's fixed scratch array (noalloc.cu)
    void *noalloc_scratch = nullptr;
    // device scratch of the solver (vectors, partials, scalars); may grow
    void *d_scratch = nullptr;
    size_t d_scratch_bytes = 0;
    // fixed 4 KB of device flags (error words), never reallocated
    int *d_flags = nullptr;
    // scan workspace (grows; only the scan touches it)
    void *d_scan = nullptr;
    size_t d_scan_bytes = 0;
    // tuning knobs (0 = built-in default)
    int spmv_lpr = 0;
    int spmv_ilp = 0;       // row groups in flight per lane in the product (0: 1)
    int tail_cap = 1024;    // largest tail of the tree solve in vertices (-1: what fits)
    int bin_cap = 0;        // largest contraction subtree solved by one thread block: 0 = 1024 for the
                            // FP32 solve only, -1 = level kernels only, else that cap in both precisions
    int fused = 1;          // PCG step fused around the binned tree solve
    int small_solve = 1;    // whole mixed solves of small systems in one thread block
    int use_pdl = 1;        // programmatic dependent launch of the level kernels
    int batch_chunk = 0;    // rows per work item of the batched solver
    int num_sms = 0;
    std::vector<std::pair<const void *, int>> occupancy;  // kernel -> resident blocks/SM
    // CUDA graphs of solver chunks (captured on a private stream)
    int use_graphs = 1;
    int use_while = 1;      // device-side iteration loops (conditional graph nodes)
    cudaStream_t cap_stream = nullptr;
    std::vector<KtRec> *capture_sink = nullptr;
    std::vector<GraphEntry *> graphs;
    uint64_t graph_clock = 0;
};

// Grid of at most one full wave: min(want, SMs x resident blocks per SM of
// `kernel` at `block` threads), cached per kernel.
sgp_status resident_grid(sgp_ctx *ctx, const void *kernel, int block, int64_t want, unsigned *grid);

// Unique generation numbers for rebuilt handles (graph cache keys).
uint64_t next_generation();
sgp_status noalloc_prepare(sgp_ctx *ctx);
sgp_status graph_lookup(sgp_ctx *ctx, const uint64_t *key, int nkey, GraphEntry **out);
sgp_status graph_begin(sgp_ctx *ctx, GraphEntry *ge, cudaStream_t *saved, int64_t *l0);
sgp_status graph_end(sgp_ctx *ctx, GraphEntry *ge, cudaStream_t saved, int64_t l0, sgp_status st);
sgp_status graph_collect_timing(sgp_ctx *ctx, GraphEntry *ge);
void graph_release_all(sgp_ctx *ctx);

// A device-side loop: `fn` (one chunk of solver iterations) is captured as
// the body of a conditional WHILE node; a one-thread kernel appended to the
// body counts the executions in *bodies and keeps the loop going while *done
// is 0 and fewer than max_bodies bodies have run in this launch.
sgp_status graph_while_begin(sgp_ctx *ctx, GraphEntry *ge, cudaStream_t *saved, int64_t *l0, cudaGraph_t *g,
                             cudaGraphConditionalHandle *h);
sgp_status graph_while_end(sgp_ctx *ctx, GraphEntry *ge, cudaStream_t saved, int64_t l0, cudaGraph_t g,
                           cudaGraphConditionalHandle h, const int *done, int *bodies, int max_bodies,
                           sgp_status st);
template <typename Fn>
sgp_status graph_capture_while(sgp_ctx *ctx, GraphEntry *ge, const int *done, int *bodies, int max_bodies, Fn fn)
{
    cudaStream_t saved;
    int64_t l0;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h{};
    sgp_status st = graph_while_begin(ctx, ge, &saved, &l0, &g, &h);
    if (st != SGP_OK) return st;
    st = fn();
    return graph_while_end(ctx, ge, saved, l0, g, h, done, bodies, max_bodies, st);
}

// Capture the work `fn` enqueues on ctx->stream into ge->exec.
template <typename Fn>
sgp_status graph_capture(sgp_ctx *ctx, GraphEntry *ge, Fn fn)
{
    cudaStream_t saved;
    int64_t l0;
    sgp_status st = graph_begin(ctx, ge, &saved, &l0);
    if (st != SGP_OK) return st;
    st = fn();
    return graph_end(ctx, ge, saved, l0, st);
}

sgp_status sgp_fail(sgp_ctx *ctx, sgp_status code, const char *fmt, ...);

#define SGP_TRY(...)                          \
    do {                                      \
        sgp_status s_ = (__VA_ARGS__);        \
        if (s_ != SGP_OK) return s_;          \
    } while (0)

#define SGP_CUDA(ctx, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return sgp_fail((ctx), e_ == cudaErrorMemoryAllocation ? SGP_ERR_OOM : SGP_ERR_CUDA, \
                            "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Launch a kernel on the context stream, count it and check the launch.
template <typename... KArgs, typename... Args>
static inline sgp_status sgp_launch(sgp_ctx *ctx, const char *name, void (*k)(KArgs...), dim3 grid,
                                    dim3 block, size_t smem, Args... args)
{
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return SGP_OK;
    k<<<grid, block, smem, ctx->stream>>>(args...);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return sgp_fail(ctx, SGP_ERR_CUDA, "launch of %s failed: %s", name, cudaGetErrorString(e));
    return SGP_OK;
}
#define LAUNCH(ctx, kern, grid, block, smem, ...) \
    SGP_TRY(sgp_launch((ctx), #kern, kern, dim3(grid), dim3(block), (smem), __VA_ARGS__))

static inline unsigned grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 0 : g);
}

// Stream-ordered device buffer owned by a handle.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
};
sgp_status buf_ensure(sgp_ctx *ctx, DBuf &b, size_t bytes);
void buf_release(DBuf &b, cudaStream_t s);
template <typename T>
static inline T *bp(const DBuf &b) { return reinterpret_cast<T *>(b.p); }

// Copy `bytes` from device to host through the pinned stage and synchronise.
sgp_status read_back(sgp_ctx *ctx, void *host, const void *dev, size_t bytes);
// Ensure ctx->d_scratch has at least `bytes` (used by reductions and scans).
sgp_status scratch_ensure(sgp_ctx *ctx, size_t bytes);

// Device-wide exclusive scan of n int32 values into out[0..n]; out[n] is
// the total.  `in` and `out` may alias.  Deterministic.
sgp_status scan_exclusive_i32(sgp_ctx *ctx, const int32_t *in, int32_t *out, int64_t n);

// z = P^-1 w in place (internal cell order); kernels return at once when
// *done is set.
template <typename T>
sgp_status tree_apply_inplace(sgp_ctx *ctx, const sgp_factor *F, T *w, const int *done);

// The binned tree solve (bins.cu).  bins_build runs at the end of a factor
// build; bins_usable tells whether precision T has a layout that fits;
// bins_apply is z = P^-1 w in place; bins_pcg_step is one PCG step around
// the solve (r -= alpha q, |r|^2 and the stopping test, z = P^-1 r, r^T z and
// beta) with the scalars in `scal` (the solver's device scalar block);
// bins_check reports a bounded device wait that gave up.
// The fused solve runs in the layout's own cell order (tree order,
// BinLayout::NT cells, padding zero): bins_tree_ready tells whether the
// factor holds the matrix's rows in that order for this assembly;
// bins_to_tree / bins_from_tree move vectors between the orders;
// bins_apply_tree is z = P^-1 w on tree-order vectors.
struct sgp_factor;
struct sgp_matrix;
sgp_status bins_build(sgp_ctx *ctx, sgp_factor *F, const sgp_matrix *M);
template <typename T>
bool bins_usable(const sgp_factor *F);
template <typename T>
bool bins_tree_ready(const sgp_factor *F, const sgp_matrix *M);
template <typename T>
sgp_status bins_apply(sgp_ctx *ctx, const sgp_factor *F, T *w, const int *done);
template <typename T>
sgp_status bins_apply_tree(sgp_ctx *ctx, const sgp_factor *F, T *w, T *z, const int *done);
template <typename T>
sgp_status bins_to_tree(sgp_ctx *ctx, const sgp_factor *F, const T *src, T *dst);
template <typename T>
sgp_status bins_from_tree(sgp_ctx *ctx, const sgp_factor *F, const T *src, T *dst);
template <typename T>
sgp_status bins_pcg_step(sgp_ctx *ctx, const sgp_factor *F, T *r, const T *q, T *z, void *scal);
sgp_status bins_check(sgp_ctx *ctx, const sgp_factor *F);

// Kernel timing hooks (no-ops unless enabled on the context).
sgp_status kt_begin(sgp_ctx *ctx, int kclass, cudaEvent_t *ev);
sgp_status kt_end(sgp_ctx *ctx, int kclass, cudaEvent_t ev);
sgp_status kt_collect(sgp_ctx *ctx);  // after a stream synchronisation

// ---------------------------------------------------------------------------
// handle types
// ---------------------------------------------------------------------------
struct sgp_graph {
    int64_t n = 0, m = 0;
    DBuf ij;       // m x 2 int32, canonical (i < j), sorted
    DBuf up_ptr;   // n + 1 int32: edges of row i are [up_ptr[i], up_ptr[i+1])
    // cell-list scratch kept for reuse
    DBuf cell_id, cell_cnt, cell_start, perm, spos, spos32, cnt, bbox, inst, grids;
    DBuf int_of;   // n int32: position of each cell in grid-cell order (perm is the inverse)
    DBuf cand;     // n x 24 int32: the first contacts of each cell found by the search
};

struct sgp_matrix {
    uint64_t gen = 0;
    int64_t n = 0, m = 0;
    double gamma0 = 0;
    int32_t precision = SGP_PREC_F64;
    DBuf ij;         // m x 2 int32 (copy of the graph's edge list)
    DBuf row_ptr;    // n + 1 int32 over 2m directed slots, columns ascending in a row
    DBuf col;        // 2m int32
    DBuf blk;        // 2m x sym6 float64
    DBuf blk32;      // MIXED only: 2m float4 (g_perp, g_par - g_perp, u_x, u_y), then 2m float2 (u_z, col bits)
    DBuf edge_slot;  // m int32: slot of each edge (i, j) in row int_of[i]
    DBuf edge_slot_j;  // m int32: slot of each edge (i, j) in row int_of[j]
    DBuf w;          // m float64 tree weight min(g_par, g_perp)
    DBuf slot_edge;  // 2m int32 (scratch)
    DBuf lowcnt, cursor;
    // The matrix rows (and every vector the solvers use internally) follow
    // the grid-cell order of the collision graph, so that cells in contact
    // sit close together in memory; orig_of / int_of translate to and from
    // the caller's cell order.  ij, edge_slot and w stay in edge order.
    DBuf orig_of, int_of;  // n int32 each
    DBuf jac;        // n x sym6 float64 block-Jacobi inverse (built lazily)
    DBuf jac32;      // n x sym6 float32
    int jac_valid = 0;
};

struct sgp_tree {
    int64_t n = 0, nt = 0, ncomp = 0;
    DBuf edges;   // nt int32 tree edge ids, ascending
    DBuf comp;    // n int32 component label
    DBuf bestw, beste, hook, intree, flag, idx;
};

// The binned layout of the tree solve (bins.cu): the contraction tree cut
// into bins of subtrees with at most bmax vertices and the top part above
// them.  Per-bin arrays are padded to 4 entries so that every segment starts
// on a 16-byte boundary (bulk copies).  Index [0] of the numeric arrays is
// FP32, [1] FP64.
struct BinLayout {
    int ok32 = 0, ok64 = 0;
    int32_t nb = 0, nt = 0, LV = 0, LVP = 0, bmax = 0;
    int32_t G = 0, E = 0, Cc = 0, K = 0, Pp = 0, Z = 0;
    int32_t ntt = 0, nte = 0, ntp = 0, nly = 0, tints = 0;
    int32_t toff[9] = {0};
    int32_t NT = 0;                    // length of a tree-order vector (cells)
    size_t smA[2] = {0, 0}, smT[2] = {0, 0}, smC[2] = {0, 0};   // fused PCG step
    size_t smA0[2] = {0, 0}, smC0[2] = {0, 0};                  // plain solve
    size_t smTnd[2] = {0, 0};                                   // top without staged pivots
    DBuf hdr, elev, vlev, gvert, er, ec, cl, kl, ks, pr, pref, zi, tv, tint;
    DBuf order;                        // bins in launch order: most levels first
    DBuf c_src, k_src, p_src, d_src, t_src, tD_src;
    DBuf cL[2], kL[2], pL[2], D[2], tL[2], tD[2];
    DBuf ly[2], lsum[2], tw[2], part, err;
    // tree order <-> the matrix's internal order, and the matrix's rows in
    // tree order (FP32 eq. (1) records for MIXED, FP64 blocks and columns
    // for F64) from the assembly of generation mgen
    DBuf i_of_t, t_of_i, rpt, ma32, mb32, m64, mc64;
    uint64_t mgen = 0;
    int mat32 = 0, mat64 = 0;
    DBuf scr[64];
};

struct sgp_factor {
    uint64_t gen = 0;
    int64_t n = 0, npairs = 0;
    int32_t rounds = 0, levels = 0;
    int32_t precision = SGP_PREC_F64;
    std::vector<int32_t> lvl_ptr;   // host, levels + 1: positions of each level in ord
    std::vector<int32_t> rl_ptr;    // host, levels + 1: receivers of each level in rv
    std::vector<int32_t> pl_ptr;    // host, levels + 1: pairs of each level
    std::vector<int32_t> cl_ptr;    // host, levels + 1: contributor entries of each level
    DBuf ord;       // n int32 vertex eliminated at each position
    DBuf pr_ptr;    // n + 1 int32 pairs (receivers) of each position
    DBuf pr_q;      // npairs int32 receiver vertex of each pair
    DBuf pr_c;      // npairs int32 contributor vertex of each pair
    DBuf rv;        // receivers, level by level, ascending vertex id within a level
    DBuf rc_ptr;    // (#receivers + 1) int32 into ct
    DBuf ct;        // npairs int32 pair ids grouped by receiver
    DBuf L, Dinv;   // npairs x full9, n x sym6 (by position), float64
    DBuf L32, Dinv32;
    DBuf ctv;       // contributor vertex per contributor entry (ct order)
    DBuf Lf, Lf32;  // L blocks in ct order (forward pass streams them)
    // tail: levels >= tail_level run in one thread block (positions >= tail_P0)
    int32_t tail_level = 0, tail_P0 = 0, tail_R0 = 0, tail_C0 = 0, tail_Q0 = 0;
    DBuf tail_idx;  // level positions and receiver offsets of the tail levels
    DBuf tail_q, tail_c, tail_b;  // local indices (position - tail_P0)
    DBuf work;      // n x 3 float64 apply workspace
    DBuf orig_of;   // n int32: the matrix's internal cell order (vectors are solved in it)
    DBuf small;     // counts of the short-tail contraction kernel (header + per-level records)
    BinLayout bl;
    // structure-simulation scratch
    DBuf adj_ptr, nbr, twin, eref, deg, lev, nrec, rq, re, ren, pos, flag, alive_a, alive_b,
        acc, fill, sbuf, tmp, rflag, cnt;
};

// Vaidya's augmented spanning forest (augment.cu): the pieces of the
// forest, the edges of T' and P' = gamma0 I + block Laplacian of T' as a
// matrix in the same internal order as the matrix it was built from.
#define SGP_AUG_SCRATCH 40
struct sgp_aug {
    int64_t n = 0, m = 0;           // cells, edges of the source matrix
    int32_t t = 0, s = 0, npieces = 0;
    int64_t nedges = 0, added = 0;  // edges of T', of which not tree edges
    uint64_t mgen = 0;              // generation of the source matrix
    DBuf piece;                     // n int32: piece of each cell (caller order)
    DBuf edges;                     // nedges int32: edge ids of T', ascending
    sgp_matrix *P = nullptr;        // P' (FP64)
    DBuf scr[SGP_AUG_SCRATCH];
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#define SGP_BLOCK 256
// Shared memory budget of the single-block tail of the tree solve (all the
// tail's vectors, pivots, L blocks and index lists, sized for FP64).
#define TREE_TAIL_SMEM (200 * 1024)

// Launch with programmatic stream serialisation (the kernel may start while
// the previous one finishes; it must griddepcontrol.wait before consuming).
template <typename... KArgs, typename... Args>
static inline sgp_status sgp_launch_pdl(sgp_ctx *ctx, const char *name, void (*k)(KArgs...), dim3 grid,
                                        dim3 block, size_t smem, Args... args)
{
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return SGP_OK;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = ctx->use_pdl;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
    ctx->launches++;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess)
        return sgp_fail(ctx, SGP_ERR_CUDA, "launch of %s failed: %s", name, cudaGetErrorString(e));
    return SGP_OK;
}
// Programmatic dependent launch: a kernel launched with LAUNCH_PDL may start
// while the previous kernel in the stream is still running; pdl_wait()
// returns once that kernel has completed and its memory is visible, so
// everything that reads what earlier kernels wrote comes after it.
// pdl_trigger() lets the next kernel start early.  Both are no-ops for a
// plain launch.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

#define LAUNCH_PDL(ctx, kern, grid, block, smem, ...) \
    SGP_TRY(sgp_launch_pdl((ctx), #kern, kern, dim3(grid), dim3(block), (smem), __VA_ARGS__))

// sym6 y = S x
template <typename T, typename U>
__device__ __forceinline__ void sym_mv(const T *S, const U *x, U *y)
{
    y[0] = (U)S[0] * x[0] + (U)S[1] * x[1] + (U)S[2] * x[2];
    y[1] = (U)S[1] * x[0] + (U)S[3] * x[1] + (U)S[4] * x[2];
    y[2] = (U)S[2] * x[0] + (U)S[4] * x[1] + (U)S[5] * x[2];
}

// Inverse of a symmetric 3x3 block by its adjugate.  Returns false unless
// the leading principal minors are positive (positive definiteness).
__device__ __forceinline__ bool sym_inv(const double *S, double *R)
{
    double a = S[0], b = S[1], c = S[2], d = S[3], e = S[4], f = S[5];
    double c00 = d * f - e * e;
    double c01 = c * e - b * f;
    double c02 = b * e - c * d;
    double c11 = a * f - c * c;
    double c12 = b * c - a * e;
    double c22 = a * d - b * b;
    double det = a * c00 + b * c01 + c * c02;
    if (!(a > 0.0) || !(c22 > 0.0) || !(det > 0.0) || !isfinite(det)) return false;
    double id = 1.0 / det;
    R[0] = c00 * id; R[1] = c01 * id; R[2] = c02 * id;
    R[3] = c11 * id; R[4] = c12 * id; R[5] = c22 * id;
    return true;
}

// full9 C = A * S (S sym6)
__device__ __forceinline__ void full_mul_sym(const double *A, const double *S, double *C)
{
    double s[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = A[3 * r] * s[c] + A[3 * r + 1] * s[3 + c] + A[3 * r + 2] * s[6 + c];
}

// full9 C = A * B^T
__device__ __forceinline__ void full_mul_bt(const double *A, const double *B, double *C)
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = A[3 * r] * B[3 * c] + A[3 * r + 1] * B[3 * c + 1] + A[3 * r + 2] * B[3 * c + 2];
}

template <typename T, typename U>
__device__ __forceinline__ void full_mv(const T *A, const U *x, U *y)
{
    y[0] = (U)A[0] * x[0] + (U)A[1] * x[1] + (U)A[2] * x[2];
    y[1] = (U)A[3] * x[0] + (U)A[4] * x[1] + (U)A[5] * x[2];
    y[2] = (U)A[6] * x[0] + (U)A[7] * x[1] + (U)A[8] * x[2];
}
template <typename T, typename U>
__device__ __forceinline__ void full_mtv(const T *A, const U *x, U *y)
{
    y[0] = (U)A[0] * x[0] + (U)A[3] * x[1] + (U)A[6] * x[2];
    y[1] = (U)A[1] * x[0] + (U)A[4] * x[1] + (U)A[7] * x[2];
    y[2] = (U)A[2] * x[0] + (U)A[5] * x[1] + (U)A[8] * x[2];
}

// Deterministic block sum (fixed shuffle tree, fixed warp order).
template <int BS>
__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (l < BS / 32) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// "Last block done": every block calls this after writing its partial;
// returns true in exactly one block (the last to arrive), which may then
// read every partial.  The counter is reset by the last block.
__device__ __forceinline__ bool last_block(unsigned *counter)
{
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x - 1);
        if (am_last) *counter = 0u;
    }
    __syncthreads();
    return am_last;
}

// Sum of partials[0..n) in a fixed order by one block.
template <int BS>
__device__ __forceinline__ double sum_partials(const double *partials, int n, double *sh)
{
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += BS) v += __ldcg(partials + k);
    return block_sum<BS>(v, sh);
}

// Vectors between the caller's cell order and the solvers' internal order
// (the matrix's orig_of): dst[r] = src[orig_of[r]] and back.  One thread per
// cell, n x 3 entries.
template <typename T>
__global__ void k_to_internal(int64_t n, const int32_t *__restrict__ orig_of, const T *__restrict__ src, T *dst)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t i = orig_of[r];
    dst[3 * r] = src[3 * i];
    dst[3 * r + 1] = src[3 * i + 1];
    dst[3 * r + 2] = src[3 * i + 2];
}

template <typename T>
__global__ void k_to_caller(int64_t n, const int32_t *__restrict__ orig_of, const T *__restrict__ src, T *dst)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t i = orig_of[r];
    dst[3 * i] = src[3 * r];
    dst[3 * i + 1] = src[3 * r + 1];
    dst[3 * i + 2] = src[3 * r + 2];
}

// internal entry points shared between translation units
sgp_status matrix_block_jacobi(sgp_ctx *ctx, sgp_matrix *M);
