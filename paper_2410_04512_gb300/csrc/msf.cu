// msf.cu -- maximum spanning forest by Boruvka's algorithm (Section 3.1).
//
// Edges are ordered strictly: weight descending, then edge index ascending.
// Under a strict total order the maximum spanning forest is unique, so the
// result equals Prim's (the paper's choice) edge for edge.
//
// Each round: every component finds its best outgoing edge (a 64-bit atomic
// max on the weight bits -- positive doubles order like their bit patterns --
// then an atomic min on the index among the edges with that weight); each
// component hooks onto the component across its best edge (of a mutual pair
// the smaller label stays the root); labels are compressed by pointer
// jumping.  Rounds repeat until no component has an outgoing edge.
#include "sgp_internal.cuh"

namespace {

__global__ void k_init_comp(int32_t *comp, int64_t n)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < n) comp[v] = (int32_t)v;
}

__global__ void k_reset_best(unsigned long long *bestw, int32_t *beste, int64_t n)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < n) {
        bestw[v] = 0ull;
        beste[v] = INT32_MAX;
    }
}

// Live edges: endpoints in different components.  `live` lists edge ids;
// edges found internal are dropped from the next round's list.
__global__ void k_best_weight(const int32_t *__restrict__ ij, const double *__restrict__ w,
                              const int32_t *__restrict__ live, int32_t nlive,
                              const int32_t *__restrict__ comp, unsigned long long *bestw)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nlive) return;
    int32_t e = live[k];
    int32_t a = comp[ij[2 * e]], b = comp[ij[2 * e + 1]];
    if (a == b) return;
    unsigned long long wb = (unsigned long long)__double_as_longlong(w[e]);
    atomicMax(bestw + a, wb);
    atomicMax(bestw + b, wb);
}

__global__ void k_best_edge(const int32_t *__restrict__ ij, const double *__restrict__ w,
                            const int32_t *__restrict__ live, int32_t nlive,
                            const int32_t *__restrict__ comp,
                            const unsigned long long *__restrict__ bestw, int32_t *beste,
                            int32_t *keep)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nlive) return;
    int32_t e = live[k];
    int32_t a = comp[ij[2 * e]], b = comp[ij[2 * e + 1]];
    keep[k] = (a != b);
    if (a == b) return;
    unsigned long long wb = (unsigned long long)__double_as_longlong(w[e]);
    if (wb == bestw[a]) atomicMin(beste + a, e);
    if (wb == bestw[b]) atomicMin(beste + b, e);
}

// Roots choose their hook target.  Writes hook[c] (not comp) so that the
// labels read by other threads stay those of the round's start.
__global__ void k_hook(const int32_t *__restrict__ ij, const int32_t *__restrict__ comp,
                       const int32_t *__restrict__ beste, int64_t n, int32_t *hook,
                       uint8_t *intree, int *any)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    int32_t h = comp[c];
    if (h == (int32_t)c) {
        int32_t e = beste[c];
        if (e != INT32_MAX) {
            int32_t a = comp[ij[2 * e]], b = comp[ij[2 * e + 1]];
            int32_t d = (a == (int32_t)c) ? b : a;
            intree[e] = 1;
            *any = 1;
            bool mutual = (beste[d] == e);
            if (!(mutual && (int32_t)c < d)) h = d;
        }
    }
    hook[c] = h;
}

__global__ void k_apply_hook(const int32_t *__restrict__ hook, int32_t *comp, int64_t n)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < n && comp[v] == (int32_t)v) comp[v] = hook[v];
}

__global__ void k_jump(int32_t *comp, int64_t n)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t c = comp[v];
    int32_t cc = comp[c];
    while (c != cc) {
        c = cc;
        cc = comp[c];
    }
    comp[v] = c;
}

__global__ void k_iota(int32_t *a, int64_t n)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < n) a[v] = (int32_t)v;
}

__global__ void k_compact(const int32_t *__restrict__ src, const int32_t *__restrict__ keep,
                          const int32_t *__restrict__ off, int64_t n, int32_t *dst)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n && keep[k]) dst[off[k]] = src ? src[k] : (int32_t)k;
}

__global__ void k_u8_to_i32(const uint8_t *__restrict__ a, int32_t *b, int64_t n)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) b[k] = a[k];
}

// Small graphs: every Boruvka round in one thread block, the component
// labels, best weights and best edges in shared memory; the rounds, the
// strict order and the hooking rule are those above (the forest is the
// same).  Each round visits every kept edge.  The final labels go to
// comp_out, as the multi-launch rounds leave them in the tree.
constexpr int MSF_SMALL_N = 11264;   // 20 bytes of shared memory per cell: 220 KB
__global__ void __launch_bounds__(1024) k_msf_small(const int32_t *__restrict__ ij, const double *__restrict__ w,
                                                    int64_t m, int32_t n, const int32_t *__restrict__ leaf,
                                                    uint8_t *intree, int32_t *comp_out, int *rounds_out)
{
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long *bestw = reinterpret_cast<unsigned long long *>(sm);
    int32_t *comp = reinterpret_cast<int32_t *>(bestw + n);
    int32_t *beste = comp + n, *hook = beste + n;
    __shared__ int any;
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) comp[v] = v;
    int rounds = 0;
    for (;;) {
        for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
            bestw[v] = 0ull;
            beste[v] = INT32_MAX;
        }
        if (threadIdx.x == 0) any = 0;
        __syncthreads();
        for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
            const int32_t i = ij[2 * e], j = ij[2 * e + 1];
            if (leaf && leaf[i] != leaf[j]) continue;
            const int32_t a = comp[i], b = comp[j];
            if (a == b) continue;
            const unsigned long long wb = (unsigned long long)__double_as_longlong(w[e]);
            atomicMax(bestw + a, wb);
            atomicMax(bestw + b, wb);
        }
        __syncthreads();
        for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
            const int32_t i = ij[2 * e], j = ij[2 * e + 1];
            if (leaf && leaf[i] != leaf[j]) continue;
            const int32_t a = comp[i], b = comp[j];
            if (a == b) continue;
            const unsigned long long wb = (unsigned long long)__double_as_longlong(w[e]);
            if (wb == bestw[a]) atomicMin(beste + a, (int32_t)e);
            if (wb == bestw[b]) atomicMin(beste + b, (int32_t)e);
        }
        __syncthreads();
        for (int32_t c = threadIdx.x; c < n; c += blockDim.x) {
            int32_t h = comp[c];
            if (h == c) {
                const int32_t e = beste[c];
                if (e != INT32_MAX) {
                    const int32_t a = comp[ij[2 * (int64_t)e]], b = comp[ij[2 * (int64_t)e + 1]];
                    const int32_t d = (a == c) ? b : a;
                    intree[e] = 1;
                    any = 1;
                    const bool mutual = (beste[d] == e);
                    if (!(mutual && c < d)) h = d;
                }
            }
            hook[c] = h;
        }
        __syncthreads();
        ++rounds;
        if (!any || rounds > 64) break;
        for (int32_t v = threadIdx.x; v < n; v += blockDim.x)
            if (comp[v] == v) comp[v] = hook[v];
        __syncthreads();
        for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
            int32_t c = comp[v], cc = comp[c];
            while (c != cc) {
                c = cc;
                cc = comp[c];
            }
            comp[v] = c;
        }
        __syncthreads();
    }
    // the final component labels (the augmentation groups cells by them)
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) comp_out[v] = comp[v];
    if (threadIdx.x == 0) *rounds_out = rounds;
}

// Section 6 (partitioned forest): contacts whose two cells share a leaf.
__global__ void k_leaf_keep(const int32_t *__restrict__ ij, const int32_t *__restrict__ leaf, int64_t m,
                            int32_t *keep)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < m) keep[e] = leaf[ij[2 * e]] == leaf[ij[2 * e + 1]];
}

// Leaf of each cell in the uniform grid of side h: k = floor(x / h) per
// axis (FP64 division, correctly rounded), label = the low 10 bits of each
// k packed x | y << 10 | z << 20.  Quotients beyond +-2^62 are clamped
// before the conversion (a leaf label either way).
__global__ void k_grid_leaves(int64_t n, const double *__restrict__ pos, double h, int32_t *leaf)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t lab = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double q = floor(pos[3 * i + c] / h);
        q = fmin(fmax(q, -4.6e18), 4.6e18);
        const long long k = (long long)q;
        lab |= (int32_t)(k & 1023) << (10 * c);
    }
    leaf[i] = lab;
}

// The maximum spanning forest of the contacts whose cells share a leaf
// (all contacts when leaf is null).
sgp_status msf_build(sgp_ctx *ctx, const sgp_matrix *M, const int32_t *leaf, sgp_tree **out)
{
    const int64_t n = M->n, m = M->m;
    sgp_tree *T = *out ? *out : new sgp_tree();
    *out = T;
    T->n = n;
    SGP_TRY(buf_ensure(ctx, T->comp, sizeof(int32_t) * (n + 1)));
    SGP_TRY(buf_ensure(ctx, T->bestw, sizeof(unsigned long long) * (n + 1)));
    SGP_TRY(buf_ensure(ctx, T->beste, sizeof(int32_t) * (n + 1)));
    SGP_TRY(buf_ensure(ctx, T->hook, sizeof(int32_t) * (n + 1)));
    SGP_TRY(buf_ensure(ctx, T->intree, (size_t)m + 16));
    // idx holds: live list A, live list B, keep flags, offsets (m + 1 each)
    SGP_TRY(buf_ensure(ctx, T->idx, sizeof(int32_t) * 4 * (size_t)(m + 1)));
    SGP_TRY(buf_ensure(ctx, T->flag, 64));
    int32_t *comp = bp<int32_t>(T->comp), *beste = bp<int32_t>(T->beste),
            *hook = bp<int32_t>(T->hook);
    unsigned long long *bestw = bp<unsigned long long>(T->bestw);
    uint8_t *intree = bp<uint8_t>(T->intree);
    int32_t *liveA = bp<int32_t>(T->idx), *liveB = liveA + (m + 1), *keep = liveB + (m + 1),
            *off = keep + (m + 1);
    int *any = bp<int>(T->flag);
    const int32_t *ij = bp<const int32_t>(M->ij);
    const double *w = bp<const double>(M->w);

    if (n > 0 && n <= MSF_SMALL_N && m < INT32_MAX) {
        // one block: every round without a launch or a host read
        static int done_dev[64] = {0};
        const size_t smem = (size_t)n * (8 + 4 + 4 + 4);
        if (ctx->device >= 0 && ctx->device < 64 && !done_dev[ctx->device]) {
            SGP_CUDA(ctx, cudaFuncSetAttribute(k_msf_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               20 * MSF_SMALL_N));
            done_dev[ctx->device] = 1;
        }
        if (m > 0) SGP_CUDA(ctx, cudaMemsetAsync(intree, 0, (size_t)m, ctx->stream));
        LAUNCH(ctx, k_msf_small, 1, 1024, smem, ij, w, m, (int32_t)n, leaf, intree, comp, any + 2);
    } else {
    LAUNCH(ctx, k_init_comp, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, comp, n);
    if (m > 0) SGP_CUDA(ctx, cudaMemsetAsync(intree, 0, (size_t)m, ctx->stream));
    int64_t nlive = m;
    if (leaf) {
        LAUNCH(ctx, k_leaf_keep, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, ij, leaf, m, keep);
        SGP_TRY(scan_exclusive_i32(ctx, keep, off, m));
        LAUNCH(ctx, k_compact, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)nullptr,
               (const int32_t *)keep, (const int32_t *)off, m, liveA);
        int32_t h = 0;
        SGP_TRY(read_back(ctx, &h, off + m, sizeof(int32_t)));
        nlive = h;
    } else {
        LAUNCH(ctx, k_iota, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, liveA, m);
    }
    int rounds = 0;
    while (nlive > 0) {
        if (++rounds > 64) return sgp_fail(ctx, SGP_ERR_TIMEOUT, "spanning forest: too many rounds");
        SGP_CUDA(ctx, cudaMemsetAsync(any, 0, sizeof(int), ctx->stream));
        LAUNCH(ctx, k_reset_best, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, bestw, beste, n);
        LAUNCH(ctx, k_best_weight, grid_for(nlive, SGP_BLOCK), SGP_BLOCK, 0, ij, w,
               (const int32_t *)liveA, (int32_t)nlive, (const int32_t *)comp, bestw);
        LAUNCH(ctx, k_best_edge, grid_for(nlive, SGP_BLOCK), SGP_BLOCK, 0, ij, w,
               (const int32_t *)liveA, (int32_t)nlive, (const int32_t *)comp,
               (const unsigned long long *)bestw, beste, keep);
        LAUNCH(ctx, k_hook, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, ij, (const int32_t *)comp,
               (const int32_t *)beste, n, hook, intree, any);
        LAUNCH(ctx, k_apply_hook, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)hook,
               comp, n);
        LAUNCH(ctx, k_jump, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, comp, n);
        // drop edges that were internal at the start of this round
        SGP_TRY(scan_exclusive_i32(ctx, keep, off, nlive));
        LAUNCH(ctx, k_compact, grid_for(nlive, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)liveA,
               (const int32_t *)keep, (const int32_t *)off, nlive, liveB);
        // the live count next to the hook flag: one read per round
        SGP_CUDA(ctx, cudaMemcpyAsync(any + 1, off + nlive, sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
        int h[2] = {0, 0};
        SGP_TRY(read_back(ctx, h, any, sizeof(h)));
        std::swap(liveA, liveB);
        nlive = h[1];
        if (!h[0]) break;
    }
    }
    // tree edge ids, ascending
    LAUNCH(ctx, k_u8_to_i32, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, (const uint8_t *)intree, keep, m);
    SGP_TRY(scan_exclusive_i32(ctx, keep, off, m));
    int32_t nt = 0;
    SGP_TRY(read_back(ctx, &nt, off + m, sizeof(int32_t)));
    T->nt = nt;
    T->ncomp = n - nt;
    SGP_TRY(buf_ensure(ctx, T->edges, sizeof(int32_t) * (size_t)(nt + 1)));
    LAUNCH(ctx, k_compact, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)nullptr,
           (const int32_t *)keep, (const int32_t *)off, m, bp<int32_t>(T->edges));
    return SGP_OK;
}

}  // namespace

extern "C" {

sgp_status sgp_max_spanning_tree(sgp_ctx *ctx, const sgp_matrix *M, sgp_tree **out)
{
    if (!ctx || !M || !out) return SGP_ERR_INVALID_ARG;
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    return msf_build(ctx, M, nullptr, out);
}

sgp_status sgp_grid_leaves(sgp_ctx *ctx, int64_t n, const double *pos, double h, int32_t *leaf)
{
    if (!ctx || n < 0 || (n > 0 && (!pos || !leaf)))
        return ctx ? sgp_fail(ctx, SGP_ERR_INVALID_ARG, "grid_leaves: bad pointers or size") : SGP_ERR_INVALID_ARG;
    if (!(h > 0.0) || !std::isfinite(h))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "grid_leaves: h must be positive and finite");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    LAUNCH(ctx, k_grid_leaves, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, pos, h, leaf);
    return SGP_OK;
}

sgp_status sgp_local_spanning_forest(sgp_ctx *ctx, const sgp_matrix *M, const int32_t *leaf, sgp_tree **out)
{
    if (!ctx || !M || !out || (M->n > 0 && !leaf)) return SGP_ERR_INVALID_ARG;
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    return msf_build(ctx, M, leaf, out);
}

sgp_status sgp_tree_info(const sgp_tree *T, int64_t *n_edges, int64_t *n_comp,
                         const int32_t **edge_ids)
{
    if (!T) return SGP_ERR_INVALID_ARG;
    if (n_edges) *n_edges = T->nt;
    if (n_comp) *n_comp = T->ncomp;
    if (edge_ids) *edge_ids = bp<const int32_t>(T->edges);
    return SGP_OK;
}

void sgp_tree_destroy(sgp_tree *T)
{
    if (!T) return;
    cudaDeviceSynchronize();
    DBuf *bufs[] = {&T->edges, &T->comp, &T->bestw, &T->beste, &T->hook, &T->intree,
                    &T->flag, &T->idx};
    for (DBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    delete T;
}

}  // extern "C"
