// augment.cu -- Vaidya's augmented spanning-forest preconditioner
// (Section 3.1): the forest is cut into t pieces, and for every pair of
// pieces that the collision graph joins, the heaviest edge between them is
// added back.  P' = gamma0 I + block Laplacian of the augmented forest T'.
// Systems in P' are solved by an inner PCG preconditioned by the plain
// forest factor (Sections 3.3 and 5; the solver is sgp_fcg_solve in pcg.cu).
//
// The partition (the paper names Chen and Toledo's TreePartition without
// stating it) is defined so that it has one answer and a data-parallel
// construction: every tree is rooted at its smallest cell id; a depth-first
// preorder visits children in ascending id order and the trees in ascending
// order of their roots, numbering all n cells; with s = ceil(n/t), a piece is
// a maximal set of cells that the tree connects and whose preorder numbers
// share one block [k s, (k+1) s).  Pieces are connected subtrees of at most
// s cells, numbered in preorder of their top cell.
//
// Construction, all in caller cell ids:
//   1. sorted tree adjacency with twin slots;
//   2. an Euler tour (each slot followed by the slot after its twin, so
//      children come cyclically after the parent) ranked by pointer
//      jumping: a slot taken before its twin points down, which gives every
//      cell's parent and subtree size;
//   3. each cell's offset below its parent (1 + sizes of its smaller
//      siblings) and each tree's base (sizes of the trees with smaller
//      roots); preorder numbers are the sums along the path to the root,
//      again by pointer jumping;
//   4. piece tops (roots, and cells whose parent is in another block) and
//      every cell's top by pointer jumping; piece numbers by a scan in
//      preorder;
//   5. the heaviest edge of every pair of pieces through a hash table keyed
//      by the pair: an atomic maximum of the weight bits (weights are
//      positive, so their bit patterns order like the values), then an
//      atomic minimum of the index among the edges that attain it -- the
//      strict order (weight descending, index ascending) of the spanning
//      forest, independent of thread timing;
//   6. P' as a matrix: the kept slots of every row, in the source matrix's
//      slot order.
#include "sgp_internal.cuh"

namespace {

constexpr unsigned long long EMPTY_KEY = ~0ull;

// ---------------------------------------------------------------- adjacency
__global__ void k_ag_deg(const int32_t *__restrict__ ij, const int32_t *__restrict__ tedges, int64_t nt, int64_t m,
                         int32_t n, int32_t *deg, int *err)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const int32_t e = tedges[k];
    if (e < 0 || e >= m) {
        atomicOr(err, 1);
        return;
    }
    const int32_t a = ij[2 * (int64_t)e], b = ij[2 * (int64_t)e + 1];
    if (a < 0 || a >= n || b < 0 || b >= n) {
        atomicOr(err, 1);
        return;
    }
    atomicAdd(deg + a, 1);
    atomicAdd(deg + b, 1);
}

__global__ void k_ag_fill(const int32_t *__restrict__ ij, const int32_t *__restrict__ tedges, int64_t nt, int32_t n,
                          const int32_t *__restrict__ aptr, int32_t *cur, int32_t *nbr)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const int32_t e = tedges[k], a = ij[2 * (int64_t)e], b = ij[2 * (int64_t)e + 1];
    if (a < 0 || a >= n || b < 0 || b >= n) return;
    nbr[aptr[a] + atomicAdd(cur + a, 1)] = b;
    nbr[aptr[b] + atomicAdd(cur + b, 1)] = a;
}

// ascending neighbour ids per cell (insertion sort: tree degrees are small)
__global__ void k_ag_sort(const int32_t *__restrict__ aptr, int32_t n, int32_t *nbr)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t lo = aptr[v], hi = aptr[v + 1];
    for (int32_t i = lo + 1; i < hi; ++i) {
        const int32_t x = nbr[i];
        int32_t j = i - 1;
        while (j >= lo && nbr[j] > x) {
            nbr[j + 1] = nbr[j];
            --j;
        }
        nbr[j + 1] = x;
    }
}

// twin of slot s (v -> u): the slot of u -> v, by binary search in u's list;
// own[s] = v
__global__ void k_ag_twin(const int32_t *__restrict__ aptr, const int32_t *__restrict__ nbr, int32_t n,
                          int32_t *twin, int32_t *own, int *err)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int32_t s = aptr[v]; s < aptr[v + 1]; ++s) {
        const int32_t u = nbr[s];
        int32_t lo = aptr[u], hi = aptr[u + 1];
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (nbr[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= aptr[u + 1] || nbr[lo] != v) {
            atomicOr(err, 2);
            twin[s] = s;
        } else {
            twin[s] = lo;
        }
        own[s] = v;
    }
}

// smallest cell id of every tree (comp: the forest's component labels)
__global__ void k_ag_minid(const int32_t *__restrict__ comp, int32_t n, int32_t *minid, int *err)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t c = comp[v];
    if (c < 0 || c >= n) {
        atomicOr(err, 4);
        return;
    }
    atomicMin(minid + c, v);
}

__global__ void k_ag_root(const int32_t *__restrict__ comp, const int32_t *__restrict__ minid, int32_t n,
                          int32_t *root, int32_t *tsize)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t c = comp[v];
    const int32_t r = (c >= 0 && c < n) ? minid[c] : v;
    root[v] = (r >= 0 && r < n) ? r : v;
    atomicAdd(tsize + root[v], 1);
}

// ---------------------------------------------------------------- Euler tour
// slot s = (v -> u) is followed by the slot after twin(s) in u's list,
// cyclically; the slot that would wrap into the root's first slot ends the
// tour (dist 0), every other slot is one step from its successor
__global__ void k_ag_tour(const int32_t *__restrict__ aptr, const int32_t *__restrict__ nbr,
                          const int32_t *__restrict__ twin, const int32_t *__restrict__ root, int64_t ns,
                          int32_t *succ, int32_t *dist)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int32_t u = nbr[s], t = twin[s];
    const bool wrap = t + 1 >= aptr[u + 1];
    if (wrap && root[u] == u) {
        succ[s] = -1;
        dist[s] = 0;
    } else {
        succ[s] = wrap ? aptr[u] : t + 1;
        dist[s] = 1;
    }
}

__global__ void k_ag_jump(int64_t ns, const int32_t *__restrict__ succ, const int32_t *__restrict__ dist,
                          int32_t *succ2, int32_t *dist2)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int32_t nx = succ[s];
    if (nx < 0 || nx >= ns) {
        succ2[s] = -1;
        dist2[s] = dist[s];
    } else {
        succ2[s] = succ[nx];
        dist2[s] = dist[s] + dist[nx];
    }
}

// a slot taken before its twin points down: parent and subtree size of its head
__global__ void k_ag_parent(int64_t ns, const int32_t *__restrict__ nbr, const int32_t *__restrict__ own,
                            const int32_t *__restrict__ twin, const int32_t *__restrict__ succ,
                            const int32_t *__restrict__ dist, int32_t *parent, int32_t *size, int *err)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    if (succ[s] >= 0) atomicOr(err, 8);   // the tour was not ranked to its end
    const int32_t d = dist[s], dt = dist[twin[s]];
    if (d > dt) {
        parent[nbr[s]] = own[s];
        size[nbr[s]] = (d - dt + 1) / 2;
    }
}

// offset of every child below its parent: 1 + sizes of its smaller siblings;
// roots take their tree's size
__global__ void k_ag_off(const int32_t *__restrict__ aptr, const int32_t *__restrict__ nbr,
                         const int32_t *__restrict__ parent, const int32_t *__restrict__ root,
                         const int32_t *__restrict__ tsize, int32_t n, int32_t *size, int32_t *off, int32_t *rsz)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const bool isroot = root[v] == v;
    if (isroot) size[v] = tsize[v];
    rsz[v] = isroot ? tsize[v] : 0;
    int32_t acc = 0;
    for (int32_t s = aptr[v]; s < aptr[v + 1]; ++s) {
        const int32_t c = nbr[s];
        if (c == parent[v]) continue;
        off[c] = 1 + acc;
        acc += size[c];
    }
}

__global__ void k_ag_pre_init(const int32_t *__restrict__ parent, const int32_t *__restrict__ root,
                              const int32_t *__restrict__ base, const int32_t *__restrict__ off, int32_t n,
                              int32_t *acc, int32_t *anc)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const bool isroot = root[v] == v;
    acc[v] = isroot ? base[v] : off[v];
    anc[v] = isroot ? -1 : parent[v];
}

__global__ void k_ag_pre_jump(int32_t n, const int32_t *__restrict__ acc, const int32_t *__restrict__ anc,
                              int32_t *acc2, int32_t *anc2)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t a = anc[v];
    if (a < 0 || a >= n) {
        acc2[v] = acc[v];
        anc2[v] = -1;
    } else {
        acc2[v] = acc[v] + acc[a];
        anc2[v] = anc[a];
    }
}

// tops: roots, and cells whose parent lies in another preorder block
__global__ void k_ag_top(const int32_t *__restrict__ pre, const int32_t *__restrict__ parent,
                         const int32_t *__restrict__ root, const int32_t *__restrict__ anc, int32_t n, int32_t s,
                         int32_t *top, int32_t *pflag, int32_t *seen, int *err)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t pv = pre[v];
    if (pv < 0 || pv >= n || anc[v] != -1) {
        atomicOr(err, 16);
        top[v] = v;
        return;
    }
    if (atomicAdd(seen + pv, 1) != 0) atomicOr(err, 16);   // not a permutation
    const int32_t p = parent[v];
    const bool t = root[v] == v || p < 0 || p >= n || pre[p] / s != pv / s;
    top[v] = t ? v : p;
    pflag[pv] = t ? 1 : 0;
}

__global__ void k_ag_top_jump(int32_t n, const int32_t *__restrict__ top, int32_t *top2)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    top2[v] = top[top[v]];
}

__global__ void k_ag_label(int32_t n, const int32_t *__restrict__ top, const int32_t *__restrict__ pre,
                           const int32_t *__restrict__ pid, int32_t *piece, int *err)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t t = top[v];
    if (top[t] != t) atomicOr(err, 32);   // pointer jumping did not reach a top
    piece[v] = pid[pre[t]];
}

// ------------------------------------------------------------- augmentation
__device__ __forceinline__ unsigned long long pair_key(int32_t a, int32_t b)
{
    const uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
    return ((unsigned long long)lo << 32) | hi;
}

__device__ __forceinline__ uint32_t key_hash(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}

__global__ void k_ag_inter(const int32_t *__restrict__ ij, const int32_t *__restrict__ piece, int64_t m,
                           int32_t *flag)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    flag[e] = piece[ij[2 * e]] != piece[ij[2 * e + 1]];
}

// claim the pair's table entry (linear probing, at most cap probes) and
// raise its weight to the edge's
__global__ void k_ag_hash_w(const int32_t *__restrict__ ij, const int32_t *__restrict__ piece,
                            const double *__restrict__ w, int64_t m, uint32_t cap, unsigned long long *keys,
                            unsigned long long *bw, int32_t *slot, int *err)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t a = piece[ij[2 * e]], b = piece[ij[2 * e + 1]];
    if (a == b) {
        slot[e] = -1;
        return;
    }
    const unsigned long long key = pair_key(a, b);
    uint32_t h = key_hash(key) & (cap - 1);
    for (uint32_t probe = 0; probe < cap; ++probe) {
        const unsigned long long old = atomicCAS(keys + h, EMPTY_KEY, key);
        if (old == EMPTY_KEY || old == key) {
            atomicMax(bw + h, (unsigned long long)__double_as_longlong(w[e]));
            slot[e] = (int32_t)h;
            return;
        }
        h = (h + 1) & (cap - 1);
    }
    slot[e] = -1;
    atomicOr(err, 64);   // table full (cannot happen: cap > 2 x inter-piece edges)
}

__global__ void k_ag_hash_e(const double *__restrict__ w, int64_t m, const int32_t *__restrict__ slot,
                            const unsigned long long *__restrict__ bw, int32_t *be)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t h = slot[e];
    if (h >= 0 && (unsigned long long)__double_as_longlong(w[e]) == bw[h]) atomicMin(be + h, (int32_t)e);
}

__global__ void k_ag_keep(int64_t m, const int32_t *__restrict__ slot, const int32_t *__restrict__ be,
                          int32_t *keep)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t h = slot[e];
    if (h >= 0 && be[h] == (int32_t)e) keep[e] = 1;
}

__global__ void k_ag_keep_tree(const int32_t *__restrict__ tedges, int64_t nt, int32_t *keep)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < nt) keep[tedges[k]] = 1;
}

// --------------------------------------------------------- P' as a matrix
__global__ void k_ag_kslot(int64_t m, const int32_t *__restrict__ keep, const int32_t *__restrict__ es,
                           const int32_t *__restrict__ esj, int32_t *kslot)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m || !keep[e]) return;
    kslot[es[e]] = 1;
    kslot[esj[e]] = 1;
}

__global__ void k_ag_rowcnt(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ kslot,
                            int32_t *cnt)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = 0;
    for (int32_t s = rp[i]; s < rp[i + 1]; ++s) c += kslot[s];
    cnt[i] = c;
}

__global__ void k_ag_rowfill(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ kslot,
                             const int32_t *__restrict__ rp2, const int32_t *__restrict__ col,
                             const double *__restrict__ blk, int32_t *col2, double *blk2, int32_t *newslot)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t k = rp2[i];
    for (int32_t s = rp[i]; s < rp[i + 1]; ++s) {
        if (!kslot[s]) continue;
        col2[k] = col[s];
        for (int a = 0; a < 6; ++a) blk2[6 * (int64_t)k + a] = blk[6 * (int64_t)s + a];
        newslot[s] = k;
        ++k;
    }
}

__global__ void k_ag_edges(int64_t m, const int32_t *__restrict__ keep, const int32_t *__restrict__ kidx,
                           const int32_t *__restrict__ ij, const double *__restrict__ w,
                           const int32_t *__restrict__ es, const int32_t *__restrict__ esj,
                           const int32_t *__restrict__ newslot, int32_t *edges, int32_t *ij2, double *w2,
                           int32_t *es2, int32_t *esj2)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m || !keep[e]) return;
    const int32_t k = kidx[e];
    edges[k] = (int32_t)e;
    ij2[2 * (int64_t)k] = ij[2 * e];
    ij2[2 * (int64_t)k + 1] = ij[2 * e + 1];
    w2[k] = w[e];
    es2[k] = newslot[es[e]];
    esj2[k] = newslot[esj[e]];
}

struct Scratch {
    sgp_ctx *ctx;
    sgp_aug *A;
    int used = 0;
    void *raw(size_t bytes)
    {
        if (used >= SGP_AUG_SCRATCH) return nullptr;
        DBuf &b = A->scr[used++];
        if (buf_ensure(ctx, b, bytes + 64) != SGP_OK) return nullptr;
        return b.p;
    }
    int32_t *i32(size_t count) { return static_cast<int32_t *>(raw(sizeof(int32_t) * (count + 4))); }
};

int rounds_for(int64_t len)
{
    int r = 1;
    while ((int64_t(1) << r) < len + 1) ++r;
    return r + 1;
}

}  // namespace

extern "C" {

sgp_status sgp_augment_tree(sgp_ctx *ctx, const sgp_matrix *M, const sgp_tree *T, int32_t t, sgp_aug **out)
{
    if (!ctx || !M || !T || !out) return SGP_ERR_INVALID_ARG;
    if (T->n != M->n) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "augment_tree: size mismatch");
    if (t < 0) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "augment_tree: t must be >= 0");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int32_t n = (int32_t)M->n;
    const int64_t m = M->m, nt = T->nt, ns = 2 * nt;
    sgp_aug *A = *out ? *out : new sgp_aug();
    *out = A;
    A->n = n;
    A->m = m;
    A->mgen = M->gen;
    A->t = t > 0 ? t : std::max(1, (int)std::lround(std::pow((double)std::max(n, 1), 0.25)));
    A->s = n > 0 ? (int32_t)((n + (int64_t)A->t - 1) / A->t) : 1;
    A->npieces = 0;
    A->nedges = 0;
    A->added = 0;
    SGP_TRY(buf_ensure(ctx, A->piece, sizeof(int32_t) * ((size_t)n + 4)));
    SGP_TRY(buf_ensure(ctx, A->edges, sizeof(int32_t) * ((size_t)m + 4)));
    if (!A->P) A->P = new sgp_matrix();
    sgp_matrix *P = A->P;
    P->gen = next_generation();
    P->n = n;
    P->m = 0;
    P->gamma0 = M->gamma0;
    P->precision = SGP_PREC_F64;
    P->jac_valid = 0;
    SGP_TRY(buf_ensure(ctx, P->row_ptr, sizeof(int32_t) * ((size_t)n + 4)));
    SGP_TRY(buf_ensure(ctx, P->orig_of, sizeof(int32_t) * ((size_t)n + 4)));
    SGP_TRY(buf_ensure(ctx, P->int_of, sizeof(int32_t) * ((size_t)n + 4)));
    if (n == 0) return SGP_OK;
    SGP_CUDA(ctx, cudaMemcpyAsync(P->orig_of.p, M->orig_of.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    SGP_CUDA(ctx, cudaMemcpyAsync(P->int_of.p, M->int_of.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    Scratch S{ctx, A};
    int *err = ctx->d_flags + 24;
    SGP_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    const int32_t *ij = bp<const int32_t>(M->ij), *tedges = bp<const int32_t>(T->edges),
                  *comp = bp<const int32_t>(T->comp);
    const unsigned gn = grid_for(n, SGP_BLOCK), gs = grid_for(ns, SGP_BLOCK), gt = grid_for(nt, SGP_BLOCK),
                   gm = grid_for(m, SGP_BLOCK);

    // 1. sorted adjacency of the forest with twins
    int32_t *deg = S.i32(n + 1), *aptr = S.i32(n + 1), *cur = S.i32(n + 1), *nbr = S.i32(ns + 1),
            *twin = S.i32(ns + 1), *own = S.i32(ns + 1);
    if (!deg || !aptr || !cur || !nbr || !twin || !own) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(deg, 0, sizeof(int32_t) * (n + 1), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(cur, 0, sizeof(int32_t) * (n + 1), ctx->stream));
    if (nt > 0) LAUNCH(ctx, k_ag_deg, gt, SGP_BLOCK, 0, ij, tedges, nt, m, n, deg, err);
    SGP_TRY(scan_exclusive_i32(ctx, deg, aptr, n));
    int herr = 0;
    SGP_TRY(read_back(ctx, &herr, err, sizeof(int)));
    if (herr) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "augment_tree: the tree does not match the matrix (%d)", herr);
    if (nt > 0) {
        LAUNCH(ctx, k_ag_fill, gt, SGP_BLOCK, 0, ij, tedges, nt, n, (const int32_t *)aptr, cur, nbr);
        LAUNCH(ctx, k_ag_sort, gn, SGP_BLOCK, 0, (const int32_t *)aptr, n, nbr);
        LAUNCH(ctx, k_ag_twin, gn, SGP_BLOCK, 0, (const int32_t *)aptr, (const int32_t *)nbr, n, twin, own, err);
    }
    // roots: the smallest id of every tree, and tree sizes
    int32_t *minid = S.i32(n), *root = S.i32(n), *tsize = S.i32(n);
    if (!minid || !root || !tsize) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(minid, 0x7f, sizeof(int32_t) * n, ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(tsize, 0, sizeof(int32_t) * n, ctx->stream));
    LAUNCH(ctx, k_ag_minid, gn, SGP_BLOCK, 0, comp, n, minid, err);
    LAUNCH(ctx, k_ag_root, gn, SGP_BLOCK, 0, comp, (const int32_t *)minid, n, root, tsize);
    SGP_TRY(read_back(ctx, &herr, err, sizeof(int)));
    if (herr) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "augment_tree: the tree does not match the matrix (%d)", herr);

    // 2. Euler tour ranked by pointer jumping: parents and subtree sizes
    int32_t *parent = S.i32(n), *size = S.i32(n), *off = S.i32(n), *rsz = S.i32(n + 1), *base = S.i32(n + 1);
    if (!parent || !size || !off || !rsz || !base) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(parent, 0xff, sizeof(int32_t) * n, ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(off, 0, sizeof(int32_t) * n, ctx->stream));
    if (nt > 0) {
        int32_t *succ = S.i32(ns), *dist = S.i32(ns), *succ2 = S.i32(ns), *dist2 = S.i32(ns);
        if (!succ || !dist || !succ2 || !dist2) return SGP_ERR_OOM;
        LAUNCH(ctx, k_ag_tour, gs, SGP_BLOCK, 0, (const int32_t *)aptr, (const int32_t *)nbr, (const int32_t *)twin,
               (const int32_t *)root, ns, succ, dist);
        const int R = rounds_for(ns);
        for (int r = 0; r < R; ++r) {
            LAUNCH(ctx, k_ag_jump, gs, SGP_BLOCK, 0, ns, (const int32_t *)succ, (const int32_t *)dist, succ2, dist2);
            std::swap(succ, succ2);
            std::swap(dist, dist2);
        }
        LAUNCH(ctx, k_ag_parent, gs, SGP_BLOCK, 0, ns, (const int32_t *)nbr, (const int32_t *)own,
               (const int32_t *)twin, (const int32_t *)succ, (const int32_t *)dist, parent, size, err);
    }
    // 3. offsets below the parent, tree bases, preorder numbers
    LAUNCH(ctx, k_ag_off, gn, SGP_BLOCK, 0, (const int32_t *)aptr, (const int32_t *)nbr, (const int32_t *)parent,
           (const int32_t *)root, (const int32_t *)tsize, n, size, off, rsz);
    SGP_TRY(scan_exclusive_i32(ctx, rsz, base, n));
    int32_t *acc = S.i32(n), *anc = S.i32(n), *acc2 = S.i32(n), *anc2 = S.i32(n);
    if (!acc || !anc || !acc2 || !anc2) return SGP_ERR_OOM;
    LAUNCH(ctx, k_ag_pre_init, gn, SGP_BLOCK, 0, (const int32_t *)parent, (const int32_t *)root,
           (const int32_t *)base, (const int32_t *)off, n, acc, anc);
    const int Rn = rounds_for(n);
    for (int r = 0; r < Rn; ++r) {
        LAUNCH(ctx, k_ag_pre_jump, gn, SGP_BLOCK, 0, n, (const int32_t *)acc, (const int32_t *)anc, acc2, anc2);
        std::swap(acc, acc2);
        std::swap(anc, anc2);
    }
    const int32_t *pre = acc;
    // 4. piece tops and labels
    int32_t *top = S.i32(n), *top2 = S.i32(n), *pflag = S.i32(n + 1), *pid = S.i32(n + 1), *seen = S.i32(n);
    if (!top || !top2 || !pflag || !pid || !seen) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(pflag, 0, sizeof(int32_t) * (n + 1), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(seen, 0, sizeof(int32_t) * n, ctx->stream));
    LAUNCH(ctx, k_ag_top, gn, SGP_BLOCK, 0, pre, (const int32_t *)parent, (const int32_t *)root,
           (const int32_t *)anc, n, A->s, top, pflag, seen, err);
    for (int r = 0; r < Rn; ++r) {
        LAUNCH(ctx, k_ag_top_jump, gn, SGP_BLOCK, 0, n, (const int32_t *)top, top2);
        std::swap(top, top2);
    }
    SGP_TRY(scan_exclusive_i32(ctx, pflag, pid, n));
    SGP_TRY(read_back(ctx, &herr, err, sizeof(int)));
    if (herr) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "augment_tree: the tree edges are not a forest (%d)", herr);
    int32_t *piece = bp<int32_t>(A->piece);
    LAUNCH(ctx, k_ag_label, gn, SGP_BLOCK, 0, n, (const int32_t *)top, pre, (const int32_t *)pid, piece, err);
    int32_t np = 0;
    SGP_TRY(read_back(ctx, &np, pid + n, sizeof(int32_t)));
    A->npieces = np;

    // 5. the heaviest edge between every pair of pieces
    int32_t *keep = S.i32(m + 1), *kidx = S.i32(m + 1), *slot = S.i32(m + 1), *iflag = S.i32(m + 1),
            *ioff = S.i32(m + 1);
    if (!keep || !kidx || !slot || !iflag || !ioff) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(keep, 0, sizeof(int32_t) * (m + 1), ctx->stream));
    int32_t ninter = 0;
    if (m > 0) {
        LAUNCH(ctx, k_ag_inter, gm, SGP_BLOCK, 0, ij, (const int32_t *)piece, m, iflag);
        SGP_TRY(scan_exclusive_i32(ctx, iflag, ioff, m));
        SGP_TRY(read_back(ctx, &ninter, ioff + m, sizeof(int32_t)));
    }
    if (ninter > 0) {
        uint32_t cap = 16;
        while (cap < 2u * (uint32_t)ninter + 16u) cap <<= 1;
        unsigned long long *keys = static_cast<unsigned long long *>(S.raw(sizeof(unsigned long long) * cap));
        unsigned long long *bw = static_cast<unsigned long long *>(S.raw(sizeof(unsigned long long) * cap));
        int32_t *be = S.i32(cap);
        if (!keys || !bw || !be) return SGP_ERR_OOM;
        SGP_CUDA(ctx, cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * cap, ctx->stream));
        SGP_CUDA(ctx, cudaMemsetAsync(bw, 0, sizeof(unsigned long long) * cap, ctx->stream));
        SGP_CUDA(ctx, cudaMemsetAsync(be, 0x7f, sizeof(int32_t) * cap, ctx->stream));
        LAUNCH(ctx, k_ag_hash_w, gm, SGP_BLOCK, 0, ij, (const int32_t *)piece, bp<const double>(M->w), m, cap, keys,
               bw, slot, err);
        LAUNCH(ctx, k_ag_hash_e, gm, SGP_BLOCK, 0, bp<const double>(M->w), m, (const int32_t *)slot,
               (const unsigned long long *)bw, be);
        LAUNCH(ctx, k_ag_keep, gm, SGP_BLOCK, 0, m, (const int32_t *)slot, (const int32_t *)be, keep);
    }
    if (nt > 0) LAUNCH(ctx, k_ag_keep_tree, gt, SGP_BLOCK, 0, tedges, nt, keep);
    int32_t ne = 0;
    if (m > 0) {
        SGP_TRY(scan_exclusive_i32(ctx, keep, kidx, m));
        SGP_TRY(read_back(ctx, &ne, kidx + m, sizeof(int32_t)));
    }
    SGP_TRY(read_back(ctx, &herr, err, sizeof(int)));
    if (herr) return sgp_fail(ctx, SGP_ERR_CUDA, "augment_tree: inconsistent pieces (%d)", herr);
    A->nedges = ne;
    A->added = ne - nt;

    // 6. P' in the source matrix's row and slot order
    const int64_t s2 = 2 * m;
    int32_t *kslot = S.i32(s2 + 1), *newslot = S.i32(s2 + 1), *rcnt = S.i32(n + 1);
    if (!kslot || !newslot || !rcnt) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(kslot, 0, sizeof(int32_t) * (s2 + 1), ctx->stream));
    P->m = ne;
    SGP_TRY(buf_ensure(ctx, P->col, sizeof(int32_t) * (2 * (size_t)ne + 4)));
    SGP_TRY(buf_ensure(ctx, P->blk, sizeof(double) * 6 * (2 * (size_t)ne + 4)));
    SGP_TRY(buf_ensure(ctx, P->ij, sizeof(int32_t) * (2 * (size_t)ne + 4)));
    SGP_TRY(buf_ensure(ctx, P->w, sizeof(double) * ((size_t)ne + 4)));
    SGP_TRY(buf_ensure(ctx, P->edge_slot, sizeof(int32_t) * ((size_t)ne + 4)));
    SGP_TRY(buf_ensure(ctx, P->edge_slot_j, sizeof(int32_t) * ((size_t)ne + 4)));
    const int32_t *es = bp<const int32_t>(M->edge_slot), *esj = bp<const int32_t>(M->edge_slot_j);
    if (m > 0) LAUNCH(ctx, k_ag_kslot, gm, SGP_BLOCK, 0, m, (const int32_t *)keep, es, esj, kslot);
    LAUNCH(ctx, k_ag_rowcnt, gn, SGP_BLOCK, 0, n, bp<const int32_t>(M->row_ptr), (const int32_t *)kslot, rcnt);
    SGP_TRY(scan_exclusive_i32(ctx, rcnt, bp<int32_t>(P->row_ptr), n));
    LAUNCH(ctx, k_ag_rowfill, gn, SGP_BLOCK, 0, n, bp<const int32_t>(M->row_ptr), (const int32_t *)kslot,
           bp<const int32_t>(P->row_ptr), bp<const int32_t>(M->col), bp<const double>(M->blk), bp<int32_t>(P->col),
           bp<double>(P->blk), newslot);
    if (m > 0)
        LAUNCH(ctx, k_ag_edges, gm, SGP_BLOCK, 0, m, (const int32_t *)keep, (const int32_t *)kidx, ij,
               bp<const double>(M->w), es, esj, (const int32_t *)newslot, bp<int32_t>(A->edges), bp<int32_t>(P->ij),
               bp<double>(P->w), bp<int32_t>(P->edge_slot), bp<int32_t>(P->edge_slot_j));
    SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SGP_OK;
}

sgp_status sgp_aug_info(const sgp_aug *A, int32_t *t, int32_t *pieces, int32_t *piece_cap, int64_t *edges,
                        int64_t *added)
{
    if (!A) return SGP_ERR_INVALID_ARG;
    if (t) *t = A->t;
    if (pieces) *pieces = A->npieces;
    if (piece_cap) *piece_cap = A->s;
    if (edges) *edges = A->nedges;
    if (added) *added = A->added;
    return SGP_OK;
}

sgp_status sgp_aug_pieces(sgp_ctx *ctx, const sgp_aug *A, int32_t *piece_dev)
{
    if (!ctx || !A || (A->n > 0 && !piece_dev)) return SGP_ERR_INVALID_ARG;
    if (A->n == 0) return SGP_OK;
    SGP_CUDA(ctx, cudaMemcpyAsync(piece_dev, A->piece.p, sizeof(int32_t) * A->n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    return SGP_OK;
}

sgp_status sgp_aug_edges(sgp_ctx *ctx, const sgp_aug *A, int32_t *edges_dev)
{
    if (!ctx || !A || (A->nedges > 0 && !edges_dev)) return SGP_ERR_INVALID_ARG;
    if (A->nedges == 0) return SGP_OK;
    SGP_CUDA(ctx, cudaMemcpyAsync(edges_dev, A->edges.p, sizeof(int32_t) * A->nedges, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    return SGP_OK;
}

const sgp_matrix *sgp_aug_matrix(const sgp_aug *A)
{
    return A ? A->P : nullptr;
}

void sgp_aug_destroy(sgp_aug *A)
{
    if (!A) return;
    cudaDeviceSynchronize();
    for (DBuf *b : {&A->piece, &A->edges})
        if (b->p) cudaFree(b->p);
    for (DBuf &b : A->scr)
        if (b.p) cudaFree(b.p);
    if (A->P) sgp_matrix_destroy(A->P);
    delete A;
}

}  // extern "C"
