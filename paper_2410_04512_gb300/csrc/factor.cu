// factor.cu -- block LDL^T of the spanning-forest preconditioner and its
// solve (Section 3.3, Algorithm 2; Appendix B.1), scheduled by rake/compress
// tree contraction.
//
// P = gamma0 I + block Laplacian of the forest (self-loops kept, Section 3.1).
// Eliminating a vertex c whose current neighbours are q (one or two of them)
// is a block Gaussian elimination step:
//     D_c       = A_cc                         (pivot, final once c's turn comes)
//     L_qc      = A_qc D_c^-1
//     A_qq     -= A_qc D_c^-1 A_cq             (Schur complement)
//     A_q0q1    = -A_q0c D_c^-1 A_cq1          (fill, only when c had two neighbours)
// Algorithm 2 eliminates children before parents, one vertex at a time.  Here
// each level eliminates, at once, every leaf (rake) and an independent set of
// degree-2 vertices (compress, each splicing its two neighbours together with
// the fill block): the degree-2 vertices without a leaf neighbour that are
// local minima of a per-level hash among their degree-2 neighbours.  Chains
// shrink by a constant fraction per level, so any tree needs O(log n) levels
// (about 23 for the spanning tree of a 1e6-cell spheroid).  Every elimination
// keeps the graph a forest, so the factor is exact: P^-1 is the same operator
// as with the paper's order (only rounding differs).
//
// Structure (which vertex goes when, with which neighbours) is computed first
// with integer kernels, level by level.  The numeric factorisation then
// replays the levels; the solve
// replays them forward (receivers gather L_qc z_c) and backward (each
// eliminated vertex gathers from its receivers).  All sums run in a fixed
// order, so results are bitwise reproducible.

#include "sgp_internal.cuh"
#include "tail.cuh"

namespace {

// ------------------------------------------------------------------ adjacency
// The factor works in the matrix's internal cell order: tree edge endpoints
// are mapped through int_of.
__global__ void k_tdeg(const int32_t *__restrict__ ij, const int32_t *__restrict__ edges, int64_t nt,
                       const int32_t *__restrict__ int_of, int32_t *deg)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int32_t e = edges[t];
    atomicAdd(deg + int_of[ij[2 * e]], 1);
    atomicAdd(deg + int_of[ij[2 * e + 1]], 1);
}

__global__ void k_adj_fill(const int32_t *__restrict__ ij, const int32_t *__restrict__ edges,
                           int64_t nt, const int32_t *__restrict__ int_of, const int32_t *__restrict__ adj_ptr,
                           int32_t *cursor, int32_t *nbr, int32_t *eref)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int32_t e = edges[t];
    int32_t a = int_of[ij[2 * e]], b = int_of[ij[2 * e + 1]];
    int32_t sa = adj_ptr[a] + atomicAdd(cursor + a, 1);
    int32_t sb = adj_ptr[b] + atomicAdd(cursor + b, 1);
    nbr[sa] = b;
    eref[sa] = (int32_t)t;
    nbr[sb] = a;
    eref[sb] = (int32_t)t;
}

__global__ void k_adj_sort(const int32_t *__restrict__ adj_ptr, int64_t n, int32_t *nbr,
                           int32_t *eref)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t b0 = adj_ptr[v], k = adj_ptr[v + 1] - b0;
    for (int32_t a = 1; a < k; ++a) {
        int32_t x = nbr[b0 + a], y = eref[b0 + a];
        int32_t b = a - 1;
        while (b >= 0 && nbr[b0 + b] > x) {
            nbr[b0 + b + 1] = nbr[b0 + b];
            eref[b0 + b + 1] = eref[b0 + b];
            --b;
        }
        nbr[b0 + b + 1] = x;
        eref[b0 + b + 1] = y;
    }
}

// twin[s] = the entry of the same edge in the neighbour's (sorted) list
__global__ void k_twin(const int32_t *__restrict__ adj_ptr, int64_t n, const int32_t *__restrict__ nbr,
                       int32_t *twin)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int32_t s = adj_ptr[v]; s < adj_ptr[v + 1]; ++s) {
        int32_t u = nbr[s];
        int32_t lo = adj_ptr[u], hi = adj_ptr[u + 1] - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi) >> 1;
            if (nbr[mid] < (int32_t)v) lo = mid + 1;
            else hi = mid;
        }
        twin[s] = lo;
    }
}

// A_vv = gamma0 I + sum of the tree blocks at v (sym6), in list order
__global__ void k_acc_init(const int32_t *__restrict__ adj_ptr, int64_t n,
                           const int32_t *__restrict__ eref, const int32_t *__restrict__ edges,
                           const int32_t *__restrict__ edge_slot, const double *__restrict__ blk,
                           double gamma0, double *acc, int32_t *deg, int32_t *lev, int32_t *alive)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    double S[6] = {gamma0, 0.0, 0.0, gamma0, 0.0, gamma0};
    for (int32_t s = adj_ptr[v]; s < adj_ptr[v + 1]; ++s) {
        const double *U = blk + 6 * (int64_t)edge_slot[edges[eref[s]]];
#pragma unroll
        for (int k = 0; k < 6; ++k) S[k] += U[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[6 * v + k] = S[k];
    deg[v] = adj_ptr[v + 1] - adj_ptr[v];
    lev[v] = -1;
    alive[v] = (int32_t)v;
}

// -------------------------------------------------------- structure: select
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ bool key_less(int32_t a, int32_t b, uint32_t salt)
{
    uint32_t ha = mix32((uint32_t)a ^ salt), hb = mix32((uint32_t)b ^ salt);
    return ha < hb || (ha == hb && a < b);
}

struct Sim {
    const int32_t *adj_ptr;
    int32_t *nbr, *twin, *eref, *deg, *lev, *nrec;
    int2 *rq, *re, *ren;
};

// One level eliminating rake and compress candidates together: every
// vertex of degree 0, every leaf (of two adjacent leaves only the larger
// id), and every degree-2 vertex that has no leaf neighbour and beats its
// degree-2 neighbours by the level's hash.  No two chosen vertices are
// adjacent, and each has at most two neighbours, so eliminating them all at
// once equals eliminating them one by one: the forest stays a forest.
__device__ __forceinline__ void select_vertex(const Sim &S, int32_t v, int32_t level, uint32_t salt)
{
    const int32_t d = S.deg[v];
    if (d == 0) {
        S.lev[v] = level;
        S.nrec[v] = 0;
        return;
    }
    if (d > 2) return;
    int32_t e1 = -1, e2 = -1;
    for (int32_t s = S.adj_ptr[v]; s < S.adj_ptr[v + 1]; ++s)
        if (S.nbr[s] >= 0) {
            if (e1 < 0) e1 = s;
            else { e2 = s; break; }
        }
    const int32_t a = S.nbr[e1];
    if (d == 1) {
        if (S.deg[a] == 1 && a > v) return;
        S.lev[v] = level;
        S.nrec[v] = 1;
        S.rq[v] = make_int2(a, -1);
        S.re[v] = make_int2(S.eref[e1], -1);
        S.ren[v] = make_int2(e1, -1);
        return;
    }
    const int32_t b = S.nbr[e2];
    const int32_t da = S.deg[a], db = S.deg[b];
    if (da == 1 || db == 1) return;
    if (da == 2 && key_less(a, v, salt)) return;
    if (db == 2 && key_less(b, v, salt)) return;
    const bool sw = a > b;
    S.lev[v] = level;
    S.nrec[v] = 2;
    S.rq[v] = sw ? make_int2(b, a) : make_int2(a, b);
    S.re[v] = sw ? make_int2(S.eref[e2], S.eref[e1]) : make_int2(S.eref[e1], S.eref[e2]);
    S.ren[v] = sw ? make_int2(e2, e1) : make_int2(e1, e2);
}

__global__ void k_select(Sim S, const int32_t *__restrict__ A, int32_t na, int32_t level, uint32_t salt)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < na) select_vertex(S, A[k], level, salt);
}

// ----------------------------------------------------- structure: bookkeeping
// mode 0: eliminated at `level`; mode 1: flagged receiver; mode 2: still alive
__global__ void k_flags(const int32_t *__restrict__ A, int32_t na, int mode, int32_t level,
                        const int32_t *__restrict__ lev, const int32_t *__restrict__ rflag,
                        int32_t *flag)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    int32_t v = A[k];
    int32_t f;
    if (mode == 0) f = (lev[v] == level);
    else if (mode == 1) f = (rflag[v] != 0);
    else f = (lev[v] == -1);
    flag[k] = f;
}

// Structural update of a merged level: a leaf leaves its neighbour's list;
// a degree-2 vertex splices its two neighbours together (fill edge nt + v).
__device__ __forceinline__ void apply_vertex(const Sim &S, int32_t v, int32_t nt)
{
    const int32_t r = S.nrec[v];
    if (r == 1) {
        S.nbr[S.twin[S.ren[v].x]] = -1;
        atomicSub(S.deg + S.rq[v].x, 1);
    } else if (r == 2) {
        int2 q = S.rq[v], en = S.ren[v];
        int32_t ta = S.twin[en.x], tb = S.twin[en.y];
        S.nbr[ta] = q.y;
        S.nbr[tb] = q.x;
        S.twin[ta] = tb;
        S.twin[tb] = ta;
        S.eref[ta] = nt + v;
        S.eref[tb] = nt + v;
    }
}


// ------------------------- structure: a level with its counts on the device
// The same steps as above for a level whose counts stay on the device until
// its end (one host read per level): grids are sized by the alive count na,
// the kernels read the actual counts from dc = (eliminated, pairs,
// receivers, contributor entries, alive), and the scans run over na entries
// with zeros past the count.  The stable compaction's scatter records the
// count of its list in *count.
__global__ void k_scatter_list_d(const int32_t *__restrict__ A, int32_t na, const int32_t *__restrict__ flag,
                                 const int32_t *__restrict__ off, int32_t *dst, int32_t base, int mode,
                                 int32_t *pos, int32_t *rflag, int32_t *count)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) *count = off[na];
    if (k >= na || !flag[k]) return;
    int32_t v = A[k];
    int32_t at = base + off[k];
    dst[at] = v;
    if (mode == 0) pos[v] = at;
    if (mode == 1) rflag[v] = 0;
}

__global__ void k_level_nrec_d(const int32_t *__restrict__ ord, int32_t p0, int32_t bound,
                               const int32_t *__restrict__ dc, const int32_t *__restrict__ nrec, int32_t *tmp)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < bound) tmp[k] = k < dc[0] ? nrec[ord[p0 + k]] : 0;
}

__global__ void k_level_pairs_d(const int32_t *__restrict__ ord, int32_t p0, int32_t bound, int32_t *dc,
                                const int32_t *__restrict__ off, int32_t pair0, const int32_t *__restrict__ nrec,
                                const int2 *__restrict__ rq, int32_t *pr_ptr, int32_t *pr_q, int32_t *pr_c,
                                int32_t *rflag)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) dc[1] = off[bound];
    if (k >= dc[0]) return;
    int32_t c = ord[p0 + k];
    int32_t p = pair0 + off[k];
    pr_ptr[p0 + k] = p;
    int32_t r = nrec[c];
    int2 q = rq[c];
    if (r > 0) { pr_q[p] = q.x; pr_c[p] = c; rflag[q.x] = 1; }
    if (r > 1) { pr_q[p + 1] = q.y; pr_c[p + 1] = c; rflag[q.y] = 1; }
}

template <bool FILL>
__global__ void k_contrib_d(Sim S, const int32_t *__restrict__ rv, int32_t r0, int32_t bound, int32_t *dc,
                            int32_t level, const int32_t *__restrict__ pos, const int32_t *__restrict__ pr_ptr,
                            int32_t *count, const int32_t *__restrict__ off, int32_t ct0, int32_t *rc_ptr,
                            int32_t *ct)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (FILL && k == 0) dc[3] = off[bound];
    if (k >= bound) return;
    if (k >= dc[2]) {
        if (!FILL) count[k] = 0;
        return;
    }
    int32_t q = rv[r0 + k];
    int32_t c_n = 0;
    int32_t at = FILL ? ct0 + off[k] : 0;
    if (FILL) rc_ptr[r0 + k] = at;
    for (int32_t s = S.adj_ptr[q]; s < S.adj_ptr[q + 1]; ++s) {
        int32_t c = S.nbr[s];
        if (c < 0 || S.lev[c] != level) continue;
        if (FILL) {
            int32_t which = (S.rq[c].x == q) ? 0 : 1;
            ct[at + c_n] = pr_ptr[pos[c]] + which;
        }
        ++c_n;
    }
    if (!FILL) count[k] = c_n;
}

__global__ void k_apply_d(Sim S, const int32_t *__restrict__ ord, int32_t p0, const int32_t *__restrict__ dc,
                          int32_t nt)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < dc[0]) apply_vertex(S, ord[p0 + k], nt);
}

// ------------------------------------------------- structure: the short tail
// Once the alive list is short (at most SMALL_NA vertices) the remaining
// levels run in one block of SB threads: the same selection, the same stable
// compactions and the same contributor lists as the per-level kernels above
// (hence the same structure), with block-wide scans and __syncthreads()
// between the steps instead of kernel boundaries and a host round trip per
// count.  Thread t owns a contiguous chunk of every list, so each compaction
// keeps list order.  rec[l] = (eliminated, pairs, receivers, contributor
// entries) of the l-th level run here; hdr = (levels run, vertices still
// alive, error: 1 = a level eliminated nothing, 2 = inconsistent contributor
// count).
constexpr int SMALL_NA = 8192;
constexpr int SMALL_MAXL = 96;
constexpr int SB = 1024;

__device__ __forceinline__ int32_t sb_scan(int32_t v, int32_t *sh, int32_t *total)
{
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (l >= o) x += y;
    }
    if (l == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t u = sh[l];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, u, o);
            if (l >= o) u += y;
        }
        sh[l] = u;
    }
    __syncthreads();
    const int32_t before = (w > 0 ? sh[w - 1] : 0) + x - v;
    *total = sh[SB / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SB) k_levels_small(Sim S, int32_t *A, int32_t *Bl, int32_t na, int32_t level,
                                                     int32_t phase, int32_t *rflag, int32_t *ord, int32_t npos,
                                                     int32_t *pos, int32_t *pr_ptr, int32_t *pr_q, int32_t *pr_c,
                                                     int32_t npair, int32_t *rv, int32_t nrecv, int32_t *rc_ptr,
                                                     int32_t *ct, int32_t ncontrib, int32_t nt, int4 *rec,
                                                     int32_t *hdr)
{
    __shared__ int32_t sh[SB / 32];
    const int32_t t = threadIdx.x;
    int32_t done = 0, err = 0;
    auto chunk = [&](int32_t cnt, int32_t &lo, int32_t &hi) {
        const int32_t per = (cnt + SB - 1) / SB;
        lo = min(cnt, t * per);
        hi = min(cnt, lo + per);
    };
    while (na > 0 && done < SMALL_MAXL) {
        const uint32_t salt = 0x9E3779B9u * (uint32_t)(phase + 1);
        int32_t lo, hi;
        chunk(na, lo, hi);
        for (int32_t k = lo; k < hi; ++k) select_vertex(S, A[k], level, salt);
        __syncthreads();
        // eliminated vertices -> ord, pos
        int32_t c = 0, ne;
        for (int32_t k = lo; k < hi; ++k) c += (S.lev[A[k]] == level);
        int32_t off = sb_scan(c, sh, &ne);
        for (int32_t k = lo; k < hi; ++k) {
            const int32_t v = A[k];
            if (S.lev[v] == level) {
                const int32_t at = npos + off++;
                ord[at] = v;
                pos[v] = at;
            }
        }
        if (ne == 0) { err = 1; break; }
        __syncthreads();
        // pairs of the eliminated vertices; receivers flagged
        int32_t elo, ehi, lp;
        chunk(ne, elo, ehi);
        c = 0;
        for (int32_t k = elo; k < ehi; ++k) c += S.nrec[ord[npos + k]];
        off = sb_scan(c, sh, &lp);
        for (int32_t k = elo; k < ehi; ++k) {
            const int32_t cv = ord[npos + k];
            const int32_t p = npair + off;
            pr_ptr[npos + k] = p;
            const int32_t r = S.nrec[cv];
            const int2 q = S.rq[cv];
            if (r > 0) { pr_q[p] = q.x; pr_c[p] = cv; rflag[q.x] = 1; }
            if (r > 1) { pr_q[p + 1] = q.y; pr_c[p + 1] = cv; rflag[q.y] = 1; }
            off += r;
        }
        __syncthreads();
        // receivers, in list order (each flag is cleared by its owner only)
        int32_t nr;
        c = 0;
        for (int32_t k = lo; k < hi; ++k) c += (rflag[A[k]] != 0);
        off = sb_scan(c, sh, &nr);
        for (int32_t k = lo; k < hi; ++k) {
            const int32_t v = A[k];
            if (rflag[v]) {
                rv[nrecv + off++] = v;
                rflag[v] = 0;
            }
        }
        __syncthreads();
        // contributors of each receiver
        int32_t rlo, rhi, lc;
        chunk(nr, rlo, rhi);
        c = 0;
        for (int32_t k = rlo; k < rhi; ++k) {
            const int32_t q = rv[nrecv + k];
            for (int32_t s = S.adj_ptr[q]; s < S.adj_ptr[q + 1]; ++s) {
                const int32_t cv = S.nbr[s];
                c += (cv >= 0 && S.lev[cv] == level);
            }
        }
        off = sb_scan(c, sh, &lc);
        for (int32_t k = rlo; k < rhi; ++k) {
            const int32_t q = rv[nrecv + k];
            rc_ptr[nrecv + k] = ncontrib + off;
            for (int32_t s = S.adj_ptr[q]; s < S.adj_ptr[q + 1]; ++s) {
                const int32_t cv = S.nbr[s];
                if (cv < 0 || S.lev[cv] != level) continue;
                const int32_t which = (S.rq[cv].x == q) ? 0 : 1;
                ct[ncontrib + off++] = pr_ptr[pos[cv]] + which;
            }
        }
        if (lc != lp) { err = 2; break; }
        __syncthreads();
        // structural update
        for (int32_t k = elo; k < ehi; ++k) apply_vertex(S, ord[npos + k], nt);
        __syncthreads();
        // the alive list of the next level
        int32_t nal;
        c = 0;
        for (int32_t k = lo; k < hi; ++k) c += (S.lev[A[k]] == -1);
        off = sb_scan(c, sh, &nal);
        for (int32_t k = lo; k < hi; ++k)
            if (S.lev[A[k]] == -1) Bl[off++] = A[k];
        if (t == 0) rec[done] = make_int4(ne, lp, nr, lc);
        npos += ne;
        npair += lp;
        nrecv += nr;
        ncontrib += lc;
        ++level;
        ++phase;
        ++done;
        int32_t *sw = A;
        A = Bl;
        Bl = sw;
        na = nal;
        __syncthreads();
    }
    if (t == 0) {
        hdr[0] = done;
        hdr[1] = na;
        hdr[2] = err;
    }
}

// ------------------------------------------------------------------ numerics
struct Num {
    const int32_t *ord, *nrec, *pr_ptr, *edges, *edge_slot;
    const int2 *rq, *re;
    const double *blk;
    double *acc, *fill, *L, *Dinv, *sbuf;
    int32_t nt;
    int *err;
};

// B = A_{q c} for the current edge `er` between q and c.
__device__ __forceinline__ void edge_block(const Num &N, int32_t er, int32_t q, double *B)
{
    if (er < N.nt) {
        const double *U = N.blk + 6 * (int64_t)N.edge_slot[N.edges[er]];
        B[0] = -U[0]; B[1] = -U[1]; B[2] = -U[2];
        B[3] = -U[1]; B[4] = -U[3]; B[5] = -U[4];
        B[6] = -U[2]; B[7] = -U[4]; B[8] = -U[5];
    } else {
        int32_t x = er - N.nt;
        const double *F = N.fill + 9 * (int64_t)x;
        if (N.rq[x].x == q) {
#pragma unroll
            for (int k = 0; k < 9; ++k) B[k] = F[k];
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) B[3 * r + c] = F[3 * c + r];
        }
    }
}

__global__ void k_factor_elim(Num N, int32_t p0, int32_t cnt)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    int32_t t = p0 + k;
    int32_t c = N.ord[t];
    double D[6], Di[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) D[a] = N.acc[6 * (int64_t)c + a];
    if (!sym_inv(D, Di)) {
        atomicOr(N.err, 1);
        Di[0] = Di[3] = Di[5] = 1.0;
        Di[1] = Di[2] = Di[4] = 0.0;
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) N.Dinv[6 * (int64_t)t + a] = Di[a];
    int32_t r = N.nrec[c];
    if (r == 0) return;
    int2 q = N.rq[c], er = N.re[c];
    int32_t p = N.pr_ptr[t];
    double B0[9], L0[9], C[9];
    edge_block(N, er.x, q.x, B0);
    full_mul_sym(B0, Di, L0);
#pragma unroll
    for (int a = 0; a < 9; ++a) N.L[9 * (int64_t)p + a] = L0[a];
    full_mul_bt(L0, B0, C);
    double *S0 = N.sbuf + 6 * (int64_t)p;
    S0[0] = C[0]; S0[1] = C[1]; S0[2] = C[2]; S0[3] = C[4]; S0[4] = C[5]; S0[5] = C[8];
    if (r == 2) {
        double B1[9], L1[9];
        edge_block(N, er.y, q.y, B1);
        full_mul_sym(B1, Di, L1);
#pragma unroll
        for (int a = 0; a < 9; ++a) N.L[9 * (int64_t)(p + 1) + a] = L1[a];
        full_mul_bt(L1, B1, C);
        double *S1 = N.sbuf + 6 * (int64_t)(p + 1);
        S1[0] = C[0]; S1[1] = C[1]; S1[2] = C[2]; S1[3] = C[4]; S1[4] = C[5]; S1[5] = C[8];
        // fill A_{q0 q1} = -A_{q0 c} D^-1 A_{c q1} = -L0 B1^T
        full_mul_bt(L0, B1, C);
        double *Fo = N.fill + 9 * (int64_t)c;
#pragma unroll
        for (int a = 0; a < 9; ++a) Fo[a] = -C[a];
    }
}

__global__ void k_factor_recv(Num N, const int32_t *__restrict__ rv, const int32_t *__restrict__ rc_ptr,
                              const int32_t *__restrict__ ct, int32_t r0, int32_t cnt)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    int32_t q = rv[r0 + k];
    double A[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) A[a] = N.acc[6 * (int64_t)q + a];
    for (int32_t j = rc_ptr[r0 + k]; j < rc_ptr[r0 + k + 1]; ++j) {
        const double *S = N.sbuf + 6 * (int64_t)ct[j];
#pragma unroll
        for (int a = 0; a < 6; ++a) A[a] -= S[a];
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) N.acc[6 * (int64_t)q + a] = A[a];
}

__global__ void k_to_f32(const double *__restrict__ a, float *b, int64_t n)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) b[k] = (float)a[k];
}

}  // namespace

// --------------------------------------------------------------------- solve
// Programmatic dependent launch: a level kernel lets the next one start its
// prologue at once (launch_dependents) and waits for the previous level's
// results (wait) only before it touches the solution vector.

// Forward substitution of one level: each receiver q subtracts
// sum_c L_qc w_c over this level's contributors c (fixed order).  Lf holds
// the L blocks in contributor-list order and ctv the contributor vertices,
// so the level streams both arrays.
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 12 : 8) k_tree_fwd(const int32_t *__restrict__ rv, const int32_t *__restrict__ rc_ptr,
                           const int32_t *__restrict__ ctv, const T *__restrict__ Lf, int32_t r0,
                           int32_t cnt, T *w, const int *done)
{
    pdl_trigger();
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt || (done && *done)) return;
    const int32_t q = rv[r0 + k];
    const int32_t j0 = rc_ptr[r0 + k], j1 = rc_ptr[r0 + k + 1];
    // Contributor ids and L blocks do not depend on the previous level: load
    // the first FWD_PRE of them before waiting, so that after the wait all
    // their w loads go out together (one memory round trip per level).
    constexpr int FWD_PRE = 2;
    T Lr[FWD_PRE][9];
    int32_t cr[FWD_PRE];
#pragma unroll
    for (int e = 0; e < FWD_PRE; ++e) {
        const int32_t j = j0 + e;
        cr[e] = j < j1 ? ctv[j] : -1;
#pragma unroll
        for (int a = 0; a < 9; ++a) Lr[e][a] = j < j1 ? Lf[9 * (int64_t)j + a] : T(0);
    }
    pdl_wait();
    T x[FWD_PRE][3];
#pragma unroll
    for (int e = 0; e < FWD_PRE; ++e) {
        const int64_t c = cr[e] >= 0 ? cr[e] : q;
        x[e][0] = w[3 * c];
        x[e][1] = w[3 * c + 1];
        x[e][2] = w[3 * c + 2];
    }
    T s[3] = {0, 0, 0};
#pragma unroll
    for (int e = 0; e < FWD_PRE; ++e) {
        if (cr[e] < 0) break;
        T y[3];
        full_mv(Lr[e], x[e], y);
        s[0] += y[0]; s[1] += y[1]; s[2] += y[2];
    }
    for (int32_t j = j0 + FWD_PRE; j < j1; ++j) {
        int32_t c = ctv[j];
        T xx[3] = {w[3 * (int64_t)c], w[3 * (int64_t)c + 1], w[3 * (int64_t)c + 2]};
        T y[3];
        full_mv(Lf + 9 * (int64_t)j, xx, y);
        s[0] += y[0]; s[1] += y[1]; s[2] += y[2];
    }
    w[3 * (int64_t)q] -= s[0];
    w[3 * (int64_t)q + 1] -= s[1];
    w[3 * (int64_t)q + 2] -= s[2];
}

// Diagonal solve and backward substitution of one level:
// z_c = D_c^-1 w_c - sum_q L_qc^T z_q, in place.
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 12 : 8) k_tree_bwd(const int32_t *__restrict__ ord, const int32_t *__restrict__ pr_ptr,
                           const int32_t *__restrict__ pr_q, const T *__restrict__ L,
                           const T *__restrict__ Dinv, int32_t p0, int32_t cnt, T *w, const int *done)
{
    pdl_trigger();
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt || (done && *done)) return;
    const int32_t t = p0 + k;
    const int32_t c = ord[t];
    const int32_t pa = pr_ptr[t], pb = pr_ptr[t + 1];
    // An eliminated vertex has at most two receivers (a leaf one, a
    // compressed vertex two): load their ids, L blocks and D^-1 before
    // waiting; after the wait the three vector loads go out together.
    T Di[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) Di[a] = Dinv[6 * (int64_t)t + a];
    int32_t qr[2];
    T Lr[2][9];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int32_t p = pa + e;
        qr[e] = p < pb ? pr_q[p] : -1;
#pragma unroll
        for (int a = 0; a < 9; ++a) Lr[e][a] = p < pb ? L[9 * (int64_t)p + a] : T(0);
    }
    pdl_wait();
    T x[3] = {w[3 * (int64_t)c], w[3 * (int64_t)c + 1], w[3 * (int64_t)c + 2]};
    T y[2][3];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int64_t q = qr[e] >= 0 ? qr[e] : c;
        y[e][0] = w[3 * q];
        y[e][1] = w[3 * q + 1];
        y[e][2] = w[3 * q + 2];
    }
    T z[3];
    sym_mv(Di, x, z);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        if (qr[e] < 0) break;
        T u[3];
        full_mtv(Lr[e], y[e], u);
        z[0] -= u[0]; z[1] -= u[1]; z[2] -= u[2];
    }
    for (int32_t p = pa + 2; p < pb; ++p) {   // not reached for a forest
        int32_t q = pr_q[p];
        T yy[3] = {w[3 * (int64_t)q], w[3 * (int64_t)q + 1], w[3 * (int64_t)q + 2]};
        T u[3];
        full_mtv(L + 9 * (int64_t)p, yy, u);
        z[0] -= u[0]; z[1] -= u[1]; z[2] -= u[2];
    }
    w[3 * (int64_t)c] = z[0];
    w[3 * (int64_t)c + 1] = z[1];
    w[3 * (int64_t)c + 2] = z[2];
}

template <typename T, bool STAGE>
__global__ void __launch_bounds__(1024) k_tree_tail(Tail tl, const int32_t *__restrict__ ord,
                                                    const int32_t *__restrict__ rc_ptr,
                                                    const int32_t *__restrict__ pr_ptr,
                                                    const T *__restrict__ L, const T *__restrict__ Lf,
                                                    const T *__restrict__ Dinv, T *w, const int *done)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();
    if (done && *done) return;
    unsigned char *cur = smem_raw;
    auto take = [&](size_t b) { unsigned char *p = cur; cur += tail_align(b); return p; };
    T *sw = reinterpret_cast<T *>(take(sizeof(T) * 3 * tl.n));
    int32_t *spr = reinterpret_cast<int32_t *>(take(4 * (tl.n + 1)));
    int32_t *stb = reinterpret_cast<int32_t *>(take(4 * tl.np));
    int32_t *spc = reinterpret_cast<int32_t *>(take(4 * tl.np));
    int32_t *sct = reinterpret_cast<int32_t *>(take(4 * tl.np));
    int32_t *src = reinterpret_cast<int32_t *>(take(4 * (tl.nr + 1)));
    int32_t *stq = reinterpret_cast<int32_t *>(take(4 * tl.nr));
    const T *Lt = L + 9 * (int64_t)tl.Q0, *Lft = Lf + 9 * (int64_t)tl.C0, *Dt = Dinv + 6 * (int64_t)tl.P0;
    T *sD = nullptr, *sL = nullptr;
    if (STAGE) {
        sD = reinterpret_cast<T *>(take(sizeof(T) * 6 * tl.n));
        sL = reinterpret_cast<T *>(take(sizeof(T) * 9 * tl.np));
        for (int32_t i = threadIdx.x; i < 6 * tl.n; i += blockDim.x) sD[i] = Dt[i];
        for (int32_t i = threadIdx.x; i < 9 * tl.np; i += blockDim.x) sL[i] = Lt[i];
    }
    // stage the index lists (independent of the previous kernel)
    for (int32_t i = threadIdx.x; i <= tl.n; i += blockDim.x) spr[i] = pr_ptr[tl.P0 + i] - tl.Q0;
    for (int32_t i = threadIdx.x; i < tl.np; i += blockDim.x) {
        stb[i] = tl.tb[i];
        spc[i] = tl.tpc[i];
        sct[i] = tl.tct[i];
    }
    for (int32_t i = threadIdx.x; i <= tl.nr; i += blockDim.x) src[i] = rc_ptr[tl.R0 + i] - tl.C0;
    for (int32_t i = threadIdx.x; i < tl.nr; i += blockDim.x) stq[i] = tl.tq[i];
    pdl_wait();
    for (int32_t i = threadIdx.x; i < tl.n; i += blockDim.x) {
        int64_t v = ord[tl.P0 + i];
        sw[3 * i] = w[3 * v];
        sw[3 * i + 1] = w[3 * v + 1];
        sw[3 * i + 2] = w[3 * v + 2];
    }
    __syncthreads();
    for (int l = 0; l < tl.nlev; ++l) {
        const int32_t k0 = tl.lvl_rv[l] - tl.R0, k1 = tl.lvl_rv[l + 1] - tl.R0;
        for (int32_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            T s[3] = {0, 0, 0};
            for (int32_t j = src[k]; j < src[k + 1]; ++j) {
                const int32_t p = sct[j];
                T y[3];
                full_mv(STAGE ? sL + 9 * p : Lft + 9 * (int64_t)j, sw + 3 * spc[p], y);
                s[0] += y[0]; s[1] += y[1]; s[2] += y[2];
            }
            const int32_t q = stq[k];
            sw[3 * q] -= s[0];
            sw[3 * q + 1] -= s[1];
            sw[3 * q + 2] -= s[2];
        }
        __syncthreads();
    }
    for (int l = tl.nlev - 1; l >= 0; --l) {
        const int32_t i0 = tl.lvl_pos[l] - tl.P0, i1 = tl.lvl_pos[l + 1] - tl.P0;
        for (int32_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            T z[3];
            sym_mv(STAGE ? sD + 6 * i : Dt + 6 * (int64_t)i, sw + 3 * i, z);
            for (int32_t p = spr[i]; p < spr[i + 1]; ++p) {
                T u[3];
                full_mtv(STAGE ? sL + 9 * p : Lt + 9 * (int64_t)p, sw + 3 * stb[p], u);
                z[0] -= u[0]; z[1] -= u[1]; z[2] -= u[2];
            }
            sw[3 * i] = z[0];
            sw[3 * i + 1] = z[1];
            sw[3 * i + 2] = z[2];
        }
        __syncthreads();
    }
    for (int32_t i = threadIdx.x; i < tl.n; i += blockDim.x) {
        int64_t v = ord[tl.P0 + i];
        w[3 * v] = sw[3 * i];
        w[3 * v + 1] = sw[3 * i + 1];
        w[3 * v + 2] = sw[3 * i + 2];
    }
}

Tail tail_of(const sgp_factor *F)
{
    Tail t;
    t.nlev = F->levels - F->tail_level;
    t.n = (int32_t)(F->n - F->tail_P0);
    t.np = (int32_t)(F->npairs - F->tail_Q0);
    t.nr = F->rl_ptr[F->levels] - F->tail_R0;
    t.P0 = F->tail_P0;
    t.Q0 = F->tail_Q0;
    t.R0 = F->tail_R0;
    t.C0 = F->tail_C0;
    const int32_t *tlp = bp<const int32_t>(F->tail_idx);
    t.lvl_pos = tlp;
    t.lvl_rv = tlp + (t.nlev + 1);
    t.tq = bp<const int32_t>(F->tail_q);
    t.tb = bp<const int32_t>(F->tail_b);
    t.tpc = bp<const int32_t>(F->tail_c);
    t.tct = bp<const int32_t>(F->tail_c) + t.np;
    return t;
}

// In-place P^-1 w (T = double uses the FP64 factor, float the FP32 copies):
// the binned solve when the factor has a layout for T, else one launch per
// contraction level below the tail, the tail kernel, one launch per level
// back down.
template <typename T>
sgp_status tree_apply_inplace(sgp_ctx *ctx, const sgp_factor *F, T *w, const int *done)
{
    if (bins_usable<T>(F)) return bins_apply<T>(ctx, F, w, done);
    const bool f64 = sizeof(T) == 8;
    const T *L = reinterpret_cast<const T *>(f64 ? F->L.p : F->L32.p);
    const T *Lf = reinterpret_cast<const T *>(f64 ? F->Lf.p : F->Lf32.p);
    const T *Dinv = reinterpret_cast<const T *>(f64 ? F->Dinv.p : F->Dinv32.p);
    const int32_t *rv = bp<const int32_t>(F->rv), *rc = bp<const int32_t>(F->rc_ptr),
                  *ctv = bp<const int32_t>(F->ctv), *ord = bp<const int32_t>(F->ord),
                  *prp = bp<const int32_t>(F->pr_ptr), *prq = bp<const int32_t>(F->pr_q);
    const int B = 128;
    // the tail was sized for the factor's own precision; an FP64 apply of a
    // MIXED factor whose tail does not fit runs every level as its own kernel
    int lt = F->tail_level;
    if (lt < F->levels) {
        const Tail tl = tail_of(F);
        if (tail_smem_bytes<T>(tl.n, tl.np, tl.nr) > (size_t)TREE_TAIL_SMEM) lt = F->levels;
    }
    for (int l = 0; l < lt; ++l) {
        int32_t r0 = F->rl_ptr[l], cnt = F->rl_ptr[l + 1] - r0;
        if (cnt > 0) LAUNCH_PDL(ctx, k_tree_fwd<T>, grid_for(cnt, B), B, 0, rv, rc, ctv, Lf, r0, cnt, w, done);
    }
    if (lt < F->levels) {
        const Tail tl = tail_of(F);
        const size_t staged = tail_smem_staged<T>(tl.n, tl.np, tl.nr);
        if (staged <= (size_t)TREE_TAIL_SMEM)
            LAUNCH_PDL(ctx, (k_tree_tail<T, true>), 1, 1024, staged, tl, ord, rc, prp, L, Lf, Dinv, w, done);
        else
            LAUNCH_PDL(ctx, (k_tree_tail<T, false>), 1, 1024, tail_smem_bytes<T>(tl.n, tl.np, tl.nr), tl, ord, rc,
                       prp, L, Lf, Dinv, w, done);
    }
    for (int l = lt - 1; l >= 0; --l) {
        int32_t p0 = F->lvl_ptr[l], cnt = F->lvl_ptr[l + 1] - p0;
        if (cnt > 0) LAUNCH_PDL(ctx, k_tree_bwd<T>, grid_for(cnt, B), B, 0, ord, prp, prq, L, Dinv, p0, cnt, w, done);
    }
    return SGP_OK;
}
template sgp_status tree_apply_inplace<double>(sgp_ctx *, const sgp_factor *, double *, const int *);
template sgp_status tree_apply_inplace<float>(sgp_ctx *, const sgp_factor *, float *, const int *);

// Shared memory of the tail kernel must be opted in above 48 KB, once per device.
static sgp_status tail_smem_optin(sgp_ctx *ctx)
{
    static int done_dev[64] = {0};
    if (ctx->device >= 0 && ctx->device < 64 && done_dev[ctx->device]) return SGP_OK;
    const int bytes = TREE_TAIL_SMEM;
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_tree_tail<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_tree_tail<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_tree_tail<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_tree_tail<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    if (ctx->device >= 0 && ctx->device < 64) done_dev[ctx->device] = 1;
    return SGP_OK;
}

namespace {
// Forward-ordered layout: contributor vertex and L block per contributor entry.
template <typename T>
__global__ void k_forward_layout(const int32_t *__restrict__ ct, const int32_t *__restrict__ pr_c,
                                 const double *__restrict__ L, int32_t nct, int32_t *ctv, T *Lf)
{
    int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nct) return;
    int32_t p = ct[j];
    if (ctv) ctv[j] = pr_c[p];
#pragma unroll
    for (int a = 0; a < 9; ++a) Lf[9 * (int64_t)j + a] = (T)L[9 * (int64_t)p + a];
}

// Local (tail) indices: positions minus P0.
__global__ void k_tail_index(const int32_t *__restrict__ src, const int32_t *__restrict__ pos,
                             int32_t first, int32_t count, int32_t P0, int32_t *dst)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) dst[k] = pos[src[first + k]] - P0;
}

// Local pair of each tail contributor entry.
__global__ void k_tail_pairs(const int32_t *__restrict__ ct, int32_t first, int32_t count, int32_t Q0,
                             int32_t *dst)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) dst[k] = ct[first + k] - Q0;
}
}  // namespace

// ------------------------------------------------------------------- factor
// Stable compaction of the flagged entries of the alive list A (k_flags'
// modes) to dst[base + ...], the count left on the device (*count).
static sgp_status compact_dev(sgp_ctx *ctx, const int32_t *A, int32_t na, int mode, int32_t level,
                              const int32_t *lev, int32_t *rflag, int32_t *flag, int32_t *off, int32_t *dst,
                              int32_t base, int32_t *pos, int32_t *count)
{
    LAUNCH(ctx, k_flags, grid_for(na, SGP_BLOCK), SGP_BLOCK, 0, A, na, mode, level, lev,
           (const int32_t *)rflag, flag);
    SGP_TRY(scan_exclusive_i32(ctx, flag, off, na));
    LAUNCH(ctx, k_scatter_list_d, grid_for(na, SGP_BLOCK), SGP_BLOCK, 0, A, na, (const int32_t *)flag,
           (const int32_t *)off, dst, base, mode, pos, rflag, count);
    return SGP_OK;
}

extern "C" {

sgp_status sgp_tree_factor(sgp_ctx *ctx, const sgp_matrix *M, const sgp_tree *T, sgp_factor **out)
{
    if (!ctx || !M || !T || !out) return SGP_ERR_INVALID_ARG;
    if (T->n != M->n) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "tree_factor: size mismatch");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = M->n, nt = T->nt;
    sgp_factor *F = *out ? *out : new sgp_factor();
    *out = F;
    F->n = n;
    F->precision = M->precision;
    F->levels = 0;
    F->gen = next_generation();
    F->rounds = 0;
    F->lvl_ptr.assign(1, 0);
    F->rl_ptr.assign(1, 0);
    F->pl_ptr.assign(1, 0);
    F->cl_ptr.assign(1, 0);
    F->tail_level = 0;
    const size_t n1 = (size_t)n + 1, P = 2 * (size_t)n + 2;
    SGP_TRY(buf_ensure(ctx, F->adj_ptr, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->nbr, sizeof(int32_t) * (2 * nt + 1)));
    SGP_TRY(buf_ensure(ctx, F->twin, sizeof(int32_t) * (2 * nt + 1)));
    SGP_TRY(buf_ensure(ctx, F->eref, sizeof(int32_t) * (2 * nt + 1)));
    SGP_TRY(buf_ensure(ctx, F->deg, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->lev, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->nrec, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->rq, sizeof(int2) * n1));
    SGP_TRY(buf_ensure(ctx, F->re, sizeof(int2) * n1));
    SGP_TRY(buf_ensure(ctx, F->ren, sizeof(int2) * n1));
    SGP_TRY(buf_ensure(ctx, F->pos, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->flag, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->tmp, sizeof(int32_t) * (n1 + 1)));
    SGP_TRY(buf_ensure(ctx, F->alive_a, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->alive_b, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->rflag, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->cnt, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->acc, sizeof(double) * 6 * n1));
    SGP_TRY(buf_ensure(ctx, F->fill, sizeof(double) * 9 * n1));
    SGP_TRY(buf_ensure(ctx, F->sbuf, sizeof(double) * 6 * P));
    SGP_TRY(buf_ensure(ctx, F->ord, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->pr_ptr, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->pr_q, sizeof(int32_t) * P));
    SGP_TRY(buf_ensure(ctx, F->pr_c, sizeof(int32_t) * P));
    SGP_TRY(buf_ensure(ctx, F->rv, sizeof(int32_t) * P));
    SGP_TRY(buf_ensure(ctx, F->rc_ptr, sizeof(int32_t) * (P + 1)));
    SGP_TRY(buf_ensure(ctx, F->ct, sizeof(int32_t) * P));
    SGP_TRY(buf_ensure(ctx, F->L, sizeof(double) * 9 * P));
    SGP_TRY(buf_ensure(ctx, F->Dinv, sizeof(double) * 6 * n1));
    SGP_TRY(buf_ensure(ctx, F->work, sizeof(double) * 3 * n1));
    SGP_TRY(buf_ensure(ctx, F->orig_of, sizeof(int32_t) * n1));
    SGP_TRY(buf_ensure(ctx, F->small, sizeof(int32_t) * (4 + 4 * SMALL_MAXL + 8)));
    if (n == 0) return SGP_OK;
    SGP_CUDA(ctx, cudaMemcpyAsync(F->orig_of.p, M->orig_of.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));

    int32_t *adj_ptr = bp<int32_t>(F->adj_ptr), *deg = bp<int32_t>(F->deg);
    int32_t *nbr = bp<int32_t>(F->nbr), *twin = bp<int32_t>(F->twin), *eref = bp<int32_t>(F->eref);
    int32_t *lev = bp<int32_t>(F->lev), *nrec = bp<int32_t>(F->nrec), *pos = bp<int32_t>(F->pos);
    int32_t *flag = bp<int32_t>(F->flag), *tmp = bp<int32_t>(F->tmp), *rflag = bp<int32_t>(F->rflag);
    int32_t *cnt = bp<int32_t>(F->cnt);
    int32_t *A = bp<int32_t>(F->alive_a), *Bl = bp<int32_t>(F->alive_b);
    int32_t *ord = bp<int32_t>(F->ord), *pr_ptr = bp<int32_t>(F->pr_ptr), *pr_q = bp<int32_t>(F->pr_q),
            *pr_c = bp<int32_t>(F->pr_c), *rv = bp<int32_t>(F->rv), *rc_ptr = bp<int32_t>(F->rc_ptr),
            *ct = bp<int32_t>(F->ct);
    const int32_t *ij = bp<const int32_t>(M->ij), *edges = bp<const int32_t>(T->edges);

    // adjacency of the forest, sorted by neighbour, with twin entries
    SGP_CUDA(ctx, cudaMemsetAsync(deg, 0, sizeof(int32_t) * n1, ctx->stream));
    const int32_t *int_of = bp<const int32_t>(M->int_of), *orig_of = bp<const int32_t>(M->orig_of);
    LAUNCH(ctx, k_tdeg, grid_for(nt, SGP_BLOCK), SGP_BLOCK, 0, ij, edges, nt, int_of, deg);
    SGP_TRY(scan_exclusive_i32(ctx, deg, adj_ptr, n));
    SGP_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n1, ctx->stream));
    LAUNCH(ctx, k_adj_fill, grid_for(nt, SGP_BLOCK), SGP_BLOCK, 0, ij, edges, nt, int_of,
           (const int32_t *)adj_ptr, cnt, nbr, eref);
    LAUNCH(ctx, k_adj_sort, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)adj_ptr, n, nbr, eref);
    LAUNCH(ctx, k_twin, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)adj_ptr, n,
           (const int32_t *)nbr, twin);
    LAUNCH(ctx, k_acc_init, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)adj_ptr, n,
           (const int32_t *)eref, edges, bp<const int32_t>(M->edge_slot), bp<const double>(M->blk),
           M->gamma0, bp<double>(F->acc), deg, lev, A);
    SGP_CUDA(ctx, cudaMemsetAsync(rflag, 0, sizeof(int32_t) * n1, ctx->stream));

    Sim S{adj_ptr, nbr, twin, eref, deg, lev, nrec, bp<int2>(F->rq), bp<int2>(F->re), bp<int2>(F->ren)};
    int32_t na = (int32_t)n, npos = 0, npair = 0, nrecv = 0, ncontrib = 0, level = 0;
    const int max_phases = 4 * 64 + 8 * 32;
    for (int phase = 0; na > 0; ++phase) {
        if (phase > max_phases)
            return sgp_fail(ctx, SGP_ERR_TIMEOUT, "tree_factor: contraction did not finish");
        if (na <= SMALL_NA) {
            // the short tail: all remaining levels in one block, one read-back
            int32_t *hdr = bp<int32_t>(F->small);
            int4 *rec = reinterpret_cast<int4 *>(hdr + 4);
            LAUNCH(ctx, k_levels_small, 1, SB, 0, S, A, Bl, na, level, phase, rflag, ord, npos, pos, pr_ptr, pr_q,
                   pr_c, npair, rv, nrecv, rc_ptr, ct, ncontrib, (int32_t)nt, rec, hdr);
            std::vector<int32_t> h(4 + 4 * SMALL_MAXL);
            SGP_TRY(read_back(ctx, h.data(), hdr, sizeof(int32_t) * h.size()));
            if (h[2] == 1) return sgp_fail(ctx, SGP_ERR_CUDA, "tree_factor: a contraction level eliminated nothing");
            if (h[2] == 2) return sgp_fail(ctx, SGP_ERR_CUDA, "tree_factor: inconsistent contraction");
            const int32_t done = h[0];
            if (done < 1 || done > SMALL_MAXL) return sgp_fail(ctx, SGP_ERR_CUDA, "tree_factor: short tail failed");
            for (int32_t l = 0; l < done; ++l) {
                const int32_t *r = &h[4 + 4 * l];
                npos += r[0];
                npair += r[1];
                nrecv += r[2];
                ncontrib += r[3];
                F->lvl_ptr.push_back(npos);
                F->rl_ptr.push_back(nrecv);
                F->pl_ptr.push_back(npair);
                F->cl_ptr.push_back(ncontrib);
                F->rounds++;
                level++;
            }
            if (done & 1) std::swap(A, Bl);
            na = h[1];
            phase += done - 1;
            continue;
        }
        // a large level: every count stays on the device until one read at its end
        const uint32_t salt = 0x9E3779B9u * (uint32_t)(phase + 1);
        int32_t *dc = bp<int32_t>(F->small) + 4 + 4 * SMALL_MAXL;
        const unsigned gn = grid_for(na, SGP_BLOCK);
        LAUNCH(ctx, k_select, gn, SGP_BLOCK, 0, S, (const int32_t *)A, na, level, salt);
        F->rounds++;
        SGP_TRY(compact_dev(ctx, A, na, 0, level, lev, rflag, flag, tmp, ord, npos, pos, dc + 0));
        LAUNCH(ctx, k_level_nrec_d, gn, SGP_BLOCK, 0, (const int32_t *)ord, npos, na, (const int32_t *)dc,
               (const int32_t *)nrec, flag);
        SGP_TRY(scan_exclusive_i32(ctx, flag, tmp, na));
        LAUNCH(ctx, k_level_pairs_d, gn, SGP_BLOCK, 0, (const int32_t *)ord, npos, na, dc, (const int32_t *)tmp,
               npair, (const int32_t *)nrec, (const int2 *)S.rq, pr_ptr, pr_q, pr_c, rflag);
        SGP_TRY(compact_dev(ctx, A, na, 1, level, lev, rflag, flag, tmp, rv, nrecv, pos, dc + 2));
        LAUNCH(ctx, k_contrib_d<false>, gn, SGP_BLOCK, 0, S, (const int32_t *)rv, nrecv, na, dc, level,
               (const int32_t *)pos, (const int32_t *)pr_ptr, flag, (const int32_t *)nullptr, 0,
               (int32_t *)nullptr, (int32_t *)nullptr);
        SGP_TRY(scan_exclusive_i32(ctx, flag, tmp, na));
        LAUNCH(ctx, k_contrib_d<true>, gn, SGP_BLOCK, 0, S, (const int32_t *)rv, nrecv, na, dc, level,
               (const int32_t *)pos, (const int32_t *)pr_ptr, flag, (const int32_t *)tmp, ncontrib, rc_ptr, ct);
        LAUNCH(ctx, k_apply_d, gn, SGP_BLOCK, 0, S, (const int32_t *)ord, npos, (const int32_t *)dc,
               (int32_t)nt);
        level++;
        SGP_TRY(compact_dev(ctx, A, na, 2, level, lev, rflag, flag, tmp, Bl, 0, pos, dc + 4));
        int32_t h[5] = {0, 0, 0, 0, 0};
        SGP_TRY(read_back(ctx, h, dc, sizeof(h)));
        const int32_t ne = h[0], lp = h[1], nr = h[2], lc = h[3], nalive = h[4];
        if (ne == 0) return sgp_fail(ctx, SGP_ERR_CUDA, "tree_factor: a contraction level eliminated nothing");
        if (lc != lp)
            return sgp_fail(ctx, SGP_ERR_CUDA, "tree_factor: inconsistent contraction (%d/%d)", lc, lp);
        npos += ne;
        npair += lp;
        nrecv += nr;
        ncontrib += lc;
        F->lvl_ptr.push_back(npos);
        F->rl_ptr.push_back(nrecv);
        F->pl_ptr.push_back(npair);
        F->cl_ptr.push_back(ncontrib);
        std::swap(A, Bl);
        na = nalive;
    }
    if (npos != n) return sgp_fail(ctx, SGP_ERR_CUDA, "tree_factor: %d of %lld eliminated", npos, (long long)n);
    F->levels = level;
    F->npairs = npair;
    // closing entries of the pointer arrays
    const int32_t np32 = npair;
    SGP_CUDA(ctx, cudaMemcpyAsync(pr_ptr + n, &np32, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    SGP_CUDA(ctx, cudaMemcpyAsync(rc_ptr + nrecv, &ncontrib, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));

    // numeric factorisation, level by level
    int *err = ctx->d_flags;
    SGP_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    Num N{ord, nrec, pr_ptr, edges, bp<const int32_t>(M->edge_slot), bp<const int2>(F->rq),
          bp<const int2>(F->re), bp<const double>(M->blk), bp<double>(F->acc), bp<double>(F->fill),
          bp<double>(F->L), bp<double>(F->Dinv), bp<double>(F->sbuf), (int32_t)nt, err};
    for (int l = 0; l < F->levels; ++l) {
        int32_t p0 = F->lvl_ptr[l], c = F->lvl_ptr[l + 1] - p0;
        LAUNCH(ctx, k_factor_elim, grid_for(c, 128), 128, 0, N, p0, c);
        int32_t r0 = F->rl_ptr[l], rc = F->rl_ptr[l + 1] - r0;
        if (rc > 0)
            LAUNCH(ctx, k_factor_recv, grid_for(rc, 128), 128, 0, N, (const int32_t *)rv,
                   (const int32_t *)rc_ptr, (const int32_t *)ct, r0, rc);
    }
    if (F->precision == SGP_PREC_MIXED) {
        SGP_TRY(buf_ensure(ctx, F->L32, sizeof(float) * 9 * P));
        SGP_TRY(buf_ensure(ctx, F->Dinv32, sizeof(float) * 6 * n1));
        LAUNCH(ctx, k_to_f32, grid_for(9 * (int64_t)npair, SGP_BLOCK), SGP_BLOCK, 0,
               bp<const double>(F->L), bp<float>(F->L32), 9 * (int64_t)npair);
        LAUNCH(ctx, k_to_f32, grid_for(6 * n, SGP_BLOCK), SGP_BLOCK, 0, bp<const double>(F->Dinv),
               bp<float>(F->Dinv32), 6 * n);
    }
    // forward-ordered copies for the solve
    const size_t nct = (size_t)std::max<int32_t>(ncontrib, 1);
    SGP_TRY(buf_ensure(ctx, F->ctv, sizeof(int32_t) * nct));
    SGP_TRY(buf_ensure(ctx, F->Lf, sizeof(double) * 9 * nct));
    LAUNCH(ctx, k_forward_layout<double>, grid_for(ncontrib, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)ct,
           (const int32_t *)pr_c, bp<const double>(F->L), ncontrib, bp<int32_t>(F->ctv), bp<double>(F->Lf));
    if (F->precision == SGP_PREC_MIXED) {
        SGP_TRY(buf_ensure(ctx, F->Lf32, sizeof(float) * 9 * nct));
        LAUNCH(ctx, k_forward_layout<float>, grid_for(ncontrib, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)ct,
               (const int32_t *)pr_c, bp<const double>(F->L), ncontrib, (int32_t *)nullptr,
               bp<float>(F->Lf32));
    }
    // the tail: the first level from which everything left fits in the
    // tail kernel's shared memory
    int lt = 0;
    auto tail_bytes = [&](int l) {
        const int32_t tn = (int32_t)(n - F->lvl_ptr[l]), tp = npair - F->pl_ptr[l], tr = nrecv - F->rl_ptr[l];
        return F->precision == SGP_PREC_MIXED ? tail_smem_bytes<float>(tn, tp, tr)
                                              : tail_smem_bytes<double>(tn, tp, tr);
    };
    while (lt < F->levels && (tail_bytes(lt) > (size_t)TREE_TAIL_SMEM ||
                              (ctx->tail_cap >= 0 && n - F->lvl_ptr[lt] > ctx->tail_cap)))
        ++lt;
    F->tail_level = lt;
    // the tail's local index lists for levels >= t
    auto build_tail = [&](int t) -> sgp_status {
        SGP_TRY(tail_smem_optin(ctx));
        const int nl = F->levels - t;
        F->tail_P0 = F->lvl_ptr[t];
        F->tail_R0 = F->rl_ptr[t];
        F->tail_C0 = F->cl_ptr[t];
        F->tail_Q0 = F->pl_ptr[t];
        std::vector<int32_t> idx(2 * (nl + 1));
        for (int l = 0; l <= nl; ++l) {
            idx[l] = F->lvl_ptr[t + l];
            idx[nl + 1 + l] = F->rl_ptr[t + l];
        }
        SGP_TRY(buf_ensure(ctx, F->tail_idx, sizeof(int32_t) * idx.size()));
        SGP_CUDA(ctx, cudaMemcpyAsync(F->tail_idx.p, idx.data(), sizeof(int32_t) * idx.size(),
                                      cudaMemcpyHostToDevice, ctx->stream));
        // every pair of the tail is one contributor entry of the tail
        const int32_t nq = nrecv - F->tail_R0, nc = ncontrib - F->tail_C0, nb = npair - F->tail_Q0;
        if (nc != nb) return sgp_fail(ctx, SGP_ERR_CUDA, "tree_factor: inconsistent tail (%d/%d)", nc, nb);
        SGP_TRY(buf_ensure(ctx, F->tail_q, sizeof(int32_t) * std::max(nq, 1)));
        SGP_TRY(buf_ensure(ctx, F->tail_c, sizeof(int32_t) * 2 * std::max(nb, 1)));
        SGP_TRY(buf_ensure(ctx, F->tail_b, sizeof(int32_t) * std::max(nb, 1)));
        LAUNCH(ctx, k_tail_index, grid_for(nq, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)rv,
               (const int32_t *)pos, F->tail_R0, nq, F->tail_P0, bp<int32_t>(F->tail_q));
        LAUNCH(ctx, k_tail_index, grid_for(nb, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)pr_q,
               (const int32_t *)pos, F->tail_Q0, nb, F->tail_P0, bp<int32_t>(F->tail_b));
        LAUNCH(ctx, k_tail_index, grid_for(nb, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)pr_c,
               (const int32_t *)pos, F->tail_Q0, nb, F->tail_P0, bp<int32_t>(F->tail_c));
        LAUNCH(ctx, k_tail_pairs, grid_for(nb, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)ct, F->tail_C0,
               nb, F->tail_Q0, bp<int32_t>(F->tail_c) + nb);
        SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // idx lives on the host stack
        return SGP_OK;
    };
    if (lt < F->levels) SGP_TRY(build_tail(lt));
    int herr = 0;
    SGP_TRY(read_back(ctx, &herr, err, sizeof(int)));
    if (herr) return sgp_fail(ctx, SGP_ERR_NOT_SPD, "tree_factor: a pivot block is not positive definite");
    SGP_TRY(bins_build(ctx, F, M));
    return SGP_OK;
}

sgp_status sgp_tree_apply(sgp_ctx *ctx, const sgp_factor *F, const double *b, double *x)
{
    if (!ctx || !F || (F->n > 0 && (!b || !x))) return SGP_ERR_INVALID_ARG;
    if (F->n == 0) return SGP_OK;
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    // caller order -> internal order (the factor's workspace) -> caller order
    double *wi = bp<double>(F->work);
    const int32_t *orig_of = bp<const int32_t>(F->orig_of);
    LAUNCH(ctx, k_to_internal<double>, grid_for(F->n, SGP_BLOCK), SGP_BLOCK, 0, F->n, orig_of, b, wi);
    SGP_TRY(tree_apply_inplace<double>(ctx, F, wi, nullptr));
    LAUNCH(ctx, k_to_caller<double>, grid_for(F->n, SGP_BLOCK), SGP_BLOCK, 0, F->n, orig_of, (const double *)wi, x);
    if (bins_usable<double>(F)) SGP_TRY(bins_check(ctx, F));
    return SGP_OK;
}

sgp_status sgp_factor_info(const sgp_factor *F, int32_t *rounds, int32_t *levels, int64_t *l_blocks,
                           int64_t *receiver_entries)
{
    if (!F) return SGP_ERR_INVALID_ARG;
    if (rounds) *rounds = F->rounds;
    if (levels) *levels = F->levels;
    if (l_blocks) *l_blocks = F->npairs;
    if (receiver_entries) *receiver_entries = F->rl_ptr.empty() ? 0 : F->rl_ptr.back();
    return SGP_OK;
}

sgp_status sgp_factor_layout(const sgp_factor *F, int32_t *bins, int32_t *top, int32_t *leaks, int32_t *bin_cap,
                             int32_t *fp32, int32_t *fp64)
{
    if (!F) return SGP_ERR_INVALID_ARG;
    if (bins) *bins = F->bl.nb;
    if (top) *top = F->bl.nt;
    if (leaks) *leaks = F->bl.nly;
    if (bin_cap) *bin_cap = F->bl.bmax;
    if (fp32) *fp32 = F->bl.ok32;
    if (fp64) *fp64 = F->bl.ok64;
    return SGP_OK;
}

void sgp_factor_destroy(sgp_factor *F)
{
    if (!F) return;
    cudaDeviceSynchronize();
    DBuf *bufs[] = {&F->ord, &F->pr_ptr, &F->pr_q, &F->pr_c, &F->rv, &F->rc_ptr, &F->ct, &F->L,
                    &F->Dinv, &F->L32, &F->Dinv32, &F->work, &F->adj_ptr, &F->nbr, &F->twin,
                    &F->eref, &F->deg, &F->lev, &F->nrec, &F->rq, &F->re, &F->ren, &F->pos,
                    &F->flag, &F->alive_a, &F->alive_b, &F->acc, &F->fill, &F->sbuf, &F->tmp,
                    &F->rflag, &F->cnt, &F->ctv, &F->Lf, &F->Lf32, &F->tail_idx, &F->tail_q,
                    &F->tail_c, &F->tail_b, &F->orig_of, &F->small};
    for (DBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    BinLayout &B = F->bl;
    DBuf *bb[] = {&B.hdr, &B.order, &B.elev, &B.vlev, &B.gvert, &B.er, &B.ec, &B.cl, &B.kl, &B.ks, &B.pr, &B.pref, &B.zi,
                  &B.tv, &B.tint, &B.c_src, &B.k_src, &B.p_src, &B.d_src, &B.t_src, &B.tD_src, &B.part, &B.err,
                  &B.i_of_t, &B.t_of_i, &B.rpt, &B.ma32, &B.mb32, &B.m64, &B.mc64};
    for (DBuf *b : bb)
        if (b->p) cudaFree(b->p);
    for (int k = 0; k < 2; ++k) {
        DBuf *nb[] = {&B.cL[k], &B.kL[k], &B.pL[k], &B.D[k], &B.tL[k], &B.tD[k], &B.ly[k], &B.lsum[k], &B.tw[k]};
        for (DBuf *b : nb)
            if (b->p) cudaFree(b->p);
    }
    for (DBuf &b : B.scr)
        if (b.p) cudaFree(b.p);
    delete F;
}

}  // extern "C"
