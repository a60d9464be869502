// bins.cu -- the spanning-forest solve z = P^-1 w in three launches
// (Appendix B.1 forward substitution, diagonal solve, backward substitution),
// on the elimination structure of the rake/compress contraction.
//
// Every eliminated vertex c sends its forward value to its receivers (the
// one or two neighbours it had when it went); the receiver eliminated first
// is c's parent in the contraction tree, and every receiver of c is c or one
// of c's ancestors there.  So a subtree of the contraction tree is closed: the
// forward values of its vertices depend only on the subtree, and the only
// values that leave it go to at most two vertices above it.  The forest's
// solve is cut along that tree:
//
//   bottom: the maximal subtrees with at most `bmax` vertices, packed in
//           spatial order into bins of at most bmax vertices; one thread
//           block solves a bin's forward levels from shared memory (its
//           structure and L blocks staged by bulk asynchronous copies),
//           writes the forward values, and the products L_qc w_c for
//           receivers q above the bin ("leaks");
//   top:    the vertices whose subtree is larger than bmax (about
//           n / bmax of them) in one thread block: its forward levels, the
//           diagonal solve and its backward levels, all in shared memory;
//   bottom: one thread block per bin again for the backward levels.
//
// Each launch stages what does not depend on the previous launch before its
// programmatic-dependent-launch wait, so the bins' copies overlap the top
// block.  Inside a bin and inside the top every level is a block barrier,
// not a kernel boundary.  The sums of the forward substitution keep the
// contraction's contributor order except for a top receiver, which first
// subtracts the sum of all its leaks (in contributor order) and then its
// top contributors level by level: the same operator, other rounding.
//
// For PCG the three launches also carry the vector work around the solve:
// the bins and the top apply r -= alpha q and sum |r|^2 (the top block
// finishes the sum and takes the stopping decision), and the backward
// launch sums r^T z (its last block sets beta).
#include "solver_common.cuh"

namespace {

constexpr int BA = 128;    // threads of a bin block
constexpr int BT = 256;    // threads of the top block
constexpr int SMEM_MAX = 226 * 1024;
constexpr int SEGMAX = 4096;
// header of a bin (int32 each)
enum { H_VOFF, H_NV, H_EOFF, H_NE, H_COFF, H_NC, H_KOFF, H_NK, H_POFF, H_NP, H_ZOFF, H_NZ, H_NLEV, H_N = 16 };

__host__ __device__ __forceinline__ int32_t pad4(int32_t x) { return (x + 3) & ~3; }

struct BinCheck {
    const int32_t *hdr, *elev, *vlev, *gvert, *er, *ec, *cl, *kl, *ks, *pr, *pref, *zi;
    int32_t LVP, nly, nt, n;
    int32_t G, E, Cc, K, Pp, Z;   // lengths of the arrays above (padded totals)
    int *err;
};
struct TopCheck {
    const int32_t *tint, *tv;
    int32_t o[9];
    int32_t LVP, nte, ntt, nt, ntp, nly, n;
    int *err;
};

// ------------------------------------------------------------ async copies
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
// bytes: a nonzero multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
// Wait for phase 0 of the barrier with an iteration limit; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(su32(bar))
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Bytes of dynamic shared memory this launch has (the kernels check their
// own layout against it before any copy, so that a layout error can only
// raise the error flag).
__device__ __forceinline__ uint32_t dyn_smem()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// Copies issued by one thread against one barrier: the expected byte count
// first (the sum of all sizes), then each nonzero copy.  Sizes and
// addresses are kept in registers (fixed slots, unrolled).
template <int N>
struct Stage {
    void *d[N];
    const void *s[N];
    uint32_t b[N];
    __device__ __forceinline__ void issue(uint64_t *bar)
    {
        uint32_t total = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) total += b[k];
        mbar_expect(bar, total);
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (b[k]) bulk_load(d[k], s[k], b[k], bar);
    }
};

// Block-wide exclusive scan of one int per thread (BS threads); *total gets the sum.
template <int BS>
__device__ __forceinline__ int32_t bscan(int32_t v, int32_t *sh, int32_t *total)
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
        int32_t t = (l < BS / 32) ? sh[l] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (l >= o) t += y;
        }
        if (l < BS / 32) sh[l] = t;
    }
    __syncthreads();
    int32_t before = (w > 0 ? sh[w - 1] : 0) + x - v;
    *total = sh[BS / 32 - 1];
    __syncthreads();
    return before;
}

// ------------------------------------------------------- structure kernels
// level of each item from the level pointer array (items in level order)
__global__ void k_bn_level(const int32_t *__restrict__ lp, int32_t LV, int32_t n, int32_t *lev)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int32_t lo = 0, hi = LV;   // lp[lo] <= t < lp[hi]
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if (lp[mid] <= t) lo = mid; else hi = mid;
    }
    lev[t] = lo;
}

// parent in the contraction tree: the receiver eliminated first
__global__ void k_bn_parent(int32_t n, const int32_t *__restrict__ pr_ptr, const int32_t *__restrict__ pr_q,
                            const int32_t *__restrict__ pos, int32_t *par, int32_t *sz)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int32_t best = -1;
    for (int32_t p = pr_ptr[t]; p < pr_ptr[t + 1]; ++p) {
        int32_t u = pos[pr_q[p]];
        if (best < 0 || u < best) best = u;
    }
    par[t] = best;
    sz[t] = 1;
}

// subtree sizes, one level at a time (children before parents)
__global__ void k_bn_size(int32_t p0, int32_t cnt, const int32_t *__restrict__ par, int32_t *sz)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    int32_t t = p0 + k, u = par[t];
    if (u >= 0) atomicAdd(sz + u, sz[t]);
}

// top: subtree larger than bmax; root of the bottom: not top, parent top or none.
// rootv is indexed by vertex (roots are packed in the cells' spatial order).
__global__ void k_bn_class(int32_t n, int32_t bmax, const int32_t *__restrict__ sz, const int32_t *__restrict__ par,
                           const int32_t *__restrict__ ord, int32_t *top, int32_t *isroot, int32_t *rootv)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const bool tp = sz[t] > bmax;
    const int32_t u = par[t];
    const bool rt = !tp && (u < 0 || sz[u] > bmax);
    top[t] = tp;
    isroot[t] = rt;
    rootv[ord[t]] = rt;
}

// roots in vertex order: position, and size when it is a small root
__global__ void k_bn_roots(int32_t n, const int32_t *__restrict__ rootv, const int32_t *__restrict__ ridx,
                           const int32_t *__restrict__ pos, const int32_t *__restrict__ sz, int32_t half,
                           int32_t *rpos, int32_t *rsm)
{
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || !rootv[v]) return;
    int32_t i = ridx[v], t = pos[v], s = sz[t];
    rpos[i] = t;
    rsm[i] = s <= half ? s : 0;
}

// A root opens a new bin if it is big (its own bin), follows a big root, or
// its small-root prefix starts a new unit of `half` vertices: small bins
// then hold less than 2 * half vertices.
__global__ void k_bn_newbin(int32_t nr, const int32_t *__restrict__ rpre, const int32_t *__restrict__ rsm,
                            int32_t half, int32_t *nbf)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    bool nb = i == 0 || rsm[i] == 0 || rsm[i - 1] == 0 || rpre[i] / half != rpre[i - 1] / half;
    nbf[i] = nb;
}

__global__ void k_bn_rootbin(int32_t nr, const int32_t *__restrict__ rpos, const int32_t *__restrict__ bid,
                             const int32_t *__restrict__ nbf, int32_t *binroot)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    binroot[rpos[i]] = bid[i] + nbf[i] - 1;
}

__global__ void k_bn_anc_init(int32_t n, const int32_t *__restrict__ top, const int32_t *__restrict__ isroot,
                              const int32_t *__restrict__ par, int32_t *anc)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    anc[t] = (top[t] || isroot[t]) ? t : par[t];
}

__global__ void k_bn_jump(int32_t n, const int32_t *__restrict__ a, int32_t *b)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    b[t] = a[a[t]];
}

__global__ void k_bn_binp(int32_t n, const int32_t *__restrict__ top, const int32_t *__restrict__ anc,
                          const int32_t *__restrict__ binroot, int32_t *binp)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    binp[t] = top[t] ? -1 : binroot[anc[t]];
}

// ---- grouping: count, padded offsets, placement, sort by key inside each group
__global__ void k_bn_count(int32_t n, const int32_t *__restrict__ seg, int32_t *cnt)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t s = seg[i];
    if (s >= 0) atomicAdd(cnt + s, 1);
}
__global__ void k_bn_pad(int32_t ns, const int32_t *__restrict__ cnt, int pad, int32_t *out)
{
    int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    out[s] = pad ? pad4(cnt[s]) : cnt[s];
}
__global__ void k_bn_place(int32_t n, const int32_t *__restrict__ seg, const int32_t *__restrict__ key,
                           const int32_t *__restrict__ off, int32_t *fill, int32_t *kt)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t s = seg[i];
    if (s < 0) return;
    int32_t slot = off[s] + atomicAdd(fill + s, 1);
    kt[slot] = key ? key[i] : i;
}
// one block per group: rank of each key among the group's (distinct) keys
__global__ void k_bn_segsort(const int32_t *__restrict__ off, const int32_t *__restrict__ cnt,
                             const int32_t *__restrict__ kt, int32_t *out)
{
    __shared__ int32_t sk[SEGMAX];
    const int32_t s = blockIdx.x, o = off[s], c = cnt[s];
    const bool sm = c <= SEGMAX;
    if (sm)
        for (int32_t i = threadIdx.x; i < c; i += blockDim.x) sk[i] = kt[o + i];
    __syncthreads();
    for (int32_t i = threadIdx.x; i < c; i += blockDim.x) {
        const int32_t k = sm ? sk[i] : kt[o + i];
        int32_t r = 0;
        for (int32_t j = 0; j < c; ++j) r += (sm ? sk[j] : kt[o + j]) < k;
        out[o + r] = k;
    }
}

// forward entries whose receiver is in a bin
__global__ void k_bn_seg_entry(int32_t ne, const int32_t *__restrict__ rv, const int32_t *__restrict__ pos,
                               const int32_t *__restrict__ binp, int32_t *seg)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ne) seg[k] = binp[pos[rv[k]]];
}
// entry of each contributor slot
__global__ void k_bn_kofj(int32_t ne, const int32_t *__restrict__ rc_ptr, int32_t *kofj)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ne) return;
    for (int32_t j = rc_ptr[k]; j < rc_ptr[k + 1]; ++j) kofj[j] = k;
}
// leaks: contributor slots with a top receiver and a bin contributor,
// grouped by the receiver's top index
__global__ void k_bn_seg_leak(int32_t nc, const int32_t *__restrict__ kofj, const int32_t *__restrict__ rv,
                              const int32_t *__restrict__ ct, const int32_t *__restrict__ pr_c,
                              const int32_t *__restrict__ pos, const int32_t *__restrict__ top,
                              const int32_t *__restrict__ topidx, int32_t *seg)
{
    int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nc) return;
    int32_t tq = pos[rv[kofj[j]]], tc = pos[pr_c[ct[j]]];
    seg[j] = (top[tq] && !top[tc]) ? topidx[tq] : -1;
}
// leak slots grouped by the contributor's bin
__global__ void k_bn_seg_leakbin(int32_t nly, const int32_t *__restrict__ lkj, const int32_t *__restrict__ ct,
                                 const int32_t *__restrict__ pr_c, const int32_t *__restrict__ pos,
                                 const int32_t *__restrict__ binp, int32_t *seg)
{
    int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nly) return;
    seg[s] = binp[pos[pr_c[ct[lkj[s]]]]];
}

// One block per bin, over its vertices (sorted by position = level order):
// local index, vertex ids, per-level vertex offsets, pair and top-reference
// starts; records the bin's counts.
__global__ void __launch_bounds__(BA) k_bn_binvert(const int32_t *__restrict__ voff, const int32_t *__restrict__ cntv,
                                                   const int32_t *__restrict__ gpos, const int32_t *__restrict__ ord,
                                                   const int32_t *__restrict__ levp,
                                                   const int32_t *__restrict__ pr_ptr,
                                                   const int32_t *__restrict__ pr_q, const int32_t *__restrict__ pos,
                                                   const int32_t *__restrict__ top, int32_t LVP, int32_t *lpos,
                                                   int32_t *gvert, int32_t *gbin, int32_t *vlev, int32_t *pr,
                                                   int32_t *zpre, int32_t *hdr)
{
    __shared__ int32_t sh[BA / 32];
    const int32_t b = blockIdx.x, o = voff[b], nv = cntv[b];
    int32_t carry_p = 0, carry_z = 0;
    for (int32_t base = 0; base < nv; base += BA) {
        const int32_t l = base + threadIdx.x;
        int32_t np = 0, nz = 0;
        if (l < nv) {
            const int32_t t = gpos[o + l];
            lpos[t] = l;
            gvert[o + l] = ord[t];
            gbin[o + l] = b;
            for (int32_t p = pr_ptr[t]; p < pr_ptr[t + 1]; ++p) {
                ++np;
                nz += top[pos[pr_q[p]]] != 0;
            }
            const int32_t lv = levp[t], lp = l > 0 ? levp[gpos[o + l - 1]] : -1;
            for (int32_t L = lp + 1; L <= lv; ++L) vlev[(size_t)b * LVP + L] = l;
            if (l == nv - 1)
                for (int32_t L = lv + 1; L < LVP; ++L) vlev[(size_t)b * LVP + L] = nv;
        }
        int32_t tp, tz;
        const int32_t ep = bscan<BA>(np, sh, &tp);
        const int32_t ez = bscan<BA>(nz, sh, &tz);
        if (l < nv) {
            pr[o + l] = carry_p + ep;
            zpre[o + l] = carry_z + ez;
        }
        carry_p += tp;
        carry_z += tz;
    }
    if (threadIdx.x == 0) {
        int32_t *h = hdr + (size_t)H_N * b;
        h[H_VOFF] = o;
        h[H_NV] = nv;
        h[H_NP] = carry_p;
        h[H_NZ] = carry_z;
        h[H_NLEV] = nv > 0 ? levp[gpos[o + nv - 1]] + 1 : 0;
    }
}

// One block per bin, over its forward entries (sorted = level order):
// receiver's local index, contributor starts, per-level entry offsets.
__global__ void __launch_bounds__(BA) k_bn_binent(const int32_t *__restrict__ eoff, const int32_t *__restrict__ cnte,
                                                  const int32_t *__restrict__ gent, const int32_t *__restrict__ rv,
                                                  const int32_t *__restrict__ rc_ptr,
                                                  const int32_t *__restrict__ pos, const int32_t *__restrict__ lpos,
                                                  const int32_t *__restrict__ levE, int32_t LVP, int32_t *er,
                                                  int32_t *ec, int32_t *ebin, int32_t *elev, int32_t *hdr)
{
    __shared__ int32_t sh[BA / 32];
    const int32_t b = blockIdx.x, o = eoff[b], ne = cnte[b];
    int32_t carry = 0;
    if (ne == 0)
        for (int32_t L = threadIdx.x; L < LVP; L += BA) elev[(size_t)b * LVP + L] = 0;
    for (int32_t base = 0; base < ne; base += BA) {
        const int32_t e = base + threadIdx.x;
        int32_t nc = 0;
        if (e < ne) {
            const int32_t k = gent[o + e];
            er[o + e] = lpos[pos[rv[k]]];
            ebin[o + e] = b;
            nc = rc_ptr[k + 1] - rc_ptr[k];
            const int32_t lv = levE[k], lp = e > 0 ? levE[gent[o + e - 1]] : -1;
            for (int32_t L = lp + 1; L <= lv; ++L) elev[(size_t)b * LVP + L] = e;
            if (e == ne - 1)
                for (int32_t L = lv + 1; L < LVP; ++L) elev[(size_t)b * LVP + L] = ne;
        }
        int32_t tot;
        const int32_t ex = bscan<BA>(nc, sh, &tot);
        if (e < ne) ec[o + e] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        int32_t *h = hdr + (size_t)H_N * b;
        h[H_EOFF] = o;
        h[H_NE] = ne;
        h[H_NC] = carry;
    }
}

// counts of the header -> padded offsets later; read one field of every header
__global__ void k_bn_hfield(int32_t nb, const int32_t *__restrict__ hdr, int f, int32_t *out)
{
    int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) out[b] = pad4(hdr[(size_t)H_N * b + f]);
}
__global__ void k_bn_hset(int32_t nb, const int32_t *__restrict__ off, int f, int32_t *hdr)
{
    int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) hdr[(size_t)H_N * b + f] = off[b];
}

// contributors of the bins' entries
__global__ void k_bn_contrib(int32_t E, const int32_t *__restrict__ gent, const int32_t *__restrict__ ebin,
                             const int32_t *__restrict__ ec, const int32_t *__restrict__ hdr,
                             const int32_t *__restrict__ rc_ptr, const int32_t *__restrict__ ct,
                             const int32_t *__restrict__ pr_c, const int32_t *__restrict__ pos,
                             const int32_t *__restrict__ lpos, int32_t *cl, int32_t *c_src)
{
    int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int32_t k = gent[e];
    if (k < 0) return;
    const int32_t b = ebin[e], base = hdr[(size_t)H_N * b + H_COFF] + ec[e];
    for (int32_t j = rc_ptr[k]; j < rc_ptr[k + 1]; ++j) {
        const int32_t d = base + (j - rc_ptr[k]);
        cl[d] = lpos[pos[pr_c[ct[j]]]];
        c_src[d] = j;
    }
}

// the bins' leaks: local contributor, slot, source contributor entry
__global__ void k_bn_leakfill(int32_t K, const int32_t *__restrict__ kslot, const int32_t *__restrict__ lkj,
                              const int32_t *__restrict__ ct, const int32_t *__restrict__ pr_c,
                              const int32_t *__restrict__ pos, const int32_t *__restrict__ lpos, int32_t *kl,
                              int32_t *ks, int32_t *k_src)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int32_t s = kslot[k];
    if (s < 0) {
        kl[k] = 0; ks[k] = 0; k_src[k] = -1;
        return;
    }
    const int32_t j = lkj[s];
    kl[k] = lpos[pos[pr_c[ct[j]]]];
    ks[k] = s;
    k_src[k] = j;
}

// backward pairs of the bins' vertices: receiver reference and source pair
__global__ void k_bn_pairs(int32_t G, const int32_t *__restrict__ gpos, const int32_t *__restrict__ gbin,
                           const int32_t *__restrict__ pr, const int32_t *__restrict__ zpre,
                           const int32_t *__restrict__ hdr, const int32_t *__restrict__ pr_ptr,
                           const int32_t *__restrict__ pr_q, const int32_t *__restrict__ pos,
                           const int32_t *__restrict__ top, const int32_t *__restrict__ topidx,
                           const int32_t *__restrict__ lpos, int32_t *pref, int32_t *p_src, int32_t *zi)
{
    int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int32_t t = gpos[g];
    if (t < 0) return;
    const int32_t *h = hdr + (size_t)H_N * gbin[g];
    int32_t pp = h[H_POFF] + pr[g], kz = zpre[g];
    for (int32_t p = pr_ptr[t]; p < pr_ptr[t + 1]; ++p, ++pp) {
        const int32_t tq = pos[pr_q[p]];
        if (top[tq]) {
            pref[pp] = -1 - kz;
            zi[h[H_ZOFF] + kz] = topidx[tq];
            ++kz;
        } else {
            pref[pp] = lpos[tq];
        }
        p_src[pp] = p;
    }
}

// per-bin shared memory of the forward and backward kernels, FP32 and FP64:
// the vector slice and the index arrays, plus the staged suffix of L blocks
// (forward: the tail levels' contributors) or of D^-1 and L blocks
// (backward: the vertices above the last level with more than 32)
__global__ void k_bn_smem(int32_t nb, const int32_t *__restrict__ hdr, int32_t LVP, const int32_t *__restrict__ elev,
                          const int32_t *__restrict__ ec, const int32_t *__restrict__ vlev,
                          const int32_t *__restrict__ pr, int32_t *mx)
{
    int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int32_t *h = hdr + (size_t)H_N * b;
    const int32_t nv = h[H_NV], ne = h[H_NE], nc = h[H_NC], nlev = h[H_NLEV];
    const int32_t nvp = pad4(nv), nep = pad4(ne), ncp = pad4(nc), nkp = pad4(h[H_NK]), npp = pad4(h[H_NP]),
                  nzp = pad4(h[H_NZ]);
    const int32_t *el = elev + (size_t)b * LVP, *vl = vlev + (size_t)b * LVP;
    int sf = nlev;
    while (sf > 0 && el[sf] - el[sf - 1] <= 32) --sf;
    const int32_t jt = (sf < nlev && el[sf] < ne) ? (ec[h[H_EOFF] + el[sf]] & ~3) : ncp;
    int sb = nlev - 1;
    while (sb >= 0 && vl[sb + 1] - vl[sb] <= 32) --sb;
    const int32_t vs = sb < nlev - 1 ? vl[sb + 1] : nv;
    const int32_t it = vs < nv ? (vs & ~3) : nvp;
    const int32_t pt = vs < nv ? (pr[h[H_VOFF] + vs] & ~3) : npp;
    // mx[4 s + 2 f + k]: precision s (FP32, FP64), fused f, kernel k (forward, backward)
    for (int s = 0; s < 2; ++s) {
        const int32_t sz = s == 0 ? 4 : 8;
        const int32_t fa = nvp * 3 * sz + LVP * 4 + nep * 8 + ncp * 4 + nkp * 8 + (ncp - jt) * 9 * sz;
        const int32_t fc = (nvp + nzp) * 3 * sz + LVP * 4 + nvp * 4 + npp * 4 + nzp * 4 + (nvp - it) * 6 * sz +
                           (npp - pt) * 9 * sz;
        atomicMax(mx + 4 * s, fa);
        atomicMax(mx + 4 * s + 1, fc);
        atomicMax(mx + 4 * s + 2, fa);
        atomicMax(mx + 4 * s + 3, fc);
    }
}

// ---- top structure
__global__ void k_bn_topcompact(int32_t n, const int32_t *__restrict__ top, const int32_t *__restrict__ topidx,
                                const int32_t *__restrict__ ord, int32_t *tpos, int32_t *tv)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || !top[t]) return;
    tpos[topidx[t]] = t;
    tv[topidx[t]] = ord[t];
}
// level boundaries of a level-sorted list (single pass): off[L] = first index with level >= L
__global__ void k_bn_bounds(int32_t cnt, const int32_t *__restrict__ item, const int32_t *__restrict__ lev,
                            int32_t LVP, int32_t *off)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (cnt == 0) {
        if (i < LVP) off[i] = 0;
        return;
    }
    if (i >= cnt) return;
    const int32_t lv = lev[item[i]], lp = i > 0 ? lev[item[i - 1]] : -1;
    for (int32_t L = lp + 1; L <= lv; ++L) off[L] = i;
    if (i == cnt - 1)
        for (int32_t L = lv + 1; L < LVP; ++L) off[L] = cnt;
}
// top entries with at least one top contributor ("blocking": they wait for
// the top's own levels); their top-contributor counts
__global__ void k_bn_tflag(int32_t ne, const int32_t *__restrict__ rv, const int32_t *__restrict__ rc_ptr,
                           const int32_t *__restrict__ ct, const int32_t *__restrict__ pr_c,
                           const int32_t *__restrict__ pos, const int32_t *__restrict__ top, int32_t *flag,
                           int32_t *tcnt)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ne) return;
    int32_t c = 0;
    if (top[pos[rv[k]]])
        for (int32_t j = rc_ptr[k]; j < rc_ptr[k + 1]; ++j) c += top[pos[pr_c[ct[j]]]] != 0;
    flag[k] = c > 0;
    tcnt[k] = c;
}
__global__ void k_bn_tentry(int32_t ne, const int32_t *__restrict__ flag, const int32_t *__restrict__ tidx,
                            const int32_t *__restrict__ tcnt, const int32_t *__restrict__ rv,
                            const int32_t *__restrict__ pos, const int32_t *__restrict__ topidx, int32_t *tek,
                            int32_t *ter, int32_t *tc_n)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ne || !flag[k]) return;
    const int32_t e = tidx[k];
    tek[e] = k;
    ter[e] = topidx[pos[rv[k]]];
    tc_n[e] = tcnt[k];
}
__global__ void k_bn_tcontrib(int32_t nte, const int32_t *__restrict__ tek, const int32_t *__restrict__ tcp,
                              const int32_t *__restrict__ rc_ptr, const int32_t *__restrict__ ct,
                              const int32_t *__restrict__ pr_c, const int32_t *__restrict__ pos,
                              const int32_t *__restrict__ top, const int32_t *__restrict__ topidx, int32_t *tcc,
                              int32_t *t_src, int32_t *pair2tt)
{
    int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nte) return;
    const int32_t k = tek[e];
    int32_t d = tcp[e];
    for (int32_t j = rc_ptr[k]; j < rc_ptr[k + 1]; ++j) {
        const int32_t tc = pos[pr_c[ct[j]]];
        if (!top[tc]) continue;
        tcc[d] = topidx[tc];
        t_src[d] = j;
        pair2tt[ct[j]] = d;
        ++d;
    }
}
__global__ void k_bn_tpcount(int32_t nt, const int32_t *__restrict__ tpos, const int32_t *__restrict__ pr_ptr,
                             int32_t *c)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt) c[i] = pr_ptr[tpos[i] + 1] - pr_ptr[tpos[i]];
}
__global__ void k_bn_tpairs(int32_t nt, const int32_t *__restrict__ tpos, const int32_t *__restrict__ tpp,
                            const int32_t *__restrict__ pr_ptr, const int32_t *__restrict__ pr_q,
                            const int32_t *__restrict__ pos, const int32_t *__restrict__ topidx,
                            const int32_t *__restrict__ pair2tt, int32_t *tpq, int32_t *tpL, int32_t *err)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int32_t t = tpos[i];
    int32_t d = tpp[i];
    for (int32_t p = pr_ptr[t]; p < pr_ptr[t + 1]; ++p, ++d) {
        tpq[d] = topidx[pos[pr_q[p]]];
        const int32_t x = pair2tt[p];
        if (x < 0) atomicOr(err, 1);
        tpL[d] = x < 0 ? 0 : x;
    }
}

// ---- numeric layout: gathers of L (full9) and D^-1 (sym6) blocks
// (source entries outside [0, lim) -- the padding -- give zero blocks)
template <typename T, int W>
__global__ void k_bn_gather(int32_t cnt, const int32_t *__restrict__ src, int64_t lim,
                            const double *__restrict__ from, T *to)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int32_t s = src[i];
    const bool ok = s >= 0 && s < lim;
#pragma unroll
    for (int a = 0; a < W; ++a) to[(size_t)W * i + a] = ok ? (T)from[(size_t)W * s + a] : T(0);
}

// ---- consistency of the layout: every index the solve kernels use must
// lie inside the arrays they stage (checked once per build; a failure is a
// library bug and the build reports it instead of launching the solve)
__device__ __forceinline__ void bad(int *err, int code) { atomicOr(err, 1 << code); }
__global__ void __launch_bounds__(BA) k_bn_check_bins(BinCheck c)
{
    const int32_t b = blockIdx.x;
    const int32_t *h = c.hdr + (size_t)H_N * b;
    const int32_t voff = h[H_VOFF], nv = h[H_NV], eoff = h[H_EOFF], ne = h[H_NE], coff = h[H_COFF], nc = h[H_NC],
                  koff = h[H_KOFF], nk = h[H_NK], poff = h[H_POFF], np = h[H_NP], zoff = h[H_ZOFF], nz = h[H_NZ],
                  nlev = h[H_NLEV];
    // every segment inside its array (else nothing below is read)
    const bool in = nv >= 1 && nlev >= 1 && nlev <= c.LVP - 1 && voff >= 0 && voff + pad4(nv) <= c.G &&
                    ne >= 0 && eoff >= 0 && eoff + pad4(ne) <= c.E && nc >= 0 && coff >= 0 &&
                    coff + pad4(nc) <= c.Cc && nk >= 0 && koff >= 0 && koff + pad4(nk) <= c.K && np >= 0 &&
                    poff >= 0 && poff + pad4(np) <= c.Pp && nz >= 0 && zoff >= 0 && zoff + pad4(nz) <= c.Z;
    if (!in) {
        if (threadIdx.x == 0) bad(c.err, 2);
        return;
    }
    if (threadIdx.x == 0)
        if (c.elev[(size_t)b * c.LVP + nlev] != ne || c.vlev[(size_t)b * c.LVP + nlev] != nv) bad(c.err, 3);
    for (int32_t L = threadIdx.x; L + 1 < c.LVP; L += BA) {
        const int32_t *el = c.elev + (size_t)b * c.LVP, *vl = c.vlev + (size_t)b * c.LVP;
        if (el[L] < 0 || el[L] > el[L + 1] || el[L + 1] > ne) bad(c.err, 4);
        if (vl[L] < 0 || vl[L] > vl[L + 1] || vl[L + 1] > nv) bad(c.err, 5);
    }
    for (int32_t e = threadIdx.x; e < ne; e += BA) {
        const int32_t r = c.er[eoff + e], j0 = c.ec[eoff + e], j1 = e + 1 < ne ? c.ec[eoff + e + 1] : nc;
        if (r < 0 || r >= nv || j0 < 0 || j0 > j1 || j1 > nc) bad(c.err, 6);
    }
    for (int32_t j = threadIdx.x; j < nc; j += BA)
        if (c.cl[coff + j] < 0 || c.cl[coff + j] >= nv) bad(c.err, 7);
    for (int32_t k = threadIdx.x; k < nk; k += BA)
        if (c.kl[koff + k] < 0 || c.kl[koff + k] >= nv || c.ks[koff + k] < 0 || c.ks[koff + k] >= c.nly)
            bad(c.err, 8);
    for (int32_t i = threadIdx.x; i < nv; i += BA) {
        const int32_t p0 = c.pr[voff + i], p1 = i + 1 < nv ? c.pr[voff + i + 1] : np;
        if (p0 < 0 || p0 > p1 || p1 > np || p1 - p0 > 2) bad(c.err, 9);
        if (c.gvert[voff + i] < 0 || c.gvert[voff + i] >= c.n) bad(c.err, 10);
    }
    for (int32_t p = threadIdx.x; p < np; p += BA) {
        const int32_t r = c.pref[poff + p];
        if (r >= nv || (r < 0 && -1 - r >= nz)) bad(c.err, 11);
    }
    for (int32_t k = threadIdx.x; k < nz; k += BA)
        if (c.zi[zoff + k] < 0 || c.zi[zoff + k] >= c.nt) bad(c.err, 12);
}
__global__ void k_bn_check_top(TopCheck t)
{
    const int32_t *ti = t.tint;
    const int32_t *telev = ti + t.o[0], *ter = ti + t.o[1], *tcp = ti + t.o[2], *tcc = ti + t.o[3],
                  *tvlev = ti + t.o[4], *tpp = ti + t.o[5], *tpq = ti + t.o[6], *tpL = ti + t.o[7],
                  *tlk = ti + t.o[8];
    for (int32_t L = threadIdx.x; L + 1 < t.LVP; L += blockDim.x) {
        if (telev[L] < 0 || telev[L] > telev[L + 1] || telev[L + 1] > t.nte) bad(t.err, 13);
        if (tvlev[L] < 0 || tvlev[L] > tvlev[L + 1] || tvlev[L + 1] > t.nt) bad(t.err, 14);
    }
    for (int32_t e = threadIdx.x; e < t.nte; e += blockDim.x)
        if (ter[e] < 0 || ter[e] >= t.nt || tcp[e] < 0 || tcp[e] > tcp[e + 1] || tcp[e + 1] > t.ntt) bad(t.err, 15);
    for (int32_t j = threadIdx.x; j < t.ntt; j += blockDim.x)
        if (tcc[j] < 0 || tcc[j] >= t.nt) bad(t.err, 16);
    for (int32_t i = threadIdx.x; i < t.nt; i += blockDim.x) {
        if (tpp[i] < 0 || tpp[i] > tpp[i + 1] || tpp[i + 1] > t.ntp) bad(t.err, 17);
        if (tlk[i] < 0 || tlk[i] > tlk[i + 1] || tlk[i + 1] > t.nly) bad(t.err, 18);
        if (t.tv[i] < 0 || t.tv[i] >= t.n) bad(t.err, 19);
    }
    for (int32_t p = threadIdx.x; p < t.ntp; p += blockDim.x)
        if (tpq[p] < 0 || tpq[p] >= t.nt || tpL[p] < 0 || tpL[p] >= t.ntt) bad(t.err, 20);
}

// ------------------------------------------------------------ solve kernels
// The vectors of the binned solve are kept in its own order ("tree order"):
// bin b's vertices at [voff, voff + nv) in elimination order (each segment
// padded to 4 entries), then the top part at [G, G + nt).  Padding entries
// are zero and stay zero, so a bin's slice of every vector is one
// contiguous, 16-byte aligned stretch.
struct BinArgs {
    const int32_t *hdr, *order, *elev, *vlev, *er, *ec, *cl, *kl, *ks, *pr, *pref, *zi;
    int32_t LVP, nb, G;
    int *err;
};
template <typename T>
struct BinNum {
    const T *cL, *kL, *pL, *D;
    T *ly;
};
struct TopArgs {
    const int32_t *tint;
    int32_t nt, LVP, nte, ntt, ntp, tints, nly, G;
    int32_t o_telev, o_ter, o_tcp, o_tcc, o_tvlev, o_tpp, o_tpq, o_tpL, o_tlk;
    int *err;
};

// The staged copies must have landed before the block may leave (they
// write into its shared memory); returns false (error recorded) on timeout.
template <int FUSE>
__device__ __forceinline__ bool staged(uint64_t *bar, int *err, Scal *sc)
{
    if (!__syncthreads_and(mbar_wait(bar))) {
        if (threadIdx.x == 0) {
            atomicOr(err, 1);
            if (FUSE) {
                sc->status = SGP_ERR_TIMEOUT;
                sc->done = 1;
            }
        }
        return false;
    }
    return true;
}

// One forward entry held in registers: its receiver, the first two of its
// contributors (index and L block) and where the others start.  The entries
// of level l+1 are read from shared memory while level l computes, so that
// a level's critical path is only its reads of the solution vector.
template <typename T>
struct FwdEnt {
    int32_t r, j0, n, c0, c1;
    T L0[9], L1[9];
};
template <typename T>
__device__ __forceinline__ void fwd_fetch(FwdEnt<T> &f, int32_t e, int32_t e1, const int32_t *er, const int32_t *ec,
                                          int32_t ne, int32_t nc, const int32_t *cl, const T *cL)
{
    if (e >= e1) {
        f.n = -1;
        return;
    }
    f.r = er[e];
    f.j0 = ec[e];
    f.n = (e + 1 < ne ? ec[e + 1] : nc) - f.j0;
    f.c0 = f.n > 0 ? cl[f.j0] : 0;
    f.c1 = f.n > 1 ? cl[f.j0 + 1] : 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        f.L0[a] = f.n > 0 ? cL[9 * f.j0 + a] : T(0);
        f.L1[a] = f.n > 1 ? cL[9 * (f.j0 + 1) + a] : T(0);
    }
}
// w[r] -= sum over the entry's contributors c of L_rc w[c], in contributor order
template <typename T>
__device__ __forceinline__ void fwd_apply(const FwdEnt<T> &f, T *w, const int32_t *cl, const T *cL)
{
    if (f.n < 0) return;
    T s[3] = {0, 0, 0};
    if (f.n > 0) {
        T y[3];
        full_mv(f.L0, w + 3 * f.c0, y);
        s[0] += y[0]; s[1] += y[1]; s[2] += y[2];
    }
    if (f.n > 1) {
        T y[3];
        full_mv(f.L1, w + 3 * f.c1, y);
        s[0] += y[0]; s[1] += y[1]; s[2] += y[2];
    }
    for (int32_t j = f.j0 + 2; j < f.j0 + f.n; ++j) {
        T y[3];
        full_mv(cL + 9 * j, w + 3 * cl[j], y);
        s[0] += y[0]; s[1] += y[1]; s[2] += y[2];
    }
    w[3 * f.r] -= s[0]; w[3 * f.r + 1] -= s[1]; w[3 * f.r + 2] -= s[2];
}

// One backward vertex held in registers: D^-1 and its (at most two)
// receivers with their L blocks.
template <typename T>
struct BwdVtx {
    int32_t i, n, r0, r1;
    T D[6], L0[9], L1[9];
};
template <typename T>
__device__ __forceinline__ void bwd_fetch(BwdVtx<T> &v, int32_t i, int32_t i1, const int32_t *pr, int32_t nv,
                                          int32_t np, const int32_t *pref, const T *D, const T *pL)
{
    if (i >= i1) {
        v.n = -1;
        return;
    }
    v.i = i;
    const int32_t p0 = pr[i];
    v.n = (i + 1 < nv ? pr[i + 1] : np) - p0;
    v.r0 = v.n > 0 ? pref[p0] : 0;
    v.r1 = v.n > 1 ? pref[p0 + 1] : 0;
#pragma unroll
    for (int a = 0; a < 6; ++a) v.D[a] = D[6 * i + a];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        v.L0[a] = v.n > 0 ? pL[9 * p0 + a] : T(0);
        v.L1[a] = v.n > 1 ? pL[9 * (p0 + 1) + a] : T(0);
    }
}
// z_i = D_i^-1 z_i - sum over receivers q of L_qi^T z_q; a receiver ref >= 0
// is a local index, -1 - k the k-th gathered top value
template <typename T>
__device__ __forceinline__ void bwd_apply(const BwdVtx<T> &v, T *z, const T *zt)
{
    if (v.n < 0) return;
    T x[3] = {z[3 * v.i], z[3 * v.i + 1], z[3 * v.i + 2]}, zz[3];
    sym_mv(v.D, x, zz);
    if (v.n > 0) {
        const T *y = v.r0 >= 0 ? z + 3 * v.r0 : zt + 3 * (-1 - v.r0);
        T u[3];
        full_mtv(v.L0, y, u);
        zz[0] -= u[0]; zz[1] -= u[1]; zz[2] -= u[2];
    }
    if (v.n > 1) {
        const T *y = v.r1 >= 0 ? z + 3 * v.r1 : zt + 3 * (-1 - v.r1);
        T u[3];
        full_mtv(v.L1, y, u);
        zz[0] -= u[0]; zz[1] -= u[1]; zz[2] -= u[2];
    }
    z[3 * v.i] = zz[0]; z[3 * v.i + 1] = zz[1]; z[3 * v.i + 2] = zz[2];
}

// The forward levels of a bin (or of the top: only its entries with top
// contributors).  A level with more than 32 entries is shared by the warps
// that have entries in it (the others only meet the block barrier); from
// the first level after which no level has more than 32 entries, warp 0
// runs the rest alone with warp barriers.  *sw is shared scratch.
template <typename T, int NT>
__device__ __forceinline__ void fwd_levels(const int32_t *lvl, int nlev, const int32_t *er, const int32_t *ec,
                                           int32_t ne, int32_t nc, const int32_t *cl, const T *cL, T *w, int split,
                                           const FwdEnt<T> &first, const T *cLt, uint64_t *bart, bool *ok)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // each thread's first entry of the next level is fetched while the
    // current level computes
    FwdEnt<T> cur = first, nxt;
    for (int lv = 0; lv < split; ++lv) {
        const int32_t e0 = lvl[lv], e1 = lvl[lv + 1];
        if (lv + 1 < nlev) fwd_fetch(nxt, lvl[lv + 1] + (int32_t)threadIdx.x, lvl[lv + 2], er, ec, ne, nc, cl, cL);
        else nxt.n = -1;
        if (warp * 32 < e1 - e0) {
            fwd_apply(cur, w, cl, cL);
            for (int32_t e = e0 + threadIdx.x + NT; e < e1; e += NT) {
                FwdEnt<T> f;
                fwd_fetch(f, e, e1, er, ec, ne, nc, cl, cL);
                fwd_apply(f, w, cl, cL);
            }
        }
        __syncthreads();
        cur = nxt;
    }
    // the tail levels (at most 32 entries each) run in warp 0 with their L
    // blocks staged in shared memory (cLt: the same indexing as cL)
    if (warp == 0 && split < nlev) {
        const bool good = __all_sync(0xffffffffu, mbar_wait(bart));
        if (lane == 0) *ok = good;
        if (good) {
            for (int lv = split; lv < nlev; ++lv) {
                const int32_t e0 = lvl[lv], e1 = lvl[lv + 1];
                for (int32_t e = e0 + lane; e < e1; e += 32) {
                    FwdEnt<T> f;
                    fwd_fetch(f, e, e1, er, ec, ne, nc, cl, cLt);
                    fwd_apply(f, w, cl, cLt);
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
}

// The backward levels of a bin, from the last level down: warp 0 alone
// while the levels have at most 32 vertices, then the warps with vertices
// in the level, block barriers between levels.
template <typename T, int NT>
__device__ __forceinline__ void bwd_levels(const int32_t *lvl, int nlev, const int32_t *pr, int32_t nv, int32_t np,
                                           const int32_t *pref, const T *D, const T *pL, T *z, const T *zt, int split,
                                           const T *Dt, const T *pLt, uint64_t *bart, bool *ok, const BwdVtx<T> &first)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the levels above `split` (at most 32 vertices each) run in warp 0
    // with their D^-1 and L blocks staged in shared memory (Dt, pLt: the
    // same indexing as D, pL)
    if (warp == 0 && split < nlev - 1) {
        const bool good = __all_sync(0xffffffffu, mbar_wait(bart));
        if (lane == 0) *ok = good;
        if (good) {
            for (int lv = nlev - 1; lv > split; --lv) {
                const int32_t i0 = lvl[lv], i1 = lvl[lv + 1];
                for (int32_t i = i0 + lane; i < i1; i += 32) {
                    BwdVtx<T> v;
                    bwd_fetch(v, i, i1, pr, nv, np, pref, Dt, pLt);
                    bwd_apply(v, z, zt);
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    const int start = split;
    BwdVtx<T> cur = first, nxt;
    for (int lv = start; lv >= 0; --lv) {
        const int32_t i0 = lvl[lv], i1 = lvl[lv + 1];
        if (lv > 0) bwd_fetch(nxt, lvl[lv - 1] + (int32_t)threadIdx.x, lvl[lv], pr, nv, np, pref, D, pL);
        else nxt.n = -1;
        if (warp * 32 < i1 - i0) {
            bwd_apply(cur, z, zt);
            for (int32_t i = i0 + threadIdx.x + NT; i < i1; i += NT) {
                BwdVtx<T> v;
                bwd_fetch(v, i, i1, pr, nv, np, pref, D, pL);
                bwd_apply(v, z, zt);
            }
        }
        __syncthreads();
        cur = nxt;
    }
}

// Sum of each top vertex's leaks: one warp per vertex, a fixed shuffle tree.
template <typename T, int FUSE>
__global__ void __launch_bounds__(256) k_leaksum(const int32_t *__restrict__ tlk, int32_t nt,
                                                 const T *__restrict__ ly, T *lsum, const Scal *sc, const int *done)
{
    pdl_trigger();
    pdl_wait();
    if (FUSE ? sc->done != 0 : (done && *done)) return;
    const int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= nt) return;
    const int32_t k0 = tlk[i], k1 = tlk[i + 1];
    T s[3] = {0, 0, 0};
    for (int32_t k = k0 + lane; k < k1; k += 32) {
        s[0] += ly[3 * (size_t)k]; s[1] += ly[3 * (size_t)k + 1]; s[2] += ly[3 * (size_t)k + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s[0] += __shfl_xor_sync(0xffffffffu, s[0], o);
        s[1] += __shfl_xor_sync(0xffffffffu, s[1], o);
        s[2] += __shfl_xor_sync(0xffffffffu, s[2], o);
    }
    if (lane == 0) {
        lsum[3 * (size_t)i] = s[0]; lsum[3 * (size_t)i + 1] = s[1]; lsum[3 * (size_t)i + 2] = s[2];
    }
}

// Forward levels of one bin.  FUSE: w is r (r -= alpha q is applied and
// stored, |r|^2 of the bin goes to part[b]); otherwise w is the right-hand
// side.  The forward values go to z (which may alias w).
template <typename T, int FUSE>
__global__ void __launch_bounds__(BA, 7) k_bin_fwd(BinArgs a, BinNum<T> nm, T *w, const T *__restrict__ q, T *z,
                                                double *part, Scal *sc, const int *done)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint64_t bar, bart;
    __shared__ double shd[BA / 32];
    const int b = a.order[blockIdx.x];
    const int32_t *h = a.hdr + (size_t)H_N * b;
    const int32_t voff = h[H_VOFF], nv = h[H_NV], eoff = h[H_EOFF], ne = h[H_NE], coff = h[H_COFF],
                  nc = h[H_NC], koff = h[H_KOFF], nk = h[H_NK], nlev = h[H_NLEV];
    const int32_t nvp = pad4(nv), nep = pad4(ne), ncp = pad4(nc), nkp = pad4(nk);
    T *w_s = reinterpret_cast<T *>(sm);
    int32_t *elev_s = reinterpret_cast<int32_t *>(w_s + 3 * nvp);
    int32_t *er_s = elev_s + a.LVP, *ec_s = er_s + nep, *cl_s = ec_s + nep, *kl_s = cl_s + ncp, *ks_s = kl_s + nkp;
    const T *cLg = nm.cL + (size_t)9 * coff;   // the bin's L blocks stay in global memory
    const size_t base_bytes = sizeof(T) * 3 * (size_t)nvp + 4 * ((size_t)a.LVP + 2 * nep + ncp + 2 * nkp);
    if (base_bytes > dyn_smem()) {
        if (threadIdx.x == 0) {
            atomicOr(a.err, 2);
            if (FUSE) {
                sc->status = SGP_ERR_TIMEOUT;
                sc->done = 1;
            }
        }
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        mbar_init(&bart);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Stage<6> st;
        st.d[0] = elev_s; st.s[0] = a.elev + (size_t)b * a.LVP; st.b[0] = 4u * a.LVP;
        st.d[1] = er_s; st.s[1] = a.er + eoff; st.b[1] = 4u * nep;
        st.d[2] = ec_s; st.s[2] = a.ec + eoff; st.b[2] = 4u * nep;
        st.d[3] = cl_s; st.s[3] = a.cl + coff; st.b[3] = 4u * ncp;
        st.d[4] = kl_s; st.s[4] = a.kl + koff; st.b[4] = 4u * nkp;
        st.d[5] = ks_s; st.s[5] = a.ks + koff; st.b[5] = 4u * nkp;
        st.issue(&bar);
    }
    pdl_trigger();
    if (!staged<FUSE>(&bar, a.err, sc)) return;
    // tail levels: from the first level after which no level has more than
    // 32 entries; their contributors form a suffix of the bin's L blocks,
    // staged from a 16-byte aligned start
    int split = nlev;
    while (split > 0 && elev_s[split] - elev_s[split - 1] <= 32) --split;
    // (the last levels may have no entries: then nothing is staged)
    const int32_t jt = (split < nlev && elev_s[split] < ne) ? (ec_s[elev_s[split]] & ~3) : ncp;
    T *cLt_s = reinterpret_cast<T *>(ks_s + nkp) - (size_t)9 * jt;   // indexed like cLg
    const bool fits = base_bytes + sizeof(T) * 9 * (size_t)(ncp - jt) <= dyn_smem() && jt >= 0 && jt <= ncp;
    if (threadIdx.x == 0) {
        Stage<1> st;
        st.d[0] = cLt_s + (size_t)9 * jt; st.s[0] = cLg + (size_t)9 * jt;
        st.b[0] = fits ? (uint32_t)sizeof(T) * 9u * (uint32_t)(ncp - jt) : 0u;
        st.issue(&bart);
        if (!fits) {
            atomicOr(a.err, 2);
            if (FUSE) {
                sc->status = SGP_ERR_TIMEOUT;
                sc->done = 1;
            }
        }
    }
    if (!fits) return;
    // level 0's entries and their L blocks do not depend on the previous
    // kernel: fetched before waiting for it
    FwdEnt<T> first;
    first.n = -1;
    if (nlev > 0) fwd_fetch(first, elev_s[0] + (int32_t)threadIdx.x, elev_s[1], er_s, ec_s, ne, nc, cl_s, cLg);
    pdl_wait();
    if (FUSE ? sc->done != 0 : (done && *done)) {
        if (!__syncthreads_and(mbar_wait(&bart)) && threadIdx.x == 0) atomicOr(a.err, 1);
        return;
    }
    // the bin's slice of r (and q) with 16-byte loads, r -= alpha q stored
    constexpr int K = Pack<T>::K;
    const int32_t npk = 3 * nvp / K;
    double rr = 0.0;
    {
        Pack<T> *wg = reinterpret_cast<Pack<T> *>(w + 3 * (size_t)voff);
        const Pack<T> *qg = reinterpret_cast<const Pack<T> *>(q + 3 * (size_t)voff);
        Pack<T> *ws = reinterpret_cast<Pack<T> *>(w_s);
        const T al = FUSE ? (T)sc->alpha : T(0);
        for (int32_t i = threadIdx.x; i < npk; i += BA) {
            Pack<T> x = wg[i];
            if (FUSE) {
                const Pack<T> y = qg[i];
#pragma unroll
                for (int e = 0; e < K; ++e) {
                    x.v[e] = fma(-al, y.v[e], x.v[e]);
                    rr = fma((double)x.v[e], (double)x.v[e], rr);
                }
                wg[i] = x;
            }
            ws[i] = x;
        }
    }
    __syncthreads();
    __shared__ bool ok_s;
    ok_s = true;
    __syncthreads();
    fwd_levels<T, BA>(elev_s, nlev, er_s, ec_s, ne, nc, cl_s, cLg, w_s, split, first, cLt_s, &bart, &ok_s);
    if (!ok_s) {
        if (threadIdx.x == 0) {
            atomicOr(a.err, 1);
            if (FUSE) { sc->status = SGP_ERR_TIMEOUT; sc->done = 1; }
        }
        return;
    }
    const T *kLg = nm.kL + (size_t)9 * koff;
    for (int32_t k = threadIdx.x; k < nk; k += BA) {
        T y[3];
        full_mv(kLg + 9 * k, w_s + 3 * kl_s[k], y);
        T *o = nm.ly + 3 * (size_t)ks_s[k];
        o[0] = y[0]; o[1] = y[1]; o[2] = y[2];
    }
    Pack<T> *zg = reinterpret_cast<Pack<T> *>(z + 3 * (size_t)voff);
    const Pack<T> *ws = reinterpret_cast<const Pack<T> *>(w_s);
    for (int32_t i = threadIdx.x; i < npk; i += BA) zg[i] = ws[i];
    if (FUSE) {
        double s = block_sum<BA>(rr, shd);
        if (threadIdx.x == 0) part[b] = s;
    }
}

// The top: leaks, forward levels, diagonal, backward levels, in one block.
// FUSE: r -= alpha q on the top's entries, |r|^2 finished over the bins'
// partials, the iteration counted and the stopping decision taken; r^T z of
// the top to part[nb + 1 + nb].
template <typename T, int FUSE, int DST>
__global__ void __launch_bounds__(BT) k_top(TopArgs a, const T *__restrict__ tL, const T *__restrict__ tD,
                                            const T *__restrict__ lsum, T *w, const T *__restrict__ q, T *z,
                                            int32_t nb, double *part, Scal *sc, const int *done)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint64_t bar;
    __shared__ double shd[BT / 32];
    __shared__ int stop_s;
    const int32_t nt = a.nt, ntp4 = pad4(nt), nttp = pad4(a.ntt);
    T *w_s = reinterpret_cast<T *>(sm);
    int32_t *ti = reinterpret_cast<int32_t *>(w_s + 3 * ntp4);
    T *L_s = reinterpret_cast<T *>(ti + a.tints), *D_s = L_s + 9 * nttp;
    const int32_t *telev = ti + a.o_telev, *ter = ti + a.o_ter, *tcp = ti + a.o_tcp, *tcc = ti + a.o_tcc,
                  *tvlev = ti + a.o_tvlev, *tpp = ti + a.o_tpp, *tpq = ti + a.o_tpq, *tpL = ti + a.o_tpL;
    if (sizeof(T) * (3 * (size_t)ntp4 + 9 * (size_t)nttp + (DST ? 6 * (size_t)ntp4 : 0)) + 4 * (size_t)a.tints >
        dyn_smem()) {
        if (threadIdx.x == 0) {
            atomicOr(a.err, 2);
            if (FUSE) {
                sc->status = SGP_ERR_TIMEOUT;
                sc->done = 1;
            }
        }
        return;
    }
    if (threadIdx.x == 0) mbar_init(&bar);
    __syncthreads();
    if (threadIdx.x == 0) {
        Stage<3> st;
        st.d[0] = ti; st.s[0] = a.tint; st.b[0] = 4u * a.tints;
        st.d[1] = L_s; st.s[1] = tL; st.b[1] = (uint32_t)sizeof(T) * 9u * nttp;
        st.d[2] = D_s; st.s[2] = tD; st.b[2] = DST ? (uint32_t)sizeof(T) * 6u * ntp4 : 0u;
        st.issue(&bar);
    }
    pdl_trigger();
    pdl_wait();
    const bool stop = FUSE ? sc->done != 0 : (done && *done);
    if (!staged<FUSE>(&bar, a.err, sc) || stop) return;
    const T al = FUSE ? (T)sc->alpha : T(0);
    T *wt = w + 3 * (size_t)a.G;
    const T *qt = q + 3 * (size_t)a.G;
    // the bins' |r|^2 partials: sixteen loads in flight per thread
    double acc = 0.0;
    if (FUSE) {
        for (int32_t k0 = threadIdx.x; k0 < nb; k0 += 16 * BT) {
            double v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = k0 + u * BT < nb ? __ldcg(part + k0 + u * BT) : 0.0;
#pragma unroll
            for (int u = 0; u < 16; ++u) acc += v[u];
        }
    }
    // r -= alpha q on the top's entries, minus the sum of each vertex's
    // leaks; four vertices per thread with all their loads in flight
    for (int32_t i0 = threadIdx.x; i0 < nt; i0 += 4 * BT) {
        T x[4][3], y[4][3], l[4][3];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int32_t i = i0 + u * BT;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                x[u][c] = i < nt ? wt[3 * i + c] : T(0);
                y[u][c] = (FUSE && i < nt) ? qt[3 * i + c] : T(0);
                l[u][c] = i < nt ? lsum[3 * (size_t)i + c] : T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int32_t i = i0 + u * BT;
            if (i >= nt) continue;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T v = x[u][c];
                if (FUSE) {
                    v = fma(-al, y[u][c], v);
                    wt[3 * i + c] = v;
                    acc = fma((double)v, (double)v, acc);
                }
                w_s[3 * i + c] = v - l[u][c];
            }
        }
    }
    if (FUSE) {
        const double tot = block_sum<BT>(acc, shd);
        if (threadIdx.x == 0) {
            sc->rr = tot;
            sc->it += 1;
            int st = 0;
            if (tot <= sc->stop2) {
                st = 1;
            } else if (sc->it >= sc->maxit) {
                st = 1;
                sc->status = SGP_ERR_NO_CONVERGENCE;
            }
            if (st) sc->done = 1;
            stop_s = st;
        }
    }
    __syncthreads();
    if (FUSE && stop_s) return;
    // forward levels of the top (only the entries with top contributors);
    // empty levels are skipped, warps without entries only meet the
    // barrier; from the first level after which no level has more than 32
    // entries, warp 0 runs the rest alone with warp barriers
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nlv = a.LVP - 1;
    int fsplit = nlv;
    while (fsplit > 0 && telev[fsplit] - telev[fsplit - 1] <= 32) --fsplit;
    for (int lv = 0; lv < fsplit; ++lv) {
        const int32_t e0 = telev[lv], e1 = telev[lv + 1];
        if (e0 == e1) continue;
        if (warp * 32 < e1 - e0)
            for (int32_t e = e0 + threadIdx.x; e < e1; e += BT) {
                FwdEnt<T> f;
                fwd_fetch(f, e, e1, ter, tcp, a.nte, a.ntt, tcc, L_s);
                fwd_apply(f, w_s, tcc, L_s);
            }
        __syncthreads();
    }
    if (warp == 0) {
        for (int lv = fsplit; lv < nlv; ++lv) {
            const int32_t e0 = telev[lv], e1 = telev[lv + 1];
            if (e0 == e1) continue;
            if (lane < e1 - e0) {
                FwdEnt<T> f;
                fwd_fetch(f, e0 + lane, e1, ter, tcp, a.nte, a.ntt, tcc, L_s);
                fwd_apply(f, w_s, tcc, L_s);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // diagonal and backward levels: warp 0 alone while the levels have at
    // most 32 vertices, then the warps with vertices in the level
    auto bwd_vertex = [&](int32_t i) {
        T x[3] = {w_s[3 * i], w_s[3 * i + 1], w_s[3 * i + 2]}, zz[3];
        sym_mv((DST ? (const T *)D_s : tD) + 6 * i, x, zz);
        for (int32_t p = tpp[i]; p < tpp[i + 1]; ++p) {
            T u[3];
            full_mtv(L_s + 9 * tpL[p], w_s + 3 * tpq[p], u);
            zz[0] -= u[0]; zz[1] -= u[1]; zz[2] -= u[2];
        }
        w_s[3 * i] = zz[0]; w_s[3 * i + 1] = zz[1]; w_s[3 * i + 2] = zz[2];
    };
    int bsplit = nlv - 1;
    while (bsplit >= 0 && tvlev[bsplit + 1] - tvlev[bsplit] <= 32) --bsplit;
    if (warp == 0) {
        for (int lv = nlv - 1; lv > bsplit; --lv) {
            const int32_t i0 = tvlev[lv], i1 = tvlev[lv + 1];
            if (i0 == i1) continue;
            if (lane < i1 - i0) bwd_vertex(i0 + lane);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int lv = bsplit; lv >= 0; --lv) {
        const int32_t i0 = tvlev[lv], i1 = tvlev[lv + 1];
        if (i0 == i1) continue;
        if (warp * 32 < i1 - i0)
            for (int32_t i = i0 + threadIdx.x; i < i1; i += BT) bwd_vertex(i);
        __syncthreads();
    }
    T *zt = z + 3 * (size_t)a.G;
    double rz = 0.0;
    for (int32_t i = threadIdx.x; i < 3 * nt; i += BT) {
        const T v = w_s[i];
        zt[i] = v;
        if (FUSE) rz = fma((double)wt[i], (double)v, rz);
    }
    if (FUSE) {
        double s = block_sum<BT>(rz, shd);
        if (threadIdx.x == 0) part[nb + 1 + nb] = s;
    }
}

// Diagonal solve and backward levels of one bin: z holds the forward values
// on entry and the solution on exit.  FUSE: r^T z of the bin to
// part[nb + 1 + b]; the last block sums them with the top's and sets beta.
template <typename T, int FUSE>
__global__ void __launch_bounds__(BA, 7) k_bin_bwd(BinArgs a, BinNum<T> nm, T *z, const T *__restrict__ r,
                                                double *part, Scal *sc, const int *done)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint64_t bar, bart;
    __shared__ double shd[BA / 32];
    __shared__ bool ok_s;
    const int b = a.order[blockIdx.x];
    const int32_t *h = a.hdr + (size_t)H_N * b;
    const int32_t voff = h[H_VOFF], nv = h[H_NV], poff = h[H_POFF], np = h[H_NP], zoff = h[H_ZOFF],
                  nz = h[H_NZ], nlev = h[H_NLEV];
    const int32_t nvp = pad4(nv), npp = pad4(np), nzp = pad4(nz);
    T *z_s = reinterpret_cast<T *>(sm);
    T *zt_s = z_s + 3 * nvp;
    int32_t *vlev_s = reinterpret_cast<int32_t *>(zt_s + 3 * nzp);
    int32_t *pr_s = vlev_s + a.LVP, *pref_s = pr_s + nvp, *zi_s = pref_s + npp;
    const T *Dg = nm.D + (size_t)6 * voff, *pLg = nm.pL + (size_t)9 * poff;   // stay in global memory
    const size_t base_bytes = sizeof(T) * 3 * ((size_t)nvp + nzp) + 4 * ((size_t)a.LVP + nvp + npp + nzp);
    if (base_bytes > dyn_smem()) {
        if (threadIdx.x == 0) {
            atomicOr(a.err, 2);
            if (FUSE) {
                sc->status = SGP_ERR_TIMEOUT;
                sc->done = 1;
            }
        }
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        mbar_init(&bart);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Stage<4> st;
        st.d[0] = vlev_s; st.s[0] = a.vlev + (size_t)b * a.LVP; st.b[0] = 4u * a.LVP;
        st.d[1] = pr_s; st.s[1] = a.pr + voff; st.b[1] = 4u * nvp;
        st.d[2] = pref_s; st.s[2] = a.pref + poff; st.b[2] = 4u * npp;
        st.d[3] = zi_s; st.s[3] = a.zi + zoff; st.b[3] = 4u * nzp;
        st.issue(&bar);
    }
    pdl_trigger();
    if (!staged<FUSE>(&bar, a.err, sc)) return;
    // the levels above `split` have at most 32 vertices each: their vertices
    // are a suffix of the bin, whose D^-1 and L blocks are staged (from
    // 16-byte aligned starts)
    int split = nlev - 1;
    while (split >= 0 && vlev_s[split + 1] - vlev_s[split] <= 32) --split;
    const int32_t vs = split < nlev - 1 ? vlev_s[split + 1] : nv;
    const int32_t it = vs < nv ? (vs & ~3) : nvp;
    const int32_t pt = vs < nv ? (pr_s[vs] & ~3) : npp;
    T *Dt_s = reinterpret_cast<T *>(zi_s + nzp) - (size_t)6 * it;
    T *pLt_s = Dt_s + (size_t)6 * nvp - (size_t)9 * pt;
    const bool fits = it >= 0 && it <= nvp && pt >= 0 && pt <= npp &&
                      base_bytes + sizeof(T) * (6 * (size_t)(nvp - it) + 9 * (size_t)(npp - pt)) <= dyn_smem();
    if (threadIdx.x == 0) {
        Stage<2> st;
        st.d[0] = Dt_s + (size_t)6 * it; st.s[0] = Dg + (size_t)6 * it;
        st.b[0] = fits ? (uint32_t)sizeof(T) * 6u * (uint32_t)(nvp - it) : 0u;
        st.d[1] = pLt_s + (size_t)9 * pt; st.s[1] = pLg + (size_t)9 * pt;
        st.b[1] = fits ? (uint32_t)sizeof(T) * 9u * (uint32_t)(npp - pt) : 0u;
        st.issue(&bart);
        if (!fits) {
            atomicOr(a.err, 2);
            if (FUSE) {
                sc->status = SGP_ERR_TIMEOUT;
                sc->done = 1;
            }
        }
    }
    if (!fits) return;
    // the first level of the block phase (`split`) does not depend on the
    // previous kernel: its vertices, D^-1 and L blocks are fetched before
    // waiting for it
    BwdVtx<T> first;
    first.n = -1;
    if (split >= 0) bwd_fetch(first, vlev_s[split] + (int32_t)threadIdx.x, vlev_s[split + 1], pr_s, nv, np, pref_s, Dg, pLg);
    pdl_wait();
    if (FUSE ? sc->done != 0 : (done && *done)) {
        if (!__syncthreads_and(mbar_wait(&bart)) && threadIdx.x == 0) atomicOr(a.err, 1);
        return;
    }
    constexpr int K = Pack<T>::K;
    const int32_t npk = 3 * nvp / K;
    {
        const Pack<T> *zg = reinterpret_cast<const Pack<T> *>(z + 3 * (size_t)voff);
        Pack<T> *zs = reinterpret_cast<Pack<T> *>(z_s);
        for (int32_t i = threadIdx.x; i < npk; i += BA) zs[i] = zg[i];
    }
    const T *ztop = z + 3 * (size_t)a.G;
    for (int32_t k = threadIdx.x; k < nz; k += BA) {
        const T *t = ztop + 3 * (size_t)zi_s[k];
        zt_s[3 * k] = t[0]; zt_s[3 * k + 1] = t[1]; zt_s[3 * k + 2] = t[2];
    }
    __syncthreads();
    ok_s = true;
    __syncthreads();
    bwd_levels<T, BA>(vlev_s, nlev, pr_s, nv, np, pref_s, Dg, pLg, z_s, zt_s, split, Dt_s, pLt_s, &bart, &ok_s, first);
    if (!ok_s) {
        if (threadIdx.x == 0) {
            atomicOr(a.err, 1);
            if (FUSE) { sc->status = SGP_ERR_TIMEOUT; sc->done = 1; }
        }
        return;
    }
    Pack<T> *zo = reinterpret_cast<Pack<T> *>(z + 3 * (size_t)voff);
    const Pack<T> *rg = reinterpret_cast<const Pack<T> *>(r + 3 * (size_t)voff);
    const Pack<T> *zs = reinterpret_cast<const Pack<T> *>(z_s);
    double rz = 0.0;
    for (int32_t i = threadIdx.x; i < npk; i += BA) {
        const Pack<T> v = zs[i];
        zo[i] = v;
        if (FUSE) {
            const Pack<T> x = rg[i];
#pragma unroll
            for (int e = 0; e < K; ++e) rz = fma((double)x.v[e], (double)v.v[e], rz);
        }
    }
    if (FUSE) {
        double s = block_sum<BA>(rz, shd);
        if (threadIdx.x == 0) part[a.nb + 1 + b] = s;
        if (last_block(&sc->cnt)) {
            double t = 0.0;
            for (int32_t k = threadIdx.x; k <= a.nb; k += BA) t += __ldcg(part + a.nb + 1 + k);
            t = block_sum<BA>(t, shd);
            if (threadIdx.x == 0) rz_finish(sc, t);
        }
    }
}

// Vectors between the matrix's internal order and the tree order.
template <typename T>
__global__ void k_bn_to_tree(int32_t NT, const int32_t *__restrict__ i_of_t, const T *__restrict__ src, T *dst)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NT) return;
    const int32_t i = i_of_t[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[3 * (size_t)t + c] = i >= 0 ? src[3 * (size_t)i + c] : T(0);
}
template <typename T>
__global__ void k_bn_from_tree(int32_t n, const int32_t *__restrict__ t_of_i, const T *__restrict__ src, T *dst)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t t = t_of_i[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[3 * (size_t)i + c] = src[3 * (size_t)t + c];
}

// The matrix's rows in tree order (padding rows empty), columns mapped to
// tree order: FP32 eq. (1) records, or FP64 blocks and columns.
__global__ void k_bn_rowlen(int32_t NT, const int32_t *__restrict__ i_of_t, const int32_t *__restrict__ rp,
                            int32_t *len)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NT) return;
    const int32_t i = i_of_t[t];
    len[t] = i >= 0 ? rp[i + 1] - rp[i] : 0;
}
__global__ void k_bn_rows32(int32_t NT, const int32_t *__restrict__ i_of_t, const int32_t *__restrict__ t_of_i,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ rpt,
                            const float4 *__restrict__ a, const float2 *__restrict__ bb, float4 *at, float2 *bt)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NT) return;
    const int32_t i = i_of_t[t];
    if (i < 0) return;
    int32_t d = rpt[t];
    for (int32_t s = rp[i]; s < rp[i + 1]; ++s, ++d) {
        at[d] = a[s];
        const float2 y = bb[s];
        bt[d] = make_float2(y.x, __int_as_float(t_of_i[__float_as_int(y.y)]));
    }
}
__global__ void k_bn_rows64(int32_t NT, const int32_t *__restrict__ i_of_t, const int32_t *__restrict__ t_of_i,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ rpt,
                            const double *__restrict__ blk, const int32_t *__restrict__ col, double *bt, int32_t *ct)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NT) return;
    const int32_t i = i_of_t[t];
    if (i < 0) return;
    int32_t d = rpt[t];
    for (int32_t s = rp[i]; s < rp[i + 1]; ++s, ++d) {
#pragma unroll
        for (int k = 0; k < 6; ++k) bt[6 * (size_t)d + k] = blk[6 * (size_t)s + k];
        ct[d] = t_of_i[col[s]];
    }
}
__global__ void k_bn_tree_maps(int32_t G, int32_t nt, const int32_t *__restrict__ gvert,
                               const int32_t *__restrict__ tv, int32_t *i_of_t, int32_t *t_of_i)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < G) {
        const int32_t v = gvert[t];
        i_of_t[t] = v;
        if (v >= 0) t_of_i[v] = t;
    } else if (t < G + pad4(nt)) {
        const int32_t k = t - G;
        const int32_t v = k < nt ? tv[k] : -1;
        i_of_t[t] = v;
        if (v >= 0) t_of_i[v] = t;
    }
}

template <typename T>
static int pidx() { return sizeof(T) == 4 ? 0 : 1; }

static sgp_status smem_optin(sgp_ctx *ctx)
{
    static int done_dev[64] = {0};
    if (ctx->device >= 0 && ctx->device < 64 && done_dev[ctx->device]) return SGP_OK;
    const int by = SMEM_MAX;
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_bin_fwd<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_bin_fwd<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_bin_fwd<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_bin_fwd<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_top<float, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_top<float, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_top<double, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_top<double, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_top<float, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_top<float, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_top<double, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_top<double, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_bin_bwd<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_bin_bwd<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_bin_bwd<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    SGP_CUDA(ctx, cudaFuncSetAttribute(k_bin_bwd<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, by));
    if (ctx->device >= 0 && ctx->device < 64) done_dev[ctx->device] = 1;
    return SGP_OK;
}

template <typename T>
static BinArgs bin_args(const sgp_factor *F)
{
    const BinLayout &B = F->bl;
    return BinArgs{bp<const int32_t>(B.hdr), bp<const int32_t>(B.order), bp<const int32_t>(B.elev),
                   bp<const int32_t>(B.vlev),
                   bp<const int32_t>(B.er), bp<const int32_t>(B.ec), bp<const int32_t>(B.cl),
                   bp<const int32_t>(B.kl), bp<const int32_t>(B.ks), bp<const int32_t>(B.pr),
                   bp<const int32_t>(B.pref), bp<const int32_t>(B.zi), B.LVP, B.nb, B.G, bp<int>(B.err)};
}
template <typename T>
static BinNum<T> bin_num(const sgp_factor *F)
{
    const BinLayout &B = F->bl;
    const int k = pidx<T>();
    return BinNum<T>{bp<const T>(B.cL[k]), bp<const T>(B.kL[k]), bp<const T>(B.pL[k]), bp<const T>(B.D[k]),
                     bp<T>(B.ly[k])};
}
static TopArgs top_args(const sgp_factor *F)
{
    const BinLayout &B = F->bl;
    TopArgs t{bp<const int32_t>(B.tint), B.nt, B.LVP, B.nte, B.ntt, B.ntp, B.tints, B.nly, B.G,
              B.toff[0], B.toff[1], B.toff[2], B.toff[3], B.toff[4], B.toff[5], B.toff[6], B.toff[7], B.toff[8],
              bp<int>(B.err)};
    return t;
}

// The three launches on tree-order vectors: w (FUSE: r) in, z out (may alias
// w unless FUSE).
template <typename T, int FUSE>
static sgp_status launch3(sgp_ctx *ctx, const sgp_factor *F, T *w, const T *q, T *z, Scal *sc, const int *done)
{
    const BinLayout &B = F->bl;
    const int k = pidx<T>();
    SGP_TRY(smem_optin(ctx));
    const BinArgs a = bin_args<T>(F);
    const BinNum<T> nm = bin_num<T>(F);
    const TopArgs ta = top_args(F);
    double *part = bp<double>(B.part);
    const size_t smA = FUSE ? B.smA[k] : B.smA0[k], smC = FUSE ? B.smC[k] : B.smC0[k];
    LAUNCH_PDL(ctx, (k_bin_fwd<T, FUSE>), B.nb, BA, smA, a, nm, w, q, z, part, sc, done);
    T *lsum = bp<T>(B.lsum[k]);
    if (B.nt > 0)
        LAUNCH_PDL(ctx, (k_leaksum<T, FUSE>), grid_for(32 * (int64_t)B.nt, 256), 256, 0,
                   bp<const int32_t>(B.tint) + B.toff[8], B.nt, (const T *)nm.ly, lsum, (const Scal *)sc, done);
    if (B.smT[k] <= (size_t)SMEM_MAX)
        LAUNCH_PDL(ctx, (k_top<T, FUSE, 1>), 1, BT, B.smT[k], ta, bp<const T>(B.tL[k]), bp<const T>(B.tD[k]),
                   (const T *)lsum, w, q, z, B.nb, part, sc, done);
    else
        LAUNCH_PDL(ctx, (k_top<T, FUSE, 0>), 1, BT, B.smTnd[k], ta, bp<const T>(B.tL[k]), bp<const T>(B.tD[k]),
                   (const T *)lsum, w, q, z, B.nb, part, sc, done);
    LAUNCH_PDL(ctx, (k_bin_bwd<T, FUSE>), B.nb, BA, smC, a, nm, z, (const T *)w, part, sc, done);
    return SGP_OK;
}

// ---------------------------------------------------------- host: building
struct Scr {
    sgp_ctx *ctx;
    BinLayout *B;
    int nbuf = 0;
    int32_t *take(size_t count)
    {
        DBuf &b = B->scr[nbuf++];
        if (buf_ensure(ctx, b, sizeof(int32_t) * std::max<size_t>(count, 4)) != SGP_OK) return nullptr;
        return bp<int32_t>(b);
    }
};

static sgp_status ensure_i32(sgp_ctx *ctx, DBuf &b, size_t count, int32_t **p)
{
    SGP_TRY(buf_ensure(ctx, b, sizeof(int32_t) * std::max<size_t>(count, 4)));
    *p = bp<int32_t>(b);
    return SGP_OK;
}

static sgp_status read_i32(sgp_ctx *ctx, const int32_t *dev, int32_t *host)
{
    return read_back(ctx, host, dev, sizeof(int32_t));
}

// Group items i (seg[i] >= 0) by segment, each group sorted by key; offsets
// padded to 4 when `pad`.  off: nseg + 1, cnt: nseg, out: sorted keys (-1 in
// padding), total: off[nseg].
static sgp_status group(sgp_ctx *ctx, Scr &S, int32_t n, const int32_t *seg, const int32_t *key, int32_t nseg,
                        int pad, int32_t *off, int32_t *cnt, DBuf &outbuf, int32_t **out, int32_t *total)
{
    SGP_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * std::max(nseg, 1), ctx->stream));
    LAUNCH(ctx, k_bn_count, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, seg, cnt);
    int32_t *tmp = S.take((size_t)nseg + 1);
    if (!tmp) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_pad, grid_for(nseg, SGP_BLOCK), SGP_BLOCK, 0, nseg, (const int32_t *)cnt, pad, tmp);
    SGP_TRY(scan_exclusive_i32(ctx, tmp, off, nseg));
    SGP_TRY(read_i32(ctx, off + nseg, total));
    int32_t *kt = S.take((size_t)*total + 4);
    int32_t *fill = S.take((size_t)nseg + 1);
    if (!kt || !fill) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(fill, 0, sizeof(int32_t) * std::max(nseg, 1), ctx->stream));
    LAUNCH(ctx, k_bn_place, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, seg, key, (const int32_t *)off, fill, kt);
    SGP_TRY(ensure_i32(ctx, outbuf, (size_t)*total + 4, out));
    SGP_CUDA(ctx, cudaMemsetAsync(*out, 0xff, sizeof(int32_t) * ((size_t)*total + 4), ctx->stream));
    if (nseg > 0)
        LAUNCH(ctx, k_bn_segsort, nseg, SGP_BLOCK, 0, (const int32_t *)off, (const int32_t *)cnt,
               (const int32_t *)kt, *out);
    return SGP_OK;
}

}  // namespace

// Build the binned layout of a factor whose structure and numerics are done.
// Leaves F->bl.ok32 / ok64 at 0 when a part does not fit in shared memory
// (the level kernels then serve that precision).
sgp_status bins_build(sgp_ctx *ctx, sgp_factor *F, const sgp_matrix *M)
{
    BinLayout &B = F->bl;
    B.ok32 = B.ok64 = 0;
    const int32_t n = (int32_t)F->n, LV = F->levels;
    // default (0): the FP32 solve of a MIXED factor only, at 1024 -- measured,
    // FP64 bins were slower than the level kernels on the 1e6 spheroid
    const int bmax = ctx->bin_cap == 0 ? 1024 : ctx->bin_cap;
    const bool f64_bins = ctx->bin_cap > 0;
    if (n == 0 || bmax <= 0 || LV == 0) return SGP_OK;
    if (!f64_bins && F->precision != SGP_PREC_MIXED) return SGP_OK;
    // default: a factor whose every level fits the one-block tail is solved
    // by that single launch (the three bin launches measured slower on the
    // 1000-cell cube)
    if (ctx->bin_cap == 0 && F->tail_level == 0) return SGP_OK;
    B.LV = LV;
    B.LVP = pad4(LV + 1);
    B.bmax = bmax;
    const int32_t E = F->rl_ptr[LV], NC = F->cl_ptr[LV];
    const int32_t *ord = bp<const int32_t>(F->ord), *pos = bp<const int32_t>(F->pos),
                  *pr_ptr = bp<const int32_t>(F->pr_ptr), *pr_q = bp<const int32_t>(F->pr_q),
                  *pr_c = bp<const int32_t>(F->pr_c), *rv = bp<const int32_t>(F->rv),
                  *rc_ptr = bp<const int32_t>(F->rc_ptr), *ct = bp<const int32_t>(F->ct);
    Scr S{ctx, &B};
    // level of every position and of every forward entry
    int32_t *lp = S.take(LV + 1), *rp = S.take(LV + 1);
    int32_t *levp = S.take(n), *levE = S.take(E);
    if (!lp || !rp || !levp || !levE) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemcpyAsync(lp, F->lvl_ptr.data(), sizeof(int32_t) * (LV + 1), cudaMemcpyHostToDevice,
                                  ctx->stream));
    SGP_CUDA(ctx, cudaMemcpyAsync(rp, F->rl_ptr.data(), sizeof(int32_t) * (LV + 1), cudaMemcpyHostToDevice,
                                  ctx->stream));
    LAUNCH(ctx, k_bn_level, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)lp, LV, n, levp);
    LAUNCH(ctx, k_bn_level, grid_for(E, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)rp, LV, E, levE);
    // contraction-tree parents and subtree sizes
    int32_t *par = S.take(n), *sz = S.take(n);
    if (!par || !sz) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_parent, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, pr_ptr, pr_q, pos, par, sz);
    for (int l = 0; l < LV; ++l) {
        const int32_t p0 = F->lvl_ptr[l], c = F->lvl_ptr[l + 1] - p0;
        if (c > 0) LAUNCH(ctx, k_bn_size, grid_for(c, SGP_BLOCK), SGP_BLOCK, 0, p0, c, (const int32_t *)par, sz);
    }
    // classes and the bins' roots in spatial order
    int32_t *top = S.take(n), *isroot = S.take(n), *rootv = S.take(n), *ridx = S.take((size_t)n + 1);
    if (!top || !isroot || !rootv || !ridx) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_class, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, bmax, (const int32_t *)sz,
           (const int32_t *)par, ord, top, isroot, rootv);
    SGP_TRY(scan_exclusive_i32(ctx, rootv, ridx, n));
    int32_t nr = 0;
    SGP_TRY(read_i32(ctx, ridx + n, &nr));
    const int32_t half = std::max(1, bmax / 2);
    int32_t *rpos = S.take(nr), *rsm = S.take((size_t)nr + 1), *rpre = S.take((size_t)nr + 1),
            *nbf = S.take((size_t)nr + 1), *bid = S.take((size_t)nr + 1);
    if (!rpos || !rsm || !rpre || !nbf || !bid) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_roots, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, (const int32_t *)rootv, (const int32_t *)ridx,
           pos, (const int32_t *)sz, half, rpos, rsm);
    SGP_TRY(scan_exclusive_i32(ctx, rsm, rpre, nr));
    LAUNCH(ctx, k_bn_newbin, grid_for(nr, SGP_BLOCK), SGP_BLOCK, 0, nr, (const int32_t *)rpre, (const int32_t *)rsm,
           half, nbf);
    SGP_TRY(scan_exclusive_i32(ctx, nbf, bid, nr));
    int32_t nb = 0;
    SGP_TRY(read_i32(ctx, bid + nr, &nb));
    B.nb = nb;
    int32_t *binroot = S.take(n), *anc = S.take(n), *anc2 = S.take(n);
    if (!binroot || !anc || !anc2) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_rootbin, grid_for(nr, SGP_BLOCK), SGP_BLOCK, 0, nr, (const int32_t *)rpos,
           (const int32_t *)bid, (const int32_t *)nbf, binroot);
    LAUNCH(ctx, k_bn_anc_init, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, (const int32_t *)top,
           (const int32_t *)isroot, (const int32_t *)par, anc);
    for (int r = 0; (1 << r) <= LV + 1; ++r) {
        LAUNCH(ctx, k_bn_jump, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, (const int32_t *)anc, anc2);
        std::swap(anc, anc2);
    }
    int32_t *binp = S.take(n);
    if (!binp) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_binp, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, (const int32_t *)top, (const int32_t *)anc,
           (const int32_t *)binroot, binp);
    // top indices (position order)
    int32_t *topidx = S.take((size_t)n + 1);
    if (!topidx) return SGP_ERR_OOM;
    SGP_TRY(scan_exclusive_i32(ctx, top, topidx, n));
    int32_t nt = 0;
    SGP_TRY(read_i32(ctx, topidx + n, &nt));
    B.nt = nt;

    // ---- bins: vertices
    int32_t *voff = S.take((size_t)nb + 1), *cntv = S.take((size_t)nb + 1), *gpos = nullptr, G = 0;
    if (!voff || !cntv) return SGP_ERR_OOM;
    SGP_TRY(group(ctx, S, n, binp, nullptr, nb, 1, voff, cntv, B.scr[S.nbuf++], &gpos, &G));
    B.G = G;
    int32_t *lpos = S.take(n), *gvert, *gbin = S.take((size_t)G + 4), *vlev, *pr, *zpre = S.take((size_t)G + 4),
            *hdr;
    if (!lpos || !gbin || !zpre) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(lpos, 0xff, sizeof(int32_t) * (size_t)n, ctx->stream));
    SGP_TRY(ensure_i32(ctx, B.gvert, (size_t)G + 4, &gvert));
    SGP_TRY(ensure_i32(ctx, B.vlev, (size_t)nb * B.LVP + 4, &vlev));
    SGP_TRY(ensure_i32(ctx, B.pr, (size_t)G + 4, &pr));
    SGP_TRY(ensure_i32(ctx, B.hdr, (size_t)H_N * nb + 4, &hdr));
    SGP_CUDA(ctx, cudaMemsetAsync(hdr, 0, sizeof(int32_t) * ((size_t)H_N * nb + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(gvert, 0xff, sizeof(int32_t) * ((size_t)G + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(pr, 0, sizeof(int32_t) * ((size_t)G + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(gbin, 0, sizeof(int32_t) * ((size_t)G + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(zpre, 0, sizeof(int32_t) * ((size_t)G + 4), ctx->stream));
    if (nb > 0)
        LAUNCH(ctx, k_bn_binvert, nb, BA, 0, (const int32_t *)voff, (const int32_t *)cntv, (const int32_t *)gpos, ord,
               (const int32_t *)levp, pr_ptr, pr_q, pos, (const int32_t *)top, B.LVP, lpos, gvert, gbin, vlev, pr,
               zpre, hdr);
    // ---- bins: forward entries and their contributors
    int32_t *segE = S.take(E), *eoff = S.take((size_t)nb + 1), *cnte = S.take((size_t)nb + 1), *gent = nullptr,
            EE = 0;
    if (!segE || !eoff || !cnte) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_seg_entry, grid_for(E, SGP_BLOCK), SGP_BLOCK, 0, E, rv, pos, (const int32_t *)binp, segE);
    SGP_TRY(group(ctx, S, E, segE, nullptr, nb, 1, eoff, cnte, B.scr[S.nbuf++], &gent, &EE));
    B.E = EE;
    int32_t *er, *ec, *elev, *ebin = S.take((size_t)EE + 4);
    if (!ebin) return SGP_ERR_OOM;
    SGP_TRY(ensure_i32(ctx, B.er, (size_t)EE + 4, &er));
    SGP_TRY(ensure_i32(ctx, B.ec, (size_t)EE + 4, &ec));
    SGP_TRY(ensure_i32(ctx, B.elev, (size_t)nb * B.LVP + 4, &elev));
    SGP_CUDA(ctx, cudaMemsetAsync(er, 0, sizeof(int32_t) * ((size_t)EE + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(ec, 0, sizeof(int32_t) * ((size_t)EE + 4), ctx->stream));
    if (nb > 0)
        LAUNCH(ctx, k_bn_binent, nb, BA, 0, (const int32_t *)eoff, (const int32_t *)cnte, (const int32_t *)gent, rv,
               rc_ptr, pos, (const int32_t *)lpos, (const int32_t *)levE, B.LVP, er, ec, ebin, elev, hdr);
    // padded offsets of the per-bin contributor, pair and top-reference arrays
    auto offsets = [&](int f_count, int f_off, int32_t *total) -> sgp_status {
        int32_t *c = S.take((size_t)nb + 1), *o = S.take((size_t)nb + 1);
        if (!c || !o) return SGP_ERR_OOM;
        LAUNCH(ctx, k_bn_hfield, grid_for(nb, SGP_BLOCK), SGP_BLOCK, 0, nb, (const int32_t *)hdr, f_count, c);
        SGP_TRY(scan_exclusive_i32(ctx, c, o, nb));
        SGP_TRY(read_i32(ctx, o + nb, total));
        LAUNCH(ctx, k_bn_hset, grid_for(nb, SGP_BLOCK), SGP_BLOCK, 0, nb, (const int32_t *)o, f_off, hdr);
        return SGP_OK;
    };
    int32_t Cc = 0, Pp = 0, Z = 0;
    SGP_TRY(offsets(H_NC, H_COFF, &Cc));
    SGP_TRY(offsets(H_NP, H_POFF, &Pp));
    SGP_TRY(offsets(H_NZ, H_ZOFF, &Z));
    B.Cc = Cc; B.Pp = Pp; B.Z = Z;
    int32_t *cl, *c_src, *pref, *p_src, *zi;
    SGP_TRY(ensure_i32(ctx, B.cl, (size_t)Cc + 4, &cl));
    SGP_TRY(ensure_i32(ctx, B.c_src, (size_t)Cc + 4, &c_src));
    SGP_TRY(ensure_i32(ctx, B.pref, (size_t)Pp + 4, &pref));
    SGP_TRY(ensure_i32(ctx, B.p_src, (size_t)Pp + 4, &p_src));
    SGP_TRY(ensure_i32(ctx, B.zi, (size_t)Z + 4, &zi));
    SGP_CUDA(ctx, cudaMemsetAsync(cl, 0, sizeof(int32_t) * ((size_t)Cc + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(c_src, 0xff, sizeof(int32_t) * ((size_t)Cc + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(pref, 0, sizeof(int32_t) * ((size_t)Pp + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(p_src, 0xff, sizeof(int32_t) * ((size_t)Pp + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(zi, 0, sizeof(int32_t) * ((size_t)Z + 4), ctx->stream));
    LAUNCH(ctx, k_bn_contrib, grid_for(EE, SGP_BLOCK), SGP_BLOCK, 0, EE, (const int32_t *)gent,
           (const int32_t *)ebin, (const int32_t *)ec, (const int32_t *)hdr, rc_ptr, ct, pr_c, pos,
           (const int32_t *)lpos, cl, c_src);
    LAUNCH(ctx, k_bn_pairs, grid_for(G, SGP_BLOCK), SGP_BLOCK, 0, G, (const int32_t *)gpos, (const int32_t *)gbin,
           (const int32_t *)pr, (const int32_t *)zpre, (const int32_t *)hdr, pr_ptr, pr_q, pos,
           (const int32_t *)top, (const int32_t *)topidx, (const int32_t *)lpos, pref, p_src, zi);
    // ---- leaks: slots grouped by top receiver, then by contributor bin
    int32_t *kofj = S.take(NC), *segL = S.take(NC), *lcnt = S.take((size_t)nt + 1), *lkj = nullptr, nly = 0;
    if (!kofj || !segL || !lcnt) return SGP_ERR_OOM;
    int32_t *tint_tlk = S.take((size_t)nt + 2);
    if (!tint_tlk) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_kofj, grid_for(E, SGP_BLOCK), SGP_BLOCK, 0, E, rc_ptr, kofj);
    LAUNCH(ctx, k_bn_seg_leak, grid_for(NC, SGP_BLOCK), SGP_BLOCK, 0, NC, (const int32_t *)kofj, rv, ct, pr_c, pos,
           (const int32_t *)top, (const int32_t *)topidx, segL);
    SGP_TRY(group(ctx, S, NC, segL, nullptr, nt, 0, tint_tlk, lcnt, B.scr[S.nbuf++], &lkj, &nly));
    B.nly = nly;
    int32_t *segK = S.take((size_t)nly + 1), *koff = S.take((size_t)nb + 1), *cntk = S.take((size_t)nb + 1),
            *kslot = nullptr, K = 0;
    if (!segK || !koff || !cntk) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_seg_leakbin, grid_for(nly, SGP_BLOCK), SGP_BLOCK, 0, nly, (const int32_t *)lkj, ct, pr_c, pos,
           (const int32_t *)binp, segK);
    SGP_TRY(group(ctx, S, nly, segK, nullptr, nb, 1, koff, cntk, B.scr[S.nbuf++], &kslot, &K));
    B.K = K;
    LAUNCH(ctx, k_bn_hset, grid_for(nb, SGP_BLOCK), SGP_BLOCK, 0, nb, (const int32_t *)koff, (int)H_KOFF, hdr);
    LAUNCH(ctx, k_bn_hset, grid_for(nb, SGP_BLOCK), SGP_BLOCK, 0, nb, (const int32_t *)cntk, (int)H_NK, hdr);
    int32_t *kl, *ks, *k_src;
    SGP_TRY(ensure_i32(ctx, B.kl, (size_t)K + 4, &kl));
    SGP_TRY(ensure_i32(ctx, B.ks, (size_t)K + 4, &ks));
    SGP_TRY(ensure_i32(ctx, B.k_src, (size_t)K + 4, &k_src));
    SGP_CUDA(ctx, cudaMemsetAsync(k_src, 0xff, sizeof(int32_t) * ((size_t)K + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(kl, 0, sizeof(int32_t) * ((size_t)K + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(ks, 0, sizeof(int32_t) * ((size_t)K + 4), ctx->stream));
    LAUNCH(ctx, k_bn_leakfill, grid_for(K, SGP_BLOCK), SGP_BLOCK, 0, K, (const int32_t *)kslot, (const int32_t *)lkj,
           ct, pr_c, pos, (const int32_t *)lpos, kl, ks, k_src);
    // ---- top
    int32_t *tpos = S.take((size_t)nt + 4), *tv;
    if (!tpos) return SGP_ERR_OOM;
    SGP_TRY(ensure_i32(ctx, B.tv, (size_t)nt + 4, &tv));
    LAUNCH(ctx, k_bn_topcompact, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, (const int32_t *)top,
           (const int32_t *)topidx, ord, tpos, tv);
    int32_t *tflag = S.take(E), *tcnt = S.take(E), *tidx = S.take((size_t)E + 1);
    if (!tflag || !tcnt || !tidx) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_tflag, grid_for(E, SGP_BLOCK), SGP_BLOCK, 0, E, rv, rc_ptr, ct, pr_c, pos, (const int32_t *)top,
           tflag, tcnt);
    SGP_TRY(scan_exclusive_i32(ctx, tflag, tidx, E));
    int32_t nte = 0;
    SGP_TRY(read_i32(ctx, tidx + E, &nte));
    B.nte = nte;
    int32_t *tek = S.take((size_t)nte + 1), *ter = S.take((size_t)nte + 1), *tcn = S.take((size_t)nte + 1),
            *tcp = S.take((size_t)nte + 2);
    if (!tek || !ter || !tcn || !tcp) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_tentry, grid_for(E, SGP_BLOCK), SGP_BLOCK, 0, E, (const int32_t *)tflag, (const int32_t *)tidx,
           (const int32_t *)tcnt, rv, pos, (const int32_t *)topidx, tek, ter, tcn);
    SGP_TRY(scan_exclusive_i32(ctx, tcn, tcp, nte));
    int32_t ntt = 0;
    SGP_TRY(read_i32(ctx, tcp + nte, &ntt));
    B.ntt = ntt;
    const int32_t NP = (int32_t)F->npairs;
    int32_t *tcc = S.take((size_t)ntt + 1), *t_src, *pair2tt = S.take((size_t)NP + 1);
    if (!tcc || !pair2tt) return SGP_ERR_OOM;
    SGP_TRY(ensure_i32(ctx, B.t_src, (size_t)pad4(ntt) + 4, &t_src));
    SGP_CUDA(ctx, cudaMemsetAsync(t_src, 0xff, sizeof(int32_t) * ((size_t)pad4(ntt) + 4), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(pair2tt, 0xff, sizeof(int32_t) * ((size_t)NP + 1), ctx->stream));
    LAUNCH(ctx, k_bn_tcontrib, grid_for(nte, SGP_BLOCK), SGP_BLOCK, 0, nte, (const int32_t *)tek,
           (const int32_t *)tcp, rc_ptr, ct, pr_c, pos, (const int32_t *)top, (const int32_t *)topidx, tcc, t_src,
           pair2tt);
    int32_t *tpc = S.take((size_t)nt + 1), *tpp = S.take((size_t)nt + 2);
    if (!tpc || !tpp) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_tpcount, grid_for(nt, SGP_BLOCK), SGP_BLOCK, 0, nt, (const int32_t *)tpos, pr_ptr, tpc);
    SGP_TRY(scan_exclusive_i32(ctx, tpc, tpp, nt));
    int32_t ntp = 0;
    SGP_TRY(read_i32(ctx, tpp + nt, &ntp));
    B.ntp = ntp;
    int32_t *tpq = S.take((size_t)ntp + 1), *tpL = S.take((size_t)ntp + 1);
    if (!tpq || !tpL) return SGP_ERR_OOM;
    int *berr;
    SGP_TRY(buf_ensure(ctx, B.err, 64));
    berr = bp<int>(B.err);
    SGP_CUDA(ctx, cudaMemsetAsync(berr, 0, 64, ctx->stream));
    LAUNCH(ctx, k_bn_tpairs, grid_for(nt, SGP_BLOCK), SGP_BLOCK, 0, nt, (const int32_t *)tpos, (const int32_t *)tpp,
           pr_ptr, pr_q, pos, (const int32_t *)topidx, (const int32_t *)pair2tt, tpq, tpL, berr);
    int32_t *telev = S.take(B.LVP), *tvlev = S.take(B.LVP);
    if (!telev || !tvlev) return SGP_ERR_OOM;
    LAUNCH(ctx, k_bn_bounds, grid_for(std::max(nte, B.LVP), SGP_BLOCK), SGP_BLOCK, 0, nte, (const int32_t *)tek,
           (const int32_t *)levE, B.LVP, telev);
    LAUNCH(ctx, k_bn_bounds, grid_for(std::max(nt, B.LVP), SGP_BLOCK), SGP_BLOCK, 0, nt, (const int32_t *)tpos,
           (const int32_t *)levp, B.LVP, tvlev);
    // the top's int blob: telev ter tcp tcc tvlev tpp tpq tpL tlk
    {
        const int32_t lens[9] = {B.LVP, nte, nte + 1, ntt, B.LVP, nt + 1, ntp, ntp, nt + 1};
        const int32_t *srcs[9] = {telev, ter, tcp, tcc, tvlev, tpp, tpq, tpL, tint_tlk};
        int32_t o = 0;
        for (int k = 0; k < 9; ++k) {
            B.toff[k] = o;
            o += pad4(lens[k]);
        }
        B.tints = o;
        int32_t *blob;
        SGP_TRY(ensure_i32(ctx, B.tint, (size_t)o + 4, &blob));
        SGP_CUDA(ctx, cudaMemsetAsync(blob, 0, sizeof(int32_t) * ((size_t)o + 4), ctx->stream));
        for (int k = 0; k < 9; ++k)
            if (lens[k] > 0)
                SGP_CUDA(ctx, cudaMemcpyAsync(blob + B.toff[k], srcs[k], sizeof(int32_t) * lens[k],
                                              cudaMemcpyDeviceToDevice, ctx->stream));
    }
    int32_t *tD_src;
    SGP_TRY(ensure_i32(ctx, B.tD_src, (size_t)pad4(nt) + 4, &tD_src));
    SGP_CUDA(ctx, cudaMemsetAsync(tD_src, 0xff, sizeof(int32_t) * ((size_t)pad4(nt) + 4), ctx->stream));
    if (nt > 0)
        SGP_CUDA(ctx, cudaMemcpyAsync(tD_src, tpos, sizeof(int32_t) * nt, cudaMemcpyDeviceToDevice, ctx->stream));
    int32_t *d_src;
    SGP_TRY(ensure_i32(ctx, B.d_src, (size_t)G + 4, &d_src));
    SGP_CUDA(ctx, cudaMemcpyAsync(d_src, gpos, sizeof(int32_t) * ((size_t)G + 4), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    // consistency of every index the solve kernels stage
    {
        BinCheck bc{(const int32_t *)hdr, (const int32_t *)elev, (const int32_t *)vlev, (const int32_t *)gvert,
                    (const int32_t *)er, (const int32_t *)ec, (const int32_t *)cl, (const int32_t *)kl,
                    (const int32_t *)ks, (const int32_t *)pr, (const int32_t *)pref, (const int32_t *)zi,
                    B.LVP, nly, nt, n, G, EE, Cc, K, Pp, Z, berr};
        if (nb > 0) LAUNCH(ctx, k_bn_check_bins, nb, BA, 0, bc);
        TopCheck tc{bp<const int32_t>(B.tint), (const int32_t *)tv, {0}, B.LVP, nte, ntt, nt, ntp, nly, n, berr};
        for (int k = 0; k < 9; ++k) tc.o[k] = B.toff[k];
        LAUNCH(ctx, k_bn_check_top, 1, 256, 0, tc);
    }
    // shared memory of each kernel
    int32_t *mx = S.take(8);
    if (!mx) return SGP_ERR_OOM;
    SGP_CUDA(ctx, cudaMemsetAsync(mx, 0, sizeof(int32_t) * 8, ctx->stream));
    if (nb > 0)
        LAUNCH(ctx, k_bn_smem, grid_for(nb, SGP_BLOCK), SGP_BLOCK, 0, nb, (const int32_t *)hdr, B.LVP,
               (const int32_t *)elev, (const int32_t *)ec, (const int32_t *)vlev, (const int32_t *)pr, mx);
    int32_t hm[8] = {0}, herr = 0;
    SGP_TRY(read_back(ctx, hm, mx, sizeof(hm)));
    SGP_TRY(read_back(ctx, &herr, berr, sizeof(int)));
    if (herr) return sgp_fail(ctx, SGP_ERR_CUDA, "tree_factor: inconsistent binned layout (0x%x)", herr);
    for (int s = 0; s < 2; ++s) {
        const size_t sz = s == 0 ? 4 : 8;
        B.smA0[s] = (size_t)hm[4 * s];
        B.smC0[s] = (size_t)hm[4 * s + 1];
        B.smA[s] = (size_t)hm[4 * s + 2];
        B.smC[s] = (size_t)hm[4 * s + 3];
        B.smTnd[s] = (size_t)pad4(nt) * 3 * sz + (size_t)B.tints * 4 + (size_t)pad4(ntt) * 9 * sz;
        B.smT[s] = B.smTnd[s] + (size_t)pad4(nt) * 6 * sz;
    }
    // tree order: the bins' padded segments, then the top part
    const int32_t NT = G + pad4(nt);
    B.NT = NT;
    int32_t *i_of_t, *t_of_i;
    SGP_TRY(ensure_i32(ctx, B.i_of_t, (size_t)NT + 4, &i_of_t));
    SGP_TRY(ensure_i32(ctx, B.t_of_i, (size_t)n + 4, &t_of_i));
    SGP_CUDA(ctx, cudaMemsetAsync(t_of_i, 0xff, sizeof(int32_t) * ((size_t)n + 4), ctx->stream));
    LAUNCH(ctx, k_bn_tree_maps, grid_for(NT, SGP_BLOCK), SGP_BLOCK, 0, G, nt, (const int32_t *)gvert,
           (const int32_t *)tv, i_of_t, t_of_i);
    // the matrix's rows in tree order for the fused solve (its precision only)
    B.mgen = 0;
    B.mat32 = B.mat64 = 0;
    if (M && M->n == n) {
        int32_t *len = S.take((size_t)NT + 1), *rpt;
        if (!len) return SGP_ERR_OOM;
        SGP_TRY(ensure_i32(ctx, B.rpt, (size_t)NT + 4, &rpt));
        const int32_t *rp = bp<const int32_t>(M->row_ptr);
        LAUNCH(ctx, k_bn_rowlen, grid_for(NT, SGP_BLOCK), SGP_BLOCK, 0, NT, (const int32_t *)i_of_t, rp, len);
        SGP_TRY(scan_exclusive_i32(ctx, len, rpt, NT));
        const size_t m2 = 2 * (size_t)M->m + 4;
        if (M->precision == SGP_PREC_MIXED && F->precision == SGP_PREC_MIXED) {
            SGP_TRY(buf_ensure(ctx, B.ma32, sizeof(float4) * m2));
            SGP_TRY(buf_ensure(ctx, B.mb32, sizeof(float2) * m2));
            const float4 *a4 = bp<const float4>(M->blk32);
            const float2 *b2 = reinterpret_cast<const float2 *>(a4 + 2 * M->m);
            LAUNCH(ctx, k_bn_rows32, grid_for(NT, SGP_BLOCK), SGP_BLOCK, 0, NT, (const int32_t *)i_of_t,
                   (const int32_t *)t_of_i, rp, (const int32_t *)rpt, a4, b2, bp<float4>(B.ma32), bp<float2>(B.mb32));
            B.mat32 = 1;
        } else if (F->precision == SGP_PREC_F64) {
            SGP_TRY(buf_ensure(ctx, B.m64, sizeof(double) * 6 * m2));
            SGP_TRY(buf_ensure(ctx, B.mc64, sizeof(int32_t) * m2));
            LAUNCH(ctx, k_bn_rows64, grid_for(NT, SGP_BLOCK), SGP_BLOCK, 0, NT, (const int32_t *)i_of_t,
                   (const int32_t *)t_of_i, rp, (const int32_t *)rpt, bp<const double>(M->blk),
                   bp<const int32_t>(M->col), bp<double>(B.m64), bp<int32_t>(B.mc64));
            B.mat64 = 1;
        }
        B.mgen = M->gen;
    }
    // launch order: the bins with the most levels (the longest dependency
    // chains) first, so that the last wave of blocks holds the short ones
    {
        std::vector<int32_t> h((size_t)H_N * std::max(nb, 1));
        if (nb > 0) SGP_TRY(read_back(ctx, h.data(), hdr, sizeof(int32_t) * (size_t)H_N * nb));
        std::vector<int32_t> ord_h((size_t)std::max(nb, 1));
        for (int32_t b = 0; b < nb; ++b) ord_h[b] = b;
        std::stable_sort(ord_h.begin(), ord_h.begin() + nb, [&](int32_t x, int32_t y) {
            const int32_t lx = h[(size_t)H_N * x + H_NLEV], ly = h[(size_t)H_N * y + H_NLEV];
            if (lx != ly) return lx > ly;
            return h[(size_t)H_N * x + H_NV] > h[(size_t)H_N * y + H_NV];
        });
        SGP_TRY(buf_ensure(ctx, B.order, sizeof(int32_t) * ((size_t)nb + 4)));
        if (nb > 0)
            SGP_CUDA(ctx, cudaMemcpyAsync(B.order.p, ord_h.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice,
                                          ctx->stream));
        SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // ord_h lives on the host stack
    }
    // numeric layouts
    const int32_t Gp = G + 4, Cp = Cc + 4, Kp = K + 4, Pq = Pp + 4, TT = pad4(ntt) + 4, NTp = pad4(nt) + 4;
    for (int s = 0; s < 2; ++s) {
        const bool f32 = s == 0;
        if (f32 && F->precision != SGP_PREC_MIXED) continue;
        if (!f32 && !f64_bins) continue;
        const bool fits = B.smA[s] <= (size_t)SMEM_MAX && B.smC[s] <= (size_t)SMEM_MAX && B.smTnd[s] <= (size_t)SMEM_MAX &&
                          B.smA0[s] <= (size_t)SMEM_MAX && B.smC0[s] <= (size_t)SMEM_MAX;
        if (!fits) continue;
        const size_t esz = f32 ? 4 : 8;
        SGP_TRY(buf_ensure(ctx, B.cL[s], esz * 9 * Cp));
        SGP_TRY(buf_ensure(ctx, B.kL[s], esz * 9 * Kp));
        SGP_TRY(buf_ensure(ctx, B.pL[s], esz * 9 * Pq));
        SGP_TRY(buf_ensure(ctx, B.D[s], esz * 6 * Gp));
        SGP_TRY(buf_ensure(ctx, B.tL[s], esz * 9 * TT));
        SGP_TRY(buf_ensure(ctx, B.tD[s], esz * 6 * NTp));
        SGP_TRY(buf_ensure(ctx, B.ly[s], esz * 3 * ((size_t)nly + 4)));
        SGP_TRY(buf_ensure(ctx, B.lsum[s], esz * 3 * (size_t)NTp));
        SGP_TRY(buf_ensure(ctx, B.tw[s], esz * 3 * ((size_t)NT + 4)));
        const double *Lf = bp<const double>(F->Lf), *L = bp<const double>(F->L), *Di = bp<const double>(F->Dinv);
        if (f32) {
            LAUNCH(ctx, (k_bn_gather<float, 9>), grid_for(Cp, SGP_BLOCK), SGP_BLOCK, 0, Cp, (const int32_t *)c_src, (int64_t)NC, Lf, bp<float>(B.cL[s]));
            LAUNCH(ctx, (k_bn_gather<float, 9>), grid_for(Kp, SGP_BLOCK), SGP_BLOCK, 0, Kp, (const int32_t *)k_src, (int64_t)NC, Lf, bp<float>(B.kL[s]));
            LAUNCH(ctx, (k_bn_gather<float, 9>), grid_for(Pq, SGP_BLOCK), SGP_BLOCK, 0, Pq, (const int32_t *)p_src, (int64_t)NP, L, bp<float>(B.pL[s]));
            LAUNCH(ctx, (k_bn_gather<float, 6>), grid_for(Gp, SGP_BLOCK), SGP_BLOCK, 0, Gp, (const int32_t *)d_src, (int64_t)n, Di, bp<float>(B.D[s]));
            LAUNCH(ctx, (k_bn_gather<float, 9>), grid_for(TT, SGP_BLOCK), SGP_BLOCK, 0, TT, (const int32_t *)t_src, (int64_t)NC, Lf, bp<float>(B.tL[s]));
            LAUNCH(ctx, (k_bn_gather<float, 6>), grid_for(NTp, SGP_BLOCK), SGP_BLOCK, 0, NTp, (const int32_t *)tD_src, (int64_t)n, Di, bp<float>(B.tD[s]));
        } else {
            LAUNCH(ctx, (k_bn_gather<double, 9>), grid_for(Cp, SGP_BLOCK), SGP_BLOCK, 0, Cp, (const int32_t *)c_src, (int64_t)NC, Lf, bp<double>(B.cL[s]));
            LAUNCH(ctx, (k_bn_gather<double, 9>), grid_for(Kp, SGP_BLOCK), SGP_BLOCK, 0, Kp, (const int32_t *)k_src, (int64_t)NC, Lf, bp<double>(B.kL[s]));
            LAUNCH(ctx, (k_bn_gather<double, 9>), grid_for(Pq, SGP_BLOCK), SGP_BLOCK, 0, Pq, (const int32_t *)p_src, (int64_t)NP, L, bp<double>(B.pL[s]));
            LAUNCH(ctx, (k_bn_gather<double, 6>), grid_for(Gp, SGP_BLOCK), SGP_BLOCK, 0, Gp, (const int32_t *)d_src, (int64_t)n, Di, bp<double>(B.D[s]));
            LAUNCH(ctx, (k_bn_gather<double, 9>), grid_for(TT, SGP_BLOCK), SGP_BLOCK, 0, TT, (const int32_t *)t_src, (int64_t)NC, Lf, bp<double>(B.tL[s]));
            LAUNCH(ctx, (k_bn_gather<double, 6>), grid_for(NTp, SGP_BLOCK), SGP_BLOCK, 0, NTp, (const int32_t *)tD_src, (int64_t)n, Di, bp<double>(B.tD[s]));
        }
        if (f32) B.ok32 = 1; else B.ok64 = 1;
    }
    // partials: bins' |r|^2, one spare, bins' r^T z, the top's r^T z
    SGP_TRY(buf_ensure(ctx, B.part, sizeof(double) * (2 * (size_t)nb + 4)));
    SGP_CUDA(ctx, cudaMemsetAsync(B.part.p, 0, sizeof(double) * (2 * (size_t)nb + 4), ctx->stream));
    SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SGP_OK;
}

template <typename T>
bool bins_usable(const sgp_factor *F)
{
    return F && (sizeof(T) == 4 ? F->bl.ok32 : F->bl.ok64);
}
template bool bins_usable<float>(const sgp_factor *);
template bool bins_usable<double>(const sgp_factor *);

// z = P^-1 w in place (w in the matrix's internal order: taken to the tree
// order and back through the factor's workspace).
template <typename T>
sgp_status bins_apply(sgp_ctx *ctx, const sgp_factor *F, T *w, const int *done)
{
    const BinLayout &B = F->bl;
    T *tw = bp<T>(B.tw[pidx<T>()]);
    LAUNCH(ctx, k_bn_to_tree<T>, grid_for(B.NT, SGP_BLOCK), SGP_BLOCK, 0, B.NT, bp<const int32_t>(B.i_of_t),
           (const T *)w, tw);
    SGP_TRY((launch3<T, 0>(ctx, F, tw, nullptr, tw, nullptr, done)));
    LAUNCH(ctx, k_bn_from_tree<T>, grid_for(F->n, SGP_BLOCK), SGP_BLOCK, 0, (int32_t)F->n,
           bp<const int32_t>(B.t_of_i), (const T *)tw, w);
    return SGP_OK;
}

// z = P^-1 w on tree-order vectors (z may alias w).
template <typename T>
sgp_status bins_apply_tree(sgp_ctx *ctx, const sgp_factor *F, T *w, T *z, const int *done)
{
    return launch3<T, 0>(ctx, F, w, nullptr, z, nullptr, done);
}
template sgp_status bins_apply_tree<float>(sgp_ctx *, const sgp_factor *, float *, float *, const int *);
template sgp_status bins_apply_tree<double>(sgp_ctx *, const sgp_factor *, double *, double *, const int *);

// The fused solve's tree order is usable for this matrix: layout and
// tree-order rows of precision T built from this very assembly.
template <typename T>
bool bins_tree_ready(const sgp_factor *F, const sgp_matrix *M)
{
    return bins_usable<T>(F) && M && F->bl.mgen == M->gen && (sizeof(T) == 4 ? F->bl.mat32 : F->bl.mat64);
}
template bool bins_tree_ready<float>(const sgp_factor *, const sgp_matrix *);
template bool bins_tree_ready<double>(const sgp_factor *, const sgp_matrix *);

template <typename T>
sgp_status bins_to_tree(sgp_ctx *ctx, const sgp_factor *F, const T *src, T *dst)
{
    LAUNCH(ctx, k_bn_to_tree<T>, grid_for(F->bl.NT, SGP_BLOCK), SGP_BLOCK, 0, F->bl.NT,
           bp<const int32_t>(F->bl.i_of_t), src, dst);
    return SGP_OK;
}
template <typename T>
sgp_status bins_from_tree(sgp_ctx *ctx, const sgp_factor *F, const T *src, T *dst)
{
    LAUNCH(ctx, k_bn_from_tree<T>, grid_for(F->n, SGP_BLOCK), SGP_BLOCK, 0, (int32_t)F->n,
           bp<const int32_t>(F->bl.t_of_i), src, dst);
    return SGP_OK;
}
template sgp_status bins_to_tree<float>(sgp_ctx *, const sgp_factor *, const float *, float *);
template sgp_status bins_to_tree<double>(sgp_ctx *, const sgp_factor *, const double *, double *);
template sgp_status bins_from_tree<float>(sgp_ctx *, const sgp_factor *, const float *, float *);
template sgp_status bins_from_tree<double>(sgp_ctx *, const sgp_factor *, const double *, double *);
template sgp_status bins_apply<float>(sgp_ctx *, const sgp_factor *, float *, const int *);
template sgp_status bins_apply<double>(sgp_ctx *, const sgp_factor *, double *, const int *);

// One PCG step around the solve: r -= alpha q, |r|^2 and the stopping test,
// z = P^-1 r, r^T z and beta (the scalars live in *scal, a Scal).
template <typename T>
sgp_status bins_pcg_step(sgp_ctx *ctx, const sgp_factor *F, T *r, const T *q, T *z, void *scal)
{
    return launch3<T, 1>(ctx, F, r, q, z, reinterpret_cast<Scal *>(scal), nullptr);
}
template sgp_status bins_pcg_step<float>(sgp_ctx *, const sgp_factor *, float *, const float *, float *, void *);
template sgp_status bins_pcg_step<double>(sgp_ctx *, const sgp_factor *, double *, const double *, double *, void *);

// Device error word of the binned kernels (a bounded wait that gave up).
sgp_status bins_check(sgp_ctx *ctx, const sgp_factor *F)
{
    if (!F || !F->bl.err.p) return SGP_OK;
    int h = 0;
    SGP_TRY(read_back(ctx, &h, F->bl.err.p, sizeof(int)));
    if (h & 2) return sgp_fail(ctx, SGP_ERR_CUDA, "tree solve: a bin's layout exceeds its launch's shared memory");
    if (h) return sgp_fail(ctx, SGP_ERR_TIMEOUT, "tree solve: a staged copy did not complete");
    return SGP_OK;
}
