// batch.cu -- batched PCG: many independent configurations in one solve.
//
// The batch is one block-diagonal system (the union of the instances' cell
// sets, built by sgp_collision_graph_batched), so the collision graph,
// friction blocks, spanning forest and tree factor of all instances are each
// computed by one pass of the ordinary kernels, and one contraction schedule
// serves every instance.  What the instances do not share are the PCG
// scalars (Section 1.1): each instance has its own rho, alpha, beta and
// stopping test |r_s| <= tol |F_s|.
//
// Work items are (instance, chunk of <= CH rows; CH is a tuning knob).  Each reduction kernel
// writes one partial per chunk; the last chunk of an instance to arrive (a
// per-instance arrival counter) sums that instance's partials in chunk order
// and updates the instance's scalars -- deterministic, no float atomics.
// Converged instances skip their chunks; the tree solve runs on the whole
// batch until every instance has converged.
#include "solver_common.cuh"


namespace {

constexpr int BB = 256;    // threads per block (one block per chunk)
constexpr int CH_DEFAULT = 2048;   // rows per chunk unless tuned

struct BScal {
    double rho, alpha, beta, FF, stop2, rr, pq, rz;
    long long it, maxit;
    int done, status;
    unsigned cnt;
    int skip;   // converged before this inner solve started (mixed outer loop)
};

struct Batch {
    const int32_t *chunk_inst;  // nchunks: instance of each chunk
    const int32_t *chunk_row;   // nchunks + 1: first row of each chunk
    const int32_t *inst_chunk;  // n_inst + 1: first chunk of each instance
    BScal *sc;                  // n_inst
    double *part;               // 2 per chunk
    int *n_done, *all_done;
    int n_inst;
};

// Arrival of one chunk of instance s; true in the instance's last chunk.
__device__ __forceinline__ bool inst_last(const Batch &b, int s)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned nch = (unsigned)(b.inst_chunk[s + 1] - b.inst_chunk[s]);
        const unsigned t = atomicAdd(&b.sc[s].cnt, 1u);
        last = (t == nch - 1);
        if (last) b.sc[s].cnt = 0u;
    }
    __syncthreads();
    return last;
}

// Sum of the instance's chunk partials (component k of 2), in chunk order.
__device__ __forceinline__ double inst_sum(const Batch &b, int s, int k, double *sh)
{
    double v = 0.0;
    for (int c = b.inst_chunk[s] + threadIdx.x; c < b.inst_chunk[s + 1]; c += BB) v += __ldcg(b.part + 2 * c + k);
    return block_sum<BB>(v, sh);
}

__device__ __forceinline__ void mark_done(const Batch &b, int s)
{
    b.sc[s].done = 1;
    const int d = atomicAdd(b.n_done, 1) + 1;
    if (d == b.n_inst) *b.all_done = 1;
}

// r = F - Gamma x (or F), w = H r, |F|^2, |r|^2 per instance.
// PREC: 0 tree (w = r), 1 block Jacobi, 2 none (w = r).
template <typename T, int PREC>
__global__ void __launch_bounds__(BB) k_b_init(Blk<T> B, const int32_t *__restrict__ row_ptr, T g0, Batch b,
                                               const T *__restrict__ F, const T *__restrict__ x, int x_given,
                                               T *r, T *w, const T *__restrict__ jac,
                                               const double *__restrict__ tol2_inst, double tol2,
                                               long long maxit)
{
    __shared__ double sh[BB / 32];
    const int c = blockIdx.x, s = b.chunk_inst[c];
    const bool skip = b.sc[s].skip;
    double ff = 0.0, rr = 0.0;
    if (!skip)
        for (int32_t i = b.chunk_row[c] + threadIdx.x; i < b.chunk_row[c + 1]; i += BB) {
            T ri[3] = {F[3 * (int64_t)i], F[3 * (int64_t)i + 1], F[3 * (int64_t)i + 2]};
            ff += (double)fma(ri[0], ri[0], fma(ri[1], ri[1], ri[2] * ri[2]));
            if (x_given) {
                const T v0 = x[3 * (int64_t)i], v1 = x[3 * (int64_t)i + 1], v2 = x[3 * (int64_t)i + 2];
                T y0 = g0 * v0, y1 = g0 * v1, y2 = g0 * v2;
                row_accumulate(B, row_ptr[i], row_ptr[i + 1], 1, x, v0, v1, v2, y0, y1, y2);
                ri[0] -= y0; ri[1] -= y1; ri[2] -= y2;
            }
            rr += (double)fma(ri[0], ri[0], fma(ri[1], ri[1], ri[2] * ri[2]));
            T zi[3] = {ri[0], ri[1], ri[2]};
            if (PREC == 1) sym_mv(jac + 6 * (int64_t)i, ri, zi);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                r[3 * (int64_t)i + a] = ri[a];
                w[3 * (int64_t)i + a] = zi[a];
            }
        }
    double s1 = block_sum<BB>(ff, sh);
    if (threadIdx.x == 0) b.part[2 * c] = s1;
    double s2 = block_sum<BB>(rr, sh);
    if (threadIdx.x == 0) b.part[2 * c + 1] = s2;
    if (inst_last(b, s)) {
        const double FF = inst_sum(b, s, 0, sh), R = inst_sum(b, s, 1, sh);
        if (threadIdx.x == 0) {
            BScal &S = b.sc[s];
            const double t2 = tol2_inst ? tol2_inst[s] : tol2;
            S.FF = FF;
            S.rr = R;
            S.stop2 = t2 * FF;
            S.it = 0;
            S.maxit = maxit;
            S.status = 0;
            S.done = 0;
            if (skip || FF == 0.0 || R <= t2 * FF) mark_done(b, s);
        }
    }
}

// rho = r^T w, p = w
template <typename T>
__global__ void __launch_bounds__(BB) k_b_rz_init(Batch b, const T *__restrict__ r, const T *__restrict__ w, T *p)
{
    __shared__ double sh[BB / 32];
    const int c = blockIdx.x, s = b.chunk_inst[c];
    if (b.sc[s].done) return;
    double acc = 0.0;
    for (int64_t k = 3 * (int64_t)b.chunk_row[c] + threadIdx.x; k < 3 * (int64_t)b.chunk_row[c + 1]; k += BB) {
        const T wk = w[k];
        acc += (double)(r[k] * wk);
        p[k] = wk;
    }
    double v = block_sum<BB>(acc, sh);
    if (threadIdx.x == 0) b.part[2 * c] = v;
    if (inst_last(b, s)) {
        const double rz = inst_sum(b, s, 0, sh);
        if (threadIdx.x == 0) {
            BScal &S = b.sc[s];
            S.rho = rz;
            if (!(rz > 0.0) || !isfinite(rz)) {
                S.status = SGP_ERR_NOT_SPD;
                mark_done(b, s);
            }
        }
    }
}

// q = Gamma p and p^T q per instance; alpha = rho / p^T q.
template <typename T, int LPR>
__global__ void __launch_bounds__(BB) k_b_spmv(Blk<T> B, const int32_t *__restrict__ row_ptr, T g0, Batch b,
                                               const T *__restrict__ p, T *q)
{
    __shared__ double sh[BB / 32];
    const int c = blockIdx.x, s = b.chunk_inst[c];
    if (b.sc[s].done) return;
    const int lane = threadIdx.x & 31, g = lane % LPR;
    const int32_t r0 = b.chunk_row[c], r1 = b.chunk_row[c + 1];
    constexpr int RPB = BB / LPR;
    double acc = 0.0;
    for (int32_t base = r0; base < r1; base += RPB) {
        const int32_t i = base + (int32_t)threadIdx.x / LPR;
        const bool active = i < r1;
        T y0 = 0, y1 = 0, y2 = 0, v0 = 0, v1 = 0, v2 = 0;
        if (active) {
            v0 = p[3 * (int64_t)i]; v1 = p[3 * (int64_t)i + 1]; v2 = p[3 * (int64_t)i + 2];
            row_accumulate(B, row_ptr[i] + g, row_ptr[i + 1], LPR, p, v0, v1, v2, y0, y1, y2);
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
            y0 += __shfl_xor_sync(0xffffffffu, y0, o);
            y1 += __shfl_xor_sync(0xffffffffu, y1, o);
            y2 += __shfl_xor_sync(0xffffffffu, y2, o);
        }
        if (active && g == 0) {
            y0 = fma(g0, v0, y0); y1 = fma(g0, v1, y1); y2 = fma(g0, v2, y2);
            q[3 * (int64_t)i] = y0; q[3 * (int64_t)i + 1] = y1; q[3 * (int64_t)i + 2] = y2;
            acc += (double)fma(v0, y0, fma(v1, y1, v2 * y2));
        }
    }
    double v = block_sum<BB>(acc, sh);
    if (threadIdx.x == 0) b.part[2 * c] = v;
    if (inst_last(b, s)) {
        const double pq = inst_sum(b, s, 0, sh);
        if (threadIdx.x == 0) {
            BScal &S = b.sc[s];
            S.pq = pq;
            if (!(pq > 0.0) || !isfinite(pq)) {
                S.status = SGP_ERR_NOT_SPD;
                mark_done(b, s);
            } else {
                S.alpha = S.rho / pq;
            }
        }
    }
}

// x += alpha p, r -= alpha q, w = H r; |r|^2 (and r^T w); convergence.
template <typename T, int PREC>
__global__ void __launch_bounds__(BB) k_b_update(Batch b, T *x, const T *__restrict__ p, T *r,
                                                 const T *__restrict__ q, T *w, const T *__restrict__ jac)
{
    __shared__ double sh[BB / 32];
    const int c = blockIdx.x, s = b.chunk_inst[c];
    if (b.sc[s].done) return;
    const T a = (T)b.sc[s].alpha;
    double rr = 0.0, rz = 0.0;
    for (int32_t i = b.chunk_row[c] + threadIdx.x; i < b.chunk_row[c + 1]; i += BB) {
        T ri[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int64_t k = 3 * (int64_t)i + e;
            x[k] = fma(a, p[k], x[k]);
            ri[e] = fma(-a, q[k], r[k]);
            r[k] = ri[e];
        }
        T zi[3] = {ri[0], ri[1], ri[2]};
        if (PREC == 1) sym_mv(jac + 6 * (int64_t)i, ri, zi);
#pragma unroll
        for (int e = 0; e < 3; ++e) w[3 * (int64_t)i + e] = zi[e];
        rr += (double)fma(ri[0], ri[0], fma(ri[1], ri[1], ri[2] * ri[2]));
        rz += (double)fma(ri[0], zi[0], fma(ri[1], zi[1], ri[2] * zi[2]));
    }
    double s1 = block_sum<BB>(rr, sh);
    if (threadIdx.x == 0) b.part[2 * c] = s1;
    double s2 = block_sum<BB>(rz, sh);
    if (threadIdx.x == 0) b.part[2 * c + 1] = s2;
    if (inst_last(b, s)) {
        const double R = inst_sum(b, s, 0, sh), Z = inst_sum(b, s, 1, sh);
        if (threadIdx.x == 0) {
            BScal &S = b.sc[s];
            S.rr = R;
            S.it += 1;
            if (R <= S.stop2) {
                mark_done(b, s);
            } else if (S.it >= S.maxit) {
                S.status = SGP_ERR_NO_CONVERGENCE;
                mark_done(b, s);
            } else if (PREC != 0) {
                S.beta = Z / S.rho;
                S.rho = Z;
            }
        }
    }
}

// rho' = r^T w after the tree solve; beta = rho' / rho.
template <typename T>
__global__ void __launch_bounds__(BB) k_b_rz(Batch b, const T *__restrict__ r, const T *__restrict__ w)
{
    __shared__ double sh[BB / 32];
    const int c = blockIdx.x, s = b.chunk_inst[c];
    if (b.sc[s].done) return;
    double acc = 0.0;
    for (int64_t k = 3 * (int64_t)b.chunk_row[c] + threadIdx.x; k < 3 * (int64_t)b.chunk_row[c + 1]; k += BB)
        acc += (double)(r[k] * w[k]);
    double v = block_sum<BB>(acc, sh);
    if (threadIdx.x == 0) b.part[2 * c] = v;
    if (inst_last(b, s)) {
        const double rz = inst_sum(b, s, 0, sh);
        if (threadIdx.x == 0) {
            BScal &S = b.sc[s];
            if (!(rz > 0.0) || !isfinite(rz)) {
                S.status = SGP_ERR_NOT_SPD;
                mark_done(b, s);
            } else {
                S.beta = rz / S.rho;
                S.rho = rz;
            }
        }
    }
}

// p = w + beta p
template <typename T>
__global__ void __launch_bounds__(BB) k_b_pupd(Batch b, const T *__restrict__ w, T *p)
{
    const int c = blockIdx.x, s = b.chunk_inst[c];
    if (b.sc[s].done) return;
    const T beta = (T)b.sc[s].beta;
    for (int64_t k = 3 * (int64_t)b.chunk_row[c] + threadIdx.x; k < 3 * (int64_t)b.chunk_row[c + 1]; k += BB)
        p[k] = fma(beta, p[k], w[k]);
}

// FP64 residual r = F - Gamma v per instance: out[2s] = |r_s|^2, out[2s+1] = |F_s|^2.
__global__ void __launch_bounds__(BB) k_b_resid64(Blk<double> B, const int32_t *__restrict__ row_ptr, double g0,
                                                  Batch b, const double *__restrict__ F,
                                                  const double *__restrict__ v, double *r, double *out)
{
    __shared__ double sh[BB / 32];
    const int c = blockIdx.x, s = b.chunk_inst[c];
    double rr = 0.0, ff = 0.0;
    for (int32_t i = b.chunk_row[c] + threadIdx.x; i < b.chunk_row[c + 1]; i += BB) {
        const double v0 = v[3 * (int64_t)i], v1 = v[3 * (int64_t)i + 1], v2 = v[3 * (int64_t)i + 2];
        double y0 = g0 * v0, y1 = g0 * v1, y2 = g0 * v2;
        row_accumulate(B, row_ptr[i], row_ptr[i + 1], 1, v, v0, v1, v2, y0, y1, y2);
        const double yy[3] = {y0, y1, y2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double f = F[3 * (int64_t)i + a];
            const double rc = f - yy[a];
            if (r) r[3 * (int64_t)i + a] = rc;
            rr += rc * rc;
            ff += f * f;
        }
    }
    double s1 = block_sum<BB>(rr, sh);
    if (threadIdx.x == 0) b.part[2 * c] = s1;
    double s2 = block_sum<BB>(ff, sh);
    if (threadIdx.x == 0) b.part[2 * c + 1] = s2;
    if (inst_last(b, s)) {
        const double R = inst_sum(b, s, 0, sh), FF = inst_sum(b, s, 1, sh);
        if (threadIdx.x == 0) {
            out[2 * s] = R;
            out[2 * s + 1] = FF;
        }
    }
}

// mixed: r32 = r64 * scale_s, d = 0
__global__ void k_b_scale(Batch b, const double *__restrict__ r64, const double *__restrict__ scale, float *r32,
                          float *d)
{
    const int c = blockIdx.x, s = b.chunk_inst[c];
    const double sc = scale[s];
    for (int64_t k = 3 * (int64_t)b.chunk_row[c] + threadIdx.x; k < 3 * (int64_t)b.chunk_row[c + 1]; k += BB) {
        r32[k] = (float)(r64[k] * sc);
        d[k] = 0.f;
    }
}

// mixed: v += |r_s| d
__global__ void k_b_accumulate(Batch b, const float *__restrict__ d, const double *__restrict__ nrm, double *v)
{
    const int c = blockIdx.x, s = b.chunk_inst[c];
    const double a = nrm[s];
    if (a == 0.0) return;
    for (int64_t k = 3 * (int64_t)b.chunk_row[c] + threadIdx.x; k < 3 * (int64_t)b.chunk_row[c + 1]; k += BB)
        v[k] += a * (double)d[k];
}

// Every edge must join two cells of the same instance.
__global__ void k_b_check_edges(const int32_t *__restrict__ ij, int64_t m, const int32_t *__restrict__ row_inst,
                                int *err)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < m && row_inst[ij[2 * e]] != row_inst[ij[2 * e + 1]]) atomicOr(err, 1);
}

// The matrix's internal cell order must keep every instance on its own rows.
__global__ void k_b_check_order(int64_t n, const int32_t *__restrict__ orig_of, const int32_t *__restrict__ row_inst,
                                int *err)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n && row_inst[orig_of[r]] != row_inst[r]) atomicOr(err, 2);
}

__global__ void k_b_row_inst(const int32_t *__restrict__ inst_row, int32_t *row_inst)
{
    const int s = blockIdx.x;
    for (int32_t i = inst_row[s] + threadIdx.x; i < inst_row[s + 1]; i += blockDim.x) row_inst[i] = s;
}

template <typename T, int PREC>
sgp_status launch_update(sgp_ctx *ctx, unsigned G, Batch b, T *x, const T *p, T *r, const T *q, T *w, const T *jac)
{
    LAUNCH(ctx, (k_b_update<T, PREC>), G, BB, 0, b, x, p, r, q, w, jac);
    return SGP_OK;
}

// One batched PCG run in precision T from x = 0 (x given when x_given).
template <typename T>
sgp_status pcg_b_run(sgp_ctx *ctx, const sgp_matrix *M, const sgp_factor *Fac, int precond, const Batch &b,
                     unsigned nchunks, const T *F, T *x, int x_given, double tol, const double *tol2_inst,
                     int64_t maxit, T *r, T *p, T *q, T *w)
{
    const int64_t n = M->n;
    Blk<T> B = make_blk<T>(M);
    const int32_t *row_ptr = bp<const int32_t>(M->row_ptr);
    const T g0 = (T)M->gamma0;
    const T *jac = nullptr;
    if (precond == SGP_PRECOND_BLOCK_JACOBI) {
        SGP_TRY(matrix_block_jacobi(ctx, const_cast<sgp_matrix *>(M)));
        jac = reinterpret_cast<const T *>(sizeof(T) == 8 ? M->jac.p : M->jac32.p);
    }
    if (!x_given) SGP_CUDA(ctx, cudaMemsetAsync(x, 0, sizeof(T) * 3 * n, ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(b.n_done, 0, 2 * sizeof(int), ctx->stream));  // n_done, all_done
    const int pc = precond == SGP_PRECOND_TREE ? 0 : (precond == SGP_PRECOND_BLOCK_JACOBI ? 1 : 2);
    if (pc == 0)
        LAUNCH(ctx, (k_b_init<T, 0>), nchunks, BB, 0, B, row_ptr, g0, b, F, (const T *)x, x_given, r, w, jac,
               tol2_inst, tol * tol, (long long)maxit);
    else if (pc == 1)
        LAUNCH(ctx, (k_b_init<T, 1>), nchunks, BB, 0, B, row_ptr, g0, b, F, (const T *)x, x_given, r, w, jac,
               tol2_inst, tol * tol, (long long)maxit);
    else
        LAUNCH(ctx, (k_b_init<T, 2>), nchunks, BB, 0, B, row_ptr, g0, b, F, (const T *)x, x_given, r, w, jac,
               tol2_inst, tol * tol, (long long)maxit);
    if (pc == 0) SGP_TRY(tree_apply_inplace<T>(ctx, Fac, w, b.all_done));
    LAUNCH(ctx, k_b_rz_init<T>, nchunks, BB, 0, b, (const T *)r, (const T *)w, p);
    const int lpr = ctx->spmv_lpr > 0 ? ctx->spmv_lpr : (sizeof(T) == 8 ? 1 : 2);
    auto iterate = [&](int count) -> sgp_status {
        for (int it = 0; it < count; ++it) {
            switch (lpr) {
            case 1: LAUNCH(ctx, (k_b_spmv<T, 1>), nchunks, BB, 0, B, row_ptr, g0, b, (const T *)p, q); break;
            case 4: LAUNCH(ctx, (k_b_spmv<T, 4>), nchunks, BB, 0, B, row_ptr, g0, b, (const T *)p, q); break;
            default: LAUNCH(ctx, (k_b_spmv<T, 2>), nchunks, BB, 0, B, row_ptr, g0, b, (const T *)p, q); break;
            }
            if (pc == 0) SGP_TRY((launch_update<T, 0>(ctx, nchunks, b, x, p, r, q, w, jac)));
            else if (pc == 1) SGP_TRY((launch_update<T, 1>(ctx, nchunks, b, x, p, r, q, w, jac)));
            else SGP_TRY((launch_update<T, 2>(ctx, nchunks, b, x, p, r, q, w, jac)));
            if (pc == 0) {
                SGP_TRY(tree_apply_inplace<T>(ctx, Fac, w, b.all_done));
                LAUNCH(ctx, k_b_rz<T>, nchunks, BB, 0, b, (const T *)r, (const T *)w);
            }
            LAUNCH(ctx, k_b_pupd<T>, nchunks, BB, 0, b, (const T *)w, p);
        }
        return SGP_OK;
    };
    const int chunk = 8;
    int all_done = 0;
    if (!ctx->use_graphs) {
        for (;;) {
            SGP_TRY(read_back(ctx, &all_done, b.all_done, sizeof(int)));
            if (all_done) break;
            SGP_TRY(iterate(chunk));
        }
        return SGP_OK;
    }
    // device-side loop (see the single-system solver): chunks of 4
    // iterations as the body of a conditional WHILE node; the body counter
    // sits in the flag word after n_done and all_done
    if (ctx->use_while && !ctx->timing) {
        const int wchunk = 4, max_bodies = 1024;
        int *bodies = b.n_done + 3;
        const uint64_t wkey[] = {0xBA7C5ull, (uint64_t)sizeof(T), (uint64_t)pc, (uint64_t)n, (uint64_t)nchunks,
                                 M->gen, Fac ? Fac->gen : 0ull, (uint64_t)(uintptr_t)x, (uint64_t)(uintptr_t)r,
                                 (uint64_t)(uintptr_t)p, (uint64_t)(uintptr_t)q, (uint64_t)(uintptr_t)w,
                                 (uint64_t)(uintptr_t)b.sc, (uint64_t)(uintptr_t)jac, (uint64_t)wchunk,
                                 (uint64_t)lpr};
        GraphEntry *we = nullptr;
        SGP_TRY(graph_lookup(ctx, wkey, sizeof(wkey) / sizeof(wkey[0]), &we));
        if (!we->exec &&
            graph_capture_while(ctx, we, b.all_done, bodies, max_bodies, [&]() { return iterate(wchunk); }) !=
                SGP_OK) {
            ctx->use_while = 0;
            cudaGetLastError();
        }
        if (we->exec) {
            int fl[4] = {0, 0, 0, 0};   // n_done, all_done, -, bodies
            SGP_TRY(read_back(ctx, fl, b.n_done, sizeof(fl)));
            while (!fl[1]) {
                SGP_CUDA(ctx, cudaMemsetAsync(bodies, 0, sizeof(int), ctx->stream));
                SGP_CUDA(ctx, cudaGraphLaunch(we->exec, ctx->stream));
                SGP_TRY(read_back(ctx, fl, b.n_done, sizeof(fl)));
                ctx->launches += (int64_t)fl[3] * we->kernels;
            }
            return SGP_OK;
        }
    }
    const uint64_t key[] = {0xBA7C4ull, (uint64_t)sizeof(T), (uint64_t)pc, (uint64_t)n, (uint64_t)nchunks,
                            M->gen, Fac ? Fac->gen : 0ull, (uint64_t)(uintptr_t)x, (uint64_t)(uintptr_t)r,
                            (uint64_t)(uintptr_t)p, (uint64_t)(uintptr_t)q, (uint64_t)(uintptr_t)w,
                            (uint64_t)(uintptr_t)b.sc, (uint64_t)(uintptr_t)jac, (uint64_t)ctx->timing,
                            (uint64_t)lpr};
    GraphEntry *ge = nullptr;
    SGP_TRY(graph_lookup(ctx, key, sizeof(key) / sizeof(key[0]), &ge));
    if (!ge->exec) SGP_TRY(graph_capture(ctx, ge, [&]() { return iterate(chunk); }));
    for (;;) {
        SGP_TRY(read_back(ctx, &all_done, b.all_done, sizeof(int)));
        if (all_done) break;
        SGP_CUDA(ctx, cudaGraphLaunch(ge->exec, ctx->stream));
        ctx->launches += ge->kernels;
    }
    return SGP_OK;
}

}  // namespace

extern "C" {

sgp_status sgp_pcg_solve_batched(sgp_ctx *ctx, const sgp_matrix *M, const sgp_factor *Fac, int64_t n_inst,
                                 const int64_t *offsets, const double *F, double *v, const sgp_solve_opts *opts,
                                 sgp_solve_info *infos)
{
    if (!ctx || !M || !opts || !offsets || n_inst < 1) return SGP_ERR_INVALID_ARG;
    const int64_t n = M->n;
    if (offsets[0] != 0 || offsets[n_inst] != n)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: offsets must run from 0 to n");
    for (int64_t s = 0; s < n_inst; ++s)
        if (offsets[s + 1] < offsets[s])
            return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: offsets must not decrease");
    if (n > 0 && (!F || !v)) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: NULL vector");
    if (!(opts->tol > 0.0) || opts->maxit <= 0)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: tol must be > 0 and maxit >= 1");
    if (opts->stop != SGP_STOP_RESIDUAL)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: residual stopping only");
    if (opts->precond < 0 || opts->precond > 2)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: bad preconditioner");
    if (opts->precond == SGP_PRECOND_TREE && (!Fac || Fac->n != n))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: the tree preconditioner needs a factor");
    const bool mixed = opts->precision == SGP_PREC_MIXED;
    if (mixed && (M->precision != SGP_PREC_MIXED ||
                  (opts->precond == SGP_PRECOND_TREE && Fac->precision != SGP_PREC_MIXED)))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: MIXED needs a MIXED matrix and factor");
    if (n == 0) {
        if (infos) std::memset(infos, 0, sizeof(sgp_solve_info) * n_inst);
        return SGP_OK;
    }
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    // chunk table: instances cut into chunks of at most CH rows
    const int CH = ctx->batch_chunk > 0 ? ctx->batch_chunk : CH_DEFAULT;
    std::vector<int32_t> chunk_inst, chunk_row, inst_chunk(n_inst + 1), inst_row(n_inst + 1);
    for (int64_t s = 0; s < n_inst; ++s) {
        inst_chunk[s] = (int32_t)chunk_inst.size();
        inst_row[s] = (int32_t)offsets[s];
        for (int64_t r0 = offsets[s]; r0 < offsets[s + 1]; r0 += CH) {
            chunk_inst.push_back((int32_t)s);
            chunk_row.push_back((int32_t)r0);
        }
        if (offsets[s + 1] == offsets[s]) {      // an empty instance still gets a chunk
            chunk_inst.push_back((int32_t)s);
            chunk_row.push_back((int32_t)offsets[s]);
        }
    }
    inst_chunk[n_inst] = (int32_t)chunk_inst.size();
    inst_row[n_inst] = (int32_t)n;
    chunk_row.push_back((int32_t)n);
    // chunk_row must end each chunk at the next chunk's start or the instance end
    const int64_t nch = (int64_t)chunk_inst.size();
    std::vector<int32_t> row_end(nch);
    for (int64_t c = 0; c < nch; ++c) {
        const int32_t s = chunk_inst[c];
        row_end[c] = (int32_t)std::min<int64_t>(chunk_row[c] + CH, offsets[s + 1]);
    }
    for (int64_t c = 0; c + 1 < nch; ++c)
        if (row_end[c] != chunk_row[c + 1]) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: chunk table");

    // workspace
    const size_t v64 = sizeof(double) * 3 * n, v32 = sizeof(float) * 3 * n;
    const size_t tbl = sizeof(int32_t) * (2 * nch + 2 * n_inst + 4 + n);
    size_t need = 6 * v64 + (mixed ? 6 * v32 : 0) + sizeof(double) * 2 * nch + sizeof(BScal) * n_inst +
                  sizeof(double) * 6 * n_inst + tbl + 18 * 4096;
    SGP_TRY(scratch_ensure(ctx, need));
    char *base = reinterpret_cast<char *>(ctx->d_scratch) + 256;
    auto take = [&](size_t bytes) {
        char *q = base;
        base += (bytes + 255) & ~size_t(255);
        return q;
    };
    int32_t *d_chunk_inst = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * nch));
    int32_t *d_chunk_row = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (nch + 1)));
    int32_t *d_inst_chunk = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (n_inst + 1)));
    int32_t *d_inst_row = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (n_inst + 1)));
    int32_t *d_row_inst = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * n));
    BScal *d_sc = reinterpret_cast<BScal *>(take(sizeof(BScal) * n_inst));
    double *d_part = reinterpret_cast<double *>(take(sizeof(double) * 2 * nch));
    double *d_out = reinterpret_cast<double *>(take(sizeof(double) * 2 * n_inst));
    double *d_scale = reinterpret_cast<double *>(take(sizeof(double) * n_inst));
    double *d_nrm = reinterpret_cast<double *>(take(sizeof(double) * n_inst));
    double *d_tol2 = reinterpret_cast<double *>(take(sizeof(double) * n_inst));
    int *d_flags = reinterpret_cast<int *>(take(64));
    double *r = reinterpret_cast<double *>(take(v64));
    double *p = reinterpret_cast<double *>(take(v64));
    double *q = reinterpret_cast<double *>(take(v64));
    double *w = reinterpret_cast<double *>(take(v64));
    SGP_CUDA(ctx, cudaMemcpyAsync(d_chunk_inst, chunk_inst.data(), sizeof(int32_t) * nch, cudaMemcpyHostToDevice, ctx->stream));
    SGP_CUDA(ctx, cudaMemcpyAsync(d_chunk_row, chunk_row.data(), sizeof(int32_t) * (nch + 1), cudaMemcpyHostToDevice, ctx->stream));
    SGP_CUDA(ctx, cudaMemcpyAsync(d_inst_chunk, inst_chunk.data(), sizeof(int32_t) * (n_inst + 1), cudaMemcpyHostToDevice, ctx->stream));
    SGP_CUDA(ctx, cudaMemcpyAsync(d_inst_row, inst_row.data(), sizeof(int32_t) * (n_inst + 1), cudaMemcpyHostToDevice, ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(d_sc, 0, sizeof(BScal) * n_inst, ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(d_flags, 0, 64, ctx->stream));
    // block-diagonal check
    LAUNCH(ctx, k_b_row_inst, (unsigned)n_inst, BB, 0, (const int32_t *)d_inst_row, d_row_inst);
    LAUNCH(ctx, k_b_check_edges, grid_for(M->m, BB), BB, 0, bp<const int32_t>(M->ij), M->m,
           (const int32_t *)d_row_inst, d_flags + 8);
    const int32_t *orig_of = bp<const int32_t>(M->orig_of);
    LAUNCH(ctx, k_b_check_order, grid_for(n, BB), BB, 0, n, orig_of, (const int32_t *)d_row_inst, d_flags + 8);
    int herr = 0;
    SGP_TRY(read_back(ctx, &herr, d_flags + 8, sizeof(int)));
    if (herr & 1) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg_batched: an edge joins two instances");
    if (herr & 2)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG,
                        "pcg_batched: the matrix's cell order mixes instances (build its graph with "
                        "sgp_collision_graph_batched and the same offsets)");
    // the solve runs in the matrix's internal cell order, which keeps each
    // instance on the rows [offsets[s], offsets[s+1])
    const double *F_user = F;
    double *v_user = v;
    double *F_in = reinterpret_cast<double *>(take(v64));
    double *v_in = reinterpret_cast<double *>(take(v64));
    LAUNCH(ctx, k_to_internal<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, F_user, F_in);
    if (opts->x0_given)
        LAUNCH(ctx, k_to_internal<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, (const double *)v_user,
               v_in);
    F = F_in;
    v = v_in;

    Batch b{d_chunk_inst, d_chunk_row, d_inst_chunk, d_sc, d_part, d_flags, d_flags + 1, (int)n_inst};
    const unsigned G = (unsigned)nch;
    Blk<double> B64 = make_blk<double>(M);
    const int32_t *row_ptr = bp<const int32_t>(M->row_ptr);
    std::vector<BScal> hs(n_inst);
    std::vector<double> hres(2 * n_inst);
    std::vector<sgp_solve_info> inf(n_inst);
    std::memset(inf.data(), 0, sizeof(sgp_solve_info) * n_inst);
    if (!mixed) {
        SGP_TRY(pcg_b_run<double>(ctx, M, Fac, opts->precond, b, G, F, v, opts->x0_given, opts->tol, nullptr,
                                  opts->maxit, r, p, q, w));
        SGP_TRY(read_back(ctx, hs.data(), d_sc, sizeof(BScal) * n_inst));
        for (int64_t s = 0; s < n_inst; ++s) {
            inf[s].iterations = hs[s].it;
            inf[s].status = hs[s].status;
            inf[s].rel_residual = hs[s].FF > 0 ? std::sqrt(hs[s].rr / hs[s].FF) : 0.0;
        }
    } else {
        float *r32 = reinterpret_cast<float *>(take(v32));
        float *s32 = reinterpret_cast<float *>(take(v32));
        float *p32 = reinterpret_cast<float *>(take(v32));
        float *q32 = reinterpret_cast<float *>(take(v32));
        float *w32 = reinterpret_cast<float *>(take(v32));
        float *d32 = reinterpret_cast<float *>(take(v32));
        const int max_outer = opts->max_outer > 0 ? opts->max_outer : 30;
        const double itol = opts->inner_tol > 0 ? opts->inner_tol : 1e-3;
        if (!opts->x0_given) SGP_CUDA(ctx, cudaMemsetAsync(v, 0, v64, ctx->stream));
        std::vector<double> scale(n_inst), nrm(n_inst), tol2(n_inst);
        std::vector<int> active(n_inst, 1);
        for (int outer = 0;; ++outer) {
            SGP_CUDA(ctx, cudaMemsetAsync(d_out, 0, sizeof(double) * 2 * n_inst, ctx->stream));
            LAUNCH(ctx, k_b_resid64, G, BB, 0, B64, row_ptr, M->gamma0, b, F, (const double *)v, r, d_out);
            SGP_TRY(read_back(ctx, hres.data(), d_out, sizeof(double) * 2 * n_inst));
            int n_active = 0;
            for (int64_t s = 0; s < n_inst; ++s) {
                const double rr = hres[2 * s], ff = hres[2 * s + 1];
                inf[s].rel_residual = ff > 0 ? std::sqrt(rr / ff) : 0.0;
                inf[s].outer_iterations = outer;
                const bool conv = ff == 0.0 || rr <= opts->tol * opts->tol * ff;
                if (active[s] && !conv && (outer >= max_outer || inf[s].iterations >= opts->maxit)) {
                    inf[s].status = SGP_ERR_NO_CONVERGENCE;
                    active[s] = 0;
                }
                if (conv || inf[s].status) active[s] = 0;
                if (active[s]) {
                    nrm[s] = std::sqrt(rr);
                    scale[s] = 1.0 / nrm[s];
                    const double want = 0.5 * opts->tol * std::sqrt(ff) / nrm[s];
                    const double it = std::max(itol, std::min(want, 0.5));
                    tol2[s] = it * it;
                    ++n_active;
                } else {
                    nrm[s] = 0.0;
                    scale[s] = 0.0;
                    tol2[s] = 1.0;
                }
            }
            if (n_active == 0) break;
            SGP_CUDA(ctx, cudaMemcpyAsync(d_scale, scale.data(), sizeof(double) * n_inst, cudaMemcpyHostToDevice, ctx->stream));
            SGP_CUDA(ctx, cudaMemcpyAsync(d_nrm, nrm.data(), sizeof(double) * n_inst, cudaMemcpyHostToDevice, ctx->stream));
            SGP_CUDA(ctx, cudaMemcpyAsync(d_tol2, tol2.data(), sizeof(double) * n_inst, cudaMemcpyHostToDevice, ctx->stream));
            // per-instance skip flags for the inner solve
            for (int64_t s = 0; s < n_inst; ++s) {
                hs[s] = BScal{};
                hs[s].skip = active[s] ? 0 : 1;
            }
            SGP_CUDA(ctx, cudaMemcpyAsync(d_sc, hs.data(), sizeof(BScal) * n_inst, cudaMemcpyHostToDevice, ctx->stream));
            LAUNCH(ctx, k_b_scale, G, BB, 0, b, (const double *)r, (const double *)d_scale, r32, d32);
            SGP_TRY(pcg_b_run<float>(ctx, M, Fac, opts->precond, b, G, (const float *)r32, d32, 0, itol, d_tol2,
                                     opts->maxit, s32, p32, q32, w32));
            SGP_TRY(read_back(ctx, hs.data(), d_sc, sizeof(BScal) * n_inst));
            for (int64_t s = 0; s < n_inst; ++s)
                if (active[s]) {
                    inf[s].iterations += hs[s].it;
                    if (hs[s].status == SGP_ERR_NOT_SPD) {
                        inf[s].status = SGP_ERR_NOT_SPD;
                        nrm[s] = 0.0;
                        active[s] = 0;
                    }
                }
            SGP_CUDA(ctx, cudaMemcpyAsync(d_nrm, nrm.data(), sizeof(double) * n_inst, cudaMemcpyHostToDevice, ctx->stream));
            LAUNCH(ctx, k_b_accumulate, G, BB, 0, b, (const float *)d32, (const double *)d_nrm, v);
        }
    }
    // true FP64 residual per instance
    SGP_CUDA(ctx, cudaMemsetAsync(d_out, 0, sizeof(double) * 2 * n_inst, ctx->stream));
    LAUNCH(ctx, k_b_resid64, G, BB, 0, B64, row_ptr, M->gamma0, b, F, (const double *)v, (double *)nullptr, d_out);
    SGP_TRY(read_back(ctx, hres.data(), d_out, sizeof(double) * 2 * n_inst));
    LAUNCH(ctx, k_to_caller<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, (const double *)v, v_user);
    sgp_status rc = SGP_OK;
    for (int64_t s = 0; s < n_inst; ++s) {
        inf[s].true_rel_residual = hres[2 * s + 1] > 0 ? std::sqrt(hres[2 * s] / hres[2 * s + 1]) : 0.0;
        if (inf[s].status == SGP_ERR_NOT_SPD) rc = SGP_ERR_NOT_SPD;
        else if (inf[s].status && rc == SGP_OK) rc = (sgp_status)inf[s].status;
    }
    if (infos) std::memcpy(infos, inf.data(), sizeof(sgp_solve_info) * n_inst);
    if (rc == SGP_ERR_NOT_SPD) return sgp_fail(ctx, rc, "pcg_batched: breakdown in an instance");
    if (rc != SGP_OK) return sgp_fail(ctx, rc, "pcg_batched: an instance did not converge");
    return SGP_OK;
}

}  // extern "C"
