// assemble.cu -- friction blocks and the block-sparse matrix (Section 2,
// Step 3, eq. (1); Definition "Block Laplacian").
//
// For every contact e = (i, j) (i < j):
//   u = (r_j - r_i) / |r_j - r_i|,
//   Upsilon_e = g_par (u u^T) + g_perp (I - u u^T)        (eq. (1), A_ij folded in)
// evaluated entry by entry as (g_par * (u_a u_b)) + (g_perp * (delta_ab - u_a u_b))
// with explicit round-to-nearest FP64 operations.  The matrix stores, per
// directed slot of each block row, the column and the symmetric block
// (Gamma_ij = -Upsilon_e); the diagonal is never assembled -- products use the
// difference form of Appendix B.2.  Rows and columns follow the solvers'
// internal cell order (the collision graph's grid-cell order); columns are
// ascending within a row.
#include "sgp_internal.cuh"

namespace {

// Rows and columns in the solvers' internal cell order (int_of): every edge
// gives a slot in both of its rows.
__global__ void k_slot_count(const int32_t *__restrict__ ij, int64_t m, const int32_t *__restrict__ int_of,
                             int32_t *cnt)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    atomicAdd(cnt + int_of[ij[2 * e]], 1);
    atomicAdd(cnt + int_of[ij[2 * e + 1]], 1);
}

__global__ void k_slot_place(const int32_t *__restrict__ ij, int64_t m, const int32_t *__restrict__ int_of,
                             const int32_t *__restrict__ row_ptr, int32_t *cursor, int32_t *col,
                             int32_t *slot_edge)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t a = int_of[ij[2 * e]], b = int_of[ij[2 * e + 1]];
    const int32_t sa = row_ptr[a] + atomicAdd(cursor + a, 1);
    const int32_t sb = row_ptr[b] + atomicAdd(cursor + b, 1);
    col[sa] = b;
    slot_edge[sa] = (int32_t)e;
    col[sb] = a;
    slot_edge[sb] = (int32_t)e;
}

// Sort each row by column (makes the layout deterministic) and record, for
// every edge (i, j), its slot in row int_of[i] and in row int_of[j].
__global__ void k_sort_rows(const int32_t *__restrict__ row_ptr, int64_t n, const int32_t *__restrict__ ij,
                            const int32_t *__restrict__ int_of, int32_t *col, int32_t *slot_edge,
                            int32_t *edge_slot, int32_t *edge_slot_j)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t b0 = row_ptr[r], k = row_ptr[r + 1] - b0;
    for (int32_t a = 1; a < k; ++a) {
        const int32_t c = col[b0 + a], se = slot_edge[b0 + a];
        int32_t b = a - 1;
        while (b >= 0 && col[b0 + b] > c) {
            col[b0 + b + 1] = col[b0 + b];
            slot_edge[b0 + b + 1] = slot_edge[b0 + b];
            --b;
        }
        col[b0 + b + 1] = c;
        slot_edge[b0 + b + 1] = se;
    }
    for (int32_t a = 0; a < k; ++a) {
        const int32_t e = slot_edge[b0 + a];
        if (int_of[ij[2 * e]] == (int32_t)r) edge_slot[e] = b0 + a;
        else edge_slot_j[e] = b0 + a;
    }
}

// Coefficient check and the spanning-tree weight of every edge.
__global__ void k_edge_weight(int64_t m, const double *__restrict__ gpar, const double *__restrict__ gperp,
                              double *w, int *err)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    const double a = gpar[e], b = gperp[e];
    if (!(a > 0.0) || !(b > 0.0) || !isfinite(a) || !isfinite(b)) atomicOr(err, 1);
    w[e] = a < b ? a : b;  // lambda_min of the block (Lemma 2.1)
}

// eq. (1) for each edge, written to its two slots (row i and row j carry the
// same symmetric block).
__global__ void k_blocks(const int32_t *__restrict__ ij, const double *__restrict__ pos,
                         const double *__restrict__ gpar, const double *__restrict__ gperp,
                         const int32_t *__restrict__ edge_slot, const int32_t *__restrict__ edge_slot_j,
                         const int32_t *__restrict__ col, int64_t m, int64_t nslot, double *blk, float *blk32,
                         int *err)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    int32_t i = ij[2 * e], j = ij[2 * e + 1];
    double dx = __dsub_rn(pos[3 * j + 0], pos[3 * i + 0]);
    double dy = __dsub_rn(pos[3 * j + 1], pos[3 * i + 1]);
    double dz = __dsub_rn(pos[3 * j + 2], pos[3 * i + 2]);
    double q = __dmul_rn(dx, dx);
    q = __dadd_rn(q, __dmul_rn(dy, dy));
    q = __dadd_rn(q, __dmul_rn(dz, dz));
    double d = __dsqrt_rn(q);
    if (!(d > 0.0)) {
        atomicOr(err, 2);
        d = 1.0;
    }
    double u[3] = {__ddiv_rn(dx, d), __ddiv_rn(dy, d), __ddiv_rn(dz, d)};
    double gp = gpar[e], gq = gperp[e];
    double out[6];
    const int ra[6] = {0, 0, 0, 1, 1, 2}, rb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        double uu = __dmul_rn(u[ra[k]], u[rb[k]]);
        double id = (ra[k] == rb[k]) ? 1.0 : 0.0;
        out[k] = __dadd_rn(__dmul_rn(gp, uu), __dmul_rn(gq, __dsub_rn(id, uu)));
    }
    const int64_t sl[2] = {edge_slot[e], edge_slot_j[e]};
    const float4 r4 = make_float4((float)gq, (float)__dsub_rn(gp, gq), (float)u[0], (float)u[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t s = sl[h];
        double2 *o2 = reinterpret_cast<double2 *>(blk + 6 * s);
        o2[0] = make_double2(out[0], out[1]);
        o2[1] = make_double2(out[2], out[3]);
        o2[2] = make_double2(out[4], out[5]);
        if (blk32) {   // eq. (1) form: (g_perp, g_par - g_perp, u) and the column
            reinterpret_cast<float4 *>(blk32)[s] = r4;
            reinterpret_cast<float2 *>(blk32 + 4 * nslot)[s] = make_float2((float)u[2], __int_as_float(col[s]));
        }
    }
}

// Expand the block of each edge (slot (i, j) in row i) to 9 entries.
__global__ void k_edge_blocks(const int32_t *__restrict__ edge_slot, const double *__restrict__ blk,
                              int64_t m, double *out)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    const double *S = blk + 6 * (int64_t)edge_slot[e];
    double *o = out + 9 * e;
    o[0] = S[0]; o[1] = S[1]; o[2] = S[2];
    o[3] = S[1]; o[4] = S[3]; o[5] = S[4];
    o[6] = S[2]; o[7] = S[4]; o[8] = S[5];
}

// Block-Jacobi: inverse of Gamma_ii = gamma0 I + sum_j Upsilon_ij.
__global__ void k_block_jacobi(const int32_t *__restrict__ row_ptr, const double *__restrict__ blk,
                               int64_t n, double gamma0, double *jac, float *jac32, int *err)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double S[6] = {gamma0, 0.0, 0.0, gamma0, 0.0, gamma0};
    for (int32_t s = row_ptr[i]; s < row_ptr[i + 1]; ++s)
#pragma unroll
        for (int k = 0; k < 6; ++k) S[k] += blk[6 * (int64_t)s + k];
    double R[6];
    if (!sym_inv(S, R)) {
        atomicOr(err, 4);
        R[0] = R[3] = R[5] = 1.0;
        R[1] = R[2] = R[4] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        jac[6 * i + k] = R[k];
        if (jac32) jac32[6 * i + k] = (float)R[k];
    }
}

}  // namespace

sgp_status matrix_block_jacobi(sgp_ctx *ctx, sgp_matrix *M)
{
    if (M->jac_valid) return SGP_OK;
    int64_t n = M->n;
    SGP_TRY(buf_ensure(ctx, M->jac, sizeof(double) * 6 * (size_t)std::max<int64_t>(n, 1)));
    float *j32 = nullptr;
    if (M->precision == SGP_PREC_MIXED) {
        SGP_TRY(buf_ensure(ctx, M->jac32, sizeof(float) * 6 * (size_t)std::max<int64_t>(n, 1)));
        j32 = bp<float>(M->jac32);
    }
    int *err = ctx->d_flags;
    SGP_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    LAUNCH(ctx, k_block_jacobi, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, bp<const int32_t>(M->row_ptr),
           bp<const double>(M->blk), n, M->gamma0, bp<double>(M->jac), j32, err);
    int herr = 0;
    SGP_TRY(read_back(ctx, &herr, err, sizeof(int)));
    if (herr) return sgp_fail(ctx, SGP_ERR_NOT_SPD, "block Jacobi: a diagonal block is not SPD");
    M->jac_valid = 1;
    return SGP_OK;
}

extern "C" {

sgp_status sgp_friction_assemble(sgp_ctx *ctx, const sgp_graph *G, const double *pos,
                                 const double *gpar, const double *gperp, double gamma0,
                                 int32_t precision, sgp_matrix **out)
{
    if (!ctx || !G || !out) return SGP_ERR_INVALID_ARG;
    const int64_t n = G->n, m = G->m;
    if ((n > 0 && !pos) || (m > 0 && (!gpar || !gperp)))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "friction_assemble: NULL input");
    if (!(gamma0 > 0.0) || !std::isfinite(gamma0))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "friction_assemble: gamma0 must be positive");
    if (precision != SGP_PREC_F64 && precision != SGP_PREC_MIXED)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "friction_assemble: bad precision");
    if (2 * m >= (int64_t(1) << 31))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "friction_assemble: too many edges");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    sgp_matrix *M = *out ? *out : new sgp_matrix();
    *out = M;
    M->n = n;
    M->m = m;
    M->gamma0 = gamma0;
    M->precision = precision;
    M->jac_valid = 0;
    M->gen = next_generation();
    const int64_t ns = 2 * m;
    SGP_TRY(buf_ensure(ctx, M->ij, sizeof(int32_t) * 2 * m));
    SGP_TRY(buf_ensure(ctx, M->row_ptr, sizeof(int32_t) * (n + 1)));
    SGP_TRY(buf_ensure(ctx, M->col, sizeof(int32_t) * ns));
    SGP_TRY(buf_ensure(ctx, M->blk, sizeof(double) * 6 * ns));
    SGP_TRY(buf_ensure(ctx, M->edge_slot, sizeof(int32_t) * m));
    SGP_TRY(buf_ensure(ctx, M->edge_slot_j, sizeof(int32_t) * std::max<int64_t>(m, 1)));
    SGP_TRY(buf_ensure(ctx, M->w, sizeof(double) * m));
    SGP_TRY(buf_ensure(ctx, M->slot_edge, sizeof(int32_t) * ns));
    SGP_TRY(buf_ensure(ctx, M->lowcnt, sizeof(int32_t) * (n + 1)));
    SGP_TRY(buf_ensure(ctx, M->cursor, sizeof(int32_t) * (n + 1)));
    float *blk32 = nullptr;
    if (precision == SGP_PREC_MIXED) {
        SGP_TRY(buf_ensure(ctx, M->blk32, sizeof(float) * 6 * std::max<int64_t>(ns, 1)));
        blk32 = bp<float>(M->blk32);
    }
    if (m > 0)
        SGP_CUDA(ctx, cudaMemcpyAsync(M->ij.p, G->ij.p, sizeof(int32_t) * 2 * m,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    int32_t *cnt = bp<int32_t>(M->lowcnt), *cursor = bp<int32_t>(M->cursor);
    int32_t *row_ptr = bp<int32_t>(M->row_ptr), *col = bp<int32_t>(M->col);
    int32_t *slot_edge = bp<int32_t>(M->slot_edge), *edge_slot = bp<int32_t>(M->edge_slot);
    const int32_t *ij = bp<const int32_t>(M->ij);
    // the internal cell order of the graph
    SGP_TRY(buf_ensure(ctx, M->orig_of, sizeof(int32_t) * std::max<int64_t>(n, 1)));
    SGP_TRY(buf_ensure(ctx, M->int_of, sizeof(int32_t) * std::max<int64_t>(n, 1)));
    if (n > 0) {
        SGP_CUDA(ctx, cudaMemcpyAsync(M->orig_of.p, G->perm.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
        SGP_CUDA(ctx, cudaMemcpyAsync(M->int_of.p, G->int_of.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    }
    const int32_t *int_of = bp<const int32_t>(M->int_of);
    int *err = ctx->d_flags;
    SGP_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (n + 1), ctx->stream));
    LAUNCH(ctx, k_slot_count, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, ij, m, int_of, cnt);
    SGP_TRY(scan_exclusive_i32(ctx, cnt, row_ptr, n));
    LAUNCH(ctx, k_slot_place, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, ij, m, int_of, (const int32_t *)row_ptr, cursor,
           col, slot_edge);
    int32_t *edge_slot_j = bp<int32_t>(M->edge_slot_j);
    LAUNCH(ctx, k_sort_rows, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, (const int32_t *)row_ptr, n, ij, int_of, col,
           slot_edge, edge_slot, edge_slot_j);
    LAUNCH(ctx, k_edge_weight, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, m, gpar, gperp, bp<double>(M->w), err);
    LAUNCH(ctx, k_blocks, grid_for(m, SGP_BLOCK), SGP_BLOCK, 0, ij, pos, gpar, gperp,
           (const int32_t *)edge_slot, (const int32_t *)edge_slot_j, (const int32_t *)col, m, ns,
           bp<double>(M->blk), blk32, err);
    int herr = 0;
    SGP_TRY(read_back(ctx, &herr, err, sizeof(int)));
    if (herr & 1)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG,
                        "friction_assemble: friction coefficients must be positive and finite");
    if (herr & 2)
        return sgp_fail(ctx, SGP_ERR_DEGENERATE,
                        "friction_assemble: two cells in contact share a centre");
    return SGP_OK;
}

sgp_status sgp_matrix_edge_blocks(sgp_ctx *ctx, const sgp_matrix *M, double *blocks, double *w)
{
    if (!ctx || !M) return SGP_ERR_INVALID_ARG;
    if (blocks)
        LAUNCH(ctx, k_edge_blocks, grid_for(M->m, SGP_BLOCK), SGP_BLOCK, 0,
               bp<const int32_t>(M->edge_slot), bp<const double>(M->blk), M->m, blocks);
    if (w && M->m > 0)
        SGP_CUDA(ctx, cudaMemcpyAsync(w, M->w.p, sizeof(double) * M->m, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    return SGP_OK;
}

void sgp_matrix_destroy(sgp_matrix *M)
{
    if (!M) return;
    cudaDeviceSynchronize();
    DBuf *bufs[] = {&M->ij, &M->row_ptr, &M->col, &M->blk, &M->blk32, &M->edge_slot, &M->w,
                    &M->slot_edge, &M->lowcnt, &M->cursor, &M->jac, &M->jac32, &M->orig_of, &M->int_of,
                    &M->edge_slot_j};
    for (DBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    delete M;
}

}  // extern "C"
