// graph.cu -- collision graph by a uniform cell list (Section 2, Steps 1-2).
//
// Cells i < j are in contact iff |r_j - r_i| < R_i + R_j.  The distance is
// evaluated with explicit round-to-nearest FP64 operations in a fixed order,
// sqrt((dx*dx + dy*dy) + dz*dz), so the result does not depend on the
// compiler's contraction choices.  Grid cells have side >= 2 max R, so every
// contact lies in one of the 27 grid cells around a cell's own.
//
// A batch of independent configurations (instances: contiguous index ranges)
// gets one grid per instance, laid end to end in one cell array, so cells of
// different instances are never candidates.  One configuration is the
// one-instance case.
//
// Output: canonical edge list (i < j), sorted by i then j, and the row
// pointer up_ptr of that "upper" adjacency.
#include "sgp_internal.cuh"

namespace {

// Bounding box, max radius and input validity of cells [b, e), reduced by
// one or more blocks: 8 values (-lo[3], hi[3], rmax, bad) per partial.
__device__ void bbox_block(const double *__restrict__ pos, const double *__restrict__ radii, int64_t b,
                           int64_t e, int64_t stride0, int64_t stride, double *out8)
{
    __shared__ double sh[SGP_BLOCK / 32];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double rmax = 0.0, bad = 0.0;
    for (int64_t i = b + stride0; i < e; i += stride) {
        double r = radii[i];
        if (!(r > 0.0) || !isfinite(r)) bad = 1.0;
        rmax = fmax(rmax, r);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double x = pos[3 * i + a];
            if (!isfinite(x)) bad = 1.0;
            lo[a] = fmin(lo[a], x);
            hi[a] = fmax(hi[a], x);
        }
    }
    // min as -max(-x)
    double vals[8] = {-lo[0], -lo[1], -lo[2], hi[0], hi[1], hi[2], rmax, bad};
    for (int q = 0; q < 8; ++q) {
        double v = vals[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = sh[0];
            for (int w = 1; w < SGP_BLOCK / 32; ++w) t = fmax(t, sh[w]);
            out8[q] = t;
        }
    }
}

// Many blocks over one range; the last block merges the partials.
__global__ void k_bbox(const double *__restrict__ pos, const double *__restrict__ radii, int64_t n,
                       double *partials, unsigned *counter, double *out)
{
    bbox_block(pos, radii, 0, n, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
               (int64_t)gridDim.x * blockDim.x, partials + 8 * blockIdx.x);
    if (last_block(counter)) {
        if (threadIdx.x < 8) {
            double t = -INFINITY;
            for (unsigned b = 0; b < gridDim.x; ++b) t = fmax(t, __ldcg(partials + 8 * b + threadIdx.x));
            out[threadIdx.x] = t;
        }
    }
}

// One block per instance.
__global__ void k_bbox_inst(const double *__restrict__ pos, const double *__restrict__ radii,
                            const int64_t *__restrict__ off, double *out)
{
    const int s = blockIdx.x;
    bbox_block(pos, radii, off[s], off[s + 1], threadIdx.x, blockDim.x, out + 8 * s);
}

struct Grid {
    double lo[3];
    double inv_h;
    int dim[3];
    int32_t base;   // first cell of this grid in the cell array
    float delta;    // bound on the FP32 distance error of the candidate filter
};

__global__ void k_inst_of(const int64_t *__restrict__ off, int32_t *inst)
{
    const int s = blockIdx.x;
    for (int64_t i = off[s] + threadIdx.x; i < off[s + 1]; i += blockDim.x) inst[i] = s;
}

__device__ __forceinline__ int cell_coord(double x, double lo, double inv_h, int dim)
{
    int c = (int)floor((x - lo) * inv_h);
    return c < 0 ? 0 : (c >= dim ? dim - 1 : c);
}

__global__ void k_cell_id(const double *__restrict__ pos, int64_t n, const Grid *__restrict__ grids,
                          const int32_t *__restrict__ inst, int32_t *cell_id, int32_t *cell_cnt)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Grid g = grids[inst ? inst[i] : 0];
    int cx = cell_coord(pos[3 * i + 0], g.lo[0], g.inv_h, g.dim[0]);
    int cy = cell_coord(pos[3 * i + 1], g.lo[1], g.inv_h, g.dim[1]);
    int cz = cell_coord(pos[3 * i + 2], g.lo[2], g.inv_h, g.dim[2]);
    int32_t c = g.base + (int32_t)(((int64_t)cx * g.dim[1] + cy) * g.dim[2] + cz);
    cell_id[i] = c;
    atomicAdd(cell_cnt + c, 1);
}

// Scatter cells into grid-cell order.  The order inside a grid cell is not
// deterministic; nothing downstream depends on it (rows are sorted).
__global__ void k_scatter(const double *__restrict__ pos, const double *__restrict__ radii, int64_t n,
                          const int32_t *__restrict__ cell_id, const int32_t *__restrict__ cell_start,
                          int32_t *cursor, int32_t *perm, double4_32a *spos, float4 *spos32)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = cell_id[i];
    int32_t s = cell_start[c] + atomicAdd(cursor + c, 1);
    perm[s] = (int32_t)i;
    spos[s] = make_double4_32a(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], radii[i]);
    spos32[s] = make_float4((float)pos[3 * i], (float)pos[3 * i + 1], (float)pos[3 * i + 2], (float)radii[i]);
}

// Order the cells inside each grid cell by index, which makes the grid-cell
// order (the solvers' internal cell order) deterministic.
__global__ void k_sort_cells(int64_t ncell, const int32_t *__restrict__ cell_start, int32_t *perm,
                             double4_32a *spos, float4 *spos32)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int32_t b0 = cell_start[c], k = cell_start[c + 1] - b0;
    for (int32_t a = 1; a < k; ++a) {
        const int32_t v = perm[b0 + a];
        const double4_32a p = spos[b0 + a];
        const float4 f = spos32[b0 + a];
        int32_t b = a - 1;
        while (b >= 0 && perm[b0 + b] > v) {
            perm[b0 + b + 1] = perm[b0 + b];
            spos[b0 + b + 1] = spos[b0 + b];
            spos32[b0 + b + 1] = spos32[b0 + b];
            --b;
        }
        perm[b0 + b + 1] = v;
        spos[b0 + b + 1] = p;
        spos32[b0 + b + 1] = f;
    }
}

__global__ void k_inverse_perm(int64_t n, const int32_t *__restrict__ perm, int32_t *inv)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) inv[perm[t]] = (int32_t)t;
}

// The contact predicate, with explicit round-to-nearest operations in the
// order sqrt((dx*dx + dy*dy) + dz*dz) < R_i + R_j, dx = x_j - x_i.
__device__ __forceinline__ bool contact(double4_32a pi, double4_32a pj)
{
    double dx = __dsub_rn(pj.x, pi.x);
    double dy = __dsub_rn(pj.y, pi.y);
    double dz = __dsub_rn(pj.z, pi.z);
    double s = __dmul_rn(dx, dx);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    double d = __dsqrt_rn(s);
    return d < __dadd_rn(pi.w, pj.w);
}

// One thread per cell (in grid-cell order).  EMIT = false: count the
// contacts j > i of cell i; EMIT = true: write them at up_ptr[i] and sort.
// MODE 0: count the contacts j > i of cell i; MODE 1: write them at
// up_ptr[i] and sort; MODE 2: count them and keep the first CAND in the
// cell's slot of `cand` (grid-cell order), flagging a cell with more.
constexpr int CAND = 24;

template <int MODE>
__global__ void k_contacts(int64_t n, const Grid *__restrict__ grids, const int32_t *__restrict__ inst,
                           const int32_t *__restrict__ perm, const double4_32a *__restrict__ spos,
                           const float4 *__restrict__ spos32, const int32_t *__restrict__ cell_start,
                           int32_t *cnt, const int32_t *__restrict__ up_ptr, int32_t *ij, int32_t *cand,
                           int *overflow)
{
    constexpr bool EMIT = MODE == 1;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t i = perm[t];
    const double4_32a pi = spos[t];
    const float4 fi = spos32[t];
    const Grid g = grids[inst ? inst[i] : 0];
    int cx = cell_coord(pi.x, g.lo[0], g.inv_h, g.dim[0]);
    int cy = cell_coord(pi.y, g.lo[1], g.inv_h, g.dim[1]);
    int cz = cell_coord(pi.z, g.lo[2], g.inv_h, g.dim[2]);
    int32_t k = 0;
    int64_t base = EMIT ? (int64_t)up_ptr[i] : 0;
    for (int ax = max(cx - 1, 0); ax <= min(cx + 1, g.dim[0] - 1); ++ax)
        for (int ay = max(cy - 1, 0); ay <= min(cy + 1, g.dim[1] - 1); ++ay) {
            int64_t row = g.base + ((int64_t)ax * g.dim[1] + ay) * g.dim[2];
            int z0 = max(cz - 1, 0), z1 = min(cz + 1, g.dim[2] - 1);
            // grid cells (ax, ay, z0..z1) are contiguous in grid-cell order
            int32_t s0 = cell_start[row + z0], s1 = cell_start[row + z1 + 1];
            for (int32_t s = s0; s < s1; ++s) {
                // FP32 filter: a pair farther apart than R_i + R_j + delta in
                // FP32 cannot be in contact (delta bounds the FP32 error);
                // every pair that passes is decided by the exact FP64 test
                const float4 fj = spos32[s];
                const float dx = fj.x - fi.x, dy = fj.y - fi.y, dz = fj.z - fi.z;
                const float lim = fi.w + fj.w + g.delta;
                if (dx * dx + dy * dy + dz * dz > lim * lim) continue;
                int32_t j = perm[s];
                if (j <= i) continue;
                if (contact(pi, spos[s])) {
                    if (EMIT) {
                        ij[2 * (base + k)] = i;
                        ij[2 * (base + k) + 1] = j;
                    }
                    if (MODE == 2 && k < CAND) cand[t * CAND + k] = j;
                    ++k;
                }
            }
        }
    if (!EMIT) {
        cnt[i] = k;
        if (MODE == 2 && k > CAND) atomicOr(overflow, 1);
    } else {
        // insertion sort of this row's j values
        for (int32_t a = 1; a < k; ++a) {
            int32_t v = ij[2 * (base + a) + 1];
            int32_t b = a - 1;
            while (b >= 0 && ij[2 * (base + b) + 1] > v) {
                ij[2 * (base + b + 1) + 1] = ij[2 * (base + b) + 1];
                --b;
            }
            ij[2 * (base + b + 1) + 1] = v;
        }
    }
}

// The kept candidates of each cell to its rows of the edge list, sorted.
__global__ void k_cand_copy(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ cnt,
                            const int32_t *__restrict__ up_ptr, const int32_t *__restrict__ cand, int32_t *ij)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t i = perm[t], k = cnt[i];
    const int64_t base = up_ptr[i];
    for (int32_t a = 0; a < k; ++a) {
        const int32_t v = cand[t * CAND + a];
        ij[2 * (base + a)] = i;
        int32_t b = a - 1;
        while (b >= 0 && ij[2 * (base + b) + 1] > v) {
            ij[2 * (base + b + 1) + 1] = ij[2 * (base + b) + 1];
            --b;
        }
        ij[2 * (base + b + 1) + 1] = v;
    }
}

// Grid of one instance from its bounding box: side >= 2 max R (with a margin
// against rounding of the cell index), at most max(2 n_s, 4096) cells.
// Cells whose index rounds up past floor(ext/h) are clamped into the last
// layer; the margin on h keeps every contact within the 27-cell stencil.
Grid make_grid(const double *hb, int64_t n_s, int64_t base)
{
    Grid g;
    double ext[3];
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = -hb[a];
        ext[a] = hb[3 + a] - g.lo[a];
    }
    double h = 2.0 * hb[6] * (1.0 + 1e-6);
    if (!(h > 0.0)) h = 1.0;
    const double max_cells = std::max<double>(2.0 * (double)n_s, 4096.0);
    for (;;) {
        double tot = 1.0;
        for (int a = 0; a < 3; ++a) tot *= std::floor(ext[a] / h) + 1.0;
        if (tot <= max_cells) break;
        h *= std::max(1.0001, std::cbrt(tot / max_cells));
    }
    g.inv_h = 1.0 / h;
    for (int a = 0; a < 3; ++a) g.dim[a] = (int)(std::floor(ext[a] / h) + 1.0);
    g.base = (int32_t)base;
    // |x_f - x| <= X 2^-24 per coordinate (X the largest coordinate
    // magnitude), so an FP32 difference is within 3 X 2^-24 of the exact one
    // and the FP32 distance within sqrt(3) of that plus a few roundings of
    // the distance and of R_i + R_j: 16 (X + 2 max R) 2^-24 covers all
    double X = 0.0;
    for (int a = 0; a < 3; ++a) X = std::max(X, std::max(std::fabs(hb[a]), std::fabs(hb[3 + a])));
    g.delta = (float)(16.0 * (X + 2.0 * hb[6]) * std::ldexp(1.0, -24));
    return g;
}

}  // namespace

// The collision graph of n_inst instances (offsets: n_inst + 1 host values).
static sgp_status collision_graph(sgp_ctx *ctx, int64_t n, int64_t n_inst, const int64_t *offsets,
                                  const double *pos, const double *radii, sgp_graph **out)
{
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    sgp_graph *G = *out ? *out : new sgp_graph();
    *out = G;
    G->n = n;
    G->m = 0;
    SGP_TRY(buf_ensure(ctx, G->up_ptr, sizeof(int32_t) * (size_t)(n + 1)));
    if (n == 0) {
        SGP_CUDA(ctx, cudaMemsetAsync(G->up_ptr.p, 0, sizeof(int32_t), ctx->stream));
        SGP_TRY(buf_ensure(ctx, G->ij, 16));
        return SGP_OK;
    }
    // bounding boxes, max radii, input validity
    std::vector<double> hb(8 * n_inst);
    int32_t *inst = nullptr;
    if (n_inst == 1) {
        const int bb_blocks = 296;
        SGP_TRY(buf_ensure(ctx, G->bbox, sizeof(double) * (8 * bb_blocks + 8) + 64));
        double *partials = bp<double>(G->bbox);
        double *bbout = partials + 8 * bb_blocks;
        unsigned *counter = reinterpret_cast<unsigned *>(bbout + 8);
        SGP_CUDA(ctx, cudaMemsetAsync(counter, 0, 64, ctx->stream));
        unsigned nb = (unsigned)std::min<int64_t>(bb_blocks, (n + SGP_BLOCK - 1) / SGP_BLOCK);
        LAUNCH(ctx, k_bbox, nb, SGP_BLOCK, 0, pos, radii, n, partials, counter, bbout);
        SGP_TRY(read_back(ctx, hb.data(), bbout, sizeof(double) * 8));
    } else {
        SGP_TRY(buf_ensure(ctx, G->bbox, sizeof(double) * 8 * n_inst + sizeof(int64_t) * (n_inst + 1) + 64));
        double *bbout = bp<double>(G->bbox);
        int64_t *doff = reinterpret_cast<int64_t *>(bbout + 8 * n_inst);
        SGP_CUDA(ctx, cudaMemcpyAsync(doff, offsets, sizeof(int64_t) * (n_inst + 1), cudaMemcpyHostToDevice,
                                      ctx->stream));
        LAUNCH(ctx, k_bbox_inst, (unsigned)n_inst, SGP_BLOCK, 0, pos, radii, (const int64_t *)doff, bbout);
        SGP_TRY(buf_ensure(ctx, G->inst, sizeof(int32_t) * n));
        inst = bp<int32_t>(G->inst);
        LAUNCH(ctx, k_inst_of, (unsigned)n_inst, SGP_BLOCK, 0, (const int64_t *)doff, inst);
        SGP_TRY(read_back(ctx, hb.data(), bbout, sizeof(double) * 8 * n_inst));
    }
    std::vector<Grid> grids(n_inst);
    int64_t ncell = 0;
    for (int64_t s = 0; s < n_inst; ++s) {
        const int64_t n_s = offsets[s + 1] - offsets[s];
        if (n_s == 0) {
            grids[s] = Grid{{0, 0, 0}, 1.0, {1, 1, 1}, (int32_t)ncell};
            ncell += 1;
            continue;
        }
        if (hb[8 * s + 7] != 0.0)
            return sgp_fail(ctx, SGP_ERR_INVALID_ARG,
                            "collision_graph: non-finite position or non-positive radius");
        grids[s] = make_grid(&hb[8 * s], n_s, ncell);
        ncell += (int64_t)grids[s].dim[0] * grids[s].dim[1] * grids[s].dim[2];
        if (ncell >= (int64_t(1) << 31) - 1)
            return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "collision_graph: too many grid cells");
    }
    SGP_TRY(buf_ensure(ctx, G->grids, sizeof(Grid) * n_inst));
    SGP_CUDA(ctx, cudaMemcpyAsync(G->grids.p, grids.data(), sizeof(Grid) * n_inst, cudaMemcpyHostToDevice,
                                  ctx->stream));
    const Grid *dgrids = bp<const Grid>(G->grids);
    SGP_TRY(buf_ensure(ctx, G->cell_id, sizeof(int32_t) * n));
    SGP_TRY(buf_ensure(ctx, G->cell_cnt, sizeof(int32_t) * (ncell + 1)));
    SGP_TRY(buf_ensure(ctx, G->cell_start, sizeof(int32_t) * (ncell + 1)));
    SGP_TRY(buf_ensure(ctx, G->perm, sizeof(int32_t) * n));
    SGP_TRY(buf_ensure(ctx, G->spos, sizeof(double4_32a) * n));
    SGP_TRY(buf_ensure(ctx, G->spos32, sizeof(float4) * n));
    SGP_TRY(buf_ensure(ctx, G->cnt, sizeof(int32_t) * (n + 1)));
    int32_t *cell_id = bp<int32_t>(G->cell_id), *cell_cnt = bp<int32_t>(G->cell_cnt);
    int32_t *cell_start = bp<int32_t>(G->cell_start), *perm = bp<int32_t>(G->perm);
    double4_32a *spos = bp<double4_32a>(G->spos);
    float4 *spos32 = bp<float4>(G->spos32);
    int32_t *cnt = bp<int32_t>(G->cnt), *up = bp<int32_t>(G->up_ptr);
    SGP_CUDA(ctx, cudaMemsetAsync(cell_cnt, 0, sizeof(int32_t) * (ncell + 1), ctx->stream));
    LAUNCH(ctx, k_cell_id, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, pos, n, dgrids, (const int32_t *)inst, cell_id,
           cell_cnt);
    SGP_TRY(scan_exclusive_i32(ctx, cell_cnt, cell_start, ncell));
    SGP_CUDA(ctx, cudaMemsetAsync(cell_cnt, 0, sizeof(int32_t) * (ncell + 1), ctx->stream));
    LAUNCH(ctx, k_scatter, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, pos, radii, n,
           (const int32_t *)cell_id, (const int32_t *)cell_start, cell_cnt, perm, spos, spos32);
    LAUNCH(ctx, k_sort_cells, grid_for(ncell, SGP_BLOCK), SGP_BLOCK, 0, ncell, (const int32_t *)cell_start, perm,
           spos, spos32);
    SGP_TRY(buf_ensure(ctx, G->int_of, sizeof(int32_t) * n));
    LAUNCH(ctx, k_inverse_perm, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, (const int32_t *)perm, bp<int32_t>(G->int_of));
    // one search: counts plus the first CAND contacts of each cell; a second
    // search (writing straight to the edge list) only if some cell has more
    SGP_TRY(buf_ensure(ctx, G->cand, sizeof(int32_t) * CAND * (size_t)n));
    int *ovf = ctx->d_flags + 20;
    SGP_CUDA(ctx, cudaMemsetAsync(ovf, 0, sizeof(int), ctx->stream));
    LAUNCH(ctx, k_contacts<2>, grid_for(n, 128), 128, 0, n, dgrids, (const int32_t *)inst,
           (const int32_t *)perm, (const double4_32a *)spos, (const float4 *)spos32, (const int32_t *)cell_start,
           cnt, (const int32_t *)nullptr, (int32_t *)nullptr, bp<int32_t>(G->cand), ovf);
    SGP_TRY(scan_exclusive_i32(ctx, cnt, up, n));
    SGP_CUDA(ctx, cudaMemcpyAsync(ovf + 1, up + n, sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    int32_t h[2] = {0, 0};
    SGP_TRY(read_back(ctx, h, ovf, sizeof(h)));
    const int32_t m32 = h[1];
    if (m32 < 0) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "collision_graph: edge count overflow");
    G->m = m32;
    SGP_TRY(buf_ensure(ctx, G->ij, sizeof(int32_t) * 2 * (size_t)G->m));
    if (h[0] == 0)
        LAUNCH(ctx, k_cand_copy, grid_for(n, 128), 128, 0, n, (const int32_t *)perm, (const int32_t *)cnt,
               (const int32_t *)up, (const int32_t *)bp<int32_t>(G->cand), bp<int32_t>(G->ij));
    else
        LAUNCH(ctx, k_contacts<1>, grid_for(n, 128), 128, 0, n, dgrids, (const int32_t *)inst,
               (const int32_t *)perm, (const double4_32a *)spos, (const float4 *)spos32,
               (const int32_t *)cell_start, cnt, (const int32_t *)up, bp<int32_t>(G->ij), (int32_t *)nullptr,
               (int *)nullptr);
    return SGP_OK;
}

extern "C" {

sgp_status sgp_collision_graph(sgp_ctx *ctx, int64_t n, const double *pos, const double *radii,
                               sgp_graph **out)
{
    if (!ctx || !out) return SGP_ERR_INVALID_ARG;
    if (n < 0 || n >= (int64_t(1) << 30) || (n > 0 && (!pos || !radii)))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "collision_graph: bad n=%lld or NULL input",
                        (long long)n);
    const int64_t off[2] = {0, n};
    return collision_graph(ctx, n, 1, off, pos, radii, out);
}

sgp_status sgp_collision_graph_batched(sgp_ctx *ctx, int64_t n_instances, const int64_t *offsets,
                                       const double *pos, const double *radii, sgp_graph **out)
{
    if (!ctx || !out || !offsets || n_instances < 1) return SGP_ERR_INVALID_ARG;
    if (offsets[0] != 0)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "collision_graph_batched: offsets[0] must be 0");
    for (int64_t s = 0; s < n_instances; ++s)
        if (offsets[s + 1] < offsets[s])
            return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "collision_graph_batched: offsets must not decrease");
    const int64_t n = offsets[n_instances];
    if (n >= (int64_t(1) << 30) || (n > 0 && (!pos || !radii)))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "collision_graph_batched: bad n=%lld or NULL input",
                        (long long)n);
    return collision_graph(ctx, n, n_instances, offsets, pos, radii, out);
}

sgp_status sgp_graph_info(const sgp_graph *G, int64_t *n, int64_t *m, const int32_t **ij)
{
    if (!G) return SGP_ERR_INVALID_ARG;
    if (n) *n = G->n;
    if (m) *m = G->m;
    if (ij) *ij = bp<const int32_t>(G->ij);
    return SGP_OK;
}

void sgp_graph_destroy(sgp_graph *G)
{
    if (!G) return;
    cudaDeviceSynchronize();
    DBuf *bufs[] = {&G->ij, &G->up_ptr, &G->cell_id, &G->cell_cnt, &G->cell_start, &G->perm,
                    &G->spos, &G->spos32, &G->cnt, &G->bbox, &G->inst, &G->grids, &G->int_of, &G->cand};
    for (DBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    delete G;
}

}  // extern "C"
