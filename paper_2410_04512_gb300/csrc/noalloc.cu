// noalloc.cu -- y = Gamma v together with v^T Gamma v, without allocating.
//
// For callers that cannot allocate device memory while they run: code that
// executes between a cudaStreamBeginCapture and its end (allocation calls are
// not allowed there), hosts whose device memory is handed out by their own
// pool and must not be touched by a library, or real-time loops that forbid
// the synchronisation cudaMalloc/cudaFree imply.  The library's regular calls
// grow their workspace with cudaMallocAsync; this one uses only the
// fixed-size array below, which is part of the library image.
//
// The scratch -- one FP64 partial sum per thread block and the arrival
// counter of the last-block reduction -- lives in a file-scope __device__
// array of SGP_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds
// this array until the process exits.  All calls share it and it keeps the
// last call's contents; the counter is cleared at the start of every call.
// Calls whose GPU work overlaps (two streams, or two host threads) race on the
// array and must not be issued.
#include "sgp_internal.cuh"

namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_MAX_BLOCKS = 4096;
// 4096 partial sums + a 256-byte slot for the counter
constexpr size_t NA_SCRATCH_BYTES = NA_MAX_BLOCKS * sizeof(double) + 256;
static_assert(NA_SCRATCH_BYTES == 33024, "stated scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];


// Internal row r (cell orig_of[r]) of the Appendix B.2 product, same
// operation order as the solver's.  v is in the caller's cell order: the
// matrix's rows and columns are mapped through orig_of, so no permuted copy
// (and no workspace) is needed.
__device__ __forceinline__ void na_row(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                       const double *__restrict__ blk, const int32_t *__restrict__ orig_of,
                                       double gamma0, const double *__restrict__ v, int64_t r, int64_t i,
                                       double *vi, double *y)
{
    vi[0] = v[3 * i]; vi[1] = v[3 * i + 1]; vi[2] = v[3 * i + 2];
    y[0] = gamma0 * vi[0]; y[1] = gamma0 * vi[1]; y[2] = gamma0 * vi[2];
    int32_t s1 = row_ptr[r + 1];
    for (int32_t s = row_ptr[r]; s < s1; ++s) {
        const double2 *b2 = reinterpret_cast<const double2 *>(blk + 6 * (int64_t)s);
        double2 a = b2[0], b = b2[1], c = b2[2];
        double S[6] = {a.x, a.y, b.x, b.y, c.x, c.y};
        int32_t j = orig_of[col[s]];
        double d[3] = {vi[0] - v[3 * (int64_t)j], vi[1] - v[3 * (int64_t)j + 1], vi[2] - v[3 * (int64_t)j + 2]};
        double t[3];
        sym_mv(S, d, t);
        y[0] += t[0]; y[1] += t[1]; y[2] += t[2];
    }
}

// One thread per row; one partial per block in the scratch array; the last
// block to arrive sums the partials in block order and writes *dot.
__global__ void k_spmv_dot_noalloc(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                   const double *__restrict__ blk, const int32_t *__restrict__ orig_of,
                                   double gamma0, int64_t n, const double *__restrict__ v, double *y, double *dot,
                                   unsigned char *scratch)
{
    __shared__ double sh[NA_BLOCK / 32];
    double *partials = reinterpret_cast<double *>(scratch);
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + NA_MAX_BLOCKS * sizeof(double));
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (r < n) {
        const int64_t i = orig_of[r];
        double vi[3], yi[3];
        na_row(row_ptr, col, blk, orig_of, gamma0, v, r, i, vi, yi);
        y[3 * i] = yi[0]; y[3 * i + 1] = yi[1]; y[3 * i + 2] = yi[2];
        acc = vi[0] * yi[0] + vi[1] * yi[1] + vi[2] * yi[2];
    }
    double s = block_sum<NA_BLOCK>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(counter)) {
        double tot = sum_partials<NA_BLOCK>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) *dot = tot;
    }
}

}  // namespace

// Device address of the scratch array, looked up when a context is created
// (sgp_create, outside any capture) and kept in the context: a device reset
// ends every context, so no address outlives the CUDA context it came from.
sgp_status noalloc_prepare(sgp_ctx *ctx)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return sgp_fail(ctx, SGP_ERR_CUDA, "noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    }
    ctx->noalloc_scratch = p;
    return SGP_OK;
}

extern "C" {

sgp_status sgp_spmv_dot_noalloc(sgp_ctx *ctx, const sgp_matrix *M, const double *v, double *y,
                                double *dot)
{
    if (!ctx || !M || !dot || (M->n > 0 && (!v || !y)))
        return ctx ? sgp_fail(ctx, SGP_ERR_INVALID_ARG, "spmv_dot_noalloc: NULL argument")
                   : SGP_ERR_INVALID_ARG;
    if (v == y) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "spmv_dot_noalloc: v and y must differ");
    const int64_t n = M->n;
    const int64_t max_n = (int64_t)NA_MAX_BLOCKS * NA_BLOCK;
    if (n > max_n)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG,
                        "spmv_dot_noalloc: %lld cells exceed the fixed scratch limit of %lld cells",
                        (long long)n, (long long)max_n);
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    if (!ctx->noalloc_scratch) return sgp_fail(ctx, SGP_ERR_CUDA, "spmv_dot_noalloc: scratch address unknown");
    unsigned char *base = reinterpret_cast<unsigned char *>(ctx->noalloc_scratch);
    SGP_CUDA(ctx, cudaMemsetAsync(base + NA_MAX_BLOCKS * sizeof(double), 0, sizeof(unsigned), ctx->stream));
    if (n == 0) {
        SGP_CUDA(ctx, cudaMemsetAsync(dot, 0, sizeof(double), ctx->stream));
        return SGP_OK;
    }
    LAUNCH(ctx, k_spmv_dot_noalloc, grid_for(n, NA_BLOCK), NA_BLOCK, 0, bp<const int32_t>(M->row_ptr),
           bp<const int32_t>(M->col), bp<const double>(M->blk), bp<const int32_t>(M->orig_of), M->gamma0, n, v, y,
           dot, base);
    return SGP_OK;
}

}  // extern "C"
