// api.cu -- context, errors, device buffers, scans and kernel timing.
#include "sgp_internal.cuh"

#include <atomic>
#include <cstdlib>

sgp_status sgp_fail(sgp_ctx *ctx, sgp_status code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

sgp_status buf_ensure(sgp_ctx *ctx, DBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return SGP_OK;
    if (b.p) {
        cudaFreeAsync(b.p, ctx->stream);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = (bytes + 255) & ~size_t(255);
    cudaError_t e = cudaMallocAsync(&b.p, want, ctx->stream);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return sgp_fail(ctx, SGP_ERR_OOM, "device allocation of %zu bytes failed: %s", want,
                        cudaGetErrorString(e));
    }
    b.bytes = want;
    return SGP_OK;
}

void buf_release(DBuf &b, cudaStream_t s)
{
    if (b.p) cudaFreeAsync(b.p, s);
    b.p = nullptr;
    b.bytes = 0;
}

sgp_status scratch_ensure(sgp_ctx *ctx, size_t bytes)
{
    if (ctx->d_scratch && ctx->d_scratch_bytes >= bytes) return SGP_OK;
    if (ctx->d_scratch) cudaFreeAsync(ctx->d_scratch, ctx->stream);
    ctx->d_scratch = nullptr;
    size_t want = (bytes + 4095) & ~size_t(4095);
    cudaError_t e = cudaMallocAsync(&ctx->d_scratch, want, ctx->stream);
    if (e != cudaSuccess) {
        ctx->d_scratch = nullptr;
        ctx->d_scratch_bytes = 0;
        cudaGetLastError();
        return sgp_fail(ctx, SGP_ERR_OOM, "scratch allocation of %zu bytes failed", want);
    }
    SGP_CUDA(ctx, cudaMemsetAsync(ctx->d_scratch, 0, want, ctx->stream));
    ctx->d_scratch_bytes = want;
    return SGP_OK;
}

sgp_status read_back(sgp_ctx *ctx, void *host, const void *dev, size_t bytes)
{
    if (bytes > ctx->h_stage_bytes) {
        if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        size_t want = bytes < 4096 ? 4096 : bytes;
        SGP_CUDA(ctx, cudaMallocHost(&ctx->h_stage, want));
        ctx->h_stage_bytes = want;
    }
    SGP_CUDA(ctx, cudaMemcpyAsync(ctx->h_stage, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    memcpy(host, ctx->h_stage, bytes);
    SGP_TRY(kt_collect(ctx));
    return SGP_OK;
}

// ---------------------------------------------------------------------------
// exclusive scan (int32): per-block scans, a recursive scan of the block
// totals, then a uniform add.  1024 items per block of 256 threads.
// ---------------------------------------------------------------------------
#define SCAN_ITEMS 4
#define SCAN_TILE (SGP_BLOCK * SCAN_ITEMS)

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *sh, int32_t *total)
{
    int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (l >= o) x += y;
    }
    if (l == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t t = (l < SGP_BLOCK / 32) ? sh[l] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (l >= o) t += y;
        }
        if (l < SGP_BLOCK / 32) sh[l] = t;
    }
    __syncthreads();
    int32_t before = (w > 0 ? sh[w - 1] : 0) + x - v;
    *total = sh[SGP_BLOCK / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_tiles(const int32_t *in, int32_t *out, int32_t *tile_sums, int64_t n)
{
    __shared__ int32_t sh[SGP_BLOCK / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t run = block_excl_scan(s, sh, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(int32_t *out, const int32_t *tile_off, int64_t n)
{
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t add = tile_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) out[base + k] += add;
}

__global__ void k_scan_total(const int32_t *in, int32_t *out, int64_t n)
{
    // out[n] = out[n-1] + in[n-1] (in is read before out is overwritten when
    // they alias: the caller saves the last input first)
    if (threadIdx.x == 0 && blockIdx.x == 0) out[n] = (n > 0 ? out[n - 1] + in[0] : 0);
}

static sgp_status scan_rec(sgp_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int32_t *work)
{
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *sums = work;  // tiles + 1 entries
    LAUNCH(ctx, k_scan_tiles, (unsigned)tiles, SGP_BLOCK, 0, in, out, sums, n);
    if (tiles > 1) {
        SGP_TRY(scan_rec(ctx, sums, sums, tiles, work + tiles + 1));
        LAUNCH(ctx, k_scan_add, (unsigned)tiles, SGP_BLOCK, 0, out, (const int32_t *)sums, n);
    }
    return SGP_OK;
}

sgp_status scan_exclusive_i32(sgp_ctx *ctx, const int32_t *in, int32_t *out, int64_t n)
{
    if (n <= 0) {
        SGP_CUDA(ctx, cudaMemsetAsync(out, 0, sizeof(int32_t), ctx->stream));
        return SGP_OK;
    }
    // workspace for all recursion levels, plus one slot to save in[n-1]
    int64_t need = 8, t = n;
    while (t > 1) { t = (t + SCAN_TILE - 1) / SCAN_TILE; need += t + 1; }
    const size_t bytes = (size_t)(need + 64) * sizeof(int32_t) + 4096;
    if (!ctx->d_scan || ctx->d_scan_bytes < bytes) {
        if (ctx->d_scan) cudaFreeAsync(ctx->d_scan, ctx->stream);
        ctx->d_scan = nullptr;
        ctx->d_scan_bytes = 0;
        size_t want = std::max<size_t>(bytes, size_t(1) << 18);
        SGP_CUDA(ctx, cudaMallocAsync(&ctx->d_scan, want, ctx->stream));
        ctx->d_scan_bytes = want;
    }
    int32_t *work = reinterpret_cast<int32_t *>(ctx->d_scan) + 16;
    int32_t *last = reinterpret_cast<int32_t *>(ctx->d_scan) + 8;
    SGP_CUDA(ctx, cudaMemcpyAsync(last, in + (n - 1), sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    SGP_TRY(scan_rec(ctx, in, out, n, work));
    LAUNCH(ctx, k_scan_total, 1, 32, 0, (const int32_t *)last, out, n);
    return SGP_OK;
}

// ---------------------------------------------------------------------------
// kernel timing
// ---------------------------------------------------------------------------
static cudaEvent_t ev_get(sgp_ctx *ctx)
{
    if (!ctx->ev_free.empty()) {
        cudaEvent_t e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

sgp_status kt_begin(sgp_ctx *ctx, int kclass, cudaEvent_t *ev)
{
    *ev = nullptr;
    if (!ctx->timing) return SGP_OK;
    if (ctx->capture_sink) {
        // inside a capture: an event-record node owned by the graph entry
        SGP_CUDA(ctx, cudaEventCreate(ev));
        SGP_CUDA(ctx, cudaEventRecordWithFlags(*ev, ctx->stream, cudaEventRecordExternal));
        return SGP_OK;
    }
    *ev = ev_get(ctx);
    SGP_CUDA(ctx, cudaEventRecord(*ev, ctx->stream));
    return SGP_OK;
}

sgp_status kt_end(sgp_ctx *ctx, int kclass, cudaEvent_t start)
{
    if (!ctx->timing || !start) return SGP_OK;
    if (ctx->capture_sink) {
        cudaEvent_t e = nullptr;
        SGP_CUDA(ctx, cudaEventCreate(&e));
        SGP_CUDA(ctx, cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal));
        ctx->capture_sink->push_back(KtRec{kclass, start, e});
        return SGP_OK;
    }
    cudaEvent_t e = ev_get(ctx);
    SGP_CUDA(ctx, cudaEventRecord(e, ctx->stream));
    ctx->ev_pending[kclass].push_back(start);
    ctx->ev_pending[kclass].push_back(e);
    return SGP_OK;
}

sgp_status resident_grid(sgp_ctx *ctx, const void *kernel, int block, int64_t want, unsigned *grid)
{
    if (!ctx->num_sms) SGP_CUDA(ctx, cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    int per_sm = 0;
    for (auto &kv : ctx->occupancy)
        if (kv.first == kernel) per_sm = kv.second;
    if (!per_sm) {
        SGP_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0));
        per_sm = std::max(per_sm, 1);
        ctx->occupancy.push_back({kernel, per_sm});
    }
    int64_t cap = (int64_t)ctx->num_sms * per_sm;
    *grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, cap));
    return SGP_OK;
}

// ---------------------------------------------------------------------------
// CUDA graph cache
// ---------------------------------------------------------------------------
uint64_t next_generation()
{
    static std::atomic<uint64_t> g{1};
    return g.fetch_add(1);
}

static void graph_free(GraphEntry *ge)
{
    if (ge->exec) cudaGraphExecDestroy(ge->exec);
    for (auto &r : ge->ev) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete ge;
}

void graph_release_all(sgp_ctx *ctx)
{
    for (GraphEntry *ge : ctx->graphs) graph_free(ge);
    ctx->graphs.clear();
}

sgp_status graph_lookup(sgp_ctx *ctx, const uint64_t *key, int nkey, GraphEntry **out)
{
    if (nkey > 32) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "graph key too long");
    ++ctx->graph_clock;
    for (GraphEntry *ge : ctx->graphs)
        if (ge->nkey == nkey && std::memcmp(ge->key, key, sizeof(uint64_t) * nkey) == 0) {
            ge->last_use = ctx->graph_clock;
            *out = ge;
            return SGP_OK;
        }
    const size_t max_entries = 6;
    if (ctx->graphs.size() >= max_entries) {
        auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                    [](GraphEntry *a, GraphEntry *b) { return a->last_use < b->last_use; });
        SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        graph_free(*lru);
        ctx->graphs.erase(lru);
    }
    GraphEntry *ge = new GraphEntry();
    std::memcpy(ge->key, key, sizeof(uint64_t) * nkey);
    ge->nkey = nkey;
    ge->last_use = ctx->graph_clock;
    ctx->graphs.push_back(ge);
    *out = ge;
    return SGP_OK;
}

sgp_status graph_begin(sgp_ctx *ctx, GraphEntry *ge, cudaStream_t *saved, int64_t *l0)
{
    if (!ctx->cap_stream) SGP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    *saved = ctx->stream;
    *l0 = ctx->launches;
    SGP_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    ctx->stream = ctx->cap_stream;
    ctx->capture_sink = &ge->ev;
    return SGP_OK;
}

sgp_status graph_end(sgp_ctx *ctx, GraphEntry *ge, cudaStream_t saved, int64_t l0, sgp_status st)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->stream = saved;
    ctx->capture_sink = nullptr;
    ge->kernels = ctx->launches - l0;
    ctx->launches = l0;
    if (st != SGP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess || !g)
        return sgp_fail(ctx, SGP_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ge->exec = nullptr;
        return sgp_fail(ctx, SGP_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return SGP_OK;
}

__global__ void k_while_cond(cudaGraphConditionalHandle h, const int *done, int *bodies, int max_bodies)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int b = *bodies + 1;
        *bodies = b;
        cudaGraphSetConditional(h, (*done == 0 && b < max_bodies) ? 1u : 0u);
    }
}

sgp_status graph_while_begin(sgp_ctx *ctx, GraphEntry *ge, cudaStream_t *saved, int64_t *l0, cudaGraph_t *g,
                             cudaGraphConditionalHandle *h)
{
    if (!ctx->cap_stream) SGP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    SGP_CUDA(ctx, cudaGraphCreate(g, 0));
    cudaError_t e = cudaGraphConditionalHandleCreate(h, *g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp{};
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = *h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, *g, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(ctx->cap_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(*g);
        *g = nullptr;
        return sgp_fail(ctx, SGP_ERR_CUDA, "conditional graph setup failed: %s", cudaGetErrorString(e));
    }
    *saved = ctx->stream;
    *l0 = ctx->launches;
    ctx->stream = ctx->cap_stream;
    ctx->capture_sink = nullptr;
    return SGP_OK;
}

sgp_status graph_while_end(sgp_ctx *ctx, GraphEntry *ge, cudaStream_t saved, int64_t l0, cudaGraph_t g,
                           cudaGraphConditionalHandle h, const int *done, int *bodies, int max_bodies,
                           sgp_status st)
{
    if (st == SGP_OK) {
        k_while_cond<<<1, 32, 0, ctx->cap_stream>>>(h, done, bodies, max_bodies);
        ctx->launches++;
    }
    cudaGraph_t body = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &body);
    if (e == cudaSuccess) e = cudaGetLastError();
    ctx->stream = saved;
    ge->kernels = ctx->launches - l0;
    ctx->launches = l0;
    if (st != SGP_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        if (st != SGP_OK) return st;
        return sgp_fail(ctx, SGP_ERR_CUDA, "conditional graph capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&ge->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ge->exec = nullptr;
        cudaGetLastError();
        return sgp_fail(ctx, SGP_ERR_CUDA, "conditional graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return SGP_OK;
}

// After a replay has completed (the caller synchronised): add the replay's
// event-pair durations to the kernel-time totals.
sgp_status graph_collect_timing(sgp_ctx *ctx, GraphEntry *ge)
{
    if (!ctx->timing) return SGP_OK;
    for (auto &r : ge->ev) {
        float ms = 0.f;
        SGP_CUDA(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
        ctx->kt_ms[r.cls] += ms;
        ctx->kt_n[r.cls] += 1;
    }
    return SGP_OK;
}

sgp_status kt_collect(sgp_ctx *ctx)
{
    for (int k = 0; k < SGP_KT_COUNT; ++k) {
        auto &v = ctx->ev_pending[k];
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            float ms = 0.f;
            SGP_CUDA(ctx, cudaEventElapsedTime(&ms, v[i], v[i + 1]));
            ctx->kt_ms[k] += ms;
            ctx->kt_n[k] += 1;
            ctx->ev_free.push_back(v[i]);
            ctx->ev_free.push_back(v[i + 1]);
        }
        v.clear();
    }
    return SGP_OK;
}

// ---------------------------------------------------------------------------
// C ABI: context
// ---------------------------------------------------------------------------
extern "C" {

const char *sgp_version(void) { return "sgp 0.1 sm_103a"; }

sgp_status sgp_create(sgp_ctx **out, int device, void *stream)
{
    if (!out) return SGP_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SGP_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SGP_ERR_CUDA;
    sgp_ctx *ctx = new sgp_ctx();
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    const char *ng = getenv("SGP_NO_GRAPHS");
    ctx->use_graphs = (ng && ng[0] == '1') ? 0 : 1;
    const char *lpr = getenv("SGP_SPMV_LPR");
    if (lpr) ctx->spmv_lpr = atoi(lpr);
    const char *nw = getenv("SGP_NO_WHILE");
    ctx->use_while = (nw && nw[0] == '1') ? 0 : 1;
    const char *np = getenv("SGP_NO_PDL");
    ctx->use_pdl = (np && np[0] == '1') ? 0 : 1;
    const char *tc = getenv("SGP_TAIL_CAP");
    if (tc) ctx->tail_cap = atoi(tc);
    const char *bc = getenv("SGP_BIN_CAP");
    if (bc) ctx->bin_cap = atoi(bc);
    const char *ns = getenv("SGP_NO_SMALL");
    if (ns && atoi(ns)) ctx->small_solve = 0;
    const char *nf = getenv("SGP_NO_FUSE");
    if (nf && atoi(nf)) ctx->fused = 0;
    if (scratch_ensure(ctx, 1 << 20) != SGP_OK || cudaMalloc(&ctx->d_flags, 4096) != cudaSuccess ||
        cudaMemset(ctx->d_flags, 0, 4096) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_scratch) cudaFree(ctx->d_scratch);
        delete ctx;
        return SGP_ERR_OOM;
    }
    if (noalloc_prepare(ctx) != SGP_OK) {
        cudaFree(ctx->d_scratch);
        cudaFree(ctx->d_flags);
        delete ctx;
        return SGP_ERR_CUDA;
    }
    *out = ctx;
    return SGP_OK;
}

void sgp_destroy(sgp_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    graph_release_all(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->d_scratch) cudaFree(ctx->d_scratch);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    if (ctx->d_scan) cudaFree(ctx->d_scan);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    for (auto e : ctx->ev_free) cudaEventDestroy(e);
    for (int k = 0; k < SGP_KT_COUNT; ++k)
        for (auto e : ctx->ev_pending[k]) cudaEventDestroy(e);
    delete ctx;
}

const char *sgp_last_error(const sgp_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

sgp_status sgp_copy(sgp_ctx *ctx, void *dst, const void *src, int64_t bytes)
{
    if (!ctx || bytes < 0 || (bytes > 0 && (!dst || !src))) return SGP_ERR_INVALID_ARG;
    if (bytes == 0) return SGP_OK;
    SGP_CUDA(ctx, cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return SGP_OK;
}

sgp_status sgp_set_kernel_timing(sgp_ctx *ctx, int32_t enable)
{
    if (!ctx) return SGP_ERR_INVALID_ARG;
    ctx->timing = enable ? 1 : 0;
    return SGP_OK;
}

sgp_status sgp_kernel_time(sgp_ctx *ctx, int32_t kclass, double *total_ms, int64_t *launches,
                           int32_t reset)
{
    if (!ctx || kclass < 0 || kclass >= SGP_KT_COUNT) return SGP_ERR_INVALID_ARG;
    SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    SGP_TRY(kt_collect(ctx));
    if (total_ms) *total_ms = ctx->kt_ms[kclass];
    if (launches) *launches = ctx->kt_n[kclass];
    if (reset) {
        ctx->kt_ms[kclass] = 0;
        ctx->kt_n[kclass] = 0;
    }
    return SGP_OK;
}

sgp_status sgp_launch_count(sgp_ctx *ctx, int64_t *count, int32_t reset)
{
    if (!ctx) return SGP_ERR_INVALID_ARG;
    if (count) *count = ctx->launches;
    if (reset) ctx->launches = 0;
    return SGP_OK;
}

}  // extern "C"
