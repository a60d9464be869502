// tune.cu -- the autotuner: picks the lanes per block row of the PCG
// product, the launch shape of the tree solve (how many of the last
// contraction levels run in one thread block, and the size of the subtrees
// that one thread block solves in the binned layout) and the rows per work
// item of the batched solver, by timing the caller's own system for each
// candidate.
// The paper has no counterpart (its solver runs on one CPU core).
#include "sgp_internal.cuh"

namespace {

struct Run {
    sgp_ctx *ctx;
    const sgp_matrix *M;
    const sgp_factor *const *Fh;
    int64_t n_inst;
    const int64_t *offsets;
    const double *F;
    double *v;
    sgp_solve_opts opts;
    cudaEvent_t e0, e1;

    // One untimed solve (graph capture, caches), then one timed solve;
    // returns milliseconds per iteration, or per solve when `whole` is set
    // (the time then includes `extra_ms`, the factor build of the candidate).
    bool whole = false;
    double extra_ms = 0.0;
    sgp_status time_it(double *ms_per_it)
    {
        double best = 0.0;
        for (int rep = 0; rep < 2; ++rep) {
            SGP_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
            int64_t its = 0;
            sgp_status st;
            if (n_inst > 0) {
                std::vector<sgp_solve_info> inf((size_t)n_inst);
                st = sgp_pcg_solve_batched(ctx, M, *Fh, n_inst, offsets, F, v, &opts, inf.data());
                for (auto &i : inf) its = std::max<int64_t>(its, i.iterations);
            } else {
                sgp_solve_info inf{};
                st = sgp_pcg_solve(ctx, M, *Fh, F, v, &opts, &inf);
                its = inf.iterations;
            }
            if (st != SGP_OK && st != SGP_ERR_NO_CONVERGENCE) return st;
            SGP_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
            SGP_CUDA(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            SGP_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
            best = whole ? (double)ms + extra_ms : (double)ms / (double)std::max<int64_t>(its, 1);
        }
        *ms_per_it = best;
        return SGP_OK;
    }
};

}  // namespace

extern "C" {

sgp_status sgp_get_tuning(const sgp_ctx *ctx, sgp_tuning *t)
{
    if (!ctx || !t) return SGP_ERR_INVALID_ARG;
    t->spmv_lpr = ctx->spmv_lpr;
    t->tail_cap = ctx->tail_cap;
    t->batch_chunk = ctx->batch_chunk;
    t->spmv_ilp = ctx->spmv_ilp;
    t->bin_cap = ctx->bin_cap;
    t->ms_per_iteration = 0.0;
    return SGP_OK;
}

sgp_status sgp_set_tuning(sgp_ctx *ctx, const sgp_tuning *t)
{
    if (!ctx || !t) return SGP_ERR_INVALID_ARG;
    if (!(t->spmv_lpr == 0 || t->spmv_lpr == 1 || t->spmv_lpr == 2 || t->spmv_lpr == 4 || t->spmv_lpr == 8))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "set_tuning: spmv_lpr must be 0, 1, 2, 4 or 8");
    if (t->tail_cap < -1) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "set_tuning: tail_cap must be >= -1");
    if (t->spmv_ilp < 0 || t->spmv_ilp > 2)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "set_tuning: spmv_ilp must be 0, 1 or 2");
    if (t->batch_chunk != 0 && (t->batch_chunk < 256 || t->batch_chunk > 65536))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "set_tuning: batch_chunk must be 0 or in [256, 65536]");
    if (!(t->bin_cap == 0 || t->bin_cap == -1 || (t->bin_cap >= 64 && t->bin_cap <= 8192)))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "set_tuning: bin_cap must be 0, -1 or in [64, 8192]");
    ctx->spmv_lpr = t->spmv_lpr;
    ctx->bin_cap = t->bin_cap;
    ctx->tail_cap = t->tail_cap;
    ctx->spmv_ilp = t->spmv_ilp;
    ctx->batch_chunk = t->batch_chunk;
    return SGP_OK;
}

sgp_status sgp_autotune(sgp_ctx *ctx, const sgp_matrix *M, const sgp_tree *T, sgp_factor **factor,
                        int64_t n_instances, const int64_t *offsets, const double *F,
                        const sgp_solve_opts *opts, int32_t iterations, sgp_tuning *out)
{
    if (!ctx || !M || !opts || !F) return SGP_ERR_INVALID_ARG;
    if (iterations < 0 || iterations > 100000)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "autotune: iterations must be in [0, 100000]");
    const bool tree = opts->precond == SGP_PRECOND_TREE;
    if (tree && (!T || !factor || !*factor))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "autotune: the tree preconditioner needs the tree and a factor");
    if (n_instances > 0 && !offsets) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "autotune: offsets missing");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = M->n;
    if (n == 0) {
        if (out) SGP_TRY(sgp_get_tuning(ctx, out));
        return SGP_OK;
    }
    double *v = nullptr;
    SGP_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void **>(&v), sizeof(double) * 3 * n, ctx->stream));
    const sgp_factor *no_factor = nullptr;
    Run run{ctx, M, factor ? factor : &no_factor, n_instances, offsets, F, v, *opts, nullptr, nullptr};
    if (iterations > 0) {
        run.opts.tol = 1e-300;      // never met: every timed solve runs exactly `iterations`
        run.opts.maxit = iterations;
    } else {
        run.whole = true;           // whole solves to opts->tol, plus the factor build
    }
    run.opts.x0_given = 0;
    // factor build timed with events (its host synchronisations included)
    auto build = [&]() -> sgp_status {
        SGP_CUDA(ctx, cudaEventRecord(run.e0, ctx->stream));
        SGP_TRY(sgp_tree_factor(ctx, M, T, factor));
        SGP_CUDA(ctx, cudaEventRecord(run.e1, ctx->stream));
        SGP_CUDA(ctx, cudaEventSynchronize(run.e1));
        float ms = 0.f;
        SGP_CUDA(ctx, cudaEventElapsedTime(&ms, run.e0, run.e1));
        run.extra_ms = ms;
        return SGP_OK;
    };
    sgp_tuning keep{};
    sgp_get_tuning(ctx, &keep);
    sgp_status st = SGP_OK;
    double best_ms = 0.0;
    auto finish = [&](sgp_status s) {
        if (run.e0) cudaEventDestroy(run.e0);
        if (run.e1) cudaEventDestroy(run.e1);
        cudaFreeAsync(v, ctx->stream);
        if (s != SGP_OK) sgp_set_tuning(ctx, &keep);
        return s;
    };
    if (cudaEventCreate(&run.e0) != cudaSuccess || cudaEventCreate(&run.e1) != cudaSuccess)
        return finish(sgp_fail(ctx, SGP_ERR_CUDA, "autotune: event creation failed"));

    // 1. tail size, then bin size (each candidate rebuilds the factor)
    if (tree) {
        auto pick = [&](int *knob, const int *cand, int nc) -> sgp_status {
            int best = *knob;
            best_ms = 1e300;
            for (int k = 0; k < nc; ++k) {
                *knob = cand[k];
                SGP_TRY(build());
                double ms;
                SGP_TRY(run.time_it(&ms));
                if (ms < best_ms) best_ms = ms, best = cand[k];
            }
            *knob = best;
            return SGP_OK;
        };
        const int caps[] = {0, 256, 512, 1024, 2048, 4096, -1};
        if ((st = pick(&ctx->tail_cap, caps, 7)) != SGP_OK) return finish(st);
        const int bins[] = {0, -1, 512, 1024, 2048};
        if ((st = pick(&ctx->bin_cap, bins, 5)) != SGP_OK) return finish(st);
        if ((st = build()) != SGP_OK) return finish(st);
    }
    // 2. lanes per block row of the product and rows in flight per lane
    {
        const int lprs[] = {1, 2, 4, 8};
        int best_lpr = ctx->spmv_lpr, best_ilp = ctx->spmv_ilp;
        best_ms = 1e300;
        for (int ilp = 1; ilp <= (n_instances > 0 ? 1 : 2); ++ilp)
            for (int lpr : lprs) {
                if (n_instances > 0 && lpr == 8) continue;   // the batched product stops at 4
                ctx->spmv_lpr = lpr;
                ctx->spmv_ilp = ilp;
                double ms;
                if ((st = run.time_it(&ms)) != SGP_OK) return finish(st);
                if (ms < best_ms) best_ms = ms, best_lpr = lpr, best_ilp = ilp;
            }
        ctx->spmv_lpr = best_lpr;
        ctx->spmv_ilp = best_ilp;
    }
    // 3. rows per work item of the batched solver
    if (n_instances > 0) {
        const int chunks[] = {512, 1024, 2048, 4096, 8192};
        int best_ch = ctx->batch_chunk;
        best_ms = 1e300;
        for (int ch : chunks) {
            ctx->batch_chunk = ch;
            double ms;
            if ((st = run.time_it(&ms)) != SGP_OK) return finish(st);
            if (ms < best_ms) best_ms = ms, best_ch = ch;
        }
        ctx->batch_chunk = best_ch;
    }
    if (out) {
        sgp_get_tuning(ctx, out);
        out->ms_per_iteration = best_ms;
    }
    return finish(SGP_OK);
}

}  // extern "C"
