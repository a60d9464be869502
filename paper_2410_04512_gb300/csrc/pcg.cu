// pcg.cu -- products with Gamma and preconditioned conjugate gradients
// (Section 1.1; Appendix B.2 for the product).
//
// y = Gamma v is evaluated in the difference form of Appendix B.2,
//   y_i = gamma0 v_i + sum_{j ~ i} Upsilon_ij (v_i - v_j),
// which annihilates rigid translations exactly and never forms the diagonal
// block (whose FP32 rounding would swamp a small gamma0).
//
// PCG scalars (rho, alpha, beta, convergence) live on the device; each
// reduction kernel ends with a "last block" step that sums the per-block
// partials in a fixed order and updates them, so no host round trip is
// needed per iteration and results are bitwise reproducible.  Iterations run
// as a device-side loop (a conditional WHILE graph node over chunks of 4) or,
// with per-kernel timing on, as replayed chunk graphs with the host polling
// the `done` word between chunks.
#include "solver_common.cuh"
#include "tail.cuh"

namespace {

constexpr int RB = 256;        // block size of reduction kernels
constexpr int MAXP = 4096;     // max blocks (partials) of a reduction kernel

// y_i of the Appendix B.2 product for row i
template <typename T>
__device__ __forceinline__ void row_product(const Blk<T> &B, const int32_t *__restrict__ row_ptr,
                                            T gamma0, const T *__restrict__ v, int64_t i, T *vi, T *y)
{
    vi[0] = v[3 * i]; vi[1] = v[3 * i + 1]; vi[2] = v[3 * i + 2];
    y[0] = gamma0 * vi[0]; y[1] = gamma0 * vi[1]; y[2] = gamma0 * vi[2];
    int32_t s1 = row_ptr[i + 1];
    for (int32_t s = row_ptr[i]; s < s1; ++s) {
        T S[6];
        int32_t j;
        B.load(s, S, j);
        T d[3] = {vi[0] - v[3 * (int64_t)j], vi[1] - v[3 * (int64_t)j + 1], vi[2] - v[3 * (int64_t)j + 2]};
        T t[3];
        sym_mv(S, d, t);
        y[0] += t[0]; y[1] += t[1]; y[2] += t[2];
    }
}

// y = Gamma v  (plain)
template <typename T>
__global__ void k_spmv(Blk<T> B, const int32_t *__restrict__ row_ptr, T gamma0, int64_t n,
                       const T *__restrict__ v, T *y)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T vi[3], yi[3];
    row_product(B, row_ptr, gamma0, v, i, vi, yi);
    y[3 * i] = yi[0]; y[3 * i + 1] = yi[1]; y[3 * i + 2] = yi[2];
}

// PCG product q = Gamma p with p^T q; the last block sets alpha = rho / p^T q.
// LPR lanes share a block row: lane g takes the row's slots g, g+LPR, ...,
// so a warp's 16-byte block loads cover a contiguous stretch of the slot
// array; the lanes' partial sums meet by shuffles.  The difference form is
// accumulated with fused multiply-adds (9 FMA + 3 subtractions per slot).
// Loops are warp-uniform so the shuffles always see all 32 lanes.
// ILP row groups are in flight per lane at once (their slot loads and
// gathers interleave), which hides the block-load -> gather latency chain.
template <typename T, int LPR, int ILP>
__global__ void __launch_bounds__(RB, sizeof(T) == 4 ? (ILP == 1 ? 6 : 4) : (ILP == 1 ? 4 : 2)) k_spmv_pq(Blk<T> B, const int32_t *__restrict__ row_ptr, T gamma0,
                                                int64_t n, const T *__restrict__ p, T *q, double *partials,
                                                Scal *sc)
{
    __shared__ double sh[RB / 32];
    if (sc->done) return;
    constexpr int RPW = 32 / LPR;  // rows per warp per sweep
    const int lane = threadIdx.x & 31, g = lane % LPR;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t stride = nwarps * RPW;
    double acc = 0.0;
    for (int64_t base = warp * RPW; base < n; base += ILP * stride) {
        int64_t i[ILP];
        bool active[ILP];
        T y0[ILP], y1[ILP], y2[ILP], v0[ILP], v1[ILP], v2[ILP];
        int32_t s[ILP], e[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            i[u] = base + u * stride + lane / LPR;
            active[u] = i[u] < n;
            y0[u] = y1[u] = y2[u] = v0[u] = v1[u] = v2[u] = 0;
            s[u] = e[u] = 0;
            if (active[u]) {
                v0[u] = p[3 * i[u]]; v1[u] = p[3 * i[u] + 1]; v2[u] = p[3 * i[u] + 2];
                s[u] = row_ptr[i[u]] + g;
                e[u] = row_ptr[i[u] + 1];
            }
        }
        // each lane's next slot record is loaded while the current slot's
        // gather and products run
        typename Blk<T>::Raw R[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u)
            if (s[u] < e[u]) R[u] = B.fetch(s[u]);
        bool more = true;
        while (more) {
            more = false;
            T S[ILP][6];
            int32_t j[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (s[u] < e[u]) B.expand(R[u], S[u], j[u]);
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (s[u] + LPR < e[u]) R[u] = B.fetch(s[u] + LPR);
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (s[u] < e[u]) {
                    const T d0 = v0[u] - p[3 * (int64_t)j[u]], d1 = v1[u] - p[3 * (int64_t)j[u] + 1],
                            d2 = v2[u] - p[3 * (int64_t)j[u] + 2];
                    y0[u] = fma(S[u][0], d0, y0[u]); y0[u] = fma(S[u][1], d1, y0[u]); y0[u] = fma(S[u][2], d2, y0[u]);
                    y1[u] = fma(S[u][1], d0, y1[u]); y1[u] = fma(S[u][3], d1, y1[u]); y1[u] = fma(S[u][4], d2, y1[u]);
                    y2[u] = fma(S[u][2], d0, y2[u]); y2[u] = fma(S[u][4], d1, y2[u]); y2[u] = fma(S[u][5], d2, y2[u]);
                    s[u] += LPR;
                    more = more || s[u] < e[u];
                }
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) {
                y0[u] += __shfl_xor_sync(0xffffffffu, y0[u], o);
                y1[u] += __shfl_xor_sync(0xffffffffu, y1[u], o);
                y2[u] += __shfl_xor_sync(0xffffffffu, y2[u], o);
            }
            if (active[u]) {
                const T a0 = fma(gamma0, v0[u], y0[u]);
                const T a1 = fma(gamma0, v1[u], y1[u]);
                const T a2 = fma(gamma0, v2[u], y2[u]);
                if (LPR >= 3) {
                    if (g < 3) q[3 * i[u] + g] = g == 0 ? a0 : (g == 1 ? a1 : a2);
                } else if (g == 0) {
                    q[3 * i[u]] = a0; q[3 * i[u] + 1] = a1; q[3 * i[u] + 2] = a2;
                }
                // the row's three products are summed in T, the running sum
                // in FP64 (one conversion per row keeps FP32 rows off the
                // FP64 pipe)
                if (g == 0) acc += (double)fma(v0[u], a0, fma(v1[u], a1, v2[u] * a2));
            }
        }
    }
    double s = block_sum<RB>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->cnt)) {
        double pq = sum_partials<RB>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->pq = pq;
            if (!(pq > 0.0) || !isfinite(pq)) {
                sc->status = SGP_ERR_NOT_SPD;
                sc->done = 1;
            } else {
                sc->alpha = sc->rho / pq;
                sc->xpend = 1;
            }
        }
    }
}

// Start of a solve: r = F - Gamma x (or r = F when x starts at 0), w = H r
// for the diagonal preconditioners (w = r for the tree, applied after),
// |F|^2 and |r|^2; the last block sets the stopping threshold.
// PREC: 0 tree (w = r), 1 block Jacobi, 2 none.
template <typename T, int PREC>
__global__ void k_init(Blk<T> B, const int32_t *__restrict__ row_ptr, T gamma0, int64_t n,
                       const T *__restrict__ F, const T *__restrict__ x, int x_given, T *r, T *w,
                       const T *__restrict__ jac, double tol2, long long maxit, double *partials,
                       Scal *sc, double mu, int stopE, double tolE2)
{
    __shared__ double sh[RB / 32];
    double ff = 0.0, rr = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T ri[3] = {F[3 * i], F[3 * i + 1], F[3 * i + 2]};
        ff += (double)ri[0] * ri[0] + (double)ri[1] * ri[1] + (double)ri[2] * ri[2];
        if (x_given) {
            T vi[3], yi[3];
            row_product(B, row_ptr, gamma0, x, i, vi, yi);
            ri[0] -= yi[0]; ri[1] -= yi[1]; ri[2] -= yi[2];
        }
        rr += (double)ri[0] * ri[0] + (double)ri[1] * ri[1] + (double)ri[2] * ri[2];
        r[3 * i] = ri[0]; r[3 * i + 1] = ri[1]; r[3 * i + 2] = ri[2];
        T zi[3] = {ri[0], ri[1], ri[2]};
        if (PREC == 1) sym_mv(jac + 6 * i, ri, zi);
        w[3 * i] = zi[0]; w[3 * i + 1] = zi[1]; w[3 * i + 2] = zi[2];
    }
    double s1 = block_sum<RB>(ff, sh);
    if (threadIdx.x == 0) partials[2 * blockIdx.x] = s1;
    double s2 = block_sum<RB>(rr, sh);
    if (threadIdx.x == 0) partials[2 * blockIdx.x + 1] = s2;
    if (last_block(&sc->cnt)) {
        double a = 0.0, b = 0.0;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += RB) {
            a += __ldcg(partials + 2 * k);
            b += __ldcg(partials + 2 * k + 1);
        }
        a = block_sum<RB>(a, sh);
        b = block_sum<RB>(b, sh);
        if (threadIdx.x == 0) {
            sc->FF = a;
            sc->rr = b;
            sc->stop2 = tol2 * a;
            sc->it = 0;
            sc->maxit = maxit;
            sc->status = 0;
            sc->done = (a == 0.0 || b <= tol2 * a) ? 1 : 0;
            sc->mu = mu;
            sc->phi = mu > 0.0 ? 1.0 / mu : 0.0;
            sc->gsum = 0.0;
            sc->est = 0.0;
            sc->stopE = stopE;
            sc->tolE2 = tolE2;
        }
    }
}

// rho = r^T w, p = w (after the first preconditioner application)
template <typename T>
__global__ void k_rz_init(int64_t n, const T *__restrict__ r, const T *__restrict__ w, T *p,
                          double *partials, Scal *sc)
{
    __shared__ double sh[RB / 32];
    if (sc->done) return;
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 3 * n;
         k += (int64_t)gridDim.x * blockDim.x) {
        T wk = w[k];
        acc += (double)r[k] * (double)wk;
        p[k] = wk;
    }
    double s = block_sum<RB>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->cnt)) {
        double rz = sum_partials<RB>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->rho = rz;
            sc->rz = rz;
            sc->est = sc->phi * rz;
            if (!(rz > 0.0) || !isfinite(rz)) {
                sc->status = SGP_ERR_NOT_SPD;
                sc->done = 1;
            }
        }
    }
}

// x += alpha p, r -= alpha q, then w = H r (PREC 1, 2) or w = r (PREC 0);
// |r|^2 (and r^T w for PREC 1, 2).  Last block: iteration count,
// convergence test, and for PREC 1, 2 also beta and rho.
template <typename T, typename X, int PREC>
__global__ void k_update(int64_t n, X *x, const T *__restrict__ p, T *r, const T *__restrict__ q, T *w,
                         const T *__restrict__ jac, double *partials, Scal *sc)
{
    __shared__ double sh[RB / 32];
    if (sc->done) return;
    const double alpha = sc->alpha;
    const T a = (T)alpha;
    double rr = 0.0, rz = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T ri[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int64_t k = 3 * i + c;
            x[k] += (X)alpha * (X)p[k];
            ri[c] = r[k] - a * q[k];
            r[k] = ri[c];
            rr += (double)ri[c] * (double)ri[c];
        }
        T zi[3] = {ri[0], ri[1], ri[2]};
        if (PREC == 1) sym_mv(jac + 6 * i, ri, zi);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w[3 * i + c] = zi[c];
            rz += (double)ri[c] * (double)zi[c];
        }
    }
    double s1 = block_sum<RB>(rr, sh);
    if (threadIdx.x == 0) partials[2 * blockIdx.x] = s1;
    double s2 = block_sum<RB>(rz, sh);
    if (threadIdx.x == 0) partials[2 * blockIdx.x + 1] = s2;
    if (last_block(&sc->cnt)) {
        double A = 0.0, Bz = 0.0;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += RB) {
            A += __ldcg(partials + 2 * k);
            Bz += __ldcg(partials + 2 * k + 1);
        }
        A = block_sum<RB>(A, sh);
        Bz = block_sum<RB>(Bz, sh);
        if (threadIdx.x == 0) {
            sc->rr = A;
            sc->it += 1;
            if (A <= sc->stop2) sc->done = 1;
            else if (sc->it >= sc->maxit) {
                sc->done = 1;
                sc->status = SGP_ERR_NO_CONVERGENCE;
            } else if (PREC != 0) {
                rz_finish(sc, Bz);
            }
        }
    }
}

// x += alpha p, r -= alpha q, w = r, |r|^2 (tree and identity
// preconditioners, which need no per-cell block), 16-byte accesses.
template <typename T, int PREC>
__global__ void __launch_bounds__(RB) k_update_v(int64_t n, T *x, const T *__restrict__ p, T *r,
                                                 const T *__restrict__ q, T *w, double *partials, Scal *sc)
{
    __shared__ double sh[RB / 32];
    if (sc->done) return;
    constexpr int K = Pack<T>::K;
    const T a = (T)sc->alpha;
    const int64_t n3 = 3 * n, np = n3 / K;
    const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    double rr = 0.0;
    for (int64_t i = g0; i < np; i += gs) {
        Pack<T> pv = reinterpret_cast<const Pack<T> *>(p)[i];
        Pack<T> qv = reinterpret_cast<const Pack<T> *>(q)[i];
        Pack<T> rv = reinterpret_cast<const Pack<T> *>(r)[i];
        Pack<T> xv = reinterpret_cast<const Pack<T> *>(x)[i];
        T s = 0;
#pragma unroll
        for (int e = 0; e < K; ++e) {
            xv.v[e] = fma(a, pv.v[e], xv.v[e]);
            rv.v[e] = fma(-a, qv.v[e], rv.v[e]);
            s = fma(rv.v[e], rv.v[e], s);
        }
        rr += (double)s;  // pack sums in T, running sum in FP64
        reinterpret_cast<Pack<T> *>(x)[i] = xv;
        reinterpret_cast<Pack<T> *>(r)[i] = rv;
        reinterpret_cast<Pack<T> *>(w)[i] = rv;
    }
    for (int64_t k = np * K + g0; k < n3; k += gs) {
        x[k] = fma(a, p[k], x[k]);
        T rk = fma(-a, q[k], r[k]);
        r[k] = rk;
        w[k] = rk;
        rr += (double)rk * (double)rk;
    }
    double s1 = block_sum<RB>(rr, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s1;
    if (last_block(&sc->cnt)) {
        double A = sum_partials<RB>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->rr = A;
            sc->it += 1;
            if (A <= sc->stop2) sc->done = 1;
            else if (sc->it >= sc->maxit) {
                sc->done = 1;
                sc->status = SGP_ERR_NO_CONVERGENCE;
            } else if (PREC != 0) {  // identity: z = r, so r^T z = |r|^2
                rz_finish(sc, A);
            }
        }
    }
}

// rho' = r^T w after the tree solve; beta = rho'/rho.
template <typename T>
__global__ void __launch_bounds__(RB, sizeof(T) == 4 ? 8 : 4) k_rz(int64_t n, const T *__restrict__ r, const T *__restrict__ w,
                                           double *partials, Scal *sc)
{
    __shared__ double sh[RB / 32];
    if (sc->done) return;
    constexpr int K = Pack<T>::K;
    const int64_t n3 = 3 * n, np = n3 / K;
    const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (int64_t i = g0; i < np; i += gs) {
        Pack<T> a = reinterpret_cast<const Pack<T> *>(r)[i];
        Pack<T> b = reinterpret_cast<const Pack<T> *>(w)[i];
        T s = 0;
#pragma unroll
        for (int e = 0; e < K; ++e) s = fma(a.v[e], b.v[e], s);
        acc += (double)s;  // pack sums in T, running sum in FP64
    }
    for (int64_t k = np * K + g0; k < n3; k += gs) acc += (double)r[k] * (double)w[k];
    double s = block_sum<RB>(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->cnt)) {
        double rz = sum_partials<RB>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) rz_finish(sc, rz);
    }
}

// p = w + beta p
template <typename T>
__global__ void __launch_bounds__(RB, sizeof(T) == 4 ? 6 : 4) k_pupd(int64_t n, const T *__restrict__ w, T *p, const Scal *sc)
{
    if (sc->done) return;
    constexpr int K = Pack<T>::K;
    const T beta = (T)sc->beta;
    const int64_t n3 = 3 * n, np = n3 / K;
    const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = g0; i < np; i += gs) {
        Pack<T> a = reinterpret_cast<const Pack<T> *>(w)[i];
        Pack<T> b = reinterpret_cast<const Pack<T> *>(p)[i];
#pragma unroll
        for (int e = 0; e < K; ++e) b.v[e] = fma(beta, b.v[e], a.v[e]);
        reinterpret_cast<Pack<T> *>(p)[i] = b;
    }
    for (int64_t k = np * K + g0; k < n3; k += gs) p[k] = fma(beta, p[k], w[k]);
}

// End of a fused PCG step (after the binned tree solve has set beta, or
// stopped): x += alpha p, and p = z + beta p while the solve goes on.  Runs
// once per step: the last block clears the pending flag that the product set.
template <typename T>
__global__ void __launch_bounds__(RB) k_pupd_x(int64_t n, T *x, T *p, const T *__restrict__ z, Scal *sc)
{
    if (!sc->xpend) return;
    constexpr int K = Pack<T>::K;
    const T a = (T)sc->alpha, beta = (T)sc->beta;
    const bool live = !sc->done;
    const int64_t n3 = 3 * n, np = n3 / K;
    const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = g0; i < np; i += gs) {
        Pack<T> xv = reinterpret_cast<const Pack<T> *>(x)[i];
        Pack<T> pv = reinterpret_cast<const Pack<T> *>(p)[i];
        Pack<T> zv = reinterpret_cast<const Pack<T> *>(z)[i];
#pragma unroll
        for (int e = 0; e < K; ++e) {
            xv.v[e] = fma(a, pv.v[e], xv.v[e]);
            pv.v[e] = fma(beta, pv.v[e], zv.v[e]);
        }
        reinterpret_cast<Pack<T> *>(x)[i] = xv;
        if (live) reinterpret_cast<Pack<T> *>(p)[i] = pv;
    }
    for (int64_t k = np * K + g0; k < n3; k += gs) {
        const T pk = p[k];
        x[k] = fma(a, pk, x[k]);
        if (live) p[k] = fma(beta, pk, z[k]);
    }
    if (last_block(&sc->cnt) && threadIdx.x == 0) sc->xpend = 0;
}

// FP64 residual r = F - Gamma x with |r|^2 and |F|^2 (exit check, outer loop)
// ZX: the iterate is zero, so r = F without the product.
template <bool ZX>
__global__ void __launch_bounds__(RB) k_resid64(Blk<double> B, const int32_t *__restrict__ row_ptr, double gamma0,
                                                int64_t n, const double *__restrict__ F,
                                                const double *__restrict__ x, double *r, double *partials,
                                                double *out2)
{
    __shared__ double sh[RB / 32];
    double rr = 0.0, ff = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double vi[3], yi[3] = {0.0, 0.0, 0.0};
        if (!ZX) row_product(B, row_ptr, gamma0, x, i, vi, yi);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double f = F[3 * i + c];
            double rc = f - yi[c];
            if (r) r[3 * i + c] = rc;
            rr += rc * rc;
            ff += f * f;
        }
    }
    double s1 = block_sum<RB>(rr, sh);
    if (threadIdx.x == 0) partials[2 * blockIdx.x] = s1;
    double s2 = block_sum<RB>(ff, sh);
    if (threadIdx.x == 0) partials[2 * blockIdx.x + 1] = s2;
    unsigned *cnt = reinterpret_cast<unsigned *>(out2 + 2);
    if (last_block(cnt)) {
        double A = 0.0, Bf = 0.0;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += RB) {
            A += __ldcg(partials + 2 * k);
            Bf += __ldcg(partials + 2 * k + 1);
        }
        A = block_sum<RB>(A, sh);
        Bf = block_sum<RB>(Bf, sh);
        if (threadIdx.x == 0) {
            out2[0] = A;
            out2[1] = Bf;
        }
    }
}

// mixed: r32 = r64 * s, d = 0
__global__ void k_scale_to32(int64_t n3, const double *__restrict__ r64, double s, float *r32, float *d)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n3) {
        r32[k] = (float)(r64[k] * s);
        d[k] = 0.f;
    }
}

// mixed: v += scale * d
__global__ void k_accumulate(int64_t n3, const float *__restrict__ d, double scale, double *v)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n3) v[k] += scale * (double)d[k];
}

// Flexible CG (sgp_fcg_solve).  beta = -z^T q_prev / p_prev^T q_prev, the
// previous step's p^T q being sc->pq.
__global__ void __launch_bounds__(RB) k_fcg_zq(int64_t n3, const double *__restrict__ z,
                                               const double *__restrict__ q, double *partials, Scal *sc)
{
    __shared__ double sh[RB / 32];
    if (sc->done) return;
    double a = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
        a = fma(z[k], q[k], a);
    const double s = block_sum<RB>(a, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->cnt)) {
        const double zq = sum_partials<RB>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) sc->beta = -zq / sc->pq;
    }
}

// p = z (FIRST) or z + beta p, and rho = p^T r for alpha = p^T r / p^T q
template <bool FIRST>
__global__ void __launch_bounds__(RB) k_fcg_dir(int64_t n3, const double *__restrict__ z,
                                                const double *__restrict__ r, double *p, double *partials, Scal *sc)
{
    __shared__ double sh[RB / 32];
    if (sc->done) return;
    const double beta = FIRST ? 0.0 : sc->beta;
    double a = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double pk = FIRST ? z[k] : fma(beta, p[k], z[k]);
        p[k] = pk;
        a = fma(pk, r[k], a);
    }
    const double s = block_sum<RB>(a, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->cnt)) {
        const double pr = sum_partials<RB>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) sc->rho = pr;
    }
}

// v += alpha p, r -= alpha q, |r|^2 and the stopping test
__global__ void __launch_bounds__(RB) k_fcg_upd(int64_t n3, const double *__restrict__ p,
                                                const double *__restrict__ q, double *x, double *r,
                                                double *partials, Scal *sc)
{
    __shared__ double sh[RB / 32];
    if (sc->done) return;
    const double alpha = sc->alpha;
    double a = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3;
         k += (int64_t)gridDim.x * blockDim.x) {
        x[k] = fma(alpha, p[k], x[k]);
        const double rk = fma(-alpha, q[k], r[k]);
        r[k] = rk;
        a = fma(rk, rk, a);
    }
    const double s = block_sum<RB>(a, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(&sc->cnt)) {
        const double rr = sum_partials<RB>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->rr = rr;
            sc->it += 1;
            if (!isfinite(rr)) {
                sc->status = SGP_ERR_NOT_SPD;
                sc->done = 1;
            } else if (rr <= sc->stop2) {
                sc->done = 1;
            } else if (sc->it >= sc->maxit) {
                sc->status = SGP_ERR_NO_CONVERGENCE;
                sc->done = 1;
            }
        }
    }
}


// ---------------------------------------------------------------------------
// Small systems: the whole mixed-precision solve in one thread block.  When
// the factor's one-block tail holds every contraction level (a few thousand
// cells at most), the FP64 residual, the FP32 inner PCG (product, tree
// solve, updates, reductions) and the FP64 accumulation all run in one
// launch with every vector in shared memory: no launch or host round trip
// per iteration.  The arithmetic is that of the multi-launch path: eq. (1)
// FP32 records and FP64 blocks for the product, the tail's level solve with
// FP32 L and D^-1, FP64 accumulators for the dot products.
// ---------------------------------------------------------------------------
constexpr int SB = 512;

struct SmallOut {
    long long it;
    int outer, status;
    double rr, ff;
};

struct SmallArgs {
    int32_t n;
    double gamma0, tol, itol;
    long long maxit;
    int max_outer, x_given;
    Blk<float> B32;
    Blk<double> B64;
    const int32_t *row_ptr;
    Tail tl;
    const int32_t *ord, *rc_ptr, *pr_ptr;
    const float *L, *Lf, *Dinv;
    const double *F;
    double *v;
    SmallOut *out;
};

__host__ __device__ inline size_t small_smem_bytes(int32_t n, int32_t np, int32_t nr)
{
    // the tail's staged arrays, the position -> cell map, r, p, q (FP32),
    // and one FP64 vector whose storage also holds z and d (FP32)
    return tail_smem_staged<float>(n, np, nr) + tail_align(4 * (size_t)n) + 3 * tail_align(12 * (size_t)n) +
           tail_align(24 * (size_t)n);
}

// Block sums whose total only thread 0 needs (it takes the scalar
// decisions and broadcasts them): FP32 partials are summed within each warp
// in FP32 and across warps in FP64; FP64 partials in FP64.  One SM's FP64
// rate is low, so FP64 work per thread is kept to the partials that need
// it.  The caller synchronises before the scratch is used again.
__device__ __forceinline__ double small_red32(float x, double *shd)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = (double)x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < SB / 32 ? shd[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}
__device__ __forceinline__ double small_red64(double x, double *shd)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < SB / 32 ? shd[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

__global__ void __launch_bounds__(SB, 1) k_pcg_small(SmallArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double shd[SB / 32];
    // scalars decided by thread 0 and read by all
    __shared__ double b_nr;
    __shared__ float b_al, b_be;
    __shared__ int b_go;
    const Tail &tl = a.tl;
    const int32_t n = a.n, n3 = 3 * n;
    unsigned char *cur = smem_raw;
    auto take = [&](size_t b) { unsigned char *p = cur; cur += tail_align(b); return p; };
    float *sw = reinterpret_cast<float *>(take(12 * (size_t)tl.n));
    int32_t *spr = reinterpret_cast<int32_t *>(take(4 * (size_t)(tl.n + 1)));
    int32_t *stb = reinterpret_cast<int32_t *>(take(4 * (size_t)tl.np));
    int32_t *spc = reinterpret_cast<int32_t *>(take(4 * (size_t)tl.np));
    int32_t *sct = reinterpret_cast<int32_t *>(take(4 * (size_t)tl.np));
    int32_t *src = reinterpret_cast<int32_t *>(take(4 * (size_t)(tl.nr + 1)));
    int32_t *stq = reinterpret_cast<int32_t *>(take(4 * (size_t)tl.nr));
    float *sD = reinterpret_cast<float *>(take(24 * (size_t)tl.n));
    float *sL = reinterpret_cast<float *>(take(36 * (size_t)tl.np));
    int32_t *sord = reinterpret_cast<int32_t *>(take(4 * (size_t)n));
    float *r = reinterpret_cast<float *>(take(12 * (size_t)n));
    float *p = reinterpret_cast<float *>(take(12 * (size_t)n));
    float *q = reinterpret_cast<float *>(take(12 * (size_t)n));
    double *r64 = reinterpret_cast<double *>(take(24 * (size_t)n));
    float *z = reinterpret_cast<float *>(r64), *d = z + n3;   // share r64's storage
    // stage the tail (it covers every position: P0 = Q0 = R0 = C0 = 0)
    const float *Lt = a.L + 9 * (int64_t)tl.Q0, *Dt = a.Dinv + 6 * (int64_t)tl.P0;
    for (int32_t i = threadIdx.x; i < 6 * tl.n; i += SB) sD[i] = Dt[i];
    for (int32_t i = threadIdx.x; i < 9 * tl.np; i += SB) sL[i] = Lt[i];
    for (int32_t i = threadIdx.x; i <= tl.n; i += SB) spr[i] = a.pr_ptr[tl.P0 + i] - tl.Q0;
    for (int32_t i = threadIdx.x; i < tl.np; i += SB) {
        stb[i] = tl.tb[i];
        spc[i] = tl.tpc[i];
        sct[i] = tl.tct[i];
    }
    for (int32_t i = threadIdx.x; i <= tl.nr; i += SB) src[i] = a.rc_ptr[tl.R0 + i] - tl.C0;
    for (int32_t i = threadIdx.x; i < tl.nr; i += SB) stq[i] = tl.tq[i];
    for (int32_t i = threadIdx.x; i < n; i += SB) sord[i] = a.ord[i];
    __syncthreads();

    // z = P^-1 r: gather r into elimination order, forward levels,
    // diagonal and backward levels, scatter back (the tail's level solve).
    // Levels with at most 32 receivers (forward: the last ones; backward:
    // the first ones) run in warp 0 alone with warp barriers.
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int fsplit = tl.nlev;
    while (fsplit > 0 && tl.lvl_rv[fsplit] - tl.lvl_rv[fsplit - 1] <= 32) --fsplit;
    int bsplit = tl.nlev;
    while (bsplit > 0 && tl.lvl_pos[bsplit] - tl.lvl_pos[bsplit - 1] <= 32) --bsplit;
    auto fwd_recv = [&](int32_t k) {
        float s3[3] = {0.f, 0.f, 0.f};
        for (int32_t j = src[k]; j < src[k + 1]; ++j) {
            const int32_t pp = sct[j];
            float y[3];
            full_mv(sL + 9 * pp, sw + 3 * spc[pp], y);
            s3[0] += y[0]; s3[1] += y[1]; s3[2] += y[2];
        }
        const int32_t qq = stq[k];
        sw[3 * qq] -= s3[0]; sw[3 * qq + 1] -= s3[1]; sw[3 * qq + 2] -= s3[2];
    };
    auto bwd_vert = [&](int32_t i) {
        float zz[3];
        sym_mv(sD + 6 * i, sw + 3 * i, zz);
        for (int32_t pp = spr[i]; pp < spr[i + 1]; ++pp) {
            float u[3];
            full_mtv(sL + 9 * pp, sw + 3 * stb[pp], u);
            zz[0] -= u[0]; zz[1] -= u[1]; zz[2] -= u[2];
        }
        sw[3 * i] = zz[0]; sw[3 * i + 1] = zz[1]; sw[3 * i + 2] = zz[2];
    };
    auto tree_solve = [&]() {
        for (int32_t i = threadIdx.x; i < n; i += SB) {
            const int32_t c = sord[i];
            sw[3 * i] = r[3 * c]; sw[3 * i + 1] = r[3 * c + 1]; sw[3 * i + 2] = r[3 * c + 2];
        }
        __syncthreads();
        for (int l = 0; l < fsplit; ++l) {
            const int32_t k0 = tl.lvl_rv[l] - tl.R0, k1 = tl.lvl_rv[l + 1] - tl.R0;
            for (int32_t k = k0 + threadIdx.x; k < k1; k += SB) fwd_recv(k);
            __syncthreads();
        }
        if (warp == 0) {
            for (int l = fsplit; l < tl.nlev; ++l) {
                const int32_t k0 = tl.lvl_rv[l] - tl.R0, k1 = tl.lvl_rv[l + 1] - tl.R0;
                if (k0 + lane < k1) fwd_recv(k0 + lane);
                __syncwarp();
            }
            for (int l = tl.nlev - 1; l >= bsplit; --l) {
                const int32_t i0 = tl.lvl_pos[l] - tl.P0, i1 = tl.lvl_pos[l + 1] - tl.P0;
                if (i0 + lane < i1) bwd_vert(i0 + lane);
                __syncwarp();
            }
        }
        __syncthreads();
        for (int l = bsplit - 1; l >= 0; --l) {
            const int32_t i0 = tl.lvl_pos[l] - tl.P0, i1 = tl.lvl_pos[l + 1] - tl.P0;
            for (int32_t i = i0 + threadIdx.x; i < i1; i += SB) bwd_vert(i);
            __syncthreads();
        }
        for (int32_t i = threadIdx.x; i < n; i += SB) {
            const int32_t c = sord[i];
            z[3 * c] = sw[3 * i]; z[3 * c + 1] = sw[3 * i + 1]; z[3 * c + 2] = sw[3 * i + 2];
        }
        __syncthreads();
    };

    double ff = 0.0;
    {
        double x = 0.0;
        for (int32_t k = threadIdx.x; k < n3; k += SB) x += a.F[k] * a.F[k];
        ff = small_red64(x, shd);   // thread 0
    }
    if (!a.x_given)
        for (int32_t k = threadIdx.x; k < n3; k += SB) a.v[k] = 0.0;
    __syncthreads();
    // thread 0's state
    long long total = 0;
    int outer = 0, status = SGP_OK;
    double rr = 0.0, fi = 0.0, stop2 = 0.0, rho = 0.0;
    long long it = 0;
    const float g32 = (float)a.gamma0;
    for (;;) {
        // FP64 residual r = F - Gamma v
        double acc = 0.0;
        for (int32_t i = threadIdx.x; i < n; i += SB) {
            double vi[3], yi[3];
            row_product(a.B64, a.row_ptr, a.gamma0, (const double *)a.v, i, vi, yi);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double rc = a.F[3 * i + c] - yi[c];
                r64[3 * i + c] = rc;
                acc += rc * rc;
            }
        }
        acc = small_red64(acc, shd);
        if (threadIdx.x == 0) {
            rr = acc;
            int go = 1;
            if (ff == 0.0) {
                rr = 0.0;
                go = 2;                 // v = 0
            } else if (rr <= a.tol * a.tol * ff) {
                go = 0;
            } else if (outer >= a.max_outer || total >= a.maxit) {
                status = SGP_ERR_NO_CONVERGENCE;
                go = 0;
            }
            b_go = go;
            b_nr = sqrt(rr);
        }
        __syncthreads();
        const int go = b_go;
        if (go == 2)
            for (int32_t k = threadIdx.x; k < n3; k += SB) a.v[k] = 0.0;
        if (go != 1) break;
        const double nr = b_nr, inv = 1.0 / nr;
        float fx = 0.f;
        for (int32_t k = threadIdx.x; k < n3; k += SB) {
            const float rk = (float)(r64[k] * inv);
            r[k] = rk;
            fx = fmaf(rk, rk, fx);
        }
        fx = (float)small_red32(fx, shd);   // r64's storage becomes z and d below
        if (threadIdx.x == 0) {
            fi = (double)fx;
            const double need = 0.5 * a.tol * sqrt(ff) / nr;
            const double itk = fmax(a.itol, fmin(need, 0.5));
            stop2 = itk * itk * fi;
            it = 0;
            b_go = fi > stop2;
        }
        __syncthreads();
        for (int32_t k = threadIdx.x; k < n3; k += SB) d[k] = 0.f;
        // inner FP32 PCG on Gamma d = r from d = 0
        if (b_go) {
            tree_solve();
            float x = 0.f;
            for (int32_t k = threadIdx.x; k < n3; k += SB) {
                p[k] = z[k];
                x = fmaf(r[k], z[k], x);
            }
            const double t = small_red32(x, shd);
            if (threadIdx.x == 0) {
                rho = t;
                b_go = rho > 0.0 ? 1 : 3;    // 3: breakdown
            }
            __syncthreads();
            while (b_go == 1) {
                float xp = 0.f;
                for (int32_t i = threadIdx.x; i < n; i += SB) {
                    float vi[3], yi[3];
                    row_product(a.B32, a.row_ptr, g32, (const float *)p, i, vi, yi);
                    q[3 * i] = yi[0]; q[3 * i + 1] = yi[1]; q[3 * i + 2] = yi[2];
                    xp += fmaf(vi[0], yi[0], fmaf(vi[1], yi[1], vi[2] * yi[2]));
                }
                const double pq = small_red32(xp, shd);
                if (threadIdx.x == 0) {
                    if (!(pq > 0.0) || !isfinite(pq)) b_go = 3;
                    else b_al = (float)(rho / pq);
                }
                __syncthreads();
                if (b_go != 1) break;
                const float al = b_al;
                float xr = 0.f;
                for (int32_t k = threadIdx.x; k < n3; k += SB) {
                    d[k] = fmaf(al, p[k], d[k]);
                    const float rk = fmaf(-al, q[k], r[k]);
                    r[k] = rk;
                    xr = fmaf(rk, rk, xr);
                }
                const double rl = small_red32(xr, shd);
                if (threadIdx.x == 0) {
                    ++it;
                    if (rl <= stop2) b_go = 0;
                    else if (total + it >= a.maxit) b_go = 4;   // inner cap
                }
                __syncthreads();
                if (b_go != 1) break;
                tree_solve();
                float xz = 0.f;
                for (int32_t k = threadIdx.x; k < n3; k += SB) xz = fmaf(r[k], z[k], xz);
                const double rz = small_red32(xz, shd);
                if (threadIdx.x == 0) {
                    if (!(rz > 0.0)) {
                        b_go = 3;
                    } else {
                        b_be = (float)(rz / rho);
                        rho = rz;
                    }
                }
                __syncthreads();
                if (b_go != 1) break;
                const float be = b_be;
                for (int32_t k = threadIdx.x; k < n3; k += SB) p[k] = fmaf(be, p[k], z[k]);
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) {
            total += it;
            ++outer;
            if (b_go == 3) status = SGP_ERR_NOT_SPD;
        }
        __syncthreads();
        if (b_go == 3) break;
        // v += |r| d (FP64)
        for (int32_t k = threadIdx.x; k < n3; k += SB) a.v[k] += nr * (double)d[k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.out->it = total;
        a.out->outer = outer;
        a.out->status = status;
        a.out->rr = rr;
        a.out->ff = ff;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
namespace {

// Lanes per block row of the product (SGP_SPMV_LPR overrides): FP64 is
// bound by the FP64 issue rate, where idle lanes of a warp instruction are
// wasted, so one lane per row; FP32 is bound by memory, where more lanes per
// row give longer contiguous loads.
template <typename T>
sgp_status launch_spmv_pq(sgp_ctx *ctx, Blk<T> B, const int32_t *row_ptr, T g0, int64_t n, const T *p,
                          T *q, double *partials, Scal *sc)
{
    const int lpr = ctx->spmv_lpr > 0 ? ctx->spmv_lpr : (sizeof(T) == 8 ? 1 : 2);
    const int ilp = ctx->spmv_ilp > 0 ? ctx->spmv_ilp : 1;
    const int64_t want = (n * lpr + RB - 1) / RB;
    auto go = [&](auto kern) -> sgp_status {
        unsigned G;
        SGP_TRY(resident_grid(ctx, (const void *)kern, RB, want, &G));
        LAUNCH(ctx, kern, G, RB, 0, B, row_ptr, g0, n, p, q, partials, sc);
        return SGP_OK;
    };
    if (ilp == 2) {
        switch (lpr) {
        case 1: return go(k_spmv_pq<T, 1, 2>);
        case 2: return go(k_spmv_pq<T, 2, 2>);
        case 8: return go(k_spmv_pq<T, 8, 2>);
        default: return go(k_spmv_pq<T, 4, 2>);
        }
    }
    switch (lpr) {
    case 1: return go(k_spmv_pq<T, 1, 1>);
    case 2: return go(k_spmv_pq<T, 2, 1>);
    case 8: return go(k_spmv_pq<T, 8, 1>);
    default: return go(k_spmv_pq<T, 4, 1>);
    }
}

static unsigned red_grid(int64_t n)
{
    int64_t g = (n + RB - 1) / RB;
    if (g > 4 * 152) g = 4 * 152;  // a few blocks per SM; grid-stride beyond
    return (unsigned)std::max<int64_t>(g, 1);
}


// The factor's copy of the matrix rows in tree order.
template <typename T>
Blk<T> tree_blk(const sgp_factor *F);
template <>
inline Blk<double> tree_blk<double>(const sgp_factor *F)
{
    return Blk<double>{bp<const int32_t>(F->bl.mc64), bp<const double>(F->bl.m64)};
}
template <>
inline Blk<float> tree_blk<float>(const sgp_factor *F)
{
    return Blk<float>{bp<const float4>(F->bl.ma32), bp<const float2>(F->bl.mb32)};
}

// One PCG run in precision T on Gamma(T) x = F(T) over n rows of the
// product B/row_ptr.  X is the type of the iterate x.  `tree`: the vectors
// are in the binned solve's tree order and every step is fused around it.
// Returns the device scalar block's final state in *hs.
template <typename T, typename X>
sgp_status pcg_core(sgp_ctx *ctx, const sgp_matrix *M, const sgp_factor *Fac, int precond, Blk<T> B,
                    const int32_t *row_ptr, int64_t n, bool tree, const T *F, X *x, int x_given, double tol,
                    int64_t maxit, T *r, T *p, T *q, T *w, double *partials, Scal *sc, Scal *hs, double mu = 0.0,
                    int stopE = 0)
{
    const T g0 = (T)M->gamma0;
    const T *jac = nullptr;
    if (precond == SGP_PRECOND_BLOCK_JACOBI) {
        SGP_TRY(matrix_block_jacobi(ctx, const_cast<sgp_matrix *>(M)));
        jac = reinterpret_cast<const T *>(sizeof(T) == 8 ? M->jac.p : M->jac32.p);
    }
    const unsigned G = red_grid(n);
    SGP_CUDA(ctx, cudaMemsetAsync(sc, 0, sizeof(Scal), ctx->stream));
    if (!x_given) SGP_CUDA(ctx, cudaMemsetAsync(x, 0, sizeof(X) * 3 * n, ctx->stream));
    const T *xin = reinterpret_cast<const T *>(x);
    if (x_given && sizeof(X) != sizeof(T))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: initial guess precision mismatch");
    // error mode: the residual test never fires (stop2 = -|F|^2); the
    // Gauss-Radau test in rz_finish decides
    const double tol2 = stopE ? -1.0 : tol * tol;
    cudaEvent_t ev;
    SGP_TRY(kt_begin(ctx, SGP_KT_PCG_VECTOR, &ev));
    if (precond == SGP_PRECOND_TREE)
        LAUNCH(ctx, (k_init<T, 0>), G, RB, 0, B, row_ptr, g0, n, F, xin, x_given, r, w, jac, tol2,
               (long long)maxit, partials, sc, mu, stopE, tol * tol);
    else if (precond == SGP_PRECOND_BLOCK_JACOBI)
        LAUNCH(ctx, (k_init<T, 1>), G, RB, 0, B, row_ptr, g0, n, F, xin, x_given, r, w, jac, tol2,
               (long long)maxit, partials, sc, mu, stopE, tol * tol);
    else
        LAUNCH(ctx, (k_init<T, 2>), G, RB, 0, B, row_ptr, g0, n, F, xin, x_given, r, w, jac, tol2,
               (long long)maxit, partials, sc, mu, stopE, tol * tol);
    SGP_TRY(kt_end(ctx, SGP_KT_PCG_VECTOR, ev));
    SGP_TRY(read_back(ctx, hs, sc, sizeof(Scal)));
    if (hs->done) return SGP_OK;
    if (precond == SGP_PRECOND_TREE) {
        SGP_TRY(kt_begin(ctx, SGP_KT_TREE_SOLVE, &ev));
        if (tree) SGP_TRY(bins_apply_tree<T>(ctx, Fac, w, w, &sc->done));
        else SGP_TRY(tree_apply_inplace<T>(ctx, Fac, w, &sc->done));
        SGP_TRY(kt_end(ctx, SGP_KT_TREE_SOLVE, ev));
    }
    LAUNCH(ctx, k_rz_init<T>, G, RB, 0, n, (const T *)r, (const T *)w, p, partials, sc);
    // streaming kernels: one full wave of resident blocks
    static_assert(sizeof(X) == sizeof(T), "iterate and vectors share one precision");
    T *xt = reinterpret_cast<T *>(x);
    unsigned Gv = 1;
    SGP_TRY(resident_grid(ctx, (const void *)k_update_v<T, 0>, RB,
                          (3 * n / Pack<T>::K + RB - 1) / RB, &Gv));
    // One PCG iteration per call; kernels return at once after convergence.
    // With the binned tree solve the step is five launches: the product, the
    // three launches of the solve carrying r -= alpha q, the stopping test
    // and r^T z, and the x / p update.
    const bool fused = tree;
    auto iterate = [&](int count) -> sgp_status {
        cudaEvent_t ev;
        if (fused) {
            for (int it = 0; it < count; ++it) {
                SGP_TRY(kt_begin(ctx, SGP_KT_SPMV, &ev));
                SGP_TRY(launch_spmv_pq<T>(ctx, B, row_ptr, g0, n, (const T *)p, q, partials, sc));
                SGP_TRY(kt_end(ctx, SGP_KT_SPMV, ev));
                SGP_TRY(kt_begin(ctx, SGP_KT_TREE_SOLVE, &ev));
                SGP_TRY(bins_pcg_step<T>(ctx, Fac, r, (const T *)q, w, sc));
                SGP_TRY(kt_end(ctx, SGP_KT_TREE_SOLVE, ev));
                SGP_TRY(kt_begin(ctx, SGP_KT_PCG_VECTOR, &ev));
                LAUNCH(ctx, k_pupd_x<T>, Gv, RB, 0, n, xt, p, (const T *)w, sc);
                SGP_TRY(kt_end(ctx, SGP_KT_PCG_VECTOR, ev));
            }
            return SGP_OK;
        }
        for (int it = 0; it < count; ++it) {
            SGP_TRY(kt_begin(ctx, SGP_KT_SPMV, &ev));
            SGP_TRY(launch_spmv_pq<T>(ctx, B, row_ptr, g0, n, (const T *)p, q, partials, sc));
            SGP_TRY(kt_end(ctx, SGP_KT_SPMV, ev));
            SGP_TRY(kt_begin(ctx, SGP_KT_PCG_VECTOR, &ev));
            if (precond == SGP_PRECOND_TREE)
                LAUNCH(ctx, (k_update_v<T, 0>), Gv, RB, 0, n, xt, (const T *)p, r, (const T *)q, w, partials, sc);
            else if (precond == SGP_PRECOND_BLOCK_JACOBI)
                LAUNCH(ctx, (k_update<T, X, 1>), G, RB, 0, n, x, (const T *)p, r, (const T *)q, w, jac,
                       partials, sc);
            else
                LAUNCH(ctx, (k_update_v<T, 2>), Gv, RB, 0, n, xt, (const T *)p, r, (const T *)q, w, partials, sc);
            SGP_TRY(kt_end(ctx, SGP_KT_PCG_VECTOR, ev));
            if (precond == SGP_PRECOND_TREE) {
                SGP_TRY(kt_begin(ctx, SGP_KT_TREE_SOLVE, &ev));
                SGP_TRY(tree_apply_inplace<T>(ctx, Fac, w, &sc->done));
                SGP_TRY(kt_end(ctx, SGP_KT_TREE_SOLVE, ev));
                SGP_TRY(kt_begin(ctx, SGP_KT_PCG_VECTOR, &ev));
                LAUNCH(ctx, k_rz<T>, Gv, RB, 0, n, (const T *)r, (const T *)w, partials, sc);
            } else {
                SGP_TRY(kt_begin(ctx, SGP_KT_PCG_VECTOR, &ev));
            }
            LAUNCH(ctx, k_pupd<T>, Gv, RB, 0, n, (const T *)w, p, (const Scal *)sc);
            SGP_TRY(kt_end(ctx, SGP_KT_PCG_VECTOR, ev));
        }
        return SGP_OK;
    };
    const int chunk = 8;
    if (!ctx->use_graphs) {
        for (;;) {
            SGP_TRY(iterate(chunk));
            SGP_TRY(read_back(ctx, hs, sc, sizeof(Scal)));
            if (hs->done) break;
        }
        return SGP_OK;
    }
    // Without per-kernel timing the iterations run as a device-side loop:
    // chunks of 4 iterations form the body of a conditional WHILE graph node
    // that repeats until the done word is set (or 1024 bodies have run), so
    // the host waits once per launch instead of once per chunk.
    if (ctx->use_while && !ctx->timing) {
        const int wchunk = 4, max_bodies = 1024;
        const uint64_t wkey[] = {0x5748494c45ull, (uint64_t)sizeof(T), (uint64_t)sizeof(X), (uint64_t)precond,
                                 (uint64_t)n, M->gen, Fac ? Fac->gen : 0ull, (uint64_t)(uintptr_t)x,
                                 (uint64_t)(uintptr_t)r, (uint64_t)(uintptr_t)p, (uint64_t)(uintptr_t)q,
                                 (uint64_t)(uintptr_t)w, (uint64_t)(uintptr_t)partials, (uint64_t)(uintptr_t)sc,
                                 (uint64_t)(uintptr_t)jac, (uint64_t)wchunk, (uint64_t)ctx->spmv_lpr,
                                 (uint64_t)ctx->spmv_ilp, (uint64_t)fused};
        GraphEntry *we = nullptr;
        SGP_TRY(graph_lookup(ctx, wkey, sizeof(wkey) / sizeof(wkey[0]), &we));
        if (!we->exec &&
            graph_capture_while(ctx, we, &sc->done, &sc->pad, max_bodies, [&]() { return iterate(wchunk); }) !=
                SGP_OK) {
            ctx->use_while = 0;   // not supported here: chunked graphs from now on
            cudaGetLastError();
        }
        if (we->exec) {
            for (;;) {
                SGP_CUDA(ctx, cudaMemsetAsync(&sc->pad, 0, sizeof(int), ctx->stream));
                SGP_CUDA(ctx, cudaGraphLaunch(we->exec, ctx->stream));
                SGP_TRY(read_back(ctx, hs, sc, sizeof(Scal)));
                ctx->launches += (int64_t)hs->pad * we->kernels;
                if (hs->done) break;
            }
            return SGP_OK;
        }
    }
    // Chunks of iterations are captured once into a CUDA graph and replayed;
    // the graph is keyed by everything its nodes point at.
    const uint64_t key[] = {(uint64_t)sizeof(T), (uint64_t)sizeof(X), (uint64_t)precond, (uint64_t)n,
                            M->gen, Fac ? Fac->gen : 0ull, (uint64_t)(uintptr_t)x, (uint64_t)(uintptr_t)r,
                            (uint64_t)(uintptr_t)p, (uint64_t)(uintptr_t)q, (uint64_t)(uintptr_t)w,
                            (uint64_t)(uintptr_t)partials, (uint64_t)(uintptr_t)sc,
                            (uint64_t)(uintptr_t)jac, (uint64_t)ctx->timing, (uint64_t)chunk,
                            (uint64_t)ctx->spmv_lpr, (uint64_t)ctx->spmv_ilp, (uint64_t)fused};
    GraphEntry *ge = nullptr;
    SGP_TRY(graph_lookup(ctx, key, sizeof(key) / sizeof(key[0]), &ge));
    if (!ge->exec) SGP_TRY(graph_capture(ctx, ge, [&]() { return iterate(chunk); }));
    for (;;) {
        SGP_CUDA(ctx, cudaGraphLaunch(ge->exec, ctx->stream));
        ctx->launches += ge->kernels;
        SGP_TRY(read_back(ctx, hs, sc, sizeof(Scal)));
        SGP_TRY(graph_collect_timing(ctx, ge));
        if (hs->done) break;
    }
    return SGP_OK;
}

// One PCG run on Gamma x = F in the matrix's internal order.  With the
// tree preconditioner and a binned factor built from this assembly, the run
// takes F (and x) to the factor's tree order, solves there with the fused
// steps, and brings x back; Ft and xt are tree-order workspaces (NT cells).
template <typename T, typename X>
sgp_status pcg_run(sgp_ctx *ctx, const sgp_matrix *M, const sgp_factor *Fac, int precond, const T *F, X *x,
                   int x_given, double tol, int64_t maxit, T *r, T *p, T *q, T *w, T *Ft, T *xt,
                   double *partials, Scal *sc, Scal *hs, double mu = 0.0, int stopE = 0)
{
    static_assert(sizeof(X) == sizeof(T), "iterate and vectors share one precision");
    const bool tree = precond == SGP_PRECOND_TREE && ctx->fused && Ft && xt && bins_tree_ready<T>(Fac, M);
    if (!tree)
        return pcg_core<T, X>(ctx, M, Fac, precond, make_blk<T>(M), bp<const int32_t>(M->row_ptr), M->n, false, F,
                              x, x_given, tol, maxit, r, p, q, w, partials, sc, hs, mu, stopE);
    SGP_TRY(bins_to_tree<T>(ctx, Fac, F, Ft));
    if (x_given) SGP_TRY(bins_to_tree<T>(ctx, Fac, reinterpret_cast<const T *>(x), xt));
    SGP_TRY((pcg_core<T, T>(ctx, M, Fac, precond, tree_blk<T>(Fac), bp<const int32_t>(Fac->bl.rpt), Fac->bl.NT,
                            true, Ft, xt, x_given, tol, maxit, r, p, q, w, partials, sc, hs, mu, stopE)));
    return bins_from_tree<T>(ctx, Fac, xt, reinterpret_cast<T *>(x));
}

}  // namespace


// The one-block solve applies: MIXED, tree preconditioner, residual
// stopping, the factor's tail covering every level, and everything fitting
// in one block's shared memory.
static bool small_pcg_fits(const sgp_ctx *ctx, const sgp_matrix *M, const sgp_factor *Fac, const sgp_solve_opts *o)
{
    if (!ctx->small_solve || o->precision != SGP_PREC_MIXED || o->precond != SGP_PRECOND_TREE ||
        o->stop != SGP_STOP_RESIDUAL || !Fac || Fac->precision != SGP_PREC_MIXED || M->precision != SGP_PREC_MIXED)
        return false;
    if (Fac->levels == 0 || Fac->tail_level != 0 || Fac->tail_P0 != 0 || !Fac->L32.p || !Fac->Dinv32.p) return false;
    const Tail tl = tail_of(Fac);
    if (tl.n != M->n) return false;
    return small_smem_bytes(tl.n, tl.np, tl.nr) <= (size_t)TREE_TAIL_SMEM;
}

static sgp_status small_pcg(sgp_ctx *ctx, const sgp_matrix *M, const sgp_factor *Fac, const double *F, double *v,
                     const sgp_solve_opts *o, SmallOut *dout, SmallOut *hout)
{
    static int done_dev[64] = {0};
    if (ctx->device >= 0 && ctx->device < 64 && !done_dev[ctx->device]) {
        SGP_CUDA(ctx, cudaFuncSetAttribute(k_pcg_small, cudaFuncAttributeMaxDynamicSharedMemorySize, TREE_TAIL_SMEM));
        done_dev[ctx->device] = 1;
    }
    const Tail tl = tail_of(Fac);
    SmallArgs a{};
    a.n = (int32_t)M->n;
    a.gamma0 = M->gamma0;
    a.tol = o->tol;
    a.itol = o->inner_tol > 0 ? o->inner_tol : 1e-3;
    a.maxit = o->maxit;
    a.max_outer = o->max_outer > 0 ? o->max_outer : 30;
    a.x_given = o->x0_given;
    a.B32 = make_blk<float>(M);
    a.B64 = make_blk<double>(M);
    a.row_ptr = bp<const int32_t>(M->row_ptr);
    a.tl = tl;
    a.ord = bp<const int32_t>(Fac->ord);
    a.rc_ptr = bp<const int32_t>(Fac->rc_ptr);
    a.pr_ptr = bp<const int32_t>(Fac->pr_ptr);
    a.L = bp<const float>(Fac->L32);
    a.Lf = bp<const float>(Fac->Lf32);
    a.Dinv = bp<const float>(Fac->Dinv32);
    a.F = F;
    a.v = v;
    a.out = dout;
    LAUNCH(ctx, k_pcg_small, 1, SB, small_smem_bytes(tl.n, tl.np, tl.nr), a);
    return read_back(ctx, hout, dout, sizeof(SmallOut));
}

// FP64 product y = Gamma v without the timing hooks (used by the warm-start
// network's loss and scaling).
sgp_status spmv64(sgp_ctx *ctx, const sgp_matrix *M, const double *v, double *y)
{
    LAUNCH(ctx, k_spmv<double>, grid_for(M->n, 128), 128, 0, make_blk<double>(M), bp<const int32_t>(M->row_ptr),
           M->gamma0, M->n, v, y);
    return SGP_OK;
}

// Warm-start acceptance: keep v0 only if |F - Gamma v0| <= |F| (otherwise
// the zero guess has the smaller residual and v0 is cleared).
sgp_status mpnn_residual_check(sgp_ctx *ctx, const sgp_matrix *M, const double *F, double *v0, int *used,
                               int kclass, cudaEvent_t ev)
{
    const int64_t n = M->n;
    *used = 0;
    if (n == 0) return SGP_OK;
    SGP_TRY(scratch_ensure(ctx, sizeof(double) * 2 * MAXP + 512));
    double *partials = reinterpret_cast<double *>(ctx->d_scratch);
    double *o2 = partials + 2 * MAXP;
    SGP_CUDA(ctx, cudaMemsetAsync(o2, 0, 32, ctx->stream));
    unsigned Gr = 1;
    SGP_TRY(resident_grid(ctx, (const void *)k_resid64<false>, RB, (n + RB - 1) / RB, &Gr));
    LAUNCH(ctx, k_resid64<false>, Gr, RB, 0, make_blk<double>(M), bp<const int32_t>(M->row_ptr), M->gamma0,
           n, F, (const double *)v0, (double *)nullptr, partials, o2);
    SGP_TRY(kt_end(ctx, kclass, ev));
    double h[2] = {0, 0};
    SGP_TRY(read_back(ctx, h, o2, sizeof(h)));
    if (h[0] <= h[1] && std::isfinite(h[0])) {
        *used = 1;
        return SGP_OK;
    }
    SGP_CUDA(ctx, cudaMemsetAsync(v0, 0, sizeof(double) * 3 * n, ctx->stream));
    return SGP_OK;
}

extern "C" {

sgp_status sgp_spmv(sgp_ctx *ctx, const sgp_matrix *M, const double *v, double *y)
{
    if (!ctx || !M || (M->n > 0 && (!v || !y))) return SGP_ERR_INVALID_ARG;
    if (v == y) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "spmv: v and y must differ");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = M->n;
    if (n == 0) return SGP_OK;
    // caller order -> internal order -> product -> caller order
    SGP_TRY(scratch_ensure(ctx, sizeof(double) * 6 * n + 1024));
    double *vi = reinterpret_cast<double *>(ctx->d_scratch), *yi = vi + 3 * n;
    const int32_t *orig_of = bp<const int32_t>(M->orig_of);
    LAUNCH(ctx, k_to_internal<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, v, vi);
    cudaEvent_t ev;
    SGP_TRY(kt_begin(ctx, SGP_KT_SPMV, &ev));
    LAUNCH(ctx, k_spmv<double>, grid_for(n, 128), 128, 0, make_blk<double>(M), bp<const int32_t>(M->row_ptr),
           M->gamma0, n, (const double *)vi, yi);
    SGP_TRY(kt_end(ctx, SGP_KT_SPMV, ev));
    LAUNCH(ctx, k_to_caller<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, (const double *)yi, y);
    return SGP_OK;
}

sgp_status sgp_pcg_solve(sgp_ctx *ctx, const sgp_matrix *M, const sgp_factor *Fac, const double *F,
                         double *v, const sgp_solve_opts *opts, sgp_solve_info *info)
{
    if (!ctx || !M || !opts) return SGP_ERR_INVALID_ARG;
    const int64_t n = M->n;
    if (n > 0 && (!F || !v)) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: NULL vector");
    if (!(opts->tol > 0.0) || opts->maxit <= 0)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: tol must be > 0 and maxit >= 1");
    if (opts->precond < 0 || opts->precond > 2)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: bad preconditioner");
    if (opts->precond == SGP_PRECOND_TREE && (!Fac || Fac->n != n))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: the tree preconditioner needs a factor of this matrix");
    const bool mixed = opts->precision == SGP_PREC_MIXED;
    if (mixed && M->precision != SGP_PREC_MIXED)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: MIXED needs a matrix assembled with MIXED");
    if (mixed && opts->precond == SGP_PRECOND_TREE && Fac->precision != SGP_PREC_MIXED)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: MIXED needs a factor of a MIXED matrix");
    if (opts->stop != SGP_STOP_RESIDUAL && opts->stop != SGP_STOP_ERROR)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: bad stopping rule");
    const bool stopE = opts->stop == SGP_STOP_ERROR;
    if (stopE && mixed) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: error-bound stopping is FP64 only");
    if (!std::isfinite(opts->mu))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: mu must be finite");
    // lower bound of lambda_min(H Gamma) for the Gauss-Radau rule
    double mu = opts->mu;
    if (!(mu > 0.0)) {
        if (opts->precond == SGP_PRECOND_TREE) mu = 1.0;            // Section 4
        else if (opts->precond == SGP_PRECOND_NONE) mu = M->gamma0;  // Lemma 2.4
        else if (stopE)
            return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "pcg: block Jacobi error-bound stopping needs mu > 0");
        else mu = 0.0;
    }
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    sgp_solve_info inf{};
    if (n == 0) {
        if (info) *info = inf;
        return SGP_OK;
    }
    // workspace: FP64 r, p, q, w and the tree-order F and x (6 x 3nv), F and
    // v in the internal order (2 x 3n), FP32 rhs, r, p, q, w, d and the
    // tree-order pair (8 x 3nv), partials, scalars; nv covers the binned
    // solve's tree order (a little longer than n: padding)
    const int64_t nv = (opts->precond == SGP_PRECOND_TREE && Fac && Fac->bl.NT > n) ? Fac->bl.NT : n;
    const size_t v64 = sizeof(double) * 3 * nv, v32 = sizeof(float) * 3 * nv;
    size_t need = 8 * v64 + (mixed ? 8 * v32 : 0) + sizeof(double) * 2 * MAXP + 2 * sizeof(Scal) + 8192;
    SGP_TRY(scratch_ensure(ctx, need + 4096));
    char *base = reinterpret_cast<char *>(ctx->d_scratch) + 256;
    auto take = [&](size_t b) {
        char *p = base;
        base += (b + 255) & ~size_t(255);
        return p;
    };
    double *partials = reinterpret_cast<double *>(take(sizeof(double) * 2 * MAXP));
    Scal *sc = reinterpret_cast<Scal *>(take(sizeof(Scal)));
    double *o2 = reinterpret_cast<double *>(take(64));
    double *r = reinterpret_cast<double *>(take(v64));
    double *p = reinterpret_cast<double *>(take(v64));
    double *q = reinterpret_cast<double *>(take(v64));
    double *w = reinterpret_cast<double *>(take(v64));
    double *Ft64 = reinterpret_cast<double *>(take(v64));
    double *xt64 = reinterpret_cast<double *>(take(v64));
    // the solve runs in the matrix's internal cell order
    const double *F_user = F;
    double *v_user = v;
    double *F_in = reinterpret_cast<double *>(take(v64));
    double *v_in = reinterpret_cast<double *>(take(v64));
    const int32_t *orig_of = bp<const int32_t>(M->orig_of);
    LAUNCH(ctx, k_to_internal<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, F_user, F_in);
    if (opts->x0_given)
        LAUNCH(ctx, k_to_internal<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, (const double *)v_user,
               v_in);
    F = F_in;
    v = v_in;
    Scal hs{};
    sgp_status rc = SGP_OK;
    Blk<double> B64 = make_blk<double>(M);
    const int32_t *row_ptr = bp<const int32_t>(M->row_ptr);
    const unsigned G = red_grid(n);
    unsigned Gr = 1;
    SGP_TRY(resident_grid(ctx, (const void *)k_resid64<false>, RB, (n + RB - 1) / RB, &Gr));
    double hres[2] = {0, 0};
    if (!mixed) {
        SGP_TRY(pcg_run<double, double>(ctx, M, Fac, opts->precond, F, v, opts->x0_given, opts->tol,
                                        opts->maxit, r, p, q, w, Ft64, xt64, partials, sc, &hs, mu, stopE ? 1 : 0));
        inf.iterations = hs.it;
        inf.err_bound = (mu > 0.0 && hs.gsum > 0.0) ? std::sqrt(std::max(hs.est, 0.0) / hs.gsum) : 0.0;
        inf.status = hs.status;
        inf.rel_residual = hs.FF > 0 ? std::sqrt(hs.rr / hs.FF) : 0.0;
        if (hs.FF == 0.0) SGP_CUDA(ctx, cudaMemsetAsync(v, 0, v64, ctx->stream));
    } else {
        float *r32 = reinterpret_cast<float *>(take(v32));
        float *s32 = reinterpret_cast<float *>(take(v32));
        float *p32 = reinterpret_cast<float *>(take(v32));
        float *q32 = reinterpret_cast<float *>(take(v32));
        float *w32 = reinterpret_cast<float *>(take(v32));
        float *d32 = reinterpret_cast<float *>(take(v32));
        float *Ft32 = reinterpret_cast<float *>(take(v32));
        float *xt32 = reinterpret_cast<float *>(take(v32));
        const int max_outer = opts->max_outer > 0 ? opts->max_outer : 30;
        const double itol = opts->inner_tol > 0 ? opts->inner_tol : 1e-3;
        if (!opts->x0_given) SGP_CUDA(ctx, cudaMemsetAsync(v, 0, v64, ctx->stream));
        int64_t total = 0;
        int outer = 0;
        const bool small = small_pcg_fits(ctx, M, Fac, opts);
        if (small) {
            SmallOut ho{};
            SGP_TRY(small_pcg(ctx, M, Fac, F, v, opts, reinterpret_cast<SmallOut *>(o2), &ho));
            total = ho.it;
            outer = ho.outer;
            inf.status = ho.status;
            hres[0] = ho.rr;
            hres[1] = ho.ff;
            inf.rel_residual = ho.ff > 0 ? std::sqrt(ho.rr / ho.ff) : 0.0;
        }
        for (; !small;) {
            SGP_CUDA(ctx, cudaMemsetAsync(o2 + 2, 0, 16, ctx->stream));
            if (outer == 0 && !opts->x0_given)
                LAUNCH(ctx, k_resid64<true>, Gr, RB, 0, B64, row_ptr, M->gamma0, n, F, (const double *)v, r,
                       partials, o2);
            else
                LAUNCH(ctx, k_resid64<false>, Gr, RB, 0, B64, row_ptr, M->gamma0, n, F, (const double *)v, r,
                       partials, o2);
            SGP_TRY(read_back(ctx, hres, o2, sizeof(hres)));
            const double rr = hres[0], ff = hres[1];
            inf.rel_residual = ff > 0 ? std::sqrt(rr / ff) : 0.0;
            if (ff == 0.0) {
                SGP_CUDA(ctx, cudaMemsetAsync(v, 0, v64, ctx->stream));
                break;
            }
            if (rr <= opts->tol * opts->tol * ff) break;
            if (outer >= max_outer || total >= opts->maxit) {
                inf.status = SGP_ERR_NO_CONVERGENCE;
                break;
            }
            const double nr = std::sqrt(rr);
            LAUNCH(ctx, k_scale_to32, grid_for(3 * n, SGP_BLOCK), SGP_BLOCK, 0, 3 * n, (const double *)r,
                   1.0 / nr, r32, d32);
            // inner solve from d = 0 on the scaled residual (|r32| ~ 1); the
            // last step only has to bring |r| to half the outer target
            const double need = 0.5 * opts->tol * std::sqrt(ff) / nr;
            const double itol_k = std::max(itol, std::min(need, 0.5));
            SGP_TRY(pcg_run<float, float>(ctx, M, Fac, opts->precond, (const float *)r32, d32, 0, itol_k,
                                          opts->maxit - total, s32, p32, q32, w32, Ft32, xt32, partials, sc,
                                          &hs));
            total += hs.it;
            ++outer;
            if (hs.status == SGP_ERR_NOT_SPD || hs.status == SGP_ERR_TIMEOUT) {
                inf.status = hs.status;
                break;
            }
            LAUNCH(ctx, k_accumulate, grid_for(3 * n, SGP_BLOCK), SGP_BLOCK, 0, 3 * n, (const float *)d32,
                   nr, v);
        }
        inf.iterations = total;
        inf.outer_iterations = outer;
    }
    // true FP64 residual at exit (the mixed loop ends on one: the residual
    // of the final v, from the FP64 product)
    if (!mixed) {
        SGP_CUDA(ctx, cudaMemsetAsync(o2 + 2, 0, 16, ctx->stream));
        LAUNCH(ctx, k_resid64<false>, Gr, RB, 0, B64, row_ptr, M->gamma0, n, F, (const double *)v,
               (double *)nullptr, partials, o2);
        SGP_TRY(read_back(ctx, hres, o2, sizeof(hres)));
    }
    inf.true_rel_residual = hres[1] > 0 ? std::sqrt(hres[0] / hres[1]) : 0.0;
    LAUNCH(ctx, k_to_caller<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, (const double *)v, v_user);
    if (info) *info = inf;
    if (opts->precond == SGP_PRECOND_TREE) SGP_TRY(bins_check(ctx, Fac));
    if (inf.status == SGP_ERR_TIMEOUT)
        rc = sgp_fail(ctx, SGP_ERR_TIMEOUT, "pcg: a bounded device wait gave up");
    else if (inf.status == SGP_ERR_NOT_SPD)
        rc = sgp_fail(ctx, SGP_ERR_NOT_SPD, "pcg: breakdown (p^T Gamma p or r^T z not positive)");
    else if (inf.status == SGP_ERR_NO_CONVERGENCE)
        rc = sgp_fail(ctx, SGP_ERR_NO_CONVERGENCE, "pcg: no convergence after %lld iterations",
                      (long long)inf.iterations);
    return rc;
}


sgp_status sgp_fcg_solve(sgp_ctx *ctx, const sgp_matrix *M, const sgp_aug *A, const sgp_factor *Fac,
                         const double *F, double *v, const sgp_solve_opts *opts, int64_t inner_maxit,
                         sgp_solve_info *info)
{
    if (!ctx || !M || !A || !Fac || !opts) return SGP_ERR_INVALID_ARG;
    const int64_t n = M->n;
    if (n > 0 && (!F || !v)) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "fcg: NULL vector");
    if (!(opts->tol > 0.0) || opts->maxit <= 0 || inner_maxit <= 0)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "fcg: tol must be > 0, maxit and inner_maxit >= 1");
    if (!(opts->inner_tol >= 0.0 && opts->inner_tol < 1.0))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "fcg: inner_tol must be in [0, 1)");
    if (opts->precond != SGP_PRECOND_TREE || opts->precision != SGP_PREC_F64)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "fcg: the nested solve is FP64 with the tree preconditioner");
    if (opts->stop != SGP_STOP_RESIDUAL)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "fcg: residual stopping only");
    if (A->n != n || A->mgen != M->gen || !A->P)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "fcg: the augmented forest was built from another matrix");
    if (Fac->n != n) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "fcg: the factor has another size");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    sgp_solve_info inf{};
    if (n == 0) {
        if (info) *info = inf;
        return SGP_OK;
    }
    const double itol = opts->inner_tol > 0.0 ? opts->inner_tol : 0.1;
    const size_t v64 = sizeof(double) * 3 * n;
    SGP_TRY(scratch_ensure(ctx, 10 * (v64 + 256) + sizeof(double) * 2 * MAXP + 4 * sizeof(Scal) + 8192));
    char *base = reinterpret_cast<char *>(ctx->d_scratch) + 256;
    auto take = [&](size_t b) {
        char *p = base;
        base += (b + 255) & ~size_t(255);
        return p;
    };
    double *partials = reinterpret_cast<double *>(take(sizeof(double) * 2 * MAXP));
    Scal *sco = reinterpret_cast<Scal *>(take(sizeof(Scal)));
    Scal *sci = reinterpret_cast<Scal *>(take(sizeof(Scal)));
    double *o2 = reinterpret_cast<double *>(take(64));
    double *r = reinterpret_cast<double *>(take(v64)), *p = reinterpret_cast<double *>(take(v64)),
           *q = reinterpret_cast<double *>(take(v64)), *z = reinterpret_cast<double *>(take(v64)),
           *Fi = reinterpret_cast<double *>(take(v64)), *x = reinterpret_cast<double *>(take(v64)),
           *ri = reinterpret_cast<double *>(take(v64)), *pi = reinterpret_cast<double *>(take(v64)),
           *qi = reinterpret_cast<double *>(take(v64)), *wi = reinterpret_cast<double *>(take(v64));
    const int32_t *orig_of = bp<const int32_t>(M->orig_of);
    LAUNCH(ctx, k_to_internal<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, F, Fi);
    if (opts->x0_given)
        LAUNCH(ctx, k_to_internal<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, (const double *)v, x);
    else
        SGP_CUDA(ctx, cudaMemsetAsync(x, 0, v64, ctx->stream));
    Blk<double> B64 = make_blk<double>(M);
    const int32_t *row_ptr = bp<const int32_t>(M->row_ptr);
    unsigned Gr = 1;
    SGP_TRY(resident_grid(ctx, (const void *)k_resid64<false>, RB, (n + RB - 1) / RB, &Gr));
    double hres[2] = {0, 0};
    SGP_CUDA(ctx, cudaMemsetAsync(o2 + 2, 0, 16, ctx->stream));
    if (opts->x0_given)
        LAUNCH(ctx, k_resid64<false>, Gr, RB, 0, B64, row_ptr, M->gamma0, n, (const double *)Fi, (const double *)x, r,
               partials, o2);
    else
        LAUNCH(ctx, k_resid64<true>, Gr, RB, 0, B64, row_ptr, M->gamma0, n, (const double *)Fi, (const double *)x, r,
               partials, o2);
    SGP_TRY(read_back(ctx, hres, o2, sizeof(hres)));
    const double ff = hres[1];
    Scal h{};
    h.FF = ff;
    h.rr = hres[0];
    h.stop2 = opts->tol * opts->tol * ff;
    h.maxit = opts->maxit;
    h.done = ff == 0.0 || h.rr <= h.stop2;
    if (ff == 0.0) SGP_CUDA(ctx, cudaMemsetAsync(x, 0, v64, ctx->stream));
    SGP_CUDA(ctx, cudaMemcpyAsync(sco, &h, sizeof(Scal), cudaMemcpyHostToDevice, ctx->stream));
    const sgp_matrix *P = A->P;
    const unsigned G = red_grid(n);
    const int64_t n3 = 3 * n;
    int64_t inner = 0;
    for (int64_t k = 0; !h.done; ++k) {
        // z ~ P'^-1 r: PCG on P' with the forest factor, from z = 0
        Scal hi{};
        SGP_TRY((pcg_core<double, double>(ctx, P, Fac, SGP_PRECOND_TREE, make_blk<double>(P),
                                          bp<const int32_t>(P->row_ptr), n, false, (const double *)r, z, 0, itol,
                                          inner_maxit, ri, pi, qi, wi, partials, sci, &hi)));
        inner += hi.it;
        if (hi.status == SGP_ERR_NOT_SPD || hi.status == SGP_ERR_TIMEOUT) {
            h.status = hi.status;
            break;
        }
        cudaEvent_t ev;
        SGP_TRY(kt_begin(ctx, SGP_KT_PCG_VECTOR, &ev));
        if (k == 0) {
            LAUNCH(ctx, k_fcg_dir<true>, G, RB, 0, n3, (const double *)z, (const double *)r, p, partials, sco);
        } else {
            LAUNCH(ctx, k_fcg_zq, G, RB, 0, n3, (const double *)z, (const double *)q, partials, sco);
            LAUNCH(ctx, k_fcg_dir<false>, G, RB, 0, n3, (const double *)z, (const double *)r, p, partials, sco);
        }
        SGP_TRY(kt_end(ctx, SGP_KT_PCG_VECTOR, ev));
        SGP_TRY(kt_begin(ctx, SGP_KT_SPMV, &ev));
        SGP_TRY(launch_spmv_pq<double>(ctx, B64, row_ptr, M->gamma0, n, (const double *)p, q, partials, sco));
        SGP_TRY(kt_end(ctx, SGP_KT_SPMV, ev));
        SGP_TRY(kt_begin(ctx, SGP_KT_PCG_VECTOR, &ev));
        LAUNCH(ctx, k_fcg_upd, G, RB, 0, n3, (const double *)p, (const double *)q, x, r, partials, sco);
        SGP_TRY(kt_end(ctx, SGP_KT_PCG_VECTOR, ev));
        SGP_TRY(read_back(ctx, &h, sco, sizeof(Scal)));
        SGP_TRY(kt_collect(ctx));
    }
    inf.iterations = inner;
    inf.outer_iterations = (int32_t)h.it;
    inf.status = h.status;
    inf.rel_residual = ff > 0 ? std::sqrt(h.rr / ff) : 0.0;
    SGP_CUDA(ctx, cudaMemsetAsync(o2 + 2, 0, 16, ctx->stream));
    LAUNCH(ctx, k_resid64<false>, Gr, RB, 0, B64, row_ptr, M->gamma0, n, (const double *)Fi, (const double *)x,
           (double *)nullptr, partials, o2);
    SGP_TRY(read_back(ctx, hres, o2, sizeof(hres)));
    inf.true_rel_residual = hres[1] > 0 ? std::sqrt(hres[0] / hres[1]) : 0.0;
    LAUNCH(ctx, k_to_caller<double>, grid_for(n, SGP_BLOCK), SGP_BLOCK, 0, n, orig_of, (const double *)x, v);
    if (info) *info = inf;
    if (inf.status == SGP_ERR_TIMEOUT) return sgp_fail(ctx, SGP_ERR_TIMEOUT, "fcg: a bounded device wait gave up");
    if (inf.status == SGP_ERR_NOT_SPD)
        return sgp_fail(ctx, SGP_ERR_NOT_SPD, "fcg: breakdown (p^T Gamma p not positive)");
    if (inf.status == SGP_ERR_NO_CONVERGENCE)
        return sgp_fail(ctx, SGP_ERR_NO_CONVERGENCE, "fcg: no convergence after %d outer iterations",
                        inf.outer_iterations);
    return SGP_OK;
}

}  // extern "C"
