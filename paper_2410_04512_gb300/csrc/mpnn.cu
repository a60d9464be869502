// mpnn.cu -- learned warm start: a message-passing network over the
// collision graph that predicts the PCG initial guess v0 (the paper has no
// learned component; the solver's own iterations measure the prediction).
//
// Network (width 64, 3 message-passing layers, BF16 weights, FP32
// activations and accumulation):
//   basis  b0 = D^-1 F (block Jacobi), b1 = P^-1 F (spanning forest),
//          b2 = previous velocity (or 0)
//   x_i    = (|b0|, |b1|, |b2|, b0.b1, b0.b2, b1.b2) / (mean |b1|)^(1|2),
//            deg_i / 6, 1
//   h0     = relu(W_in x + b_in)
//   h_l+1  = relu(W_l [h_l ; mean_{j~i} h_l,j] + c_l),   l = 0, 1, 2
//   c      = W_out h3 + b_out,   v0_i = sum_k c_ik b_i^(k)
// Every feature is rotation invariant and v0 is a scalar mix of equivariant
// fields, so the prediction rotates with the configuration.
//
// Training (online, on solutions of earlier steps): loss
// |v0 - v*|^2 / |v*|^2, hand-written backward kernels, Adam on FP32 master
// weights, BF16 copies refreshed after every step.  Weight gradients are
// reduced per block and then in block order (deterministic).
#include <cuda_bf16.h>

#include "sgp_internal.cuh"

sgp_status spmv64(sgp_ctx *ctx, const sgp_matrix *M, const double *v, double *y);

namespace {

constexpr int H = 64, KB = 3, DIN = 8, H2 = 2 * H;
// parameter layout (FP32 master, flat): W_in, b_in, {W_l, c_l} x 3, W_out, b_out
constexpr int OFF_WIN = 0, OFF_BIN = OFF_WIN + H * DIN;
constexpr int OFF_L0 = OFF_BIN + H;
constexpr int LAYER = H * H2 + H;
constexpr int OFF_WOUT = OFF_L0 + 3 * LAYER, OFF_BOUT = OFF_WOUT + KB * H;
constexpr int NPARAM = OFF_BOUT + KB;
static_assert(NPARAM == SGP_MPNN_PARAMS, "parameter layout");
constexpr int TB = 256;          // threads per block
constexpr int CHUNK = 256;       // nodes per block in the weight-gradient reductions

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int k) { return __bfloat162float(w[k]); }

// ---------------------------------------------------------------- features
// b0 = D^-1 F with the block-Jacobi inverse (sym6 per row)
__global__ void k_mp_jacobi(int64_t n, const double *__restrict__ jac, const double *__restrict__ F, double *b0)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) sym_mv(jac + 6 * i, F + 3 * i, b0 + 3 * i);
}

// sum_i |b1_i|, reduced by blocks then by the last block (fixed order)
__global__ void k_mp_norm_sum(int64_t n, const double *__restrict__ b1, double *partials, unsigned *counter,
                              double *out)
{
    __shared__ double sh[TB / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += sqrt(b1[3 * i] * b1[3 * i] + b1[3 * i + 1] * b1[3 * i + 1] + b1[3 * i + 2] * b1[3 * i + 2]);
    s = block_sum<TB>(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (last_block(counter)) {
        double t = sum_partials<TB>(partials, gridDim.x, sh);
        if (threadIdx.x == 0) out[0] = t / (double)(n > 0 ? n : 1);
    }
}

__global__ void k_mp_features(int64_t n, const double *__restrict__ b0, const double *__restrict__ b1,
                              const double *__restrict__ b2, const int32_t *__restrict__ row_ptr,
                              const double *__restrict__ mean_b1, float *x)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = mean_b1[0];
    if (!(s > 0.0)) s = 1.0;
    const double *a = b0 + 3 * i, *b = b1 + 3 * i, *c = b2 + 3 * i;
    auto dot = [](const double *u, const double *v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
    float *o = x + DIN * i;
    o[0] = (float)(sqrt(dot(a, a)) / s);
    o[1] = (float)(sqrt(dot(b, b)) / s);
    o[2] = (float)(sqrt(dot(c, c)) / s);
    o[3] = (float)(dot(a, b) / (s * s));
    o[4] = (float)(dot(a, c) / (s * s));
    o[5] = (float)(dot(b, c) / (s * s));
    o[6] = (float)((row_ptr[i + 1] - row_ptr[i]) / 6.0);
    o[7] = 1.0f;
}

// ------------------------------------------------------------ dense layers
// Y (n x DOUT) = act(X Wt + bias) where X = [X1 (n x D1), X2 (n x D2)] and the
// BF16 matrix W is DOUT x (D1 + D2) (TRANS = false), or Y = X W with W of
// shape (D1 + D2) x DOUT read transposed (TRANS = true, no bias/act: the
// backward product dX = dZ W).  The weights are staged transposed in shared
// memory as FP32 so that the threads of a node read consecutive outputs.
template <int D1, int D2, int DOUT, bool TRANS, bool RELU>
__global__ void __launch_bounds__(TB) k_mp_dense(int64_t n, const float *__restrict__ X1,
                                                 const float *__restrict__ X2,
                                                 const __nv_bfloat16 *__restrict__ W,
                                                 const __nv_bfloat16 *__restrict__ bias, float *Y)
{
    constexpr int DI = D1 + D2;
    constexpr int NPB = TB / DOUT > 0 ? TB / DOUT : 1;   // nodes per pass
    __shared__ float wt[DI * DOUT];
    __shared__ float xs[NPB][DI];
    for (int t = threadIdx.x; t < DI * DOUT; t += TB) {
        const int k = t / DOUT, o = t % DOUT;             // wt[k][o]
        wt[t] = TRANS ? bf(W, k * DOUT + o) : bf(W, o * DI + k);
    }
    const int o = threadIdx.x % DOUT, slot = threadIdx.x / DOUT;
    const float b = (!TRANS && bias && threadIdx.x < NPB * DOUT) ? bf(bias, o) : 0.f;
    for (int64_t base = (int64_t)blockIdx.x * NPB; base < n; base += (int64_t)gridDim.x * NPB) {
        __syncthreads();
        for (int t = threadIdx.x; t < NPB * DI; t += TB) {
            const int s = t / DI, k = t % DI;
            const int64_t i = base + s;
            float v = 0.f;
            if (i < n) v = k < D1 ? X1[i * D1 + k] : X2[i * D2 + (k - D1)];
            xs[s][k] = v;
        }
        __syncthreads();
        const int64_t i = base + slot;
        if (slot < NPB && threadIdx.x < NPB * DOUT && i < n) {
            float acc = b;
#pragma unroll 8
            for (int k = 0; k < DI; ++k) acc = fmaf(xs[slot][k], wt[k * DOUT + o], acc);
            if (RELU) acc = fmaxf(acc, 0.f);
            Y[i * DOUT + o] = acc;
        }
    }
}

// The forward layers (TRANS = false, DOUT = H) as a register-tiled product:
// a block holds all weights (FP32, [k][o]) and a tile of 64 nodes' inputs
// (row-major, padded) in shared memory; each thread computes 4 nodes x 4
// outputs, reading four inputs of each of its nodes and four outputs' weights
// per 16-byte load (64 FMAs per 8 shared loads).  Each output accumulates
// bias + sum_k x_k w_k in ascending k with FMAs: the same order, so the same
// bits, as k_mp_dense.
constexpr int DT_NODES = 64;
template <int D1, int D2, bool RELU>
__global__ void __launch_bounds__(TB) k_mp_dense_tiled(int64_t n, const float *__restrict__ X1,
                                                       const float *__restrict__ X2,
                                                       const __nv_bfloat16 *__restrict__ W,
                                                       const __nv_bfloat16 *__restrict__ bias, float *Y)
{
    constexpr int DI = D1 + D2, XP = DI + 4;
    static_assert(DI % 4 == 0 && H == 64, "tile shape");
    extern __shared__ __align__(16) float dsm[];
    float *wt = dsm;                 // [DI][H]
    float *xs = dsm + DI * H;        // [DT_NODES][XP]
    for (int t = threadIdx.x; t < DI * H; t += TB) {
        const int k = t / H, o = t % H;
        wt[t] = bf(W, o * DI + k);
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float bv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) bv[v] = bias ? bf(bias, 4 * tx + v) : 0.f;
    const int64_t ntiles = (n + DT_NODES - 1) / DT_NODES;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * DT_NODES;
        __syncthreads();
        for (int c = threadIdx.x; c < DT_NODES * (DI / 4); c += TB) {
            const int node = c / (DI / 4), kq = c % (DI / 4), k = 4 * kq;
            const int64_t i = base + node;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n) v = k < D1 ? *reinterpret_cast<const float4 *>(X1 + i * D1 + k)
                                  : *reinterpret_cast<const float4 *>(X2 + i * D2 + (k - D1));
            *reinterpret_cast<float4 *>(xs + node * XP + k) = v;
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = bv[v];
#pragma unroll 2
        for (int k = 0; k < DI; k += 4) {
            float4 xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = *reinterpret_cast<const float4 *>(xs + (4 * ty + u) * XP + k);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float4 wv = *reinterpret_cast<const float4 *>(wt + (k + kk) * H + 4 * tx);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float xk = kk == 0 ? xv[u].x : kk == 1 ? xv[u].y : kk == 2 ? xv[u].z : xv[u].w;
                    acc[u][0] = fmaf(xk, wv.x, acc[u][0]);
                    acc[u][1] = fmaf(xk, wv.y, acc[u][1]);
                    acc[u][2] = fmaf(xk, wv.z, acc[u][2]);
                    acc[u][3] = fmaf(xk, wv.w, acc[u][3]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = base + 4 * ty + u;
            if (i >= n) continue;
            float4 o4 = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
            if (RELU) o4 = make_float4(fmaxf(o4.x, 0.f), fmaxf(o4.y, 0.f), fmaxf(o4.z, 0.f), fmaxf(o4.w, 0.f));
            *reinterpret_cast<float4 *>(Y + i * H + 4 * tx) = o4;
        }
    }
}

// A_i = mean_{j ~ i} H_j (0 for an isolated cell); one warp per node, two
// features per lane.  Neighbours in ascending column order.
__global__ void k_mp_agg(int64_t n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                         const float *__restrict__ Hm, float *A)
{
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const int32_t s0 = row_ptr[w], s1 = row_ptr[w + 1];
    float a0 = 0.f, a1 = 0.f;
    for (int32_t s = s0; s < s1; ++s) {
        const float2 v = reinterpret_cast<const float2 *>(Hm + (int64_t)col[s] * H)[lane];
        a0 += v.x;
        a1 += v.y;
    }
    const float inv = 1.0f / (float)max(s1 - s0, 1);
    reinterpret_cast<float2 *>(A + w * H)[lane] = make_float2(a0 * inv, a1 * inv);
}

// Transpose of the mean: dH_j = dSelf_j + sum_{i ~ j} dA_i / deg_i.
__global__ void k_mp_agg_t(int64_t n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                           const float *__restrict__ dU, float *dH)
{
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const float2 self = reinterpret_cast<const float2 *>(dU + w * H2)[lane];
    float a0 = self.x, a1 = self.y;
    for (int32_t s = row_ptr[w]; s < row_ptr[w + 1]; ++s) {
        const int32_t i = col[s];
        const float inv = 1.0f / (float)max(row_ptr[i + 1] - row_ptr[i], 1);
        const float2 v = reinterpret_cast<const float2 *>(dU + (int64_t)i * H2 + H)[lane];
        a0 = fmaf(v.x, inv, a0);
        a1 = fmaf(v.y, inv, a1);
    }
    reinterpret_cast<float2 *>(dH + w * H)[lane] = make_float2(a0, a1);
}

// c = W_out h3 + b_out (kept), v0 = sum_k c_k b^(k) in FP64.
__global__ void k_mp_out(int64_t n, const float *__restrict__ h3, const __nv_bfloat16 *__restrict__ Wout,
                         const __nv_bfloat16 *__restrict__ bout, const double *__restrict__ b0,
                         const double *__restrict__ b1, const double *__restrict__ b2, float *c, double *v0)
{
    __shared__ float w[KB * H + KB];
    for (int t = threadIdx.x; t < KB * H; t += blockDim.x) w[t] = bf(Wout, t);
    if (threadIdx.x < KB) w[KB * H + threadIdx.x] = bf(bout, threadIdx.x);
    __syncthreads();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float ck[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        float acc = w[KB * H + k];
        for (int f = 0; f < H; ++f) acc = fmaf(h3[i * H + f], w[k * H + f], acc);
        ck[k] = acc;
        c[i * KB + k] = acc;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        v0[3 * i + d] = (double)ck[0] * b0[3 * i + d] + (double)ck[1] * b1[3 * i + d] + (double)ck[2] * b2[3 * i + d];
}

// out[0] = x . y, out[1] = z . w over 3n values (blocks, then the last
// block in a fixed order)
__global__ void k_mp_dot2(int64_t n3, const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, const double *__restrict__ w, double *partials,
                          unsigned *counter, double *out)
{
    __shared__ double sh[TB / 32];
    double e = 0.0, t = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x) {
        e = fma(x[k], y[k], e);
        t = fma(z[k], w[k], t);
    }
    double a = block_sum<TB>(e, sh);
    if (threadIdx.x == 0) partials[2 * blockIdx.x] = a;
    double b = block_sum<TB>(t, sh);
    if (threadIdx.x == 0) partials[2 * blockIdx.x + 1] = b;
    if (last_block(counter)) {
        double A = 0.0, B = 0.0;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += TB) {
            A += __ldcg(partials + 2 * k);
            B += __ldcg(partials + 2 * k + 1);
        }
        A = block_sum<TB>(A, sh);
        B = block_sum<TB>(B, sh);
        if (threadIdx.x == 0) {
            out[0] = A;
            out[1] = B;
        }
    }
}

__global__ void k_mp_diff(int64_t n3, const double *__restrict__ a, const double *__restrict__ b, double *e)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n3) e[k] = a[k] - b[k];
}

// dc_ik = dv_i . b^(k)_i with dv = 2 g / nd[1] (g = v0 - v* for the l2
// loss, Gamma (v0 - v*) for the energy loss; nd[1] the normaliser)
__global__ void k_mp_dc(int64_t n, const double *__restrict__ g, const double *__restrict__ b0,
                        const double *__restrict__ b1, const double *__restrict__ b2, const double *__restrict__ nd,
                        float *dc)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = nd[1] > 0 ? 2.0 / nd[1] : 0.0;
    double dv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) dv[d] = s * g[3 * i + d];
    const double *bb[3] = {b0, b1, b2};
#pragma unroll
    for (int k = 0; k < KB; ++k)
        dc[i * KB + k] = (float)(dv[0] * bb[k][3 * i] + dv[1] * bb[k][3 * i + 1] + dv[2] * bb[k][3 * i + 2]);
}

// L = nd[0] / nd[1]
__global__ void k_mp_ratio(const double *__restrict__ nd, double *L)
{
    if (threadIdx.x == 0) L[0] = nd[1] > 0 ? nd[0] / nd[1] : 0.0;
}

// v0 *= alpha with alpha = nd[0] / nd[1] (the minimal-residual step), kept
// as is when the denominator vanishes or alpha is not finite
__global__ void k_mp_scale(int64_t n3, const double *__restrict__ nd, double *v0)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n3) return;
    const double den = nd[1];
    if (!(den > 0.0)) return;
    const double alpha = nd[0] / den;
    if (isfinite(alpha)) v0[k] *= alpha;
}

// dZ = dY * (Y > 0) in place (ReLU derivative from the stored activation)
__global__ void k_mp_relu_mask(int64_t cnt, const float *__restrict__ y, float *dy)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < cnt && !(y[k] > 0.f)) dy[k] = 0.f;
}

// Per-block partial of G[o][k] = sum_n dZ[n][o] X[n][k] over the block's
// CHUNK nodes, plus the bias gradient sum_n dZ[n][o] in G[DOUT][...].
template <int D1, int D2, int DOUT>
__global__ void __launch_bounds__(TB) k_mp_wgrad(int64_t n, const float *__restrict__ dZ, const float *__restrict__ X1,
                                                 const float *__restrict__ X2, float *partial)
{
    constexpr int DI = D1 + D2;
    constexpr int NG = DOUT * DI + DOUT;
    constexpr int PER = (NG + TB - 1) / TB;
    constexpr int TILE = 32;
    __shared__ float zs[TILE][DOUT];
    __shared__ float xs[TILE][DI];
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = 0.f;
    const int64_t n0 = (int64_t)blockIdx.x * CHUNK;
    const int64_t n1 = n < n0 + CHUNK ? n : n0 + CHUNK;
    for (int64_t t0 = n0; t0 < n1; t0 += TILE) {
        __syncthreads();
        for (int t = threadIdx.x; t < TILE * DOUT; t += TB) {
            const int s = t / DOUT, o = t % DOUT;
            const int64_t i = t0 + s;
            zs[s][o] = i < n1 ? dZ[i * DOUT + o] : 0.f;
        }
        for (int t = threadIdx.x; t < TILE * DI; t += TB) {
            const int s = t / DI, k = t % DI;
            const int64_t i = t0 + s;
            float v = 0.f;
            if (i < n1) v = k < D1 ? X1[i * D1 + k] : X2[i * D2 + (k - D1)];
            xs[s][k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int g = threadIdx.x + q * TB;
            if (g < NG) {
                float a = acc[q];
                if (g < DOUT * DI) {
                    const int o = g / DI, k = g % DI;
                    for (int s = 0; s < TILE; ++s) a = fmaf(zs[s][o], xs[s][k], a);
                } else {
                    const int o = g - DOUT * DI;
                    for (int s = 0; s < TILE; ++s) a += zs[s][o];
                }
                acc[q] = a;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int g = threadIdx.x + q * TB;
        if (g < NG) partial[(int64_t)blockIdx.x * NG + g] = acc[q];
    }
}

// grad[off + g] = sum over blocks (in order) of partial[b][g]
__global__ void k_mp_wsum(int nblocks, int NG, const float *__restrict__ partial, int off_w, int off_b, int nw,
                          float *grad)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= NG) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * NG + g];
    if (g < nw) grad[off_w + g] = s;
    else grad[off_b + (g - nw)] = s;
}

// Adam on the FP32 master weights; refresh the BF16 copies.
__global__ void k_mp_adam(int np, float *p, const float *__restrict__ g, float *m, float *v, __nv_bfloat16 *pb,
                          float lr, float b1, float b2, float eps, float c1, float c2)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    if (lr > 0.f) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
    pb[k] = __float2bfloat16_rn(p[k]);
}

}  // namespace

struct sgp_mpnn {
    int64_t n = 0;
    int64_t steps = 0;
    DBuf p, pb, g, m, v;              // master, BF16, gradient, Adam moments
    DBuf basis, x, hs, aggs, c, v0w;  // activations of the last prediction
    DBuf dh, du, dc, part, red;
    DBuf tmp;                         // 3 x 3n float64: e, Gamma e, Gamma v*
    const sgp_matrix *M = nullptr;
};

static sgp_status mpnn_ensure(sgp_ctx *ctx, sgp_mpnn *N, int64_t n)
{
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    SGP_TRY(buf_ensure(ctx, N->basis, sizeof(double) * 9 * nn));
    SGP_TRY(buf_ensure(ctx, N->x, sizeof(float) * DIN * nn));
    SGP_TRY(buf_ensure(ctx, N->hs, sizeof(float) * 4 * H * nn));
    SGP_TRY(buf_ensure(ctx, N->aggs, sizeof(float) * 3 * H * nn));
    SGP_TRY(buf_ensure(ctx, N->c, sizeof(float) * KB * nn));
    SGP_TRY(buf_ensure(ctx, N->v0w, sizeof(double) * 3 * nn));
    SGP_TRY(buf_ensure(ctx, N->dh, sizeof(float) * H * nn));
    SGP_TRY(buf_ensure(ctx, N->du, sizeof(float) * H2 * nn));
    SGP_TRY(buf_ensure(ctx, N->dc, sizeof(float) * KB * nn));
    const int64_t nblk = (n + CHUNK - 1) / CHUNK + 1;
    SGP_TRY(buf_ensure(ctx, N->part, sizeof(float) * (size_t)nblk * (H * H2 + H)));
    SGP_TRY(buf_ensure(ctx, N->red, sizeof(double) * 2 * 1024 + 256));
    SGP_TRY(buf_ensure(ctx, N->tmp, sizeof(double) * 12 * nn));
    N->n = n;
    return SGP_OK;
}

static unsigned red_blocks(int64_t cnt)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (cnt + TB - 1) / TB));
}

template <int D1, int D2, int DOUT, bool TRANS, bool RELU>
static sgp_status dense(sgp_ctx *ctx, int64_t n, const float *X1, const float *X2, const __nv_bfloat16 *W,
                        const __nv_bfloat16 *b, float *Y)
{
    if constexpr (!TRANS && DOUT == H && (D1 + D2) % 4 == 0 && D1 % 4 == 0) {
        // forward layers: the register-tiled kernel (shared memory above
        // 48 KB opted in once per device)
        constexpr int DI = D1 + D2;
        constexpr size_t smem = sizeof(float) * ((size_t)DI * H + (size_t)DT_NODES * (DI + 4));
        static bool opted[64] = {false};
        auto kern = k_mp_dense_tiled<D1, D2, RELU>;
        if (ctx->device >= 0 && ctx->device < 64 && !opted[ctx->device]) {
            SGP_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            opted[ctx->device] = true;
        }
        unsigned G = 1;
        SGP_TRY(resident_grid(ctx, (const void *)kern, TB, (n + DT_NODES - 1) / DT_NODES, &G));
        LAUNCH(ctx, kern, G, TB, smem, n, X1, X2, W, b, Y);
        return SGP_OK;
    }
    constexpr int NPB = TB / DOUT > 0 ? TB / DOUT : 1;
    const int64_t want = (n + NPB - 1) / NPB;
    const unsigned G = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 152 * 16));
    LAUNCH(ctx, (k_mp_dense<D1, D2, DOUT, TRANS, RELU>), G, TB, 0, n, X1, X2, W, b, Y);
    return SGP_OK;
}

template <int D1, int D2, int DOUT>
static sgp_status wgrad(sgp_ctx *ctx, sgp_mpnn *N, int64_t n, const float *dZ, const float *X1, const float *X2,
                        int off_w, int off_b)
{
    constexpr int DI = D1 + D2;
    constexpr int NG = DOUT * DI + DOUT;
    const unsigned nb = (unsigned)((n + CHUNK - 1) / CHUNK);
    float *part = bp<float>(N->part);
    LAUNCH(ctx, (k_mp_wgrad<D1, D2, DOUT>), nb, TB, 0, n, dZ, X1, X2, part);
    LAUNCH(ctx, k_mp_wsum, grid_for(NG, TB), TB, 0, (int)nb, NG, (const float *)part, off_w, off_b, DOUT * DI,
           bp<float>(N->g));
    return SGP_OK;
}

extern "C" {

sgp_status sgp_mpnn_create(sgp_ctx *ctx, const float *params, int64_t count, sgp_mpnn **out)
{
    if (!ctx || !out || !params) return SGP_ERR_INVALID_ARG;
    if (count != NPARAM)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "mpnn_create: expected %d parameters, got %lld", NPARAM,
                        (long long)count);
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    sgp_mpnn *N = new sgp_mpnn();
    *out = N;
    SGP_TRY(buf_ensure(ctx, N->p, sizeof(float) * NPARAM));
    SGP_TRY(buf_ensure(ctx, N->pb, sizeof(__nv_bfloat16) * NPARAM));
    SGP_TRY(buf_ensure(ctx, N->g, sizeof(float) * NPARAM));
    SGP_TRY(buf_ensure(ctx, N->m, sizeof(float) * NPARAM));
    SGP_TRY(buf_ensure(ctx, N->v, sizeof(float) * NPARAM));
    SGP_CUDA(ctx, cudaMemcpyAsync(N->p.p, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(N->g.p, 0, sizeof(float) * NPARAM, ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(N->m.p, 0, sizeof(float) * NPARAM, ctx->stream));
    SGP_CUDA(ctx, cudaMemsetAsync(N->v.p, 0, sizeof(float) * NPARAM, ctx->stream));
    LAUNCH(ctx, k_mp_adam, grid_for(NPARAM, TB), TB, 0, NPARAM, bp<float>(N->p), (const float *)bp<float>(N->g),
           bp<float>(N->m), bp<float>(N->v), bp<__nv_bfloat16>(N->pb), 0.f, 0.9f, 0.999f, 1e-8f, 1.f, 1.f);
    SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // params lives in caller memory
    return SGP_OK;
}

void sgp_mpnn_destroy(sgp_mpnn *N)
{
    if (!N) return;
    cudaDeviceSynchronize();
    DBuf *bufs[] = {&N->p, &N->pb, &N->g, &N->m, &N->v, &N->basis, &N->x, &N->hs, &N->aggs,
                    &N->c, &N->v0w, &N->dh, &N->du, &N->dc, &N->part, &N->red, &N->tmp};
    for (DBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    delete N;
}

sgp_status sgp_mpnn_params(sgp_ctx *ctx, const sgp_mpnn *N, float *params, float *grads)
{
    if (!ctx || !N) return SGP_ERR_INVALID_ARG;
    if (params) SGP_CUDA(ctx, cudaMemcpyAsync(params, N->p.p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, ctx->stream));
    if (grads) SGP_CUDA(ctx, cudaMemcpyAsync(grads, N->g.p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, ctx->stream));
    SGP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SGP_OK;
}

}  // extern "C"

// The forward pass in the matrix's internal cell order: F (and v_prev) are
// taken from the caller's order into N->tmp[9n, 12n) (and the third basis
// vector); the output stays in N->v0w, in internal order.
static sgp_status mpnn_forward_internal(sgp_ctx *ctx, sgp_mpnn *N, const sgp_matrix *M, const sgp_factor *Fh,
                                        const double *F, const double *v_prev)
{
    if (!ctx || !N || !M || !Fh || !F) return SGP_ERR_INVALID_ARG;
    if (Fh->n != M->n) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "mpnn_forward: factor and matrix differ in size");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = M->n;
    SGP_TRY(mpnn_ensure(ctx, N, n));
    N->M = M;
    if (n == 0) return SGP_OK;
    double *b0 = bp<double>(N->basis), *b1 = b0 + 3 * n, *b2 = b1 + 3 * n;
    double *Fi = bp<double>(N->tmp) + 9 * n;
    const int32_t *orig_of = bp<const int32_t>(M->orig_of);
    cudaEvent_t ev;
    SGP_TRY(kt_begin(ctx, SGP_KT_WARM_BASIS, &ev));
    LAUNCH(ctx, k_to_internal<double>, grid_for(n, TB), TB, 0, n, orig_of, F, Fi);
    // basis: block-Jacobi solve, spanning-forest solve, previous velocity
    SGP_TRY(matrix_block_jacobi(ctx, const_cast<sgp_matrix *>(M)));
    LAUNCH(ctx, k_mp_jacobi, grid_for(n, TB), TB, 0, n, bp<const double>(M->jac), (const double *)Fi, b0);
    SGP_CUDA(ctx, cudaMemcpyAsync(b1, Fi, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    SGP_TRY(tree_apply_inplace<double>(ctx, Fh, b1, nullptr));
    if (v_prev) LAUNCH(ctx, k_to_internal<double>, grid_for(n, TB), TB, 0, n, orig_of, v_prev, b2);
    else SGP_CUDA(ctx, cudaMemsetAsync(b2, 0, sizeof(double) * 3 * n, ctx->stream));
    double *red = bp<double>(N->red);
    unsigned *counter = reinterpret_cast<unsigned *>(red + 2 * 1024 + 8);
    double *mean_b1 = red + 2 * 1024;
    SGP_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx->stream));
    const unsigned G = (unsigned)std::min<int64_t>(1024, (n + TB - 1) / TB);
    LAUNCH(ctx, k_mp_norm_sum, G, TB, 0, n, (const double *)b1, red, counter, mean_b1);
    float *x = bp<float>(N->x);
    LAUNCH(ctx, k_mp_features, grid_for(n, TB), TB, 0, n, (const double *)b0, (const double *)b1,
           (const double *)b2, bp<const int32_t>(M->row_ptr), (const double *)mean_b1, x);
    SGP_TRY(kt_end(ctx, SGP_KT_WARM_BASIS, ev));
    SGP_TRY(kt_begin(ctx, SGP_KT_WARM_LAYERS, &ev));
    // forward
    const __nv_bfloat16 *pb = bp<const __nv_bfloat16>(N->pb);
    float *hs = bp<float>(N->hs), *aggs = bp<float>(N->aggs);
    SGP_TRY((dense<DIN, 0, H, false, true>(ctx, n, x, nullptr, pb + OFF_WIN, pb + OFF_BIN, hs)));
    for (int l = 0; l < 3; ++l) {
        float *h = hs + (int64_t)l * H * n, *a = aggs + (int64_t)l * H * n, *hn = hs + (int64_t)(l + 1) * H * n;
        LAUNCH(ctx, k_mp_agg, grid_for(32 * n, TB), TB, 0, n, bp<const int32_t>(M->row_ptr),
               bp<const int32_t>(M->col), (const float *)h, a);
        const int off = OFF_L0 + l * LAYER;
        SGP_TRY((dense<H, H, H, false, true>(ctx, n, h, a, pb + off, pb + off + H * H2, hn)));
    }
    LAUNCH(ctx, k_mp_out, grid_for(n, TB), TB, 0, n, (const float *)(hs + 3 * H * n), pb + OFF_WOUT, pb + OFF_BOUT,
           (const double *)b0, (const double *)b1, (const double *)b2, bp<float>(N->c), bp<double>(N->v0w));
    SGP_TRY(kt_end(ctx, SGP_KT_WARM_LAYERS, ev));
    return SGP_OK;
}

extern "C" {

sgp_status sgp_mpnn_forward(sgp_ctx *ctx, sgp_mpnn *N, const sgp_matrix *M, const sgp_factor *Fh,
                            const double *F, const double *v_prev, double *v0)
{
    if (!v0) return SGP_ERR_INVALID_ARG;
    SGP_TRY(mpnn_forward_internal(ctx, N, M, Fh, F, v_prev));
    const int64_t n = M->n;
    if (n > 0)
        LAUNCH(ctx, k_to_caller<double>, grid_for(n, TB), TB, 0, n, bp<const int32_t>(M->orig_of),
               bp<const double>(N->v0w), v0);
    return SGP_OK;
}

sgp_status sgp_mpnn_backward(sgp_ctx *ctx, sgp_mpnn *N, const double *v_target, int32_t loss_kind, double *loss)
{
    if (!ctx || !N || !N->M) return SGP_ERR_INVALID_ARG;
    if (loss_kind != SGP_MPNN_LOSS_L2 && loss_kind != SGP_MPNN_LOSS_ENERGY)
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "mpnn_backward: unknown loss");
    if (N->n > 0 && !v_target) return SGP_ERR_INVALID_ARG;
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = N->n;
    if (n == 0) {
        SGP_CUDA(ctx, cudaMemsetAsync(N->g.p, 0, sizeof(float) * NPARAM, ctx->stream));
        if (loss) *loss = 0.0;
        return SGP_OK;
    }
    const sgp_matrix *M = N->M;
    const double *b0 = bp<const double>(N->basis), *b1 = b0 + 3 * n, *b2 = b1 + 3 * n;
    const double *v0 = bp<const double>(N->v0w);
    double *red = bp<double>(N->red);
    unsigned *counter = reinterpret_cast<unsigned *>(red + 2 * 1024 + 8);
    double *nd = red + 2 * 1024 + 2, *lossout = red + 2 * 1024 + 4;
    double *e = bp<double>(N->tmp), *Ge = e + 3 * n, *Gt = Ge + 3 * n, *vt = Gt + 3 * n;
    LAUNCH(ctx, k_to_internal<double>, grid_for(n, TB), TB, 0, n, bp<const int32_t>(M->orig_of), v_target, vt);
    v_target = vt;
    const unsigned G = red_blocks(3 * n);
    LAUNCH(ctx, k_mp_diff, grid_for(3 * n, TB), TB, 0, 3 * n, v0, v_target, e);
    const double *g = e;
    if (loss_kind == SGP_MPNN_LOSS_ENERGY) {
        SGP_TRY(spmv64(ctx, M, e, Ge));
        SGP_TRY(spmv64(ctx, M, v_target, Gt));
        LAUNCH(ctx, k_mp_dot2, G, TB, 0, 3 * n, (const double *)e, (const double *)Ge, v_target, (const double *)Gt,
               red, counter, nd);
        g = Ge;
    } else {
        LAUNCH(ctx, k_mp_dot2, G, TB, 0, 3 * n, (const double *)e, (const double *)e, v_target, v_target, red,
               counter, nd);
    }
    LAUNCH(ctx, k_mp_ratio, 1, 32, 0, (const double *)nd, lossout);
    float *dc = bp<float>(N->dc), *dh = bp<float>(N->dh), *du = bp<float>(N->du);
    const float *hs = bp<const float>(N->hs), *aggs = bp<const float>(N->aggs), *x = bp<const float>(N->x);
    const __nv_bfloat16 *pb = bp<const __nv_bfloat16>(N->pb);
    LAUNCH(ctx, k_mp_dc, grid_for(n, TB), TB, 0, n, g, b0, b1, b2, (const double *)nd, dc);
    // output layer
    SGP_TRY((wgrad<H, 0, KB>(ctx, N, n, dc, hs + 3 * H * n, nullptr, OFF_WOUT, OFF_BOUT)));
    SGP_TRY((dense<KB, 0, H, true, false>(ctx, n, dc, nullptr, pb + OFF_WOUT, nullptr, dh)));
    for (int l = 2; l >= 0; --l) {
        const float *hn = hs + (int64_t)(l + 1) * H * n, *h = hs + (int64_t)l * H * n, *a = aggs + (int64_t)l * H * n;
        LAUNCH(ctx, k_mp_relu_mask, grid_for(H * n, TB), TB, 0, H * n, hn, dh);
        const int off = OFF_L0 + l * LAYER;
        SGP_TRY((wgrad<H, H, H>(ctx, N, n, dh, h, a, off, off + H * H2)));
        SGP_TRY((dense<H, 0, H2, true, false>(ctx, n, dh, nullptr, pb + off, nullptr, du)));
        LAUNCH(ctx, k_mp_agg_t, grid_for(32 * n, TB), TB, 0, n, bp<const int32_t>(M->row_ptr),
               bp<const int32_t>(M->col), (const float *)du, dh);
    }
    LAUNCH(ctx, k_mp_relu_mask, grid_for(H * n, TB), TB, 0, H * n, hs, dh);
    SGP_TRY((wgrad<DIN, 0, H>(ctx, N, n, dh, x, nullptr, OFF_WIN, OFF_BIN)));
    if (loss) SGP_TRY(read_back(ctx, loss, lossout, sizeof(double)));
    return SGP_OK;
}

sgp_status sgp_mpnn_step(sgp_ctx *ctx, sgp_mpnn *N, float lr)
{
    if (!ctx || !N) return SGP_ERR_INVALID_ARG;
    if (!(lr > 0.f) || !std::isfinite(lr))
        return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "mpnn_step: learning rate must be positive");
    SGP_CUDA(ctx, cudaSetDevice(ctx->device));
    N->steps++;
    const float c1 = 1.f - powf(0.9f, (float)N->steps);
    const float c2 = 1.f - powf(0.999f, (float)N->steps);
    LAUNCH(ctx, k_mp_adam, grid_for(NPARAM, TB), TB, 0, NPARAM, bp<float>(N->p), bp<const float>(N->g),
           bp<float>(N->m), bp<float>(N->v), bp<__nv_bfloat16>(N->pb), lr, 0.9f, 0.999f, 1e-8f, c1, c2);
    return SGP_OK;
}

}  // extern "C"

// The residual check of the warm start lives with the solver's product; it
// closes the timing bracket `ev` of class kclass before its read-back.
sgp_status mpnn_residual_check(sgp_ctx *ctx, const sgp_matrix *M, const double *F, double *v0, int *used,
                               int kclass, cudaEvent_t ev);

extern "C" sgp_status sgp_warm_start(sgp_ctx *ctx, sgp_mpnn *N, const sgp_matrix *M, const sgp_factor *Fh,
                                     const double *F, const double *v_prev, double *v0, int32_t flags,
                                     int32_t *used)
{
    if (flags & ~SGP_WARM_MR_SCALE) return sgp_fail(ctx, SGP_ERR_INVALID_ARG, "warm_start: unknown flags");
    if (!v0) return SGP_ERR_INVALID_ARG;
    SGP_TRY(mpnn_forward_internal(ctx, N, M, Fh, F, v_prev));
    const int64_t n = M->n;
    if (n == 0) {
        if (used) *used = 0;
        return SGP_OK;
    }
    // scaling and acceptance on a copy of the network output (internal order);
    // N->v0w stays the network's own output for a following backward pass
    double *Gv = bp<double>(N->tmp), *w = Gv + 3 * n;
    const double *Fi = bp<const double>(N->tmp) + 9 * n;
    cudaEvent_t ev;
    SGP_TRY(kt_begin(ctx, SGP_KT_WARM_CHECK, &ev));
    SGP_CUDA(ctx, cudaMemcpyAsync(w, N->v0w.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    int u = 0;
    bool checked = false;
    if (flags & SGP_WARM_MR_SCALE) {
        double *red = bp<double>(N->red);
        unsigned *counter = reinterpret_cast<unsigned *>(red + 2 * 1024 + 8);
        double *nd = red + 2 * 1024 + 2;
        SGP_TRY(spmv64(ctx, M, w, Gv));
        LAUNCH(ctx, k_mp_dot2, red_blocks(3 * n), TB, 0, 3 * n, (const double *)Gv, Fi, (const double *)Gv,
               (const double *)Gv, red, counter, nd);
        LAUNCH(ctx, k_mp_scale, grid_for(3 * n, TB), TB, 0, 3 * n, (const double *)nd, w);
        // with a finite step alpha = (Gamma v0)^T F / |Gamma v0|^2 the scaled
        // guess has |F - alpha Gamma v0|^2 = |F|^2 - ((Gamma v0)^T F)^2 /
        // |Gamma v0|^2 <= |F|^2: the acceptance test holds without a second
        // product
        SGP_TRY(kt_end(ctx, SGP_KT_WARM_CHECK, ev));
        double h[2] = {0.0, 0.0};
        SGP_TRY(read_back(ctx, h, nd, sizeof(h)));
        if (h[1] > 0.0 && std::isfinite(h[0] / h[1])) {
            u = 1;
            checked = true;
        } else {
            SGP_TRY(kt_begin(ctx, SGP_KT_WARM_CHECK, &ev));
        }
    }
    if (!checked) SGP_TRY(mpnn_residual_check(ctx, M, Fi, w, &u, SGP_KT_WARM_CHECK, ev));
    LAUNCH(ctx, k_to_caller<double>, grid_for(n, TB), TB, 0, n, bp<const int32_t>(M->orig_of), (const double *)w,
           v0);
    if (used) *used = u;
    return SGP_OK;
}
