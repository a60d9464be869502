// solver_common.cuh -- device helpers shared by the single and the batched
// PCG drivers: loads of one directed slot's block, and 16-byte packs of
// vector entries.
#pragma once

#include "sgp_internal.cuh"

namespace {

// The device scalars of one PCG run (rho = r^T z, the step lengths, the
// stopping test, the arrival counter of the last-block reductions, the body
// count of a device-side iteration loop).
struct Scal {
    double rho, alpha, beta, FF, stop2, rr, rz, pq;
    long long it, maxit;
    int done, status;
    unsigned cnt;
    int pad;
    int xpend;   // the step's x += alpha p is still to be applied
    // Gauss-Radau bound of the Gamma-norm error (mu > 0): phi, the sum of
    // alpha_j rho_j so far, the bound phi rho; stopE: stop on it (tolE2 = tol^2)
    double mu, phi, gsum, est, tolE2;
    int stopE;
};

// The end of a step's r^T z reduction: beta = rz / rho, rho = rz, or a
// breakdown when rz is not positive.  Also the Gauss-Radau recursion of the
// Gamma-norm error (phi <- (phi - alpha) / (mu (phi - alpha) + beta), bound
// phi rho) and, in error mode, the stopping test on it.
__device__ __forceinline__ void rz_finish(Scal *sc, double rz)
{
    if (!(rz > 0.0) || !isfinite(rz)) {
        sc->done = 1;
        if (!(sc->stopE && rz == 0.0)) sc->status = SGP_ERR_NOT_SPD;   // rz = 0: solved exactly
        return;
    }
    const double alpha = sc->alpha, rho = sc->rho;
    sc->beta = rz / rho;
    sc->rho = rz;
    sc->rz = rz;
    if (sc->mu > 0.0) {
        sc->gsum += alpha * rho;
        const double d = sc->phi - alpha;
        sc->phi = d / (sc->mu * d + sc->beta);
        sc->est = sc->phi * rz;
        if (sc->stopE && sc->est <= sc->tolE2 * sc->gsum) sc->done = 1;
    }
}

// One directed slot of the block-sparse rows: the symmetric 3x3 block and
// the column.  FP64: 6 doubles (three 16-byte loads) plus the column array;
// FP32: an 8-float record (6 floats, the column's bits, pad; two loads).
template <typename T> struct Blk;
// fetch() issues a slot's loads, expand() turns them into the six entries
// and the column (split so that the next slot's loads can be in flight
// while the current one is used).
template <> struct Blk<double> {
    const int32_t *col;
    const double *blk;
    struct Raw {
        double2 a, b, c;
        int32_t j;
    };
    __device__ __forceinline__ Raw fetch(int32_t s) const
    {
        const double2 *b2 = reinterpret_cast<const double2 *>(blk + 6 * (int64_t)s);
        return Raw{b2[0], b2[1], b2[2], col[s]};
    }
    __device__ __forceinline__ void expand(const Raw &r, double *S, int32_t &j) const
    {
        S[0] = r.a.x; S[1] = r.a.y; S[2] = r.b.x; S[3] = r.b.y; S[4] = r.c.x; S[5] = r.c.y;
        j = r.j;
    }
    __device__ __forceinline__ void load(int32_t s, double *S, int32_t &j) const { expand(fetch(s), S, j); }
};
// FP32: the block is kept in the form of eq. (1), Upsilon = g_perp I +
// (g_par - g_perp) u u^T: a 16-byte record (g_perp, g_par - g_perp, u_x, u_y)
// and an 8-byte record (u_z, the column as int bits), 24 bytes per slot
// instead of 32 for the six entries plus column; the entries are rebuilt in
// registers.
template <> struct Blk<float> {
    const float4 *a;
    const float2 *b;
    struct Raw {
        float4 x;
        float2 y;
    };
    __device__ __forceinline__ Raw fetch(int32_t s) const { return Raw{a[s], b[s]}; }
    __device__ __forceinline__ void load(int32_t s, float *S, int32_t &j) const { expand(fetch(s), S, j); }
    __device__ __forceinline__ void expand(const Raw &r, float *S, int32_t &j) const
    {
        const float4 x = r.x;
        const float2 y = r.y;
        const float gq = x.x, dg = x.y, ux = x.z, uy = x.w, uz = y.x;
        const float dx = dg * ux, dy = dg * uy;
        S[0] = fmaf(dx, ux, gq);
        S[1] = dx * uy;
        S[2] = dx * uz;
        S[3] = fmaf(dy, uy, gq);
        S[4] = dy * uz;
        S[5] = fmaf(dg * uz, uz, gq);
        j = __float_as_int(y.y);
    }
};

template <typename T>
Blk<T> make_blk(const sgp_matrix *M);
template <>
inline Blk<double> make_blk<double>(const sgp_matrix *M)
{
    return Blk<double>{bp<const int32_t>(M->col), bp<const double>(M->blk)};
}
template <>
inline Blk<float> make_blk<float>(const sgp_matrix *M)
{
    const float4 *a = bp<const float4>(M->blk32);
    return Blk<float>{a, reinterpret_cast<const float2 *>(a + 2 * M->m)};
}

// Row i of the Appendix B.2 product accumulated with fused multiply-adds:
// y += sum over the row's slots s0, s0+step, ... of Upsilon (v_i - v_j).
template <typename T>
__device__ __forceinline__ void row_accumulate(const Blk<T> &B, int32_t s0, int32_t s1, int step,
                                               const T *__restrict__ p, T v0, T v1, T v2, T &y0, T &y1,
                                               T &y2)
{
    for (int32_t s = s0; s < s1; s += step) {
        T S[6];
        int32_t j;
        B.load(s, S, j);
        const T d0 = v0 - p[3 * (int64_t)j], d1 = v1 - p[3 * (int64_t)j + 1], d2 = v2 - p[3 * (int64_t)j + 2];
        y0 = fma(S[0], d0, y0); y0 = fma(S[1], d1, y0); y0 = fma(S[2], d2, y0);
        y1 = fma(S[1], d0, y1); y1 = fma(S[3], d1, y1); y1 = fma(S[4], d2, y1);
        y2 = fma(S[2], d0, y2); y2 = fma(S[4], d1, y2); y2 = fma(S[5], d2, y2);
    }
}

// 16-byte packs of vector entries (4 floats or 2 doubles): streaming
// kernels treat the n x 3 vectors as flat arrays of 3n entries.
template <typename T>
struct alignas(16) Pack {
    static constexpr int K = 16 / sizeof(T);
    T v[K];
};

}  // namespace
