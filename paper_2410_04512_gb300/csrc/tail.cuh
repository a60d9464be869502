// tail.cuh -- the tree solve's one-block "tail" (the last contraction
// levels solved by one thread block with its arrays in shared memory):
// its description and shared-memory sizes, shared by the level solve and
// the one-block PCG of small systems.
#pragma once
#include "sgp_internal.cuh"

// shared-memory carving: every piece starts on a 16-byte boundary
__host__ __device__ inline size_t tail_align(size_t b) { return (b + 15) & ~size_t(15); }

// The last levels (the vertices at elimination positions >= P0) in one
// thread block with every array they use staged in shared memory: vectors,
// D^-1 and L blocks by local index (position - P0, pair - Q0), and the local
// index lists built at factorisation time.  Levels are separated by block
// barriers; forward upwards, then backward downwards.
struct Tail {
    int32_t nlev, n, np, nr, P0, Q0, R0, C0;
    const int32_t *lvl_pos;   // nlev + 1 absolute positions
    const int32_t *lvl_rv;    // nlev + 1 absolute receiver-list offsets
    const int32_t *tq;        // nr: local receiver of each receiver entry
    const int32_t *tb;        // np: local receiver of each pair
    const int32_t *tpc;       // np: local contributor of each pair
    const int32_t *tct;       // np: local pair of each contributor entry
};


template <typename T>
__host__ __device__ inline size_t tail_smem_bytes(int32_t n, int32_t np, int32_t nr)
{
    return tail_align(sizeof(T) * 3 * (size_t)n) + tail_align(4 * (size_t)(n + 1)) + 3 * tail_align(4 * (size_t)np) +
           tail_align(4 * (size_t)(nr + 1)) + tail_align(4 * (size_t)nr);
}

// The vectors and the local index lists live in shared memory; when they fit
// (STAGE), D^-1 and the L blocks are staged there as well before the wait on
// the previous kernel, otherwise they stream from global memory in level
// order (each is read once per direction).
template <typename T>
__host__ __device__ inline size_t tail_smem_staged(int32_t n, int32_t np, int32_t nr)
{
    return tail_smem_bytes<T>(n, np, nr) + tail_align(sizeof(T) * 6 * (size_t)n) + tail_align(sizeof(T) * 9 * (size_t)np);
}

// The tail of a factor (built at factorisation time).
Tail tail_of(const sgp_factor *F);
