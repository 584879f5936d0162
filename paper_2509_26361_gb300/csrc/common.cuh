// common.cuh -- grid indexing and shared device helpers for the EBIT kernels.
//
// The whole EBIT translation unit is compiled with --fmad=false: every product
// and sum is its own IEEE double operation in the written order, and double
// division and square root are IEEE round-to-nearest (CUDA defaults).  The
// floating-point decisions of the method (which node a marker crossed, which
// circle root lies on an edge, the colour of a saddle face) therefore do not
// depend on compiler contraction.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ebit {

constexpr double ONE_MINUS = 0.99999999999999988898;  // 1 - 2^-53, largest offset below 1
constexpr int TILE = 8;                               // tile edge (cells)
constexpr int TILE_CELLS = TILE * TILE * TILE;

enum Counter { C_MARKERS = 0, C_ANNIHILATE = 1, C_MULTI = 2, C_INCONSISTENT = 3, C_CFL = 4, C_N = 5 };
// extra device counters after the event counters
enum { C_F2V_BAD = C_N, C_TILES = C_N + 1, C_TOTAL = C_N + 2 };

struct Grid {
    int n[3];        // cells per axis
    int td[3];       // tiles per axis
    int ntiles;
};

__host__ __device__ inline int wrapc(int v, int n) {
    // v is within a few cells of [0, n)
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

__device__ __forceinline__ int lin(const Grid &g, int x, int y, int z) {
    return (wrapc(z, g.n[2]) * g.n[1] + wrapc(y, g.n[1])) * g.n[0] + wrapc(x, g.n[0]);
}

__device__ __forceinline__ int lin3(const Grid &g, const int q[3]) { return lin(g, q[0], q[1], q[2]); }

// tile id -> origin of its cells
__device__ __forceinline__ void tile_origin(const Grid &g, int t, int o[3]) {
    int tx = t % g.td[0];
    int r = t / g.td[0];
    int ty = r % g.td[1];
    int tz = r / g.td[1];
    o[0] = tx * TILE;
    o[1] = ty * TILE;
    o[2] = tz * TILE;
}

// one atomicAdd per warp for a per-thread counter increment
__device__ __forceinline__ void warp_count(unsigned long long *ctr, unsigned v) {
    unsigned m = __activemask();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    int leader = __ffs(m) - 1;
    if ((int)(threadIdx.x & 31) == leader && v) atomicAdd(ctr, (unsigned long long)v);
}

}  // namespace ebit
