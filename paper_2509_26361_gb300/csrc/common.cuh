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

// Programmatic dependent launch.  The kernels of a step are launched with
// programmatic stream serialization, so the next kernel in the stream is
// launched as the blocks of the current one exit, overlapping its launch with
// the current kernel's tail.  Every such kernel calls pdl_wait() before its
// first access to global memory: it returns once the preceding kernel has
// completed and its writes are visible (and so, by induction, every earlier
// one).  None of them releases its dependents early
// (griddepcontrol.launch_dependents): grids sized to full occupancy then had
// the next kernel's waiting blocks take the slots of exiting ones unevenly,
// which measured slower than the release at exit.  For an ordinary launch
// pdl_wait() is a no-op.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Entry of a compacted work list for this thread in iteration `it` of a
// grid-stride loop over the list.  Whole warps of consecutive entries are dealt
// to the blocks in turn (warp slot 0 of every block, then slot 1, ...), so a
// list much shorter than the grid spreads over all SMs instead of filling the
// first blocks; every entry maps to one thread of one iteration.
__device__ __forceinline__ int list_item(int it) {
    const int gw = (it * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5)) * (int)gridDim.x + (int)blockIdx.x;
    return gw * 32 + (int)(threadIdx.x & 31);
}

constexpr double ONE_MINUS = 0.99999999999999988898;  // 1 - 2^-53, largest offset below 1
constexpr int TILE = 8;                               // tile edge of a single grid (cells)
constexpr int TILE_CELLS = TILE * TILE * TILE;          // cells of every tile shape

// Tile shapes (cells per tile edge along x, y, z; 512 cells each).  A single
// grid uses shape 0; a batch may use any (chosen by its autotuner).  Every
// edge is at least 4 cells, more than the NEAR = 3 layers of the proximity
// mask, so a marker can only touch its own tile and the 26 adjacent ones.
constexpr int N_TILE_SHAPES = 3;
__host__ __device__ constexpr int tile_log2(int sh, int a) {
    return sh == 0 ? 3 : (sh == 1 ? (a == 0 ? 4 : (a == 1 ? 3 : 2)) : (a == 0 ? 5 : 2));
}
template <int SH>
struct TileShape {
    static constexpr int LX = tile_log2(SH, 0), LY = tile_log2(SH, 1), LZ = tile_log2(SH, 2);
    static constexpr int TX = 1 << LX, TY = 1 << LY, TZ = 1 << LZ;
    static_assert(TX * TY * TZ == TILE_CELLS, "512 cells per tile");
    static_assert(TX >= 4 && TY >= 4 && TZ >= 4, "tile edges of at least 4 cells");
    static constexpr int t(int a) { return a == 0 ? TX : (a == 1 ? TY : TZ); }
    // cell c of a tile -> its local coordinates (x fastest)
    __device__ static void cell(int c, int l[3]) {
        l[0] = c & (TX - 1);
        l[1] = (c >> LX) & (TY - 1);
        l[2] = c >> (LX + LY);
    }
};

// Tile proximity mask: bit near_bit(dx, dy, dz) is set when a marker owned by a
// node of the tile lies within NEAR cells of the neighbour tile in direction
// (dx, dy, dz) (the owner node in the NEAR layers next to that neighbour, along
// every axis with a non-zero step); bit near_bit(0, 0, 0) whenever the tile
// owns a marker.  A sweep changes a node's byte or edges only if a marker is
// owned by a node within one cell behind or two cells ahead of it (the window of
// the band pass), and Front2VOF reads a cell's corners one cell ahead, so a
// tile next to a marker tile needs the sweep (and Front2VOF) only where that
// neighbour owns a marker within three cells of it.
constexpr int NEAR = 3;
__host__ __device__ inline int near_bit(int dx, int dy, int dz) { return 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1); }
// (lx, ly, lz: the node's place in a tile of tx x ty x tz cells)
__host__ __device__ inline unsigned near_bits(int lx, int ly, int lz, int tx = TILE, int ty = TILE, int tz = TILE) {
    unsigned m = 0;
    for (int dz = -1; dz <= 1; dz++) {
        if ((dz < 0 && lz >= NEAR) || (dz > 0 && lz < tz - NEAR)) continue;
        for (int dy = -1; dy <= 1; dy++) {
            if ((dy < 0 && ly >= NEAR) || (dy > 0 && ly < ty - NEAR)) continue;
            for (int dx = -1; dx <= 1; dx++) {
                if ((dx < 0 && lx >= NEAR) || (dx > 0 && lx < tx - NEAR)) continue;
                m |= 1u << near_bit(dx, dy, dz);
            }
        }
    }
    return m;
}

enum Counter { C_MARKERS = 0, C_ANNIHILATE = 1, C_MULTI = 2, C_INCONSISTENT = 3, C_CFL = 4, C_N = 5 };
// extra device counters after the event counters (C_NONFINITE: markers whose
// displacement u dt / h was not finite; they are left in place)
enum { C_F2V_BAD = C_N, C_TILES = C_N + 1, C_NONFINITE = C_N + 2, C_TOTAL = C_N + 3 };

struct Grid {
    int n[3];        // cells per axis
    int td[3];       // tiles per axis
    int ntiles;
    int tl[3];       // log2 of the tile edge per axis (3, 3, 3 for 8^3 tiles)
};

// tiles per axis and in total for tile shape sh
__host__ __device__ inline void grid_tiles(Grid &g, int sh) {
    g.ntiles = 1;
    for (int a = 0; a < 3; a++) {
        g.tl[a] = tile_log2(sh, a);
        g.td[a] = (g.n[a] + (1 << g.tl[a]) - 1) >> g.tl[a];
        g.ntiles *= g.td[a];
    }
}

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
    o[0] = tx << g.tl[0];
    o[1] = ty << g.tl[1];
    o[2] = tz << g.tl[2];
}

// cell c (0 .. 511) of a tile of g's shape -> its local coordinates
__device__ __forceinline__ void tile_cell(const Grid &g, int c, int l[3]) {
    l[0] = c & ((1 << g.tl[0]) - 1);
    l[1] = (c >> g.tl[0]) & ((1 << g.tl[1]) - 1);
    l[2] = c >> (g.tl[0] + g.tl[1]);
}

// one atomicAdd per warp for a per-thread counter increment
__device__ __forceinline__ void warp_count(unsigned long long *ctr, unsigned v) {
    unsigned m = __activemask();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    int leader = __ffs(m) - 1;
    if ((int)(threadIdx.x & 31) == leader && v) atomicAdd(ctr, (unsigned long long)v);
}

// Is tile (tx, ty, tz) in the band: does it own a marker, or does a neighbour
// own one within NEAR cells of it (that neighbour's proximity bit toward it)?
// (the 27 loads are independent: no early exit)
__device__ __forceinline__ bool in_band(const Grid &g, const uint32_t *__restrict__ mask, int tx, int ty, int tz) {
    unsigned on = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; dz++)
#pragma unroll
        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
            for (int dx = -1; dx <= 1; dx++) {
                const int nx = wrapc(tx + dx, g.td[0]), ny = wrapc(ty + dy, g.td[1]), nz = wrapc(tz + dz, g.td[2]);
                on |= mask[(nz * g.td[1] + ny) * g.td[0] + nx] >> near_bit(-dx, -dy, -dz);
            }
    return on & 1u;
}

// Youngs normal n = -grad C of a 3x3x3 block (1-2-1 weights, b2 outer, b1
// inner), in the type T of the block values.
template <typename T>
__device__ __forceinline__ void youngs(const T (&v)[27], T n[3]) {
    const T w[3] = {T(1), T(2), T(1)};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        T gsum = T(0);
#pragma unroll
        for (int b2 = -1; b2 <= 1; b2++)
#pragma unroll
            for (int b1 = -1; b1 <= 1; b1++) {
                int op[3] = {1, 1, 1}, om[3] = {1, 1, 1};
                op[d] += 1;
                om[d] -= 1;
                op[t1] += b1;
                om[t1] += b1;
                op[t2] += b2;
                om[t2] += b2;
                gsum += (w[b1 + 1] * w[b2 + 1]) * (v[op[2] * 9 + op[1] * 3 + op[0]] - v[om[2] * 9 + om[1] * 3 + om[0]]);
            }
        n[d] = -gsum;
    }
}

// Bound on |n_float - n| for values rounded to float: 8 additions below 64
// (half an ulp, 2^-19, each) and the inputs' rounding (2^-25 each, weights
// summing to 16, three roundings per difference) stay under 1.7e-5.
constexpr float CANON_EPS = 3.0e-5f;

}  // namespace ebit
