// amr.cuh -- the AMR refinement rule of 3D EBIT (arxiv 2509.26361, Sec. 2.5)
// and a narrow-band brick store of the state built on it.
//
// Sec. 2.5: with one marker per edge, cells of two refinement levels must
// never share the interface, so every cell within the 3x3x3 block around an
// interfacial cell is refined to the finest level.  A cell is interfacial when
// its eight corner colours differ (an edge carries a marker exactly when its
// end colours differ).  The brick store keeps the state of the 8^3 tiles that
// hold a refined cell, and one colour per other tile: such a tile contains no
// interfacial cell, so its cells share one colour, its edges carry no marker
// and its faces store their corner colour.
#pragma once
#include "common.cuh"

namespace ebit {

constexpr int AMR_R = TILE + 3;   // staged nodes per axis: -1 .. TILE + 1
constexpr int AMR_F = TILE + 2;   // interfacial flags of cells -1 .. TILE

// Per tile: the refinement mask of its cells (mask may be null), whether any
// of them is refined (flag), the colour of its origin node (bg), and the
// number of refined cells (count).  One block of 256 threads per tile.
__global__ void __launch_bounds__(256) refine_kernel(Grid g, const uint8_t *__restrict__ cb, uint8_t *__restrict__ mask,
                                                     int *__restrict__ flag, uint8_t *__restrict__ bg,
                                                     unsigned long long *__restrict__ count) {
    __shared__ uint8_t s_c[AMR_R * AMR_R * AMR_R];
    __shared__ uint8_t s_f[AMR_F * AMR_F * AMR_F];
    for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        int o[3];
        tile_origin(g, tile, o);
        int seen = 0;
        for (int r = threadIdx.x; r < AMR_R * AMR_R * AMR_R; r += blockDim.x) {
            const int rx = r % AMR_R, ry = (r / AMR_R) % AMR_R, rz = r / (AMR_R * AMR_R);
            const uint8_t c = __ldg(cb + lin(g, o[0] + rx - 1, o[1] + ry - 1, o[2] + rz - 1)) & 1;
            s_c[r] = c;
            seen |= c ? 1 : 2;
        }
        const int has1 = __syncthreads_or(seen & 1), has0 = __syncthreads_or(seen & 2);
        if (threadIdx.x == 0) bg[tile] = s_c[1 + AMR_R * (1 + AMR_R)];  // the origin node
        unsigned nref = 0;
        int any = 0;
        if (has1 && has0) {
            // interfacial flags of the cells -1 .. TILE around the tile
            for (int r = threadIdx.x; r < AMR_F * AMR_F * AMR_F; r += blockDim.x) {
                const int fx = r % AMR_F, fy = (r / AMR_F) % AMR_F, fz = r / (AMR_F * AMR_F);
                int lo = 1, hi = 0;
#pragma unroll
                for (int d = 0; d < 8; d++) {
                    const int c = s_c[(fx + (d & 1)) + AMR_R * ((fy + ((d >> 1) & 1)) + AMR_R * (fz + (d >> 2)))];
                    lo &= c;
                    hi |= c;
                }
                s_f[r] = (uint8_t)(hi & ~lo);
            }
            __syncthreads();
            for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
                const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
                const bool valid = o[0] + lx < g.n[0] && o[1] + ly < g.n[1] && o[2] + lz < g.n[2];
                int ref = 0;
#pragma unroll
                for (int d = 0; d < 27; d++)
                    ref |= s_f[(lx + d % 3) + AMR_F * ((ly + (d / 3) % 3) + AMR_F * (lz + d / 9))];
                ref = valid ? ref : 0;
                if (valid && mask) mask[lin(g, o[0] + lx, o[1] + ly, o[2] + lz)] = (uint8_t)ref;
                nref += ref;
                any |= ref;
            }
        } else if (mask) {
            for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
                const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
                if (o[0] + lx < g.n[0] && o[1] + ly < g.n[1] && o[2] + lz < g.n[2])
                    mask[lin(g, o[0] + lx, o[1] + ly, o[2] + lz)] = 0;
            }
        }
        const int tile_any = __syncthreads_or(any);
        const unsigned v = __reduce_add_sync(0xffffffffu, nref);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(count, (unsigned long long)v);
        if (threadIdx.x == 0) flag[tile] = tile_any ? 1 : 0;
        __syncthreads();  // the staging is rewritten by the next tile
    }
}

// Ascending ids of the flagged tiles into out[0 .. cap) and their number into
// *n_out (one block: each thread scans a contiguous run of tiles).
__global__ void __launch_bounds__(1024) compact_tiles_kernel(const int *__restrict__ flag, int nt,
                                                             int *__restrict__ out, int cap, int *__restrict__ n_out) {
    __shared__ int s_w[32];
    const int per = (nt + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(nt, b0 + per);
    int cnt = 0;
    for (int t = b0; t < b1; t++) cnt += flag[t];
    // block-wide exclusive scan of cnt
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += v;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += v;
        }
        s_w[lane] = w;  // inclusive prefix over warps
    }
    __syncthreads();
    int pos = (wid ? s_w[wid - 1] : 0) + inc - cnt;
    for (int t = b0; t < b1; t++)
        if (flag[t]) {
            if (pos < cap) out[pos] = t;
            pos++;
        }
    if (threadIdx.x == blockDim.x - 1) *n_out = pos;
}

// Brick k of the store: tile tiles[k]'s colour bytes cb[k][c] and canonical
// offsets s[k][a][c] (0 on an edge without a marker), c = cell index in the
// tile (x fastest); cells outside the grid give 0.
__global__ void __launch_bounds__(256) pack_kernel(Grid g, const uint8_t *__restrict__ cb, const double *__restrict__ s0,
                                                   const double *__restrict__ s1, const double *__restrict__ s2,
                                                   const int *__restrict__ tiles, int n, uint8_t *__restrict__ out_cb,
                                                   double *__restrict__ out_s) {
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        int o[3];
        tile_origin(g, tiles[k], o);
        for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
            const int x = o[0] + (c & 7), y = o[1] + ((c >> 3) & 7), z = o[2] + (c >> 6);
            uint8_t b = 0;
            double v[3] = {0.0, 0.0, 0.0};
            if (x < g.n[0] && y < g.n[1] && z < g.n[2]) {
                const int id = lin(g, x, y, z);
                b = __ldg(cb + id);
                const int nb[3] = {lin(g, x + 1, y, z), lin(g, x, y + 1, z), lin(g, x, y, z + 1)};
                const double *sa[3] = {s0, s1, s2};
#pragma unroll
                for (int a = 0; a < 3; a++)
                    if (((__ldg(cb + nb[a]) ^ b) & 1) != 0) v[a] = __ldg(sa[a] + id);
            }
            out_cb[(size_t)k * TILE_CELLS + c] = b;
#pragma unroll
            for (int a = 0; a < 3; a++) out_s[((size_t)k * 3 + a) * TILE_CELLS + c] = v[a];
        }
    }
}

// slot[t] = k for tile t = tiles[k], -1 for the other tiles; ids out of range
// are counted in *bad and skipped.
__global__ void brick_slots_kernel(const int *__restrict__ tiles, int n, int nt, int *__restrict__ slot,
                                   int *__restrict__ bad) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int t = tiles[k];
        if (t < 0 || t >= nt) atomicAdd(bad, 1);
        else slot[t] = k;
    }
}

// The state from a brick store: bricks copied in, every other tile filled
// with its colour (bg: bit 0), face colours equal to it, offsets 0.
__global__ void __launch_bounds__(256) unpack_kernel(Grid g, const int *__restrict__ slot, const uint8_t *__restrict__ in_cb,
                                                     const double *__restrict__ in_s, const uint8_t *__restrict__ bg,
                                                     uint8_t *__restrict__ cb, double *__restrict__ s0,
                                                     double *__restrict__ s1, double *__restrict__ s2) {
    for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        int o[3];
        tile_origin(g, tile, o);
        const int k = slot[tile];
        const uint8_t fill = (bg[tile] & 1) ? 0x0F : 0x00;
        for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
            const int x = o[0] + (c & 7), y = o[1] + ((c >> 3) & 7), z = o[2] + (c >> 6);
            if (x >= g.n[0] || y >= g.n[1] || z >= g.n[2]) continue;
            const int id = lin(g, x, y, z);
            if (k >= 0) {
                cb[id] = in_cb[(size_t)k * TILE_CELLS + c];
                s0[id] = in_s[((size_t)k * 3 + 0) * TILE_CELLS + c];
                s1[id] = in_s[((size_t)k * 3 + 1) * TILE_CELLS + c];
                s2[id] = in_s[((size_t)k * 3 + 2) * TILE_CELLS + c];
            } else {
                cb[id] = fill;
                s0[id] = 0.0;
                s1[id] = 0.0;
                s2[id] = 0.0;
            }
        }
    }
}

}  // namespace ebit
