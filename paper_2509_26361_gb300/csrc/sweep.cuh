// sweep.cuh -- one split advection sweep of the 3D EBIT method.
//
// Method (arxiv 2509.26361): markers move along the sweep axis D by explicit
// Euler with the interpolated velocity (Sec. 2.1, Eqs. 1-2).  Markers on D-edges
// (aligned) stay on their grid line; a node's colour flips once per marker that
// crosses it (Sec. 2.2, Fig. 4); an edge keeps a marker iff its end colours
// differ, so two markers meeting on one edge both vanish (Fig. 5).  Markers on
// the two other edge families (unaligned) are rebuilt in the two face families
// that contain D (Sec. 2.3, Fig. 6): the old polyline of each plane (connectivity
// from the corner colours, and from the face-centre colour on saddle faces) is
// advected, and each unaligned edge whose new end colours differ receives the
// crossing of that polyline with its grid line, refined by two circle fits with
// the radius-ratio rule (Sec. 2.1, Fig. 2).
//
// GPU organisation.  GB300's FP64 pipe is narrow and a warp-level FP64
// instruction costs its issue slots whatever the number of active lanes, so all
// FP64 arithmetic runs from compacted lists with full warps, and the band pass
// over the cells is integer work:
//   advect_kernel -- per band tile, the markers owned by the tile are listed in
//                    shared memory and each is moved once (trilinear velocity):
//                    adv = its advected coordinate along D relative to its node
//                    (s + u dt/h for an aligned marker, u dt/h for an unaligned
//                    one) and bin = floor(2 adv), both in scratch arrays.
//   sweep_kernel  -- per band tile, one thread per cell, integer only: new node
//                    colours, aligned edges, canonical face colours; unaligned
//                    edges that carry a marker and saddle faces are appended to
//                    global work lists (with six lists, also the unaligned
//                    edges whose annihilation count needs their crossings).
//   fp64_kernel   -- one thread per list entry (two per unaligned edge when
//                    the lists are short, the circle fits split between them):
//                    crossings, circle fits, face phases, crossing counts.
// Every crossing decision compares an advected coordinate da + adv with 0 or
// 1/2; for the integers da that occur the sum is exact near those thresholds,
// so "da + adv < 0" equals "bin < -2 da" and "da + adv < 1/2" equals
// "bin < 1 - 2 da" exactly, and the integer test gives the same answer as the
// floating-point one.  Every output word has one owner thread (face bits of
// saddle faces are OR-ed into the byte written by the band pass), and old and
// new state live in separate buffers.
#pragma once
#include "common.cuh"

namespace ebit {

struct SweepArgs {
    Grid g;
    const uint8_t *__restrict__ cb;  // old colour bytes
    uint8_t *__restrict__ cbo;       // new colour bytes
    const double *__restrict__ s[3]; // old offsets per edge axis
    double *__restrict__ so[3];      // new offsets (written only where a marker is)
    const double *__restrict__ u;    // u_D on D-faces
    double lam;                      // dt / h
    double *__restrict__ adv[3];     // advected coordinate of each marker (scratch)
    int8_t *__restrict__ bin[3];     // floor(2 adv) (scratch)
    const int *__restrict__ list;    // band tile ids
    const int *__restrict__ count;   // number of band tiles (device)
    unsigned *__restrict__ work[6];  // work lists: unaligned fam.1, fam.2, saddle fam.1, fam.2
                                     // (and, with six lists, annihilation checks fam.1, fam.2)
    int *__restrict__ wcount;        // [4] or [6] list lengths (device)
    unsigned long long *ctr;         // event counters
    uint32_t *tile_marker;           // per tile: proximity mask of its markers in the input or the output
    uint8_t *tile_dirty;             // per tile: processed since the last Front2VOF
    // Lists for the next sweep (a context's band sweeps; null elsewhere).  The
    // band pass appends every aligned edge that carries a marker after the
    // sweep to mk_out (the unaligned ones are its work lists 0 and 1) and every
    // tile whose new proximity mask is not empty to mt_out; it clears the band
    // flag of each tile it processes.  The next sweep's advection builds that
    // sweep's band from mt_out and the masks.
    unsigned *mk_out = nullptr;
    int *mk_out_count = nullptr;
    int *mt_out = nullptr;
    int *mt_out_count = nullptr;
    uint32_t *band_flag = nullptr;
    // the count of the band list the following sweep builds (cleared here)
    int *band_next_count = nullptr;
    // next band tile to take (blocks of the band pass take tiles in turn from
    // this counter; null: a fixed stride over the list)
    int *tile_next = nullptr;
};

// The markers of the state before a sweep, as node ids of their edges, one
// list per edge axis, and the tiles whose proximity mask is not empty (the
// previous sweep's band pass wrote them); the band this sweep processes is
// built from the latter into band / band_count, with band_flag against
// duplicates.
struct MarkerLists {
    const unsigned *list[3];
    const int *count[3];
    int axis[3];
    const int *mtiles;
    const int *mtiles_count;
    int *band;
    int *band_count;
};

struct P2 {
    double x, y;
};

// Loads of data produced earlier in the same launch (the persistent batched
// sweep, F = true) bypass the non-coherent read-only path and L1; separate
// launches (F = false) read them through the read-only cache.
template <bool F, typename T>
__device__ __forceinline__ T ld_in(const T *p) {
    if (F) return __ldcg(p);
    return __ldg(p);
}

// 2D cell edges in a plane spanned by (a, t): B a-edge at c00, R t-edge at c10,
// T a-edge at c01, L t-edge at c00.
enum { EB = 0, ER = 1, ET = 2, EL = 3 };

// Segments of a 2D cell from its corner colours (and the face colour on a
// saddle): returns the count, endpoints as edge codes.
__device__ __forceinline__ int cell_segs(int c00, int c10, int c01, int c11, int phif, int seg[2][2]) {
    int mB = c00 != c10, mR = c10 != c11, mT = c01 != c11, mL = c00 != c01;
    int nm = mB + mR + mT + mL;
    if (nm == 2) {
        int k = 0;
        if (mB) seg[0][k++] = EB;
        if (mR) seg[0][k++] = ER;
        if (mT) seg[0][k++] = ET;
        if (mL) seg[0][k++] = EL;
        return 1;
    }
    if (nm == 4) {
        if (c00 == phif) {
            seg[0][0] = EB; seg[0][1] = ER;
            seg[1][0] = EL; seg[1][1] = ET;
        } else {
            seg[0][0] = EB; seg[0][1] = EL;
            seg[1][0] = ER; seg[1][1] = ET;
        }
        return 2;
    }
    return 0;
}

// Circle through A, B, C meeting the grid line x = 0; only roots on the edge
// (0 <= y <= 1) count, the one nearest ylin is kept (Fig. 2).  rad2 gets the
// squared radius.
__device__ __forceinline__ bool circle_root(P2 A, P2 B, P2 C, double ylin, double *root, double *rad2) {
    double bx = B.x - A.x, by = B.y - A.y;
    double cx = C.x - A.x, cy = C.y - A.y;
    double b2 = bx * bx + by * by;
    double c2 = cx * cx + cy * cy;
    double det = 2.0 * (bx * cy - by * cx);
    if (fabs(det) <= 1e-12 * (b2 + c2)) return false;
    double ux = (cy * b2 - by * c2) / det;
    double uy = (bx * c2 - cx * b2) / det;
    double r2 = ux * ux + uy * uy;
    double dx = 0.0 - (A.x + ux);
    double disc = r2 - dx * dx;
    if (disc < 0.0) return false;
    double sq = sqrt(disc);
    double yc = A.y + uy;
    double yp = yc + sq, ym = yc - sq;
    bool okp = (yp >= 0.0 && yp <= 1.0), okm = (ym >= 0.0 && ym <= 1.0);
    if (!okp && !okm) return false;
    if (okp && okm) *root = (fabs(yp - ylin) <= fabs(ym - ylin)) ? yp : ym;
    else *root = okp ? yp : ym;
    *rad2 = r2;
    return true;
}

// The ratio rule's test rmax > 10 rmin with rmax = sqrt(r2max), rmin =
// sqrt(r2min), both rounded, as the method states it.  Away from the threshold
// the squared radii decide it (r2max against 100 r2min with a relative margin of
// 1e-12, far above the few units of rounding in the radii and the product), so
// the square roots are taken only within that margin.
__device__ __forceinline__ bool ratio_above_10(double r2max, double r2min) {
    const double t = 100.0 * r2min;
    if (r2max > t * (1.0 + 1e-12)) return true;
    if (r2max < t * (1.0 - 1e-12)) return false;
    return sqrt(r2max) > 10.0 * sqrt(r2min);
}

// The crossing of an unaligned edge from the advected points P1 P2 P3 P4
// (P2 -> P3 crosses the edge's grid line at ylin; P1, P4 their neighbours, if
// found): circles through P1 P2 P3 and P2 P3 P4; both valid -> the larger
// circle's root if its radius exceeds 10 times the smaller one, else the mean;
// one valid -> its root; none -> ylin; clamped to [0, 1-] (Fig. 2).  One
// out-of-line copy serves every edge family (the two fits are independent, so
// their FP64 chains interleave inside it).
static __device__ __noinline__ double circle_pair(P2 P1, P2 Pa, P2 Pb, P2 P4, double ylin, bool h1, bool h4) {
    double ya = 0.0, ra2 = 0.0, yb = 0.0, rb2 = 0.0;
    bool va = circle_root(P1, Pa, Pb, ylin, &ya, &ra2);
    bool vb = circle_root(Pa, Pb, P4, ylin, &yb, &rb2);
    va = va && h1;
    vb = vb && h4;
    double y;
    if (va && vb) {
        // above the ratio the radii differ, so the larger squared radius names
        // the larger circle
        const double r2max = ra2 > rb2 ? ra2 : rb2, r2min = ra2 > rb2 ? rb2 : ra2;
        if (ratio_above_10(r2max, r2min)) y = ra2 > rb2 ? ya : yb;
        else y = 0.5 * (ya + yb);
    } else if (va) {
        y = ya;
    } else if (vb) {
        y = yb;
    } else {
        y = ylin;
    }
    if (y < 0.0) y = 0.0;
    if (y > ONE_MINUS) y = ONE_MINUS;
    return y;
}

// circle_pair with one fit per lane of a lane pair (adjacent lanes of a warp;
// lane parity `half`: 0 fits P1 Pa Pb, 1 fits Pa Pb P4).  The pair exchanges
// root, squared radius and validity, and both lanes return the crossing
// circle_pair returns (the same operations, in the same order, per fit).
static __device__ __noinline__ double circle_pair_split(P2 P1, P2 Pa, P2 Pb, P2 P4, double ylin, bool h1, bool h4,
                                                        int half) {
    const unsigned pm = 3u << ((threadIdx.x & 31) & ~1u);
    const P2 A = half ? Pa : P1, B = half ? Pb : Pa, Cc = half ? P4 : Pb;
    double y = 0.0, r2 = 0.0;
    bool v = circle_root(A, B, Cc, ylin, &y, &r2);
    v = v && (half ? h4 : h1);
    const double yo = __shfl_xor_sync(pm, y, 1), r2o = __shfl_xor_sync(pm, r2, 1);
    const bool vo = __shfl_xor_sync(pm, (int)v, 1) != 0;
    const double ya = half ? yo : y, ra2 = half ? r2o : r2, yb = half ? y : yo, rb2 = half ? r2 : r2o;
    const bool va = half ? vo : v, vb = half ? v : vo;
    double res;
    if (va && vb) {
        const double r2max = ra2 > rb2 ? ra2 : rb2, r2min = ra2 > rb2 ? rb2 : ra2;
        if (ratio_above_10(r2max, r2min)) res = ra2 > rb2 ? ya : yb;
        else res = 0.5 * (ya + yb);
    } else if (va) {
        res = ya;
    } else if (vb) {
        res = yb;
    } else {
        res = ylin;
    }
    if (res < 0.0) res = 0.0;
    if (res > ONE_MINUS) res = ONE_MINUS;
    return res;
}

// trilinear u_D at node q shifted by s along axis e; lerps in x, y, z order
template <int D>
__device__ double interp_u(const Grid &g, const double *__restrict__ u, const int q[3], int e, double s) {
    int base[3];
    double t[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
        if (b == D) {
            base[b] = q[b];
            t[b] = (b == e) ? s : 0.0;
        } else if (b != e) {
            base[b] = q[b] - 1;
            t[b] = 0.5;
        } else if (s < 0.5) {
            base[b] = q[b] - 1;
            t[b] = s + 0.5;
        } else {
            base[b] = q[b];
            t[b] = s - 0.5;
        }
    }
    int x0 = wrapc(base[0], g.n[0]), x1 = wrapc(base[0] + 1, g.n[0]);
    int y0 = wrapc(base[1], g.n[1]), y1 = wrapc(base[1] + 1, g.n[1]);
    int z0 = wrapc(base[2], g.n[2]), z1 = wrapc(base[2] + 1, g.n[2]);
    int r00 = (z0 * g.n[1] + y0) * g.n[0], r10 = (z0 * g.n[1] + y1) * g.n[0];
    int r01 = (z1 * g.n[1] + y0) * g.n[0], r11 = (z1 * g.n[1] + y1) * g.n[0];
    // A marker off the sweep axis sits on a D-face plane (t[D] = 0): the lerp
    // along D gives (1 - 0) a + 0 b = a for finite b, so its upper samples are
    // not read (for a = -0 the sign of the zero may differ; nothing downstream
    // depends on it).
    const bool flatD = e != D;
    double c00, c10, c01, c11;
    if (D == 0 && flatD) {
        c00 = __ldg(u + r00 + x0);
        c10 = __ldg(u + r10 + x0);
        c01 = __ldg(u + r01 + x0);
        c11 = __ldg(u + r11 + x0);
    } else {
        c00 = (1.0 - t[0]) * __ldg(u + r00 + x0) + t[0] * __ldg(u + r00 + x1);
        c10 = (D == 1 && flatD) ? 0.0 : (1.0 - t[0]) * __ldg(u + r10 + x0) + t[0] * __ldg(u + r10 + x1);
        c01 = (D == 2 && flatD) ? 0.0 : (1.0 - t[0]) * __ldg(u + r01 + x0) + t[0] * __ldg(u + r01 + x1);
        c11 = (D != 0 && flatD) ? 0.0 : (1.0 - t[0]) * __ldg(u + r11 + x0) + t[0] * __ldg(u + r11 + x1);
    }
    const double c0 = (D == 1 && flatD) ? c00 : (1.0 - t[1]) * c00 + t[1] * c10;
    if (D == 2 && flatD) return c0;
    const double c1 = (D == 1 && flatD) ? c01 : (1.0 - t[1]) * c01 + t[1] * c11;
    return (1.0 - t[2]) * c0 + t[2] * c1;
}

// warp-aggregated append: every lane of the warp must call it
__device__ __forceinline__ int warp_append(int *counter, bool flag) {
    const unsigned full = 0xffffffffu;
    unsigned m = __ballot_sync(full, flag);
    if (!m) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(full, base, leader);
    return flag ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

// ---------------------------------------------------------------- advection
// Move every marker of one band tile once (Eq. 2).  CFL >= 1 is counted and
// clamped; a displacement that is not finite (NaN or infinite velocity) is
// counted apart and the marker stays where it is.  Called by all threads of the block; s_mk/s_c/s_n are its shared
// staging; u is u_D on the D-faces and lam = dt / h.
// Tile shape SH (TileShape<SH>); s_c holds (TX + 1) (TY + 1) (TZ + 1) colours.
template <int D, int SH = 0>
__device__ __forceinline__ void advect_tile(const SweepArgs &a, const double *__restrict__ u, double lam, int tile,
                                            uint16_t *s_mk, uint8_t *s_c, int *s_n) {
    using S = TileShape<SH>;
    constexpr int CX = S::TX + 1, CY = S::TY + 1, CZ = S::TZ + 1;
    int o[3];
    tile_origin(a.g, tile, o);
    if (threadIdx.x == 0) *s_n = 0;
    for (int r = threadIdx.x; r < CX * CY * CZ; r += blockDim.x) {
        int rx = r % CX, ry = (r / CX) % CY, rz = r / (CX * CY);
        s_c[r] = __ldg(a.cb + lin(a.g, o[0] + rx, o[1] + ry, o[2] + rz)) & 1;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
        int l[3];
        S::cell(c, l);
        int q[3] = {o[0] + l[0], o[1] + l[1], o[2] + l[2]};
        bool valid = q[0] < a.g.n[0] && q[1] < a.g.n[1] && q[2] < a.g.n[2];
        int mask = 0;
        if (valid) {
            const int r = l[0] + CX * (l[1] + CY * l[2]);
            const int c0 = s_c[r];
            mask = (s_c[r + 1] != c0) | ((s_c[r + CX] != c0) << 1) | ((s_c[r + CX * CY] != c0) << 2);
        }
        for (int e = 0; e < 3; e++) {
            int slot = warp_append(s_n, (mask >> e) & 1);
            if (slot >= 0) s_mk[slot] = (uint16_t)(c | (e << 9));
        }
    }
    __syncthreads();
    const int n = *s_n;
    unsigned hits = 0, bad = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int it = s_mk[k], c = it & 511, e = it >> 9;
        int l[3];
        S::cell(c, l);
        int q[3] = {o[0] + l[0], o[1] + l[1], o[2] + l[2]};
        const int id = lin3(a.g, q);
        double sv = __ldg(a.s[e] + id);
        double cf = interp_u<D>(a.g, u, q, e, sv) * lam;
        if (!isfinite(cf)) {
            bad++;
            cf = 0.0;
        } else if (!(fabs(cf) < 1.0)) {
            hits++;
            cf = cf > 0.0 ? ONE_MINUS : -ONE_MINUS;
        }
        double x = (e == D) ? sv + cf : cf;
        a.adv[e][id] = x;
        a.bin[e][id] = (int8_t)(int)floor(2.0 * x);
    }
    unsigned v = __reduce_add_sync(0xffffffffu, hits);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.ctr + C_CFL, (unsigned long long)v);
    v = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.ctr + C_NONFINITE, (unsigned long long)v);
    __syncthreads();
}

// the counters the band pass appends to start at zero (cleared by the launch before it)
template <int NL>
__device__ __forceinline__ void clear_sweep_counts(const SweepArgs &a) {
    if (blockIdx.x != 0) return;
    if (threadIdx.x < NL) a.wcount[threadIdx.x] = 0;
    if (threadIdx.x == 32 && a.mk_out_count) *a.mk_out_count = 0;
    if (threadIdx.x == 33 && a.mt_out_count) *a.mt_out_count = 0;
    if (threadIdx.x == 34 && a.tile_next) *a.tile_next = 0;
    if (threadIdx.x == 35 && a.band_next_count) *a.band_next_count = 0;
}

template <int D, int NL = 4>
__global__ void __launch_bounds__(256) advect_kernel(SweepArgs a) {
    __shared__ uint16_t s_mk[3 * TILE_CELLS];
    __shared__ uint8_t s_c[9 * 9 * 9];  // node colours of the tile and its +1 layer
    __shared__ int s_n;
    pdl_wait();
    const int ntl = *a.count;
    clear_sweep_counts<NL>(a);
    for (int li = blockIdx.x; li < ntl; li += gridDim.x) advect_tile<D>(a, a.u, a.lam, a.list[li], s_mk, s_c, &s_n);
}

// Advection from the marker lists (Eq. 2): one thread per marker, no tile
// staging.  Every marker of the state is on a list, so the same markers as in
// advect_tile are moved, with the same arithmetic.
template <int D, int NL = 4>
__global__ void __launch_bounds__(256) advect_list_kernel(SweepArgs a, MarkerLists m) {
    pdl_wait();
    clear_sweep_counts<NL>(a);
    // One index space: the markers, then this sweep's band items (tile of the
    // marker-tile list, direction); a thread takes one item per round, so the
    // two kinds of work run side by side rather than one after the other.
    const int n0 = *m.count[0], n1 = *m.count[1], n2 = *m.count[2];
    const int total = n0 + n1 + n2;
    const int nmt = *m.mtiles_count;
    const int all = total + 27 * nmt;
    const int stride = gridDim.x * blockDim.x;
    const int iters = (all + stride - 1) / stride;
    const int nx = a.g.n[0], nxy = a.g.n[0] * a.g.n[1];
    unsigned hits = 0, bad = 0;
    for (int it = 0; it < iters; it++) {
        const int t = list_item(it);
        if (t >= all) continue;
        if (t >= total) {
            // the band: every tile a listed tile's mask points to (bit
            // near_bit(dx, dy, dz) names the neighbour in that direction),
            // listed once
            const int tb = t - total;
            const int tile = __ldg(m.mtiles + tb / 27), b = tb % 27;
            if (!((__ldg(a.tile_marker + tile) >> b) & 1u)) continue;
            const int tx = tile % a.g.td[0], ty = (tile / a.g.td[0]) % a.g.td[1], tz = tile / (a.g.td[0] * a.g.td[1]);
            const int bx = wrapc(tx + b % 3 - 1, a.g.td[0]), by = wrapc(ty + (b / 3) % 3 - 1, a.g.td[1]),
                      bz = wrapc(tz + b / 9 - 1, a.g.td[2]);
            const int nt = (bz * a.g.td[1] + by) * a.g.td[0] + bx;
            if (atomicExch(a.band_flag + nt, 1u) == 0u) m.band[atomicAdd(m.band_count, 1)] = nt;
            continue;
        }
        // selects rather than indexing, which would copy the parameter arrays
        // to local memory
        const int k = t < n0 ? 0 : (t < n0 + n1 ? 1 : 2);
        const int j = t - (k == 0 ? 0 : (k == 1 ? n0 : n0 + n1));
        const unsigned *lst = k == 0 ? m.list[0] : (k == 1 ? m.list[1] : m.list[2]);
        const int e = k == 0 ? m.axis[0] : (k == 1 ? m.axis[1] : m.axis[2]);
        const int id = (int)__ldg(lst + j);
        const int z = id / nxy, r = id - z * nxy;
        const int y = r / nx;
        const int q[3] = {r - y * nx, y, z};
        const double *se = e == 0 ? a.s[0] : (e == 1 ? a.s[1] : a.s[2]);
        double *adv = e == 0 ? a.adv[0] : (e == 1 ? a.adv[1] : a.adv[2]);
        int8_t *bin = e == 0 ? a.bin[0] : (e == 1 ? a.bin[1] : a.bin[2]);
        const double sv = __ldg(se + id);
        double cf = interp_u<D>(a.g, a.u, q, e, sv) * a.lam;
        if (!isfinite(cf)) {
            bad++;
            cf = 0.0;
        } else if (!(fabs(cf) < 1.0)) {
            hits++;
            cf = cf > 0.0 ? ONE_MINUS : -ONE_MINUS;
        }
        const double x = (e == D) ? sv + cf : cf;
        adv[id] = x;
        bin[id] = (int8_t)(int)floor(2.0 * x);
    }
    unsigned v = __reduce_add_sync(0xffffffffu, hits);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.ctr + C_CFL, (unsigned long long)v);
    v = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.ctr + C_NONFINITE, (unsigned long long)v);
}

// ----------------------------------------------------------- cell context
template <int D, bool F = false>
struct SweepCell {
    static constexpr int A = D, T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    const SweepArgs &a;
    int p[3];
    // colour bytes of the plane window da in [-2, 2], dt in [-1, 2] of the
    // family being processed, loaded in one batch (byte (da+2) + 5 (dt+1) of
    // three 64-bit registers)
    unsigned long long w0, w1, w2;

    __device__ SweepCell(const SweepArgs &args, int x, int y, int z) : a(args) {
        p[0] = x;
        p[1] = y;
        p[2] = z;
    }
    __device__ __forceinline__ int id3(int da, int d1, int d2) const {
        int q[3];
        q[A] = p[A] + da;
        q[T1] = p[T1] + d1;
        q[T2] = p[T2] + d2;
        return lin3(a.g, q);
    }
    __device__ __forceinline__ int colid(int id) const { return __ldg(a.cb + id) & 1; }

    // plane of the face family with in-plane transverse axis TT and normal NN
    // through the cell's node; offsets (da, dt) along (A, TT)
    template <int TT, int NN>
    __device__ __forceinline__ int pid(int da, int dt) const {
        int q[3];
        q[A] = p[A] + da;
        q[TT] = p[TT] + dt;
        q[NN] = p[NN];
        return lin3(a.g, q);
    }
    template <int TT, int NN>
    __device__ __forceinline__ void loadw() {
        unsigned long long v[3] = {0ull, 0ull, 0ull};
#pragma unroll
        for (int dt = -1; dt <= 2; dt++)
#pragma unroll
            for (int da = -2; da <= 2; da++) {
                const int i = (da + 2) + 5 * (dt + 1);
                v[i >> 3] |= (unsigned long long)__ldg(a.cb + pid<TT, NN>(da, dt)) << (8 * (i & 7));
            }
        w0 = v[0];
        w1 = v[1];
        w2 = v[2];
    }
    __device__ __forceinline__ int wb(int da, int dt) const {
        const int i = (da + 2) + 5 * (dt + 1);
        const unsigned long long v = i < 8 ? w0 : (i < 16 ? w1 : w2);
        return (int)((v >> (8 * (i & 7))) & 0xFF);
    }
    template <int TT, int NN>
    __device__ int psegs(int da, int dt, int seg[2][2]) const {
        int b00 = wb(da, dt);
        return cell_segs(b00 & 1, wb(da + 1, dt) & 1, wb(da, dt + 1) & 1, wb(da + 1, dt + 1) & 1,
                         (b00 >> (1 + NN)) & 1, seg);
    }
    // bin of the advected a-coordinate of the marker on edge code e of cell
    // (da, dt), and the integer da' with x = da' + adv
    template <int TT, int NN>
    __device__ __forceinline__ int pbin(int e, int da, int dt, int *off) const {
        if (e == EB || e == ET) {
            *off = da;
            return ld_in<F>(a.bin[A] + pid<TT, NN>(da, dt + (e == ET ? 1 : 0)));
        }
        int aa = da + (e == ER ? 1 : 0);
        *off = aa;
        return ld_in<F>(a.bin[TT] + pid<TT, NN>(aa, dt));
    }
    // advected position (x along A, y along TT) relative to the cell's node
    template <int TT, int NN>
    __device__ __forceinline__ P2 ppos(int e, int da, int dt) const {
        P2 r;
        if (e == EB || e == ET) {
            int tt = dt + (e == ET ? 1 : 0);
            r.x = (double)da + ld_in<F>(a.adv[A] + pid<TT, NN>(da, tt));
            r.y = (double)tt;
        } else {
            int aa = da + (e == ER ? 1 : 0);
            int id = pid<TT, NN>(aa, dt);
            r.x = (double)aa + ld_in<F>(a.adv[TT] + id);
            r.y = (double)dt + __ldg(a.s[TT] + id);
        }
        return r;
    }
    // is the endpoint left of x = 0 (thr = 0) or of x = 1/2 (thr = 1)?
    template <int TT, int NN>
    __device__ __forceinline__ bool pleft(int e, int da, int dt, int thr) const {
        int off;
        int b = pbin<TT, NN>(e, da, dt, &off);
        return b < thr - 2 * off;
    }
    // number of segments of cells (-1, 0) and (0, 0) crossing x = 0
    template <int TT, int NN>
    __device__ int count_crossings() const {
        int n = 0;
        for (int da = -1; da <= 0; da++) {
            int seg[2][2];
            int ns = psegs<TT, NN>(da, 0, seg);
            for (int k = 0; k < ns; k++)
                n += pleft<TT, NN>(seg[k][0], da, 0, 0) != pleft<TT, NN>(seg[k][1], da, 0, 0);
        }
        return n;
    }
    // neighbour along the polyline of the marker on edge e of cell (da, dt),
    // found in the cell across that edge
    template <int TT, int NN>
    __device__ bool neighbour(int e, int da, int dt, P2 *out) const {
        int oda = da, odt = dt, oe;
        switch (e) {
        case EB: odt = dt - 1; oe = ET; break;
        case ET: odt = dt + 1; oe = EB; break;
        case EL: oda = da - 1; oe = ER; break;
        default: oda = da + 1; oe = EL; break;
        }
        int seg[2][2];
        int ns = psegs<TT, NN>(oda, odt, seg);
        for (int k = 0; k < ns; k++) {
            int other = -1;
            if (seg[k][0] == oe) other = seg[k][1];
            else if (seg[k][1] == oe) other = seg[k][0];
            if (other >= 0) {
                *out = ppos<TT, NN>(other, oda, odt);
                return true;
            }
        }
        return false;
    }

    // Crossings of the advected polyline of cells (-1, 0) and (0, 0) with the
    // grid line x = 0, in scan order (cell da = -1 then 0, segment 0 then 1):
    // their number, and for the first three their left and right endpoint
    // edges and cell (scalars, so that nothing lives in local memory).
    struct Crossings {
        int n;
        int el0, er0, da0, el1, er1, da1, el2, er2, da2;
    };
    template <int TT, int NN>
    __device__ __forceinline__ Crossings crossings() const {
        Crossings c{};
#pragma unroll
        for (int da = -1; da <= 0; da++) {
            int seg[2][2];
            const int ns = psegs<TT, NN>(da, 0, seg);
#pragma unroll
            for (int k = 0; k < 2; k++) {
                if (k >= ns) continue;
                const bool l0 = pleft<TT, NN>(seg[k][0], da, 0, 0), l1 = pleft<TT, NN>(seg[k][1], da, 0, 0);
                if (l0 == l1) continue;
                const int el = l0 ? seg[k][0] : seg[k][1], er = l0 ? seg[k][1] : seg[k][0];
                if (c.n == 0) { c.el0 = el; c.er0 = er; c.da0 = da; }
                else if (c.n == 1) { c.el1 = el; c.er1 = er; c.da1 = da; }
                else if (c.n == 2) { c.el2 = el; c.er2 = er; c.da2 = da; }
                c.n++;
            }
        }
        return c;
    }
    // the crossing's advected endpoints and its linear crossing height
    template <int TT, int NN>
    __device__ __forceinline__ double crossing_line(int el, int er, int cda, P2 &Pa, P2 &Pb) const {
        Pa = ppos<TT, NN>(el, cda, 0);
        Pb = ppos<TT, NN>(er, cda, 0);
        const double tt = (0.0 - Pa.x) / (Pb.x - Pa.x);
        return Pa.y + tt * (Pb.y - Pa.y);
    }

    // Unaligned edge of family (TT, NN) at the cell's node (carries a marker):
    // crossings of the advected polyline with the grid line x = 0 in strip 0
    // (Fig. 1c), then the two circle fits with the ratio rule (Fig. 2).
    // half: -1 one lane per edge; 0, 1 the lanes of a pair sharing the edge
    // (the even lane counts and stores).
    template <int TT, int NN>
    __device__ void unaligned(unsigned ev[C_N], int half = -1) const {
        const Crossings c = crossings<TT, NN>();
        const int myid = lin3(a.g, p);
        const bool lead = half <= 0;
        if (lead) ev[C_MARKERS]++;
        if ((c.n & 1) == 0) {
            if (lead) {
                ev[C_INCONSISTENT]++;
                a.so[TT][myid] = 0.5;
            }
            return;
        }
        int el = c.el0, er = c.er0, cda = c.da0;
        P2 Pa, Pb;
        double ylin = crossing_line<TT, NN>(el, er, cda, Pa, Pb);
        if (c.n == 3) {
            // a fold of the polyline: the crossing with the median linear
            // height, by the same three compare-exchanges as the oracle
            P2 A1, B1, A2, B2;
            const double y1 = crossing_line<TT, NN>(c.el1, c.er1, c.da1, A1, B1);
            const double y2 = crossing_line<TT, NN>(c.el2, c.er2, c.da2, A2, B2);
            // (v_k tracks yl[o_k], so the comparisons are the oracle's)
            double v0 = ylin, v1 = y1, v2 = y2, tv;
            int o0 = 0, o1 = 1, o2 = 2, tmp;
            if (v0 > v1) { tmp = o0; o0 = o1; o1 = tmp; tv = v0; v0 = v1; v1 = tv; }
            if (v1 > v2) { tmp = o1; o1 = o2; o2 = tmp; tv = v1; v1 = v2; v2 = tv; }
            if (v0 > v1) { tmp = o0; o0 = o1; o1 = tmp; tv = v0; v0 = v1; v1 = tv; }
            if (o1 == 1) { el = c.el1; er = c.er1; cda = c.da1; Pa = A1; Pb = B1; ylin = y1; }
            else if (o1 == 2) { el = c.el2; er = c.er2; cda = c.da2; Pa = A2; Pb = B2; ylin = y2; }
            if (lead) ev[C_MULTI]++;
        }
        // both neighbours first, then the two circle fits
        P2 P1 = Pa, P4 = Pb;
        const bool h1 = neighbour<TT, NN>(el, cda, 0, &P1);
        const bool h4 = neighbour<TT, NN>(er, cda, 0, &P4);
        if (lead && !h1) ev[C_INCONSISTENT]++;
        if (lead && !h4) ev[C_INCONSISTENT]++;
        if (half < 0) {
            a.so[TT][myid] = circle_pair(P1, Pa, Pb, P4, ylin, h1, h4);
        } else {
            const double y = circle_pair_split(P1, Pa, Pb, P4, ylin, h1, h4, half);
            if (lead) a.so[TT][myid] = y;
        }
    }

    // Face-centre colour of the family's 2D cell at the node (saddle faces): the
    // phase of the advected polyline at the centre, reached from the node along
    // the a-line to x = 1/2 and then up the line x = 1/2 to y = 1/2.
    template <int TT, int NN>
    __device__ int face_phase(int ncol0) const {
        int par = ncol0;
        for (int da = -1; da <= 1; da++) {
            if ((wb(da, 0) & 1) == (wb(da + 1, 0) & 1)) continue;
            int b = ld_in<F>(a.bin[A] + pid<TT, NN>(da, 0));
            if (b >= -2 * da && b < 1 - 2 * da) par ^= 1;
        }
        for (int da = -1; da <= 1; da++) {
            int seg[2][2];
            int ns = psegs<TT, NN>(da, 0, seg);
            for (int k = 0; k < ns; k++) {
                bool l0 = pleft<TT, NN>(seg[k][0], da, 0, 1), l1 = pleft<TT, NN>(seg[k][1], da, 0, 1);
                if (l0 == l1) continue;
                P2 L = ppos<TT, NN>(l0 ? seg[k][0] : seg[k][1], da, 0);
                P2 R = ppos<TT, NN>(l0 ? seg[k][1] : seg[k][0], da, 0);
                double tt = (0.5 - L.x) / (R.x - L.x);
                double yl = L.y + tt * (R.y - L.y);
                if (yl < 0.5) par ^= 1;
            }
        }
        return par;
    }
};

__device__ __forceinline__ bool saddle4(int c00, int c10, int c01, int c11) {
    return c00 == c11 && c10 == c01 && c00 != c10;
}

// ------------------------------------------------------- band pass (integer)
// staged colour region of a tile, in sweep-local axes: A in [-1, TA + 1], T1
// in [0, T1], T2 in [0, T2] relative to the tile origin (TA, T1, T2: the
// tile's edges along the sweep axis and the two others)
__host__ __device__ constexpr int tile_edge(int sh, int a) { return 1 << tile_log2(sh, a); }
__host__ __device__ constexpr int stage_n(int d, int sh) {
    return (tile_edge(sh, d) + 3) * (tile_edge(sh, (d + 1) % 3) + 1) * (tile_edge(sh, (d + 2) % 3) + 1);
}
template <int D, int SH>
struct Stage {
    static constexpr int RA = tile_edge(SH, D) + 3, R1 = tile_edge(SH, (D + 1) % 3) + 1,
                         R2 = tile_edge(SH, (D + 2) % 3) + 1;
};
// the largest staged region over directions and shapes, and the largest
// colour block of advect_tile
__host__ __device__ constexpr int stage_max() {
    int m = 0;
    for (int sh = 0; sh < N_TILE_SHAPES; sh++)
        for (int d = 0; d < 3; d++) m = stage_n(d, sh) > m ? stage_n(d, sh) : m;
    return m;
}
__host__ __device__ constexpr int adv_stage_max() {
    int m = 0;
    for (int sh = 0; sh < N_TILE_SHAPES; sh++) {
        const int v = (tile_edge(sh, 0) + 1) * (tile_edge(sh, 1) + 1) * (tile_edge(sh, 2) + 1);
        m = v > m ? v : m;
    }
    return m;
}
constexpr int RA = 11, R1 = 9, R2 = 9;  // 8^3 tiles (every direction)
static_assert(stage_n(0, 0) == RA * R1 * R2, "8^3 staging");

// One band tile, all threads of the block; s_b/s_n/s_flag are its shared
// staging (colour bytes and the A-axis bins of the same window; a bin is read
// only where its node owns a marker).
// NL = 6: an unaligned edge without a marker whose window shows a colour change
// goes to work list 4 or 5 (the crossing count of the annihilation counter is
// taken by the FP64-list kernel, with full warps); NL = 4: counted here.
template <int D, bool F, int NL = 4, int SH = 0>
__device__ __forceinline__ int sweep_tile(const SweepArgs &a, int tile, uint8_t *s_b, int8_t *s_n, unsigned *s_flag) {
    constexpr int A = D, T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    using S = TileShape<SH>;
    constexpr int RA = Stage<D, SH>::RA, R1 = Stage<D, SH>::R1, R2 = Stage<D, SH>::R2;
    {
        int o[3];
        tile_origin(a.g, tile, o);
        if (threadIdx.x == 0) *s_flag = 0;
        // walk the region in global order (x fastest), so that a warp's loads
        // fall on a few rows of the grid whatever the sweep axis; the staged
        // copy is indexed in sweep-local order (A fastest)
        constexpr int E0 = A == 0 ? RA : (T1 == 0 ? R1 : R2);
        constexpr int E1 = A == 1 ? RA : (T1 == 1 ? R1 : R2);
        int seen = 0;  // bit 0: a staged node of colour 1, bit 1: one of colour 0
        for (int r = threadIdx.x; r < RA * R1 * R2; r += blockDim.x) {
            const int gl[3] = {r % E0, (r / E0) % E1, r / (E0 * E1)};
            const int ka = gl[A], k1 = gl[T1], k2 = gl[T2];
            int q[3];
            q[A] = o[A] + ka - 1;
            q[T1] = o[T1] + k1;
            q[T2] = o[T2] + k2;
            const int id = lin3(a.g, q);
            const int sr = ka + RA * (k1 + R1 * k2);
            const uint8_t b = __ldg(a.cb + id);
            seen |= (b & 1) ? 1 : 2;
            s_b[sr] = b;
            s_n[sr] = ld_in<F>(a.bin[A] + id);
        }
        // (__syncthreads_or returns whether any thread's value is non-zero)
        const int has1 = __syncthreads_or(seen & 1), has0 = __syncthreads_or(seen & 2);
        if (!(has1 && has0)) {
            // Every staged node has one colour: no marker lies on an edge whose
            // crossing could change a node, face or edge of this tile's cells,
            // so the sweep leaves them as they are (the band pass's uniform
            // window, for the whole tile): canonical colour bytes, no markers,
            // no work, and nothing for Front2VOF to redo.
            const uint8_t byte = has1 ? 0x0F : 0x00;
            for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
                int l[3];
                S::cell(c, l);
                const int x = o[0] + l[0], y = o[1] + l[1], z = o[2] + l[2];
                if (x < a.g.n[0] && y < a.g.n[1] && z < a.g.n[2]) a.cbo[lin(a.g, x, y, z)] = byte;
            }
            if (threadIdx.x == 0) {
                a.tile_marker[tile] = 0u;
                if (a.band_flag) a.band_flag[tile] = 0u;
            }
            return -1;
        }
        unsigned ev[C_N] = {0, 0, 0, 0, 0};
        unsigned mk = 0;  // proximity mask of the markers of this thread's cells
        for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
            int l[3];
            S::cell(c, l);
            int x = o[0] + l[0], y = o[1] + l[1], z = o[2] + l[2];
            bool valid = x < a.g.n[0] && y < a.g.n[1] && z < a.g.n[2];
            bool push[6] = {false, false, false, false, false, false};
            bool push_al = false;
            int myid = 0;
            if (valid) {
                SweepCell<D, F> cell(a, x, y, z);
                myid = lin(a.g, x, y, z);
                // staged index of node (da, d1, d2) relative to the cell
                const int r0 = (l[A] + 1) + RA * (l[T1] + R1 * l[T2]);
                auto sidx = [&](int da, int d1, int d2) { return r0 + da + RA * (d1 + R1 * d2); };
                int col[4][2][2];
                const int myb = s_b[r0];
                const int c0 = myb & 1;
                int any = 0;
#pragma unroll
                for (int da = 0; da < 4; da++)
#pragma unroll
                    for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
                        for (int d2 = 0; d2 < 2; d2++) {
                            int v = s_b[sidx(da - 1, d1, d2)] & 1;
                            col[da][d1][d2] = v;
                            any |= v ^ c0;
                        }
                if (!any) {
                    a.cbo[myid] = (uint8_t)(c0 | (c0 << 1) | (c0 << 2) | (c0 << 3));
                } else {
                    bool in_marker = (c0 != col[2][0][0]) || (c0 != col[1][1][0]) || (c0 != col[1][0][1]);
                    // bins of the aligned markers on the A-edges (da in {-1,0,1}) of 4 lines
                    int bn[3][2][2];
                    bool has[3][2][2];
#pragma unroll
                    for (int da = 0; da < 3; da++)
#pragma unroll
                        for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
                            for (int d2 = 0; d2 < 2; d2++) {
                                has[da][d1][d2] = col[da][d1][d2] != col[da + 1][d1][d2];
                                bn[da][d1][d2] = has[da][d1][d2] ? (int)s_n[sidx(da - 1, d1, d2)] : 0;
                            }
                    // new colours: X >= 1 <=> bin >= 2 (crossed the right node),
                    // X < 0 <=> bin < 0 (crossed the left node)  (Fig. 4)
                    int nc[2][2][2];
#pragma unroll
                    for (int dA = 0; dA < 2; dA++)
#pragma unroll
                        for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
                            for (int d2 = 0; d2 < 2; d2++) {
                                int v = col[dA + 1][d1][d2];
                                if (has[dA][d1][d2] && bn[dA][d1][d2] >= 2) v ^= 1;
                                if (has[dA + 1][d1][d2] && bn[dA + 1][d1][d2] < 0) v ^= 1;
                                nc[dA][d1][d2] = v;
                            }
                    const int n0 = nc[0][0][0];
                    bool out_marker = false;
                    // aligned edge (Fig. 5): presence from the new colours, landing markers
                    {
                        bool present = n0 != nc[1][0][0];
                        int land[3], nl = 0;
#pragma unroll
                        for (int e = -1; e <= 1; e++) {
                            if (!has[e + 1][0][0]) continue;
                            int b = bn[e + 1][0][0];
                            int dest = (b < 0) ? -1 : (b >= 2 ? 1 : 0);
                            if (e + dest != 0) continue;
                            land[nl++] = e;
                        }
                        if (present) {
                            double v;
                            if (nl == 1 || nl == 3) {
                                double sv[3];
                                for (int k = 0; k < nl; k++) {
                                    double xv = ld_in<F>(a.adv[A] + cell.id3(land[k], 0, 0));
                                    double sn = xv - (double)(-land[k]);
                                    if (sn > ONE_MINUS) sn = ONE_MINUS;
                                    sv[k] = sn;
                                }
                                if (nl == 1) {
                                    v = sv[0];
                                } else {
                                    double a0 = sv[0], a1 = sv[1], a2 = sv[2], tmp;
                                    if (a0 > a1) { tmp = a0; a0 = a1; a1 = tmp; }
                                    if (a1 > a2) { tmp = a1; a1 = a2; a2 = tmp; }
                                    if (a0 > a1) { tmp = a0; a0 = a1; a1 = tmp; }
                                    v = a1;
                                    ev[C_MULTI]++;
                                }
                            } else {
                                v = 0.5;
                                ev[C_INCONSISTENT]++;
                            }
                            a.so[A][myid] = v;
                            ev[C_MARKERS]++;
                            out_marker = true;
                            push_al = true;
                        } else if (nl >= 2) {
                            ev[C_ANNIHILATE]++;
                        }
                    }
                    // unaligned edges: a marker -> FP64 list; none -> count the
                    // crossings that met there (topology change, Fig. 5)
                    const int m = col[0][0][0];
                    const bool pres1 = n0 != nc[0][1][0];
                    const bool pres2 = n0 != nc[0][0][1];
                    push[0] = pres1;
                    push[1] = pres2;
                    const bool chk1 = !pres1 && ((col[1][0][0] ^ m) | (col[2][0][0] ^ m) | (col[0][1][0] ^ m) |
                                                 (col[1][1][0] ^ m) | (col[2][1][0] ^ m));
                    const bool chk2 = !pres2 && ((col[1][0][0] ^ m) | (col[2][0][0] ^ m) | (col[0][0][1] ^ m) |
                                                 (col[1][0][1] ^ m) | (col[2][0][1] ^ m));
                    if (NL == 6) {
                        push[4] = chk1;
                        push[5] = chk2;
                    } else {
                        if (chk1 && (cell.template loadw<T1, T2>(), cell.template count_crossings<T1, T2>()) >= 2)
                            ev[C_ANNIHILATE]++;
                        if (chk2 && (cell.template loadw<T2, T1>(), cell.template count_crossings<T2, T1>()) >= 2)
                            ev[C_ANNIHILATE]++;
                    }
                    out_marker |= pres1 || pres2;
                    // face colours: family 1 faces are normal to T2, family 2 to T1
                    int byte = n0;
                    push[2] = saddle4(n0, nc[1][0][0], nc[0][1][0], nc[1][1][0]);
                    if (!push[2]) byte |= n0 << (1 + T2);
                    push[3] = saddle4(n0, nc[1][0][0], nc[0][0][1], nc[1][0][1]);
                    if (!push[3]) byte |= n0 << (1 + T1);
                    int fa = saddle4(n0, nc[0][1][0], nc[0][0][1], nc[0][1][1]) ? ((myb >> (1 + A)) & 1) : n0;
                    byte |= fa << (1 + A);
                    a.cbo[myid] = (uint8_t)byte;
                    if (in_marker || out_marker) mk |= near_bits(l[0], l[1], l[2], S::TX, S::TY, S::TZ);
                }
            }
            // the warp's appends to the NL work lists and the marker list: all
            // ballots first, then lane 0 reserves every list's slots with
            // independent atomics (one round trip to L2 for all of them); a
            // warp with nothing to append (cells away from the interface)
            // skips it after one vote
            bool any_push = push_al;
#pragma unroll
            for (int k = 0; k < NL; k++) any_push |= push[k];
            if (__any_sync(0xffffffffu, any_push)) {
                const unsigned full = 0xffffffffu;
                const int lane = threadIdx.x & 31;
                unsigned m[NL + 1];
                int base[NL + 1];
#pragma unroll
                for (int k = 0; k < NL; k++) m[k] = __ballot_sync(full, push[k]);
                m[NL] = a.mk_out ? __ballot_sync(full, push_al) : 0u;
#pragma unroll
                for (int k = 0; k <= NL; k++) base[k] = 0;
                if (lane == 0) {
#pragma unroll
                    for (int k = 0; k < NL; k++)
                        if (m[k]) base[k] = atomicAdd(a.wcount + k, __popc(m[k]));
                    if (m[NL]) base[NL] = atomicAdd(a.mk_out_count, __popc(m[NL]));
                }
                const unsigned below = (1u << lane) - 1u;
#pragma unroll
                for (int k = 0; k < NL; k++) {
                    const int b = __shfl_sync(full, base[k], 0);
                    if (push[k]) a.work[k][b + __popc(m[k] & below)] = (unsigned)myid;
                }
                const int b = __shfl_sync(full, base[NL], 0);
                if (push_al && a.mk_out) a.mk_out[b + __popc(m[NL] & below)] = (unsigned)myid;
            }
        }
        {
            const unsigned v = __reduce_or_sync(0xffffffffu, mk);
            if ((threadIdx.x & 31) == 0 && v) atomicOr(s_flag, v);
        }
        if (__any_sync(0xffffffffu, (ev[0] | ev[1] | ev[2] | ev[3] | ev[4]) != 0u)) {
#pragma unroll
            for (int k = 0; k < C_N; k++) {
                unsigned v = __reduce_add_sync(0xffffffffu, ev[k]);
                if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.ctr + k, (unsigned long long)v);
            }
        }
        __syncthreads();
        int pending = -1;
        if (threadIdx.x == 0) {
            const unsigned fl = *s_flag;
            a.tile_marker[tile] = fl;
            a.tile_dirty[tile] = 1;
            if (a.band_flag) a.band_flag[tile] = 0u;
            // a slot on the list of tiles with markers nearby; the caller
            // stores the tile id there later, so that nothing waits for it
            if (a.mt_out && fl) pending = atomicAdd(a.mt_out_count, 1);
        }
        __syncthreads();
        return pending;
    }
}

template <int D, int NL = 4>
__global__ void __launch_bounds__(256, 4) sweep_kernel(SweepArgs a) {
    __shared__ unsigned s_flag;
    __shared__ uint8_t s_b[RA * R1 * R2];
    __shared__ int8_t s_n[RA * R1 * R2];
    __shared__ int s_li;
    pdl_wait();
    const int ntl = *a.count;
    // the previous tile's slot on the marker-tile list (thread 0), stored one
    // tile later so that the atomic that reserved it is not waited for
    int pending = -1, pending_tile = 0;
    if (a.tile_next) {
        // tiles differ in cost (interface tiles against halo tiles): each block
        // takes the next one when it is done, the counter read one tile ahead.
        // Every thread reads s_li before the first barrier inside sweep_tile,
        // and thread 0 rewrites it only after the last one.
        int next = threadIdx.x == 0 ? atomicAdd(a.tile_next, 1) : 0;
        for (;;) {
            if (threadIdx.x == 0) s_li = next;
            __syncthreads();
            const int li = s_li;
            if (li >= ntl) break;
            if (threadIdx.x == 0) {
                next = atomicAdd(a.tile_next, 1);
                if (pending >= 0) a.mt_out[pending] = pending_tile;
            }
            pending_tile = a.list[li];
            pending = sweep_tile<D, false, NL>(a, pending_tile, s_b, s_n, &s_flag);
        }
    } else {
        for (int li = blockIdx.x; li < ntl; li += gridDim.x) {
            if (threadIdx.x == 0 && pending >= 0) a.mt_out[pending] = pending_tile;
            pending_tile = a.list[li];
            pending = sweep_tile<D, false, NL>(a, pending_tile, s_b, s_n, &s_flag);
        }
    }
    if (threadIdx.x == 0 && pending >= 0) a.mt_out[pending] = pending_tile;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.ctr + C_TILES, (unsigned long long)ntl);
}


// ------------------------------------------------- FP64 work lists
// Entry k of list `kind` (0, 1: unaligned edges of families 1, 2; 2, 3: saddle
// faces of families 1, 2).
template <int D, bool F>
__device__ __forceinline__ void fp64_item(const SweepArgs &a, int kind, int k, unsigned ev[C_N], int half = -1) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    const int id = (int)ld_in<F>(a.work[kind] + k);
    const int x = id % a.g.n[0], y = (id / a.g.n[0]) % a.g.n[1], z = id / (a.g.n[0] * a.g.n[1]);
    SweepCell<D, F> cell(a, x, y, z);
    if ((kind & 1) == 0) cell.template loadw<T1, T2>();
    else cell.template loadw<T2, T1>();
    if (kind >= 4) {
        // an even number (>= 2) of advected crossings met on an edge that keeps
        // no marker (Fig. 5)
        const int nc = (kind == 4) ? cell.template count_crossings<T1, T2>() : cell.template count_crossings<T2, T1>();
        if (nc >= 2) ev[C_ANNIHILATE]++;
    } else if (kind == 0) {
        cell.template unaligned<T1, T2>(ev, half);
    } else if (kind == 1) {
        cell.template unaligned<T2, T1>(ev, half);
    } else {
        int ncol0 = ld_in<F>(a.cbo + id) & 1;
        int bit = (kind == 2) ? (cell.template face_phase<T1, T2>(ncol0) << (1 + T2))
                              : (cell.template face_phase<T2, T1>(ncol0) << (1 + T1));
        if (bit) {
            uintptr_t addr = (uintptr_t)(a.cbo + id);
            unsigned *w = (unsigned *)(addr & ~(uintptr_t)3);
            atomicOr(w, (unsigned)bit << (8 * (addr & 3)));
        }
    }
}

template <int D, int NL = 4>
__global__ void __launch_bounds__(128, 8) fp64_kernel(SweepArgs a) {
    pdl_wait();
    const int n0 = a.wcount[0], n1 = a.wcount[1], n2 = a.wcount[2], n3 = a.wcount[3];
    const int n4 = NL == 6 ? a.wcount[4] : 0, n5 = NL == 6 ? a.wcount[5] : 0;
    const int total = n0 + n1 + n2 + n3 + n4 + n5;
    unsigned ev[C_N] = {0, 0, 0, 0, 0};
    const int stride = gridDim.x * blockDim.x;
    // Unaligned edges first, then saddle faces and annihilation checks, one lane
    // each.  When the lists fit one round of the grid with two lanes per
    // unaligned edge, each edge gets two adjacent lanes and the circle fits are
    // split between them: a shorter chain per warp where few warps run.  Long
    // lists keep one lane per edge, since the pairs repeat the work before the
    // fits.  The trip count is uniform so that every lane reaches the warp
    // reductions.
    const int nu = n0 + n1, rest = total - nu;
    const bool pairs = 2 * nu + rest <= stride;
    const int lanes_u = pairs ? 2 * nu : nu;
    const int iters = (lanes_u + rest + stride - 1) / stride;
    for (int it = 0; it < iters; it++) {
        const int t2 = list_item(it);
        int t, half;
        if (t2 < lanes_u) {
            t = pairs ? t2 >> 1 : t2;
            half = pairs ? (t2 & 1) : -1;
        } else {
            t = nu + (t2 - lanes_u);
            half = -1;
        }
        if (t >= total) continue;
        int k, kind;
        if (t < n0) { kind = 0; k = t; }
        else if (t < n0 + n1) { kind = 1; k = t - n0; }
        else if (t < n0 + n1 + n2) { kind = 2; k = t - n0 - n1; }
        else if (t < n0 + n1 + n2 + n3) { kind = 3; k = t - n0 - n1 - n2; }
        else if (t < n0 + n1 + n2 + n3 + n4) { kind = 4; k = t - n0 - n1 - n2 - n3; }
        else { kind = 5; k = t - n0 - n1 - n2 - n3 - n4; }
        fp64_item<D, false>(a, kind, k, ev, half);
    }
#pragma unroll
    for (int k = 0; k < C_N; k++) {
        unsigned v = __reduce_add_sync(0xffffffffu, ev[k]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.ctr + k, (unsigned long long)v);
    }
}

}  // namespace ebit
