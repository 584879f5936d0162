// f2v.cuh -- Front2VOF volume fractions (arxiv 2509.26361, Sec. 2.6, Eq. 7).
//
// Per cell: the corner colours (and the face colour on saddle faces) give the
// face segments of the six cube faces (Sec. 2.3, Fig. 7b); oriented so that the
// reference phase lies on their left seen from outside, they chain into closed
// loops, one loop per interface segment of the cell (separate loops are never
// merged, Sec. 2.4).  Each loop is fanned into triangles around the centroid of
// its markers (Eq. 7), and the reference-phase volume follows from Gauss's
// theorem with the cell's lowest corner as origin:
//     V = (A_x1 + A_y1 + A_z1) / 3 - sum_loops sum_i det(c, p_i, p_i+1) / 6,
// where A_a1 is the reference-phase area on the cube face a = 1 (the faces
// through the origin contribute nothing).  C = V clamped to [0, 1].
#pragma once
#include "common.cuh"

namespace ebit {

// corners of the six cube faces, counter-clockwise seen from outside
// (corner id = dx | dy<<1 | dz<<2); faces x=0, x=1, y=0, y=1, z=0, z=1
__constant__ int8_t kFaceCorner[6][4] = {
    {0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
// cube edge between consecutive face corners k and k+1 (x-edges 0-3 by dy+2dz,
// y-edges 4-7 by dx+2dz, z-edges 8-11 by dx+2dy)
__constant__ int8_t kFaceEdge[6][4] = {
    {8, 6, 10, 4}, {5, 11, 7, 9}, {0, 9, 2, 8}, {10, 3, 11, 1}, {4, 1, 5, 0}, {2, 7, 3, 6}};

struct F2VArgs {
    Grid g;
    const uint8_t *__restrict__ cb;
    const double *__restrict__ s[3];
    double *__restrict__ C;
    const int *__restrict__ list;    // tiles to recompute
    const int *__restrict__ count;
    unsigned *__restrict__ cut;      // cells cut by the interface (output list)
    int *__restrict__ ncut;
    unsigned long long *bad;
};

struct V3 {
    double x[3];
};

__device__ __forceinline__ V3 corner3(int c) {
    V3 r;
    r.x[0] = (double)(c & 1);
    r.x[1] = (double)((c >> 1) & 1);
    r.x[2] = (double)((c >> 2) & 1);
    return r;
}

__device__ __forceinline__ double det3(const V3 &c, const V3 &p, const V3 &q) {
    return c.x[0] * (p.x[1] * q.x[2] - p.x[2] * q.x[1]) + c.x[1] * (p.x[2] * q.x[0] - p.x[0] * q.x[2]) +
           c.x[2] * (p.x[0] * q.x[1] - p.x[1] * q.x[0]);
}

// |area| of a polygon on a face, projected on the face axes (u, v)
__device__ __forceinline__ double area_uv(const V3 *pts, int np, int u, int v) {
    double acc = 0.0;
    for (int i = 0; i < np; i++) {
        const V3 &a = pts[i];
        const V3 &b = pts[i + 1 == np ? 0 : i + 1];
        acc += a.x[u] * b.x[v] - b.x[u] * a.x[v];
    }
    return 0.5 * fabs(acc);
}

// volume fraction of one cell; *bad set on an inconsistent configuration
__device__ __noinline__ double cell_fraction(int K, const int F[6], const double E[12], int *bad) {
    V3 mk[12];
    for (int e = 0; e < 12; e++) {
        int ax = e >> 2, r = e & 3;
        V3 p;
        if (ax == 0) { p.x[0] = E[e]; p.x[1] = (double)(r & 1); p.x[2] = (double)(r >> 1); }
        else if (ax == 1) { p.x[0] = (double)(r & 1); p.x[1] = E[e]; p.x[2] = (double)(r >> 1); }
        else { p.x[0] = (double)(r & 1); p.x[1] = (double)(r >> 1); p.x[2] = E[e]; }
        mk[e] = p;
    }
    int8_t out[12];
    for (int e = 0; e < 12; e++) out[e] = -1;
    unsigned hasmask = 0;
    double A1[3] = {0.0, 0.0, 0.0};
    for (int f = 0; f < 6; f++) {
        int kc[4], col[4], ed[4], mm[4], nm = 0;
        for (int k = 0; k < 4; k++) {
            kc[k] = kFaceCorner[f][k];
            col[k] = (K >> kc[k]) & 1;
            ed[k] = kFaceEdge[f][k];
        }
        for (int k = 0; k < 4; k++) {
            mm[k] = col[k] != col[(k + 1) & 3];
            nm += mm[k];
            if (mm[k]) hasmask |= 1u << ed[k];
        }
        const int upper = f & 1, fa = f >> 1;
        const int u = fa == 2 ? 0 : fa + 1, v = fa == 0 ? 2 : (fa == 1 ? 0 : 1);
        double area1 = 0.0;
        if (nm == 0) {
            area1 = (double)col[0];
        } else if (nm == 2) {
            int ea = -1, eb = -1;
            for (int k = 0; k < 4; k++)
                if (mm[k]) {
                    if (ea < 0) ea = k;
                    else eb = k;
                }
            int arc = col[(ea + 1) & 3];
            if (arc) out[ed[eb]] = (int8_t)ed[ea];
            else out[ed[ea]] = (int8_t)ed[eb];
            if (upper) {
                V3 poly[6];
                int np = 0;
                poly[np++] = mk[ed[ea]];
                for (int k = ea + 1; k <= eb; k++) poly[np++] = corner3(kc[k]);
                poly[np++] = mk[ed[eb]];
                double R = area_uv(poly, np, u, v);
                area1 = arc ? R : 1.0 - R;
            }
        } else if (nm == 4) {
            int phif = F[f];
            double T = 0.0;
            for (int m = 0; m < 4; m++) {
                if (col[m] == phif) continue;
                int ep = ed[(m + 3) & 3], en = ed[m];
                if (col[m]) out[en] = (int8_t)ep;
                else out[ep] = (int8_t)en;
                if (upper) {
                    V3 tri[3] = {mk[ep], corner3(kc[m]), mk[en]};
                    T += area_uv(tri, 3, u, v);
                }
            }
            area1 = (1 - phif) ? T : 1.0 - T;
        } else {
            *bad = 1;
        }
        if (upper) A1[fa] = area1;
    }
    if (!hasmask) return (double)(K & 1);
    unsigned vis = 0;
    double acc = 0.0;
    for (int e0 = 0; e0 < 12; e0++) {
        if (!((hasmask >> e0) & 1) || ((vis >> e0) & 1)) continue;
        int idx[12];
        int len = 0, e = e0;
        while (len < 12) {
            if (e < 0 || !((hasmask >> e) & 1) || ((vis >> e) & 1)) break;
            vis |= 1u << e;
            idx[len++] = e;
            e = out[e];
            if (e == e0) break;
        }
        if (e != e0) {
            *bad = 1;
            continue;
        }
        V3 cen;
        for (int a = 0; a < 3; a++) {
            double sm = 0.0;
            for (int i = 0; i < len; i++) sm += mk[idx[i]].x[a];
            cen.x[a] = sm / (double)len;
        }
        for (int i = 0; i < len; i++) acc += det3(cen, mk[idx[i]], mk[idx[i + 1 == len ? 0 : i + 1]]);
    }
    double V = ((A1[0] + A1[1]) + A1[2]) / 3.0 - acc / 6.0;
    if (V < 0.0) V = 0.0;
    if (V > 1.0) V = 1.0;
    return V;
}

__device__ __forceinline__ void cell_ids(const Grid &g, int x, int y, int z, int ids[8]) {
#pragma unroll
    for (int cid = 0; cid < 8; cid++) ids[cid] = lin(g, x + (cid & 1), y + ((cid >> 1) & 1), z + ((cid >> 2) & 1));
}

// Band pass (integer only): a cell with eight equal corner colours holds no
// marker and its fraction is that colour (written as a bit pattern); the other
// cells go to the global cut list.
__global__ void __launch_bounds__(256) f2v_band_kernel(F2VArgs a) {
    pdl_wait();
    const int ntl = *a.count;
    for (int li = blockIdx.x; li < ntl; li += gridDim.x) {
        const int tile = a.list[li];
        int o[3];
        tile_origin(a.g, tile, o);
        for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
            int l[3];
            tile_cell(a.g, c, l);
            int x = o[0] + l[0], y = o[1] + l[1], z = o[2] + l[2];
            bool cutc = false;
            int id0 = 0;
            if (x < a.g.n[0] && y < a.g.n[1] && z < a.g.n[2]) {
                int ids[8];
                cell_ids(a.g, x, y, z, ids);
                int K = 0;
#pragma unroll
                for (int cid = 0; cid < 8; cid++) K |= (__ldg(a.cb + ids[cid]) & 1) << cid;
                id0 = ids[0];
                if (K == 0 || K == 255)
                    reinterpret_cast<unsigned long long *>(a.C)[id0] = (K & 1) ? 0x3FF0000000000000ull : 0ull;
                else
                    cutc = true;
            }
            const unsigned full = 0xffffffffu;
            unsigned m = __ballot_sync(full, cutc);
            if (m) {
                const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(a.ncut, __popc(m));
                base = __shfl_sync(full, base, leader);
                if (cutc) a.cut[base + __popc(m & ((1u << lane) - 1u))] = (unsigned)id0;
            }
        }
    }
}

// Per-cell reconstruction used by the list kernel.  Same geometry as
// cell_fraction (the reference form above, kept for the exhaustive checks), in
// a register-only formulation:
//   * face areas from closed forms -- a corner cut is the triangle l1*l2/2, a
//     cut across the face the trapezoid (l1 + l2)/2, three corners the
//     complement of a corner cut (l = distances from the cut corner or side);
//   * loops walked through successor codes packed 4 bits per edge;
//   * sum_i det(c, p_i, p_i+1) = c . sum_i (p_i x p_i+1) with c the mean of
//     the loop's markers (Eq. 7) -- the same sum reassociated, so C agrees
//     with the fan-by-fan evaluation to rounding (about 1e-16).
// face corner k -> k+1 runs along +axis when the edge goes from its lower to its
// upper node: kFaceFwd[f][k] = 1 (then the marker sits at distance s from
// corner k).
__constant__ int8_t kFaceFwd[6][4] = {
    {1, 1, 0, 0}, {1, 1, 0, 0}, {1, 1, 0, 0}, {1, 1, 0, 0}, {1, 1, 0, 0}, {1, 1, 0, 0}};

__device__ __forceinline__ double sel01(int b) { return __longlong_as_double(b ? 0x3FF0000000000000ll : 0ll); }

__device__ __forceinline__ void marker_xyz(int e, double s, double &x, double &y, double &z) {
    const int ax = e >> 2, r = e & 3;
    const double u = sel01(r & 1), v = sel01(r >> 1);
    x = ax == 0 ? s : u;
    y = ax == 1 ? s : (ax == 0 ? u : v);
    z = ax == 2 ? s : v;
}

// distance from face corner k to the marker on face edge k (corner k -> k+1)
// and from corner k+1 to it
__device__ __forceinline__ double dist_from_k(int fwd, double s) { return fwd ? s : 1.0 - s; }
__device__ __forceinline__ double dist_from_k1(int fwd, double s) { return fwd ? 1.0 - s : s; }

template <int F>
__device__ __forceinline__ double face_area_and_links(int K, int phif, const double *sE, int stride,
                                                      unsigned long long &nxt) {
    int col[4], ed[4], fw[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        col[k] = (K >> kFaceCorner[F][k]) & 1;
        ed[k] = kFaceEdge[F][k];
        fw[k] = kFaceFwd[F][k];
    }
    int mm = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) mm |= (col[k] != col[(k + 1) & 3]) << k;
    const int nm = __popc(mm);
    double area = 0.0;
    auto link = [&](int from, int to) {
        nxt = (nxt & ~(0xFull << (4 * from))) | ((unsigned long long)to << (4 * from));
    };
    if (nm == 0) {
        area = sel01(col[0]);
    } else if (nm == 2) {
        const int ea = __ffs(mm) - 1, eb = 31 - __clz(mm);
        const int arc = col[(ea + 1) & 3];
        if (arc) link(ed[eb], ed[ea]);
        else link(ed[ea], ed[eb]);
        if (F & 1) {
            const double sa = sE[ed[ea] * stride], sb = sE[ed[eb] * stride];
            double R;
            if (eb == ea + 1) {
                // triangle at corner ea+1: legs along E_ea (to corner ea+1) and E_eb (from it)
                R = 0.5 * (dist_from_k1(fw[ea], sa) * dist_from_k(fw[eb], sb));
            } else if (eb == ea + 2) {
                // corners ea+1, ea+2 on the opposite parallel edges E_ea, E_eb
                R = 0.5 * (dist_from_k1(fw[ea], sa) + dist_from_k(fw[eb], sb));
            } else {
                // three corners: complement of the triangle at corner ea (= eb + 1)
                R = 1.0 - 0.5 * (dist_from_k(fw[ea], sa) * dist_from_k1(fw[eb], sb));
            }
            area = arc ? R : 1.0 - R;
        }
    } else if (nm == 4) {
        double T = 0.0;
#pragma unroll
        for (int m = 0; m < 4; m++) {
            if (col[m] == phif) continue;
            const int ep = ed[(m + 3) & 3], en = ed[m];
            if (col[m]) link(en, ep);
            else link(ep, en);
            if (F & 1) T += 0.5 * (dist_from_k1(fw[(m + 3) & 3], sE[ep * stride]) * dist_from_k(fw[m], sE[en * stride]));
        }
        area = (1 - phif) ? T : 1.0 - T;
    }
    return area;
}

__device__ double cell_fraction_fast(int K, const int Fc[6], const double *sE, int stride, int *bad) {
    unsigned long long nxt = ~0ull;
    double A1 = 0.0, A2 = 0.0, A3 = 0.0;
    face_area_and_links<0>(K, Fc[0], sE, stride, nxt);
    A1 = face_area_and_links<1>(K, Fc[1], sE, stride, nxt);
    face_area_and_links<2>(K, Fc[2], sE, stride, nxt);
    A2 = face_area_and_links<3>(K, Fc[3], sE, stride, nxt);
    face_area_and_links<4>(K, Fc[4], sE, stride, nxt);
    A3 = face_area_and_links<5>(K, Fc[5], sE, stride, nxt);
    // markers: edges whose end colours differ
    unsigned has = 0;
    const int cx[4] = {0, 2, 4, 6}, cy[4] = {0, 1, 4, 5}, cz[4] = {0, 1, 2, 3};
#pragma unroll
    for (int r = 0; r < 4; r++) {
        has |= (unsigned)(((K >> cx[r]) ^ (K >> (cx[r] + 1))) & 1) << r;
        has |= (unsigned)(((K >> cy[r]) ^ (K >> (cy[r] + 2))) & 1) << (4 + r);
        has |= (unsigned)(((K >> cz[r]) ^ (K >> (cz[r] + 4))) & 1) << (8 + r);
    }
    if (!has) return sel01(K & 1);
    unsigned todo = has;
    double acc = 0.0;
    while (todo) {
        const int e0 = __ffs(todo) - 1;
        double x0, y0, z0;
        marker_xyz(e0, sE[e0 * stride], x0, y0, z0);
        double sx = x0, sy = y0, sz = z0;
        double px = x0, py = y0, pz = z0;
        double cxs = 0.0, cys = 0.0, czs = 0.0;
        int len = 1, e = e0;
        todo &= ~(1u << e0);
        bool closed = false;
        for (int guard = 0; guard < 12; guard++) {
            int nx_ = (int)((nxt >> (4 * e)) & 0xF);
            if (nx_ == 0xF) break;
            double qx, qy, qz;
            if (nx_ == e0) {
                qx = x0; qy = y0; qz = z0;
            } else {
                if (!((todo >> nx_) & 1)) break;
                marker_xyz(nx_, sE[nx_ * stride], qx, qy, qz);
            }
            cxs += py * qz - pz * qy;
            cys += pz * qx - px * qz;
            czs += px * qy - py * qx;
            if (nx_ == e0) {
                closed = true;
                break;
            }
            sx += qx; sy += qy; sz += qz;
            px = qx; py = qy; pz = qz;
            todo &= ~(1u << nx_);
            e = nx_;
            len++;
        }
        if (!closed) {
            *bad = 1;
            continue;
        }
        acc += (sx * cxs + sy * cys + sz * czs) / (double)len;
    }
    double V = (2.0 * ((A1 + A2) + A3) - acc) / 6.0;
    if (V < 0.0) V = 0.0;
    if (V > 1.0) V = 1.0;
    return V;
}

// FP64 pass: one thread per cut cell, full warps.
__global__ void __launch_bounds__(128) f2v_list_kernel(F2VArgs a) {
    __shared__ double sE[12 * 128];
    pdl_wait();
    const int n = *a.ncut;
    unsigned nbad = 0;
    const int stride = gridDim.x * blockDim.x;
    const int iters = (n + stride - 1) / stride;
    double *myE = sE + threadIdx.x;
    for (int it = 0; it < iters; it++) {
        const int t = list_item(it);
        if (t >= n) continue;
        const int id = (int)a.cut[t];
        const int x = id % a.g.n[0], y = (id / a.g.n[0]) % a.g.n[1], z = id / (a.g.n[0] * a.g.n[1]);
        int ids[8];
        cell_ids(a.g, x, y, z, ids);
        int K = 0;
#pragma unroll
        for (int cid = 0; cid < 8; cid++) K |= (__ldg(a.cb + ids[cid]) & 1) << cid;
        const uint8_t b0 = __ldg(a.cb + ids[0]);
        int F[6];
        F[0] = (b0 >> 1) & 1;
        F[1] = (__ldg(a.cb + ids[1]) >> 1) & 1;
        F[2] = (b0 >> 2) & 1;
        F[3] = (__ldg(a.cb + ids[2]) >> 2) & 1;
        F[4] = (b0 >> 3) & 1;
        F[5] = (__ldg(a.cb + ids[4]) >> 3) & 1;
        // x-edges at corners (0,dy,dz), y-edges at (dx,0,dz), z-edges at (dx,dy,0)
        const int cx[4] = {0, 2, 4, 6}, cy[4] = {0, 1, 4, 5}, cz[4] = {0, 1, 2, 3};
#pragma unroll
        for (int r = 0; r < 4; r++) {
            myE[r * 128] = (((K >> cx[r]) ^ (K >> (cx[r] + 1))) & 1) ? __ldg(a.s[0] + ids[cx[r]]) : 0.0;
            myE[(4 + r) * 128] = (((K >> cy[r]) ^ (K >> (cy[r] + 2))) & 1) ? __ldg(a.s[1] + ids[cy[r]]) : 0.0;
            myE[(8 + r) * 128] = (((K >> cz[r]) ^ (K >> (cz[r] + 4))) & 1) ? __ldg(a.s[2] + ids[cz[r]]) : 0.0;
        }
        int bad = 0;
        a.C[id] = cell_fraction_fast(K, F, myE, 128, &bad);
        nbad += bad;
    }
    unsigned v = __reduce_add_sync(0xffffffffu, nbad);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.bad, (unsigned long long)v);
}

}  // namespace ebit
