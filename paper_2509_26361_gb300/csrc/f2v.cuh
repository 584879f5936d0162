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
    const int *__restrict__ list;
    const int *__restrict__ count;
    uint8_t *tile_cchg;   // per tile: C rewritten (for the curvature band)
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

__global__ void __launch_bounds__(256) f2v_kernel(F2VArgs a) {
    const int ntl = *a.count;
    for (int li = blockIdx.x; li < ntl; li += gridDim.x) {
        const int tile = a.list[li];
        int o[3];
        tile_origin(a.g, tile, o);
        unsigned nbad = 0;
        for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
            int x = o[0] + (c & 7), y = o[1] + ((c >> 3) & 7), z = o[2] + (c >> 6);
            if (x >= a.g.n[0] || y >= a.g.n[1] || z >= a.g.n[2]) continue;
            int K = 0;
            int ids[8];
            for (int cid = 0; cid < 8; cid++) {
                ids[cid] = lin(a.g, x + (cid & 1), y + ((cid >> 1) & 1), z + ((cid >> 2) & 1));
                K |= (__ldg(a.cb + ids[cid]) & 1) << cid;
            }
            double val;
            if (K == 0 || K == 255) {
                val = (double)(K & 1);
            } else {
                const uint8_t b0 = __ldg(a.cb + ids[0]);
                int F[6];
                F[0] = (b0 >> 1) & 1;
                F[1] = (__ldg(a.cb + ids[1]) >> 1) & 1;
                F[2] = (b0 >> 2) & 1;
                F[3] = (__ldg(a.cb + ids[2]) >> 2) & 1;
                F[4] = (b0 >> 3) & 1;
                F[5] = (__ldg(a.cb + ids[4]) >> 3) & 1;
                double E[12];
                // x-edges at corners (0,dy,dz); y-edges at (dx,0,dz); z-edges at (dx,dy,0)
                const int xe[4] = {ids[0], ids[2], ids[4], ids[6]};
                const int xo[4] = {ids[1], ids[3], ids[5], ids[7]};
                const int ye[4] = {ids[0], ids[1], ids[4], ids[5]};
                const int yo[4] = {ids[2], ids[3], ids[6], ids[7]};
                const int ze[4] = {ids[0], ids[1], ids[2], ids[3]};
                const int zo[4] = {ids[4], ids[5], ids[6], ids[7]};
                const int cx[4] = {0, 2, 4, 6}, cxo[4] = {1, 3, 5, 7};
                const int cy[4] = {0, 1, 4, 5}, cyo[4] = {2, 3, 6, 7};
                const int cz[4] = {0, 1, 2, 3}, czo[4] = {4, 5, 6, 7};
                for (int r = 0; r < 4; r++) {
                    E[r] = (((K >> cx[r]) ^ (K >> cxo[r])) & 1) ? __ldg(a.s[0] + xe[r]) : 0.0;
                    E[4 + r] = (((K >> cy[r]) ^ (K >> cyo[r])) & 1) ? __ldg(a.s[1] + ye[r]) : 0.0;
                    E[8 + r] = (((K >> cz[r]) ^ (K >> czo[r])) & 1) ? __ldg(a.s[2] + ze[r]) : 0.0;
                }
                (void)xo; (void)yo; (void)zo;
                int bad = 0;
                val = cell_fraction(K, F, E, &bad);
                nbad += bad;
            }
            a.C[ids[0]] = val;
        }
        unsigned v = __reduce_add_sync(0xffffffffu, nbad);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.bad, (unsigned long long)v);
        if (threadIdx.x == 0 && a.tile_cchg) a.tile_cchg[tile] = 1;
    }
}

}  // namespace ebit
