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
// GPU organisation: one CTA per 8x8x8 tile of the active band, one thread per
// cell; each thread computes everything its cell owns (node colour, the three
// edges leaving its node, the three faces whose lowest corner it is) directly
// from the old state (gather form), so no two threads write the same word and
// old and new state live in separate buffers.  Cells whose 4x2x2 colour
// neighbourhood is uniform take a fast path (no marker can reach them).
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
    const int *__restrict__ list;    // band tile ids
    const int *__restrict__ count;   // number of band tiles (device)
    unsigned long long *ctr;         // event counters
    uint8_t *tile_marker;            // per tile: a marker in the input or the output
    uint8_t *tile_dirty;             // per tile: processed since the last Front2VOF
};

struct P2 {
    double x, y;
};

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
// (0 <= y <= 1) count, the one nearest ylin is kept (Fig. 2).
__device__ __noinline__ bool circle_root(P2 A, P2 B, P2 C, double ylin, double *root, double *rad) {
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
    *rad = sqrt(r2);
    return true;
}

template <int D>
struct SweepCell {
    static constexpr int A = D, T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    const SweepArgs &a;
    int p[3];
    unsigned cfl_hits;
    unsigned incons;

    __device__ SweepCell(const SweepArgs &args, int x, int y, int z) : a(args), cfl_hits(0), incons(0) {
        p[0] = x;
        p[1] = y;
        p[2] = z;
    }

    // global node for sweep-local offsets along (A, T1, T2)
    __device__ __forceinline__ void node3(int da, int d1, int d2, int q[3]) const {
        q[A] = p[A] + da;
        q[T1] = p[T1] + d1;
        q[T2] = p[T2] + d2;
    }
    __device__ __forceinline__ int id3(int da, int d1, int d2) const {
        int q[3];
        node3(da, d1, d2, q);
        return lin3(a.g, q);
    }

    // trilinear u_D at node q shifted by s along axis e; lerps in x, y, z order
    __device__ double interp(const int q[3], int e, double s) const {
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
        const Grid &g = a.g;
        int x0 = wrapc(base[0], g.n[0]), x1 = wrapc(base[0] + 1, g.n[0]);
        int y0 = wrapc(base[1], g.n[1]), y1 = wrapc(base[1] + 1, g.n[1]);
        int z0 = wrapc(base[2], g.n[2]), z1 = wrapc(base[2] + 1, g.n[2]);
        const double *u = a.u;
        int r00 = (z0 * g.n[1] + y0) * g.n[0], r10 = (z0 * g.n[1] + y1) * g.n[0];
        int r01 = (z1 * g.n[1] + y0) * g.n[0], r11 = (z1 * g.n[1] + y1) * g.n[0];
        double c00 = (1.0 - t[0]) * __ldg(u + r00 + x0) + t[0] * __ldg(u + r00 + x1);
        double c10 = (1.0 - t[0]) * __ldg(u + r10 + x0) + t[0] * __ldg(u + r10 + x1);
        double c01 = (1.0 - t[0]) * __ldg(u + r01 + x0) + t[0] * __ldg(u + r01 + x1);
        double c11 = (1.0 - t[0]) * __ldg(u + r11 + x0) + t[0] * __ldg(u + r11 + x1);
        double c0 = (1.0 - t[1]) * c00 + t[1] * c10;
        double c1 = (1.0 - t[1]) * c01 + t[1] * c11;
        return (1.0 - t[2]) * c0 + t[2] * c1;
    }

    // displacement in cells of the marker at node q on its e-edge (CFL clamp)
    __device__ double disp(const int q[3], int e, double s, bool own) {
        double c = interp(q, e, s) * a.lam;
        if (!(fabs(c) < 1.0)) {
            if (own) cfl_hits++;
            c = c > 0.0 ? ONE_MINUS : -ONE_MINUS;
        }
        return c;
    }

    __device__ __forceinline__ int colid(int id) const { return __ldg(a.cb + id) & 1; }

    // advected position (units of cells, relative to its node) of the aligned
    // marker on the A-edge of node (da, d1, d2)
    __device__ double Xa(int da, int d1, int d2, bool own) {
        int q[3];
        node3(da, d1, d2, q);
        int id = lin3(a.g, q);
        double sv = __ldg(a.s[A] + id);
        return sv + disp(q, A, sv, own);
    }

    // ---------------------------------------------------------------- planes
    // A plane of the face family with in-plane transverse axis TT and normal NN,
    // through the thread's node; offsets (da, dt) along (A, TT).
    template <int TT, int NN>
    __device__ __forceinline__ void pnode(int da, int dt, int q[3]) const {
        q[A] = p[A] + da;
        q[TT] = p[TT] + dt;
        q[NN] = p[NN];
    }
    template <int TT, int NN>
    __device__ __forceinline__ int pid(int da, int dt) const {
        int q[3];
        pnode<TT, NN>(da, dt, q);
        return lin3(a.g, q);
    }
    template <int TT, int NN>
    __device__ int psegs(int da, int dt, int seg[2][2]) const {
        int i00 = pid<TT, NN>(da, dt);
        int b00 = __ldg(a.cb + i00);
        return cell_segs(b00 & 1, colid(pid<TT, NN>(da + 1, dt)), colid(pid<TT, NN>(da, dt + 1)),
                         colid(pid<TT, NN>(da + 1, dt + 1)), (b00 >> (1 + NN)) & 1, seg);
    }
    // advected position of the marker on edge code e of the 2D cell (da, dt),
    // relative to the thread's node
    template <int TT, int NN>
    __device__ P2 ppos(int e, int da, int dt) {
        P2 r;
        int q[3];
        if (e == EB || e == ET) {
            int tt = dt + (e == ET ? 1 : 0);
            pnode<TT, NN>(da, tt, q);
            int id = lin3(a.g, q);
            double sv = __ldg(a.s[A] + id);
            double X = sv + disp(q, A, sv, false);
            r.x = (double)da + X;
            r.y = (double)tt;
        } else {
            int aa = da + (e == ER ? 1 : 0);
            pnode<TT, NN>(aa, dt, q);
            int id = lin3(a.g, q);
            double sv = __ldg(a.s[TT] + id);
            double c = disp(q, TT, sv, false);
            r.x = (double)aa + c;
            r.y = (double)dt + sv;
        }
        return r;
    }

    // The neighbour along the polyline of the marker on edge code e of cell
    // (da, dt), found in the cell across that edge.  Returns false if missing.
    template <int TT, int NN>
    __device__ bool neighbour(int e, int da, int dt, P2 *out) {
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

    // Unaligned edge (family TT/NN) of the thread's node.  Returns the number of
    // crossings; writes the reconstructed offset when present.
    template <int TT, int NN>
    __device__ void unaligned(bool present, unsigned *ev_ann, unsigned *ev_multi, double *sout) {
        // crossings of the advected polyline with the grid line x = 0 in strip 0
        P2 c2[4], c3[4];
        int e2[4], e3[4], cd[4];
        double yl[4];
        int nc = 0;
        for (int da = -1; da <= 0; da++) {
            int seg[2][2];
            int ns = psegs<TT, NN>(da, 0, seg);
            for (int k = 0; k < ns; k++) {
                P2 P = ppos<TT, NN>(seg[k][0], da, 0);
                P2 Q = ppos<TT, NN>(seg[k][1], da, 0);
                if ((P.x < 0.0) == (Q.x < 0.0)) continue;
                bool pl = P.x < 0.0;
                c2[nc] = pl ? P : Q;
                c3[nc] = pl ? Q : P;
                e2[nc] = pl ? seg[k][0] : seg[k][1];
                e3[nc] = pl ? seg[k][1] : seg[k][0];
                cd[nc] = da;
                double tt = (0.0 - c2[nc].x) / (c3[nc].x - c2[nc].x);
                yl[nc] = c2[nc].y + tt * (c3[nc].y - c2[nc].y);
                nc++;
            }
        }
        if (!present) {
            if (nc >= 2) (*ev_ann)++;
            return;
        }
        if ((nc & 1) == 0) {
            incons++;
            *sout = 0.5;
            return;
        }
        int sel = 0;
        if (nc == 3) {
            // median by ylin, equal values keep list order
            int o0 = 0, o1 = 1, o2 = 2, tmp;
            if (yl[o0] > yl[o1]) { tmp = o0; o0 = o1; o1 = tmp; }
            if (yl[o1] > yl[o2]) { tmp = o1; o1 = o2; o2 = tmp; }
            if (yl[o0] > yl[o1]) { tmp = o0; o0 = o1; o1 = tmp; }
            sel = o1;
            (*ev_multi)++;
        }
        P2 Pa = c2[sel], Pb = c3[sel];
        double ylin = yl[sel];
        P2 P1, P4;
        double ya = 0.0, ra = 0.0, yb = 0.0, rb = 0.0;
        bool va = false, vb = false;
        if (neighbour<TT, NN>(e2[sel], cd[sel], 0, &P1)) va = circle_root(P1, Pa, Pb, ylin, &ya, &ra);
        else incons++;
        if (neighbour<TT, NN>(e3[sel], cd[sel], 0, &P4)) vb = circle_root(Pa, Pb, P4, ylin, &yb, &rb);
        else incons++;
        double y;
        if (va && vb) {
            double rmax = ra > rb ? ra : rb, rmin = ra > rb ? rb : ra;
            if (rmax > 10.0 * rmin) y = ra > rb ? ya : yb;
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
        *sout = y;
    }

    // Colour of the face-centre of the family's 2D cell at the thread's node:
    // the phase of the advected polyline at the centre, reached from the node
    // along the a-line to x = 1/2 and then up the line x = 1/2 to y = 1/2.
    template <int TT, int NN>
    __device__ int face_phase(int ncol0) {
        int par = ncol0;
        for (int da = -1; da <= 1; da++) {
            int i0 = pid<TT, NN>(da, 0), i1 = pid<TT, NN>(da + 1, 0);
            if (colid(i0) == colid(i1)) continue;
            P2 P = ppos<TT, NN>(EB, da, 0);
            if (P.x >= 0.0 && P.x < 0.5) par ^= 1;
        }
        for (int da = -1; da <= 1; da++) {
            int seg[2][2];
            int ns = psegs<TT, NN>(da, 0, seg);
            for (int k = 0; k < ns; k++) {
                P2 P = ppos<TT, NN>(seg[k][0], da, 0);
                P2 Q = ppos<TT, NN>(seg[k][1], da, 0);
                if ((P.x < 0.5) == (Q.x < 0.5)) continue;
                P2 L = (P.x < 0.5) ? P : Q, R = (P.x < 0.5) ? Q : P;
                double tt = (0.5 - L.x) / (R.x - L.x);
                double yl = L.y + tt * (R.y - L.y);
                if (yl < 0.5) par ^= 1;
            }
        }
        return par;
    }

    __device__ static bool saddle(int c00, int c10, int c01, int c11) {
        return c00 == c11 && c10 == c01 && c00 != c10;
    }

    // Process the cell.  Returns whether any of its edges carries a marker in
    // the input or in the output.
    __device__ bool run(unsigned ev[C_N]) {
        const int myid = lin(a.g, p[0], p[1], p[2]);
        // old colours of the nodes (da, d1, d2), da in [-1, 2], d1, d2 in {0, 1}
        int col[4][2][2];
        int any = 0, c0 = colid(myid);
#pragma unroll
        for (int da = 0; da < 4; da++)
#pragma unroll
            for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
                for (int d2 = 0; d2 < 2; d2++) {
                    int c = (da == 1 && d1 == 0 && d2 == 0) ? c0 : colid(id3(da - 1, d1, d2));
                    col[da][d1][d2] = c;
                    any |= c ^ c0;
                }
        if (!any) {
            a.cbo[myid] = (uint8_t)(c0 | (c0 << 1) | (c0 << 2) | (c0 << 3));
            return false;
        }
        const uint8_t myb = __ldg(a.cb + myid);
        bool in_marker = (col[1][0][0] != col[2][0][0]) || (col[1][0][0] != col[1][1][0]) ||
                         (col[1][0][0] != col[1][0][1]);
        // advected aligned markers on the A-edges (da in {-1,0,1}) of the 4 lines
        double X[3][2][2];
        bool has[3][2][2];
#pragma unroll
        for (int da = 0; da < 3; da++)
#pragma unroll
            for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
                for (int d2 = 0; d2 < 2; d2++) {
                    has[da][d1][d2] = col[da][d1][d2] != col[da + 1][d1][d2];
                    X[da][d1][d2] = has[da][d1][d2] ? Xa(da - 1, d1, d2, da == 1 && d1 == 0 && d2 == 0) : 0.0;
                }
        // new colours of the nodes (dA, d1, d2), dA in {0, 1} (Fig. 4)
        int nc[2][2][2];
#pragma unroll
        for (int dA = 0; dA < 2; dA++)
#pragma unroll
            for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
                for (int d2 = 0; d2 < 2; d2++) {
                    int c = col[dA + 1][d1][d2];
                    if (has[dA][d1][d2] && X[dA][d1][d2] >= 1.0) c ^= 1;
                    if (has[dA + 1][d1][d2] && X[dA + 1][d1][d2] < 0.0) c ^= 1;
                    nc[dA][d1][d2] = c;
                }
        const int n0 = nc[0][0][0];
        bool out_marker = false;
        // aligned edge: presence from the new colours, markers landing on it (Fig. 5)
        {
            bool present = n0 != nc[1][0][0];
            double land[3];
            int nl = 0;
#pragma unroll
            for (int e = -1; e <= 1; e++) {
                if (!has[e + 1][0][0]) continue;
                double x = X[e + 1][0][0];
                int dest = (x < 0.0) ? -1 : (x >= 1.0 ? 1 : 0);
                if (e + dest != 0) continue;
                double sn = x - (double)dest;
                if (sn > ONE_MINUS) sn = ONE_MINUS;
                land[nl++] = sn;
            }
            if (present) {
                double v;
                if (nl == 1) {
                    v = land[0];
                } else if (nl == 3) {
                    double a0 = land[0], a1 = land[1], a2 = land[2], tmp;
                    if (a0 > a1) { tmp = a0; a0 = a1; a1 = tmp; }
                    if (a1 > a2) { tmp = a1; a1 = a2; a2 = tmp; }
                    if (a0 > a1) { tmp = a0; a0 = a1; a1 = tmp; }
                    v = a1;
                    ev[C_MULTI]++;
                } else {
                    v = 0.5;
                    incons++;
                }
                a.so[A][myid] = v;
                ev[C_MARKERS]++;
                out_marker = true;
            } else if (nl >= 2) {
                ev[C_ANNIHILATE]++;
            }
        }
        // unaligned edges of the two families (Fig. 1c, Fig. 2)
        {
            int qo[3];
            // own old unaligned markers: count a CFL violation once, by the owner
            if (col[1][0][0] != col[1][1][0]) {
                node3(0, 0, 0, qo);
                disp(qo, T1, __ldg(a.s[T1] + myid), true);
            }
            if (col[1][0][0] != col[1][0][1]) {
                node3(0, 0, 0, qo);
                disp(qo, T2, __ldg(a.s[T2] + myid), true);
            }
            bool pres1 = n0 != nc[0][1][0];
            bool cells1 = pres1 || col[0][0][0] != col[0][1][0] || col[0][0][0] != col[1][0][0] ||
                          col[0][0][0] != col[2][0][0] || col[0][0][0] != col[0][1][0] ||
                          col[0][0][0] != col[1][1][0] || col[0][0][0] != col[2][1][0];
            if (cells1) {
                double sv = 0.0;
                unaligned<T1, T2>(pres1, &ev[C_ANNIHILATE], &ev[C_MULTI], &sv);
                if (pres1) {
                    a.so[T1][myid] = sv;
                    ev[C_MARKERS]++;
                    out_marker = true;
                }
            }
            bool pres2 = n0 != nc[0][0][1];
            bool cells2 = pres2 || col[0][0][0] != col[0][0][1] || col[0][0][0] != col[1][0][0] ||
                          col[0][0][0] != col[2][0][0] || col[0][0][0] != col[1][0][1] ||
                          col[0][0][0] != col[2][0][1];
            if (cells2) {
                double sv = 0.0;
                unaligned<T2, T1>(pres2, &ev[C_ANNIHILATE], &ev[C_MULTI], &sv);
                if (pres2) {
                    a.so[T2][myid] = sv;
                    ev[C_MARKERS]++;
                    out_marker = true;
                }
            }
        }
        // face colours (Sec. 2.2): family 1 faces are normal to T2, family 2 to T1
        int f1 = saddle(n0, nc[1][0][0], nc[0][1][0], nc[1][1][0]) ? face_phase<T1, T2>(n0) : n0;
        int f2 = saddle(n0, nc[1][0][0], nc[0][0][1], nc[1][0][1]) ? face_phase<T2, T1>(n0) : n0;
        int fa = saddle(n0, nc[0][1][0], nc[0][0][1], nc[0][1][1]) ? ((myb >> (1 + A)) & 1) : n0;
        a.cbo[myid] = (uint8_t)(n0 | (fa << (1 + A)) | (f1 << (1 + T2)) | (f2 << (1 + T1)));
        return in_marker || out_marker;
    }
};

template <int D>
__global__ void __launch_bounds__(256) sweep_kernel(SweepArgs args) {
    __shared__ int s_flag;
    const int ntl = *args.count;
    for (int li = blockIdx.x; li < ntl; li += gridDim.x) {
        const int tile = args.list[li];
        int o[3];
        tile_origin(args.g, tile, o);
        if (threadIdx.x == 0) s_flag = 0;
        __syncthreads();
        unsigned ev[C_N] = {0, 0, 0, 0, 0};
        bool mk = false;
        for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
            int x = o[0] + (c & 7), y = o[1] + ((c >> 3) & 7), z = o[2] + (c >> 6);
            if (x >= args.g.n[0] || y >= args.g.n[1] || z >= args.g.n[2]) continue;
            SweepCell<D> cell(args, x, y, z);
            mk |= cell.run(ev);
            ev[C_INCONSISTENT] += cell.incons;
            ev[C_CFL] += cell.cfl_hits;
        }
        if (mk) s_flag = 1;
#pragma unroll
        for (int k = 0; k < C_N; k++) {
            unsigned v = __reduce_add_sync(0xffffffffu, ev[k]);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(args.ctr + k, (unsigned long long)v);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            args.tile_marker[tile] = (uint8_t)s_flag;
            args.tile_dirty[tile] = 1;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(args.ctr + C_TILES, (unsigned long long)ntl);
}

}  // namespace ebit
