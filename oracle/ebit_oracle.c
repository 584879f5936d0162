/*
 * ebit_oracle.c -- plain, slow CPU FP64 oracle for the 3D EBIT kinematics path
 * (arxiv 2509.26361).  TEST INFRASTRUCTURE ONLY: only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load this file.  The product
 * path never links it and shares no code with it.
 *
 * Compile with -ffp-contract=off: every product and sum below is a separate
 * IEEE double operation in the order written, so that decisions taken in
 * floating point (node crossings, saddle face colours, root choice) are
 * reproducible.
 *
 * What it computes (paper passages):
 *   oracle_init        -- marker initialisation from a level set: colour = (phi>=0),
 *                         marker at the linear-interpolation root of a sign-change
 *                         edge (Sec. 3.1, translation test set-up).
 *   oracle_sweep       -- one split 1D advection along axis d (Sec. 2.1 Eqs. 1-2,
 *                         Fig. 1; circle fit with the radius-ratio rule, Fig. 2;
 *                         colour vertex update and topology change, Sec. 2.2,
 *                         Figs. 4-5; 3D decomposition onto the two face families
 *                         containing d, Sec. 2.3, Fig. 6).
 *   oracle_front2vof   -- per-cell loops from the face-wise connectivity, centroid
 *                         fan (Eq. 7), exact volume by Gauss's theorem (Sec. 2.6).
 *   oracle_hf          -- height-function curvature from volume fractions
 *                         (Sec. 2.6 cites the generalised HF method; the standard
 *                         fixed 9-cell column form is used, no paraboloid fallback).
 *   oracle_surface_volume -- enclosed volume of the global fan-triangulated
 *                         surface with a single global origin (volume pin).
 *   oracle_circle_root -- the circle-fit root alone (unit pin).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   marker offset s in [0, 1-) of the edge from its lower node; colour 1 = the
 *   reference phase; a marker at X is left of node m iff X < m; an edge carries a
 *   marker iff its end colours differ, and if three markers land on one edge the
 *   median is kept; circle fit P1-P2-P3 / P2-P3-P4 around the crossing segment
 *   P2->P3, root on the target edge nearest the straight-line crossing, ratio
 *   rule r_max > 10 r_min;
 *   face-centre colour = phase of the advected polyline at the face centre,
 *   stored only for saddle faces (4 markers) -- every other face stores the colour
 *   of its lowest corner; velocity by trilinear interpolation of the MAC
 *   component; periodic grid, at least 8 cells per axis; CFL < 1.
 *
 * The paper fixes no value for the face-centre colour rule (phase of the
 * advected polyline at the face centre); the tests pin it by invariants:
 * equivariance under reflections of the grid, independence of the path along
 * which the phase is counted, and the colours of a surface moved by a uniform
 * velocity.
 *
 * Layout (shared with the product only as a documented format): node/cell index
 * idx = (k*ny + j)*nx + i.  Colour byte cb[idx]: bit0 = node colour, bit(1+a) =
 * colour of the face normal to axis a whose lowest corner is node idx.
 * s[a*N + idx] = marker offset on the a-edge from node idx (0 when absent).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>



#define HFH 4 /* height-function column half-length: columns of 2*HFH+1 cells */
#define ONE_MINUS 0.99999999999999988898 /* nextafter(1.0, 0.0) = 1 - 2^-53 */

/* counters (same order as the product's ebit_counters_t) */
enum {
    CNT_MARKERS = 0,      /* edges carrying a marker after the sweep          */
    CNT_ANNIHILATE = 1,   /* edges where an even (>=2) number of markers met    */
    CNT_MULTI = 2,        /* edges where three markers met (median kept)        */
    CNT_INCONSISTENT = 3, /* colour/crossing parity disagreement (never expected)*/
    CNT_CFL = 4,          /* markers whose displacement reached one cell        */
    CNT_N = 5
};

typedef struct {
    int n[3];
    long N;
} grid_t;

static int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

static long nid(const grid_t *g, const int p[3]) {
    int i = wrapi(p[0], g->n[0]), j = wrapi(p[1], g->n[1]), k = wrapi(p[2], g->n[2]);
    return ((long)k * g->n[1] + j) * g->n[0] + i;
}

/* offset in (-n/2, n/2] of a periodic index difference */
static int wrapd(int dlt, int n) {
    int r = wrapi(dlt, n);
    if (2 * r > n) r -= n;
    return r;
}

static void padd(int out[3], const int p[3], int a, int da) {
    out[0] = p[0];
    out[1] = p[1];
    out[2] = p[2];
    out[a] += da;
}

static int vcol(const uint8_t *cb, long id) { return cb[id] & 1; }
static int fcol(const uint8_t *cb, long id, int a) { return (cb[id] >> (1 + a)) & 1; }

/* Face normal to a at node p is a saddle iff its 4 corner colours alternate. */
static int face_is_saddle(const grid_t *g, const uint8_t *cb, const int p[3], int a) {
    int e1 = (a == 0) ? 1 : 0, e2 = (a == 2) ? 1 : 2;
    int q[3], r[3], t[3];
    padd(q, p, e1, 1);
    padd(r, p, e2, 1);
    padd(t, q, e2, 1);
    int c00 = vcol(cb, nid(g, p)), c10 = vcol(cb, nid(g, q)), c01 = vcol(cb, nid(g, r)),
        c11 = vcol(cb, nid(g, t));
    return c00 == c11 && c10 == c01 && c00 != c10;
}

/* ---------------------------------------------------------------- init (Sec. 3.1) */
void oracle_init(int nx, int ny, int nz, const double *phi, const double *phi_face,
                 const double *s_exact, uint8_t *cb, double *s) {
    grid_t g = {{nx, ny, nz}, (long)nx * ny * nz};
    for (long id = 0; id < g.N; id++) cb[id] = (phi[id] >= 0.0) ? 1 : 0;
    for (int a = 0; a < 3; a++)
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int p[3] = {i, j, k}, q[3];
                    padd(q, p, a, 1);
                    long id = nid(&g, p), iq = nid(&g, q);
                    double v = 0.0;
                    if ((cb[id] & 1) != (cb[iq] & 1)) {
                        /* linear interpolation root of phi along the edge, or a
                         * caller-given exact offset when one is supplied */
                        double ex = s_exact ? s_exact[(long)a * g.N + id] : NAN;
                        if (ex == ex) v = ex;
                        else v = phi[id] / (phi[id] - phi[iq]);
                        if (v < 0.0) v = 0.0;
                        if (v > ONE_MINUS) v = ONE_MINUS;
                    }
                    s[(long)a * g.N + id] = v;
                }
    for (int a = 0; a < 3; a++) {
        int e1 = (a == 0) ? 1 : 0, e2 = (a == 2) ? 1 : 2;
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int p[3] = {i, j, k};
                    long id = nid(&g, p);
                    int bit;
                    if (face_is_saddle(&g, cb, p, a)) {
                        double fc;
                        if (phi_face) {
                            fc = phi_face[(long)a * g.N + id];
                        } else {
                            int q[3], r[3], t[3];
                            padd(q, p, e1, 1);
                            padd(r, p, e2, 1);
                            padd(t, q, e2, 1);
                            fc = 0.25 * ((phi[id] + phi[nid(&g, q)]) + (phi[nid(&g, r)] + phi[nid(&g, t)]));
                        }
                        bit = fc >= 0.0;
                    } else {
                        bit = cb[id] & 1;
                    }
                    cb[id] = (uint8_t)(cb[id] | (bit << (1 + a)));
                }
    }
}

/* ------------------------------------------------ velocity at a marker (Eq. 2) */
/* u_d is sampled at the centres of the d-normal faces: node + 1/2 along the two
 * axes other than d.  The point is node p shifted by s along axis e (e < 0: the
 * node itself).  Trilinear interpolation, lerps in the order x, y, z. */
static double interp_u(const grid_t *g, const double *u, int d, const int p[3], int e, double s) {
    int base[3];
    double t[3];
    for (int b = 0; b < 3; b++) {
        if (b == d) {
            base[b] = p[b];
            t[b] = (b == e) ? s : 0.0;
        } else if (b != e) {
            base[b] = p[b] - 1;
            t[b] = 0.5;
        } else if (s < 0.5) {
            base[b] = p[b] - 1;
            t[b] = s + 0.5;
        } else {
            base[b] = p[b];
            t[b] = s - 0.5;
        }
    }
    double v[2][2][2];
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                int q[3] = {base[0] + dx, base[1] + dy, base[2] + dz};
                v[dz][dy][dx] = u[nid(g, q)];
            }
    double c00 = (1.0 - t[0]) * v[0][0][0] + t[0] * v[0][0][1];
    double c10 = (1.0 - t[0]) * v[0][1][0] + t[0] * v[0][1][1];
    double c01 = (1.0 - t[0]) * v[1][0][0] + t[0] * v[1][0][1];
    double c11 = (1.0 - t[0]) * v[1][1][0] + t[0] * v[1][1][1];
    double c0 = (1.0 - t[1]) * c00 + t[1] * c10;
    double c1 = (1.0 - t[1]) * c01 + t[1] * c11;
    return (1.0 - t[2]) * c0 + t[2] * c1;
}

/* -------------------------------------------------------- circle fit (Fig. 2) */
typedef struct {
    double x, y;
} pt2;

/* Circle through A, B, C intersected with the line x = x0.  Only roots on the
 * target edge (0 <= y <= 1) count; of those the one nearest ylin is taken.
 * Returns 1 and (root, radius) if valid; 0 if the points are collinear or no
 * root lies on the edge. */
static int circle_root(pt2 A, pt2 B, pt2 C, double x0, double ylin, double *root, double *rad) {
    double bx = B.x - A.x, by = B.y - A.y;
    double cx = C.x - A.x, cy = C.y - A.y;
    double b2 = bx * bx + by * by;
    double c2 = cx * cx + cy * cy;
    double det = 2.0 * (bx * cy - by * cx);
    if (fabs(det) <= 1e-12 * (b2 + c2)) return 0;
    double ux = (cy * b2 - by * c2) / det;
    double uy = (bx * c2 - cx * b2) / det;
    double r2 = ux * ux + uy * uy;
    double dx = x0 - (A.x + ux);
    double disc = r2 - dx * dx;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double yc = A.y + uy;
    double yp = yc + sq, ym = yc - sq;
    int okp = (yp >= 0.0 && yp <= 1.0), okm = (ym >= 0.0 && ym <= 1.0);
    if (!okp && !okm) return 0;
    if (okp && okm) *root = (fabs(yp - ylin) <= fabs(ym - ylin)) ? yp : ym;
    else *root = okp ? yp : ym;
    *rad = sqrt(r2);
    return 1;
}

/* Combination of the two circle fits (ratio rule, threshold 10). */
static double circle_fit(int va, double ya, double ra, int vb, double yb, double rb, double ylin) {
    if (va && vb) {
        double rmax = ra > rb ? ra : rb, rmin = ra > rb ? rb : ra;
        if (rmax > 10.0 * rmin) return ra > rb ? ya : yb;
        return 0.5 * (ya + yb);
    }
    if (va) return ya;
    if (vb) return yb;
    return ylin;
}

/* exported for the unit pin: P1..P4 as (x,y) pairs, grid line x = 0 */
double oracle_circle_root(const double *P, double ylin, int *which) {
    pt2 p1 = {P[0], P[1]}, p2 = {P[2], P[3]}, p3 = {P[4], P[5]}, p4 = {P[6], P[7]};
    double ya = 0, ra = 0, yb = 0, rb = 0;
    int va = circle_root(p1, p2, p3, 0.0, ylin, &ya, &ra);
    int vb = circle_root(p2, p3, p4, 0.0, ylin, &yb, &rb);
    if (which) *which = va + 2 * vb;
    return circle_fit(va, ya, ra, vb, yb, rb, ylin);
}

/* ------------------------------------- 2D cell connectivity (Sec. 2.2, Fig. 3) */
/* A 2D cell in a plane spanned by axes (a, t): corners c00 (lowest), c10 (+a),
 * c01 (+t), c11.  Edges: B = a-edge at c00, R = t-edge at c10, T = a-edge at
 * c01, L = t-edge at c00.  Markers sit on edges whose end colours differ.  With
 * 4 markers (saddle) the corners whose colour equals the face colour are joined
 * through the centre and the two other corners are cut off. */
enum { EB = 0, ER = 1, ET = 2, EL = 3 };

static int cell_segments(int c00, int c10, int c01, int c11, int phif, int seg[2][2]) {
    int m[4] = {c00 != c10, c10 != c11, c01 != c11, c00 != c01};
    int nm = m[0] + m[1] + m[2] + m[3];
    if (nm == 0) return 0;
    if (nm == 2) {
        int k = 0;
        for (int e = 0; e < 4; e++)
            if (m[e]) seg[0][k++] = e;
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
    return -1;
}

/* ----------------------------------------------------------- one split sweep */
/* Per-plane marker graph.  Marker ids: type 0 = a-edge, type 1 = t-edge, at
 * plane-local node (pa, pt): id = (type*Nt + pt)*Na + pa. */
typedef struct {
    int Na, Nt;
    int *nb;     /* 2 neighbour ids per marker, -1 when unset */
    double *adv; /* advected a-coordinate relative to the marker's node (a-edges:
                    s + c; t-edges: c) */
    double *sv;  /* offset along the edge (old state) */
    uint8_t *has;
} plane_t;

static long pmid(const plane_t *P, int type, int pa, int pt) {
    pa = wrapi(pa, P->Na);
    pt = wrapi(pt, P->Nt);
    return ((long)type * P->Nt + pt) * P->Na + pa;
}

static void pm_decode(const plane_t *P, long id, int *type, int *pa, int *pt) {
    *pa = (int)(id % P->Na);
    long r = id / P->Na;
    *pt = (int)(r % P->Nt);
    *type = (int)(r / P->Nt);
}

/* advected local position of marker id relative to plane node (m, q) */
static pt2 pm_pos(const plane_t *P, long id, int m, int q) {
    int type, pa, pt;
    pm_decode(P, id, &type, &pa, &pt);
    int da = wrapd(pa - m, P->Na), dt = wrapd(pt - q, P->Nt);
    pt2 r;
    if (type == 0) {
        r.x = (double)da + P->adv[id];
        r.y = (double)dt;
    } else {
        r.x = (double)da + P->adv[id];
        r.y = (double)dt + P->sv[id];
    }
    return r;
}

/* marker id of the cell edge e of the 2D cell at plane node (pa, pt) */
static long cell_edge_id(const plane_t *P, int pa, int pt, int e) {
    switch (e) {
    case EB: return pmid(P, 0, pa, pt);
    case ET: return pmid(P, 0, pa, pt + 1);
    case EL: return pmid(P, 1, pa, pt);
    default: return pmid(P, 1, pa + 1, pt);
    }
}

typedef struct {
    int d, a, t, n, r; /* sweep axis, plane axes, plane normal, plane index */
} planeinfo_t;

static void plane_node(const planeinfo_t *pi, int pa, int pt, int p[3]) {
    p[pi->a] = pa;
    p[pi->t] = pt;
    p[pi->n] = pi->r;
}

static int cell_segs_old(const grid_t *g, const planeinfo_t *pi, const uint8_t *cb, int pa, int pt,
                         int seg[2][2]) {
    int p00[3], p10[3], p01[3], p11[3];
    plane_node(pi, pa, pt, p00);
    plane_node(pi, pa + 1, pt, p10);
    plane_node(pi, pa, pt + 1, p01);
    plane_node(pi, pa + 1, pt + 1, p11);
    long i00 = nid(g, p00);
    return cell_segments(vcol(cb, i00), vcol(cb, nid(g, p10)), vcol(cb, nid(g, p01)),
                         vcol(cb, nid(g, p11)), fcol(cb, i00, pi->n), seg);
}

typedef struct {
    pt2 p2, p3;
    long id2, id3;
    double ylin;
} crossing_t;

void oracle_sweep(int nx, int ny, int nz, int d, const double *u, double lam, const uint8_t *cb,
                  const double *s, uint8_t *cb2, double *s2, long long *cnt) {
    grid_t g = {{nx, ny, nz}, (long)nx * ny * nz};
    const long N = g.N;
    long long c[CNT_N] = {0};

    /* (1) aligned markers on every d-edge: X = s + u dt/h, relative to the node */
    double *X = (double *)malloc(sizeof(double) * N);
    uint8_t *hasd = (uint8_t *)malloc(N);
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int p[3] = {i, j, k}, q[3];
                padd(q, p, d, 1);
                long id = nid(&g, p);
                hasd[id] = vcol(cb, id) != vcol(cb, nid(&g, q));
                X[id] = 0.0;
                if (hasd[id]) {
                    double sv = s[(long)d * N + id];
                    double cf = interp_u(&g, u, d, p, d, sv) * lam;
                    if (!(fabs(cf) < 1.0)) {
                        c[CNT_CFL]++;
                        cf = cf > 0.0 ? ONE_MINUS : -ONE_MINUS;
                    }
                    X[id] = sv + cf;
                }
            }

    /* (2) node colours: a node flips once per marker that crosses it (Fig. 4) */
    uint8_t *col = (uint8_t *)malloc(N);
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int p[3] = {i, j, k}, q[3];
                padd(q, p, d, -1);
                long id = nid(&g, p), iq = nid(&g, q);
                int v = vcol(cb, id);
                if (hasd[iq] && X[iq] >= 1.0) v ^= 1; /* from the left edge   */
                if (hasd[id] && X[id] < 0.0) v ^= 1;  /* from the right edge  */
                col[id] = (uint8_t)v;
            }

    /* start the output: colours, all offsets zero */
    for (long id = 0; id < N; id++) cb2[id] = col[id];
    for (long id = 0; id < 3 * N; id++) s2[id] = 0.0;

    /* (3) aligned edges: presence from the colours; landing markers (Fig. 5) */
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int p[3] = {i, j, k}, q[3];
                padd(q, p, d, 1);
                long id = nid(&g, p);
                int present = col[id] != col[nid(&g, q)];
                double land[3];
                int nl = 0;
                for (int e = -1; e <= 1; e++) {
                    int r[3];
                    padd(r, p, d, e);
                    long ir = nid(&g, r);
                    if (!hasd[ir]) continue;
                    double x = X[ir];
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
                        /* median of three */
                        double a0 = land[0], a1 = land[1], a2 = land[2], tmp;
                        if (a0 > a1) { tmp = a0; a0 = a1; a1 = tmp; }
                        if (a1 > a2) { tmp = a1; a1 = a2; a2 = tmp; }
                        if (a0 > a1) { tmp = a0; a0 = a1; a1 = tmp; }
                        v = a1;
                        c[CNT_MULTI]++;
                    } else {
                        v = 0.5;
                        c[CNT_INCONSISTENT]++;
                    }
                    s2[(long)d * N + id] = v;
                    c[CNT_MARKERS]++;
                } else if (nl >= 2) {
                    c[CNT_ANNIHILATE]++;
                }
            }

    /* (4) the two face families containing d: 2D EBIT per plane (Fig. 6) */
    for (int f = 1; f <= 2; f++) {
        planeinfo_t pi;
        pi.d = d;
        pi.a = d;
        pi.t = (d + f) % 3;
        pi.n = (d + 3 - f) % 3;
        plane_t P;
        P.Na = g.n[pi.a];
        P.Nt = g.n[pi.t];
        long M = 2L * P.Na * P.Nt;
        P.nb = (int *)malloc(sizeof(int) * 2 * M);
        P.adv = (double *)malloc(sizeof(double) * M);
        P.sv = (double *)malloc(sizeof(double) * M);
        P.has = (uint8_t *)malloc(M);
        for (int r = 0; r < g.n[pi.n]; r++) {
            pi.r = r;
            /* markers of this plane with their advected a-coordinates */
            for (long id = 0; id < M; id++) {
                P.nb[2 * id] = P.nb[2 * id + 1] = -1;
                P.has[id] = 0;
                P.adv[id] = 0.0;
                P.sv[id] = 0.0;
            }
            for (int pt = 0; pt < P.Nt; pt++)
                for (int pa = 0; pa < P.Na; pa++) {
                    int p[3];
                    plane_node(&pi, pa, pt, p);
                    long gid = nid(&g, p);
                    long ida = pmid(&P, 0, pa, pt), idt = pmid(&P, 1, pa, pt);
                    P.has[ida] = hasd[gid];
                    P.adv[ida] = X[gid];
                    P.sv[ida] = s[(long)pi.a * N + gid];
                    int q[3];
                    padd(q, p, pi.t, 1);
                    if (vcol(cb, gid) != vcol(cb, nid(&g, q))) {
                        double sv = s[(long)pi.t * N + gid];
                        double cf = interp_u(&g, u, d, p, pi.t, sv) * lam;
                        if (!(fabs(cf) < 1.0)) {
                            c[CNT_CFL]++;
                            cf = cf > 0.0 ? ONE_MINUS : -ONE_MINUS;
                        }
                        P.has[idt] = 1;
                        P.adv[idt] = cf;
                        P.sv[idt] = sv;
                    }
                }
            /* connectivity graph from the old colours */
            for (int pt = 0; pt < P.Nt; pt++)
                for (int pa = 0; pa < P.Na; pa++) {
                    int seg[2][2];
                    int ns = cell_segs_old(&g, &pi, cb, pa, pt, seg);
                    if (ns < 0) {
                        c[CNT_INCONSISTENT]++;
                        continue;
                    }
                    for (int sgi = 0; sgi < ns; sgi++) {
                        long e0 = cell_edge_id(&P, pa, pt, seg[sgi][0]);
                        long e1 = cell_edge_id(&P, pa, pt, seg[sgi][1]);
                        int k0 = P.nb[2 * e0] < 0 ? 0 : 1;
                        int k1 = P.nb[2 * e1] < 0 ? 0 : 1;
                        P.nb[2 * e0 + k0] = (int)e1;
                        P.nb[2 * e1 + k1] = (int)e0;
                    }
                }
            /* unaligned t-edges of the plane: crossings of the advected polyline
             * with the grid line, circle fit (Fig. 1c, Fig. 2) */
            for (int q = 0; q < P.Nt; q++)
                for (int m = 0; m < P.Na; m++) {
                    int p[3], pq[3];
                    plane_node(&pi, m, q, p);
                    padd(pq, p, pi.t, 1);
                    long gid = nid(&g, p);
                    int present = col[gid] != col[nid(&g, pq)];
                    crossing_t cr[8];
                    int ncr = 0;
                    for (int dl = -2; dl <= 1; dl++) {
                        int seg[2][2];
                        int ns = cell_segs_old(&g, &pi, cb, m + dl, q, seg);
                        for (int sgi = 0; sgi < ns; sgi++) {
                            long e0 = cell_edge_id(&P, m + dl, q, seg[sgi][0]);
                            long e1 = cell_edge_id(&P, m + dl, q, seg[sgi][1]);
                            pt2 A = pm_pos(&P, e0, m, q), B = pm_pos(&P, e1, m, q);
                            if ((A.x < 0.0) == (B.x < 0.0)) continue;
                            crossing_t x;
                            if (A.x < 0.0) {
                                x.p2 = A; x.id2 = e0; x.p3 = B; x.id3 = e1;
                            } else {
                                x.p2 = B; x.id2 = e1; x.p3 = A; x.id3 = e0;
                            }
                            double tt = (0.0 - x.p2.x) / (x.p3.x - x.p2.x);
                            x.ylin = x.p2.y + tt * (x.p3.y - x.p2.y);
                            if (ncr < 8) cr[ncr++] = x;
                        }
                    }
                    if (!present) {
                        if (ncr >= 2) c[CNT_ANNIHILATE]++;
                        continue;
                    }
                    c[CNT_MARKERS]++;
                    if ((ncr & 1) == 0) {
                        c[CNT_INCONSISTENT]++;
                        s2[(long)pi.t * N + gid] = 0.5;
                        continue;
                    }
                    int sel = 0;
                    if (ncr >= 3) {
                        /* median crossing by ylin; equal values keep list order */
                        int ord[8];
                        for (int a2 = 0; a2 < ncr; a2++) ord[a2] = a2;
                        for (int a2 = 1; a2 < ncr; a2++)
                            for (int b2 = a2; b2 > 0 && cr[ord[b2 - 1]].ylin > cr[ord[b2]].ylin; b2--) {
                                int tmp = ord[b2];
                                ord[b2] = ord[b2 - 1];
                                ord[b2 - 1] = tmp;
                            }
                        sel = ord[ncr / 2];
                        c[CNT_MULTI]++;
                    }
                    crossing_t x = cr[sel];
                    /* neighbours along the polyline: P1 of P2 (not P3), P4 of P3 (not P2) */
                    long n2a = P.nb[2 * x.id2], n2b = P.nb[2 * x.id2 + 1];
                    long n3a = P.nb[2 * x.id3], n3b = P.nb[2 * x.id3 + 1];
                    long id1 = (n2a == x.id3) ? n2b : n2a;
                    long id4 = (n3a == x.id2) ? n3b : n3a;
                    double ya = 0, ra = 0, yb = 0, rb = 0;
                    int va = 0, vb = 0;
                    if (id1 >= 0 && id1 != x.id3) {
                        pt2 P1 = pm_pos(&P, id1, m, q);
                        va = circle_root(P1, x.p2, x.p3, 0.0, x.ylin, &ya, &ra);
                    } else {
                        c[CNT_INCONSISTENT]++;
                    }
                    if (id4 >= 0 && id4 != x.id2) {
                        pt2 P4 = pm_pos(&P, id4, m, q);
                        vb = circle_root(x.p2, x.p3, P4, 0.0, x.ylin, &yb, &rb);
                    } else {
                        c[CNT_INCONSISTENT]++;
                    }
                    double y = circle_fit(va, ya, ra, vb, yb, rb, x.ylin);
                    if (y < 0.0) y = 0.0;
                    if (y > ONE_MINUS) y = ONE_MINUS;
                    s2[(long)pi.t * N + gid] = y;
                }
            /* face-centre colours of this family (n-normal faces): the phase of
             * the advected polyline at the face centre, for saddle faces only */
            for (int q = 0; q < P.Nt; q++)
                for (int m = 0; m < P.Na; m++) {
                    int p[3];
                    plane_node(&pi, m, q, p);
                    long gid = nid(&g, p);
                    int bit;
                    if (!face_is_saddle(&g, col, p, pi.n)) {
                        bit = col[gid] & 1;
                    } else {
                        int par = col[gid] & 1;
                        /* along the a-line of node (m, q) from x = 0 to x = 1/2 */
                        for (int dl = -2; dl <= 2; dl++) {
                            long ida = pmid(&P, 0, m + dl, q);
                            if (!P.has[ida]) continue;
                            double x = (double)dl + P.adv[ida];
                            if (x >= 0.0 && x < 0.5) par ^= 1;
                        }
                        /* up the line x = 1/2 from y = 0 to y = 1/2 */
                        for (int dl = -2; dl <= 2; dl++) {
                            int seg[2][2];
                            int ns = cell_segs_old(&g, &pi, cb, m + dl, q, seg);
                            for (int sgi = 0; sgi < ns; sgi++) {
                                long e0 = cell_edge_id(&P, m + dl, q, seg[sgi][0]);
                                long e1 = cell_edge_id(&P, m + dl, q, seg[sgi][1]);
                                pt2 A = pm_pos(&P, e0, m, q), B = pm_pos(&P, e1, m, q);
                                if ((A.x < 0.5) == (B.x < 0.5)) continue;
                                pt2 L = (A.x < 0.5) ? A : B, Rr = (A.x < 0.5) ? B : A;
                                double tt = (0.5 - L.x) / (Rr.x - L.x);
                                double yl = L.y + tt * (Rr.y - L.y);
                                if (yl < 0.5) par ^= 1;
                            }
                        }
                        bit = par;
                    }
                    cb2[gid] = (uint8_t)(cb2[gid] | (bit << (1 + pi.n)));
                }
        }
        free(P.nb);
        free(P.adv);
        free(P.sv);
        free(P.has);
    }
    /* (5) the d-normal family is not swept: its face colour is kept on saddle
     * faces and reset to the lowest-corner colour elsewhere */
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int p[3] = {i, j, k};
                long gid = nid(&g, p);
                int bit = face_is_saddle(&g, col, p, d) ? fcol(cb, gid, d) : (col[gid] & 1);
                cb2[gid] = (uint8_t)(cb2[gid] | (bit << (1 + d)));
            }
    /* markers on the two unaligned families already counted; aligned counted */
    for (int i = 0; i < CNT_N; i++) cnt[i] += c[i];
    free(X);
    free(hasd);
    free(col);
}

/* ------------------------------------------------------ Front2VOF (Sec. 2.6) */
/* Cube faces with corners in counter-clockwise order seen from outside.
 * Corner id = dx | dy<<1 | dz<<2.  Face id: 0 x=0, 1 x=1, 2 y=0, 3 y=1, 4 z=0, 5 z=1. */
static const int FACE_CORNERS[6][4] = {
    {0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};

/* cube edge id between two corners: x-edges 0-3 (dy + 2dz), y-edges 4-7
 * (dx + 2dz), z-edges 8-11 (dx + 2dy) */
static int cube_edge(int u, int v) {
    int lo = u < v ? u : v, diff = u ^ v;
    int dx = lo & 1, dy = (lo >> 1) & 1, dz = (lo >> 2) & 1;
    if (diff == 1) return dy + 2 * dz;
    if (diff == 2) return 4 + dx + 2 * dz;
    return 8 + dx + 2 * dy;
}

typedef struct {
    double x[3];
} pt3;

static pt3 corner_pos(int cid) {
    pt3 r = {{(double)(cid & 1), (double)((cid >> 1) & 1), (double)((cid >> 2) & 1)}};
    return r;
}

/* area of a planar polygon on a cube face, projected on the face axes (u, v) */
static double poly_area(const pt3 *pts, int np, int u, int v) {
    double acc = 0.0;
    for (int i = 0; i < np; i++) {
        const pt3 *a = &pts[i], *b = &pts[(i + 1) % np];
        acc += a->x[u] * b->x[v] - b->x[u] * a->x[v];
    }
    return 0.5 * fabs(acc);
}

static double det3(const pt3 *c, const pt3 *p, const pt3 *q) {
    return c->x[0] * (p->x[1] * q->x[2] - p->x[2] * q->x[1]) +
           c->x[1] * (p->x[2] * q->x[0] - p->x[0] * q->x[2]) +
           c->x[2] * (p->x[0] * q->x[1] - p->x[1] * q->x[0]);
}

/* Per-cell reconstruction.  Returns the cell's volume fraction, and (optionally)
 * the loops: loop_len[l], loop_pts (cell-local).  Sets *bad on inconsistency. */
static double cell_volume(const int K[8], const int F[6], const double E[12], int *nloops,
                          int loop_len[6], pt3 loop_pts[6][12], int *bad) {
    pt3 mk[12];
    int has[12];
    for (int e = 0; e < 12; e++) {
        has[e] = 0;
        int ax = e / 4, r = e % 4;
        pt3 p;
        if (ax == 0) { p.x[0] = E[e]; p.x[1] = (double)(r & 1); p.x[2] = (double)(r >> 1); }
        else if (ax == 1) { p.x[0] = (double)(r & 1); p.x[1] = E[e]; p.x[2] = (double)(r >> 1); }
        else { p.x[0] = (double)(r & 1); p.x[1] = (double)(r >> 1); p.x[2] = E[e]; }
        mk[e] = p;
    }
    int out[12];
    for (int e = 0; e < 12; e++) out[e] = -1;
    double A1[3] = {0.0, 0.0, 0.0};
    int nmk = 0;
    for (int f = 0; f < 6; f++) {
        int kc[4], col[4], ed[4], mm[4], nm = 0;
        for (int k = 0; k < 4; k++) {
            kc[k] = FACE_CORNERS[f][k];
            col[k] = K[kc[k]];
        }
        for (int k = 0; k < 4; k++) {
            ed[k] = cube_edge(kc[k], kc[(k + 1) & 3]);
            mm[k] = col[k] != col[(k + 1) & 3];
            nm += mm[k];
            if (mm[k]) has[ed[k]] = 1;
        }
        /* the face's phase-1 area is needed on the faces x=1, y=1, z=1 */
        int upper = f & 1, fa = f >> 1;
        int u = (fa + 1) % 3, v = (fa + 2) % 3;
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
            int arc_col = col[(ea + 1) & 3];
            if (arc_col) out[ed[eb]] = ed[ea];
            else out[ed[ea]] = ed[eb];
            if (upper) {
                pt3 poly[6];
                int np = 0;
                poly[np++] = mk[ed[ea]];
                for (int k = ea + 1; k <= eb; k++) poly[np++] = corner_pos(kc[k]);
                poly[np++] = mk[ed[eb]];
                double R = poly_area(poly, np, u, v);
                area1 = arc_col ? R : 1.0 - R;
            }
        } else if (nm == 4) {
            int phif = F[f];
            double T = 0.0;
            for (int mc = 0; mc < 4; mc++) {
                if (col[mc] == phif) continue;
                int eprev = ed[(mc + 3) & 3], enext = ed[mc];
                if (col[mc]) out[enext] = eprev;
                else out[eprev] = enext;
                if (upper) {
                    pt3 tri[3] = {mk[eprev], corner_pos(kc[mc]), mk[enext]};
                    T += poly_area(tri, 3, u, v);
                }
            }
            area1 = (1 - phif) ? T : 1.0 - T;
        } else {
            *bad = 1;
        }
        if (upper) A1[fa] = area1;
    }
    for (int e = 0; e < 12; e++) nmk += has[e];
    *nloops = 0;
    if (nmk == 0) return (double)K[0];
    int vis[12] = {0};
    double acc = 0.0;
    for (int e0 = 0; e0 < 12; e0++) {
        if (!has[e0] || vis[e0]) continue;
        int len = 0, e = e0;
        pt3 lp[12];
        while (len < 12) {
            if (e < 0 || !has[e] || vis[e]) break;
            vis[e] = 1;
            lp[len++] = mk[e];
            e = out[e];
            if (e == e0) break;
        }
        if (e != e0) {
            *bad = 1;
            continue;
        }
        /* centroid of the loop's markers (Eq. 7), then the fan of triangles */
        pt3 cen;
        for (int a = 0; a < 3; a++) {
            double sm = 0.0;
            for (int i = 0; i < len; i++) sm += lp[i].x[a];
            cen.x[a] = sm / (double)len;
        }
        for (int i = 0; i < len; i++) acc += det3(&cen, &lp[i], &lp[(i + 1) % len]);
        if (*nloops < 6) {
            loop_len[*nloops] = len;
            for (int i = 0; i < len; i++) loop_pts[*nloops][i] = lp[i];
            (*nloops)++;
        }
    }
    double V = ((A1[0] + A1[1]) + A1[2]) / 3.0 - acc / 6.0;
    if (V < 0.0) V = 0.0;
    if (V > 1.0) V = 1.0;
    return V;
}

static void gather_cell(const grid_t *g, const uint8_t *cb, const double *s, int i, int j, int k,
                        int K[8], int F[6], double E[12]) {
    for (int cid = 0; cid < 8; cid++) {
        int p[3] = {i + (cid & 1), j + ((cid >> 1) & 1), k + ((cid >> 2) & 1)};
        K[cid] = vcol(cb, nid(g, p));
    }
    int p0[3] = {i, j, k};
    for (int a = 0; a < 3; a++) {
        int q[3];
        padd(q, p0, a, 1);
        F[2 * a] = fcol(cb, nid(g, p0), a);
        F[2 * a + 1] = fcol(cb, nid(g, q), a);
    }
    for (int r = 0; r < 4; r++) {
        int dy = r & 1, dz = r >> 1;
        int px[3] = {i, j + dy, k + dz};
        E[r] = s[0 * g->N + nid(g, px)];
        int py[3] = {i + (r & 1), j, k + (r >> 1)};
        E[4 + r] = s[1 * g->N + nid(g, py)];
        int pz[3] = {i + (r & 1), j + (r >> 1), k};
        E[8 + r] = s[2 * g->N + nid(g, pz)];
    }
}

long oracle_front2vof(int nx, int ny, int nz, const uint8_t *cb, const double *s, double *C) {
    grid_t g = {{nx, ny, nz}, (long)nx * ny * nz};
    long nbad = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int K[8], F[6];
                double E[12];
                gather_cell(&g, cb, s, i, j, k, K, F, E);
                int nl, ll[6], bad = 0;
                pt3 lp[6][12];
                int p[3] = {i, j, k};
                C[nid(&g, p)] = cell_volume(K, F, E, &nl, ll, lp, &bad);
                nbad += bad;
            }
    return nbad;
}

/* single-cube entry for the exhaustive pins: K[8] corner colours, F[6] face
 * colours, E[12] edge offsets; returns C and the number of loops */
double oracle_cube_volume(const int *K, const int *F, const double *E, int *nloops, int *bad) {
    int ll[6];
    pt3 lp[6][12];
    *bad = 0;
    return cell_volume(K, F, E, nloops, ll, lp, bad);
}

/* Enclosed volume of the union of all fan triangles, computed with one global
 * origin (cell coordinates unwrapped: the surface must not cross the periodic
 * boundary).  Also returns the number of triangles.  Used by the volume pin. */
double oracle_surface_volume(int nx, int ny, int nz, const uint8_t *cb, const double *s, long *ntri) {
    grid_t g = {{nx, ny, nz}, (long)nx * ny * nz};
    double acc = 0.0;
    long nt = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int K[8], F[6];
                double E[12];
                gather_cell(&g, cb, s, i, j, k, K, F, E);
                int nl, ll[6], bad = 0;
                pt3 lp[6][12];
                cell_volume(K, F, E, &nl, ll, lp, &bad);
                for (int l = 0; l < nl; l++) {
                    pt3 cen;
                    for (int a = 0; a < 3; a++) {
                        double sm = 0.0;
                        for (int q = 0; q < ll[l]; q++) sm += lp[l][q].x[a];
                        cen.x[a] = sm / (double)ll[l];
                    }
                    pt3 gc, ga, gb;
                    for (int q = 0; q < ll[l]; q++) {
                        const pt3 *pa = &lp[l][q], *pb = &lp[l][(q + 1) % ll[l]];
                        int o[3] = {i, j, k};
                        for (int a = 0; a < 3; a++) {
                            gc.x[a] = (double)o[a] + cen.x[a];
                            ga.x[a] = (double)o[a] + pa->x[a];
                            gb.x[a] = (double)o[a] + pb->x[a];
                        }
                        acc += det3(&gc, &ga, &gb);
                        nt++;
                    }
                }
            }
    if (ntri) *ntri = nt;
    return -acc / 6.0;
}

/* --------------------------------------------- height-function curvature */
/* Columns of 9 cells (4 on each side of the cell) on a 3x3 stencil of columns.
 * Status: 0 not an interface cell, 1+d curvature from heights along axis d,
 * 4 no consistent height-function stencil (kappa*h set to 0). */
void oracle_hf(int nx, int ny, int nz, const double *C, double *kh, uint8_t *st) {
    grid_t g = {{nx, ny, nz}, (long)nx * ny * nz};
    static const double w[3] = {1.0, 2.0, 1.0};
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int p[3] = {i, j, k};
                long id = nid(&g, p);
                double c0 = C[id];
                kh[id] = 0.0;
                st[id] = 0;
                if (!(c0 > 0.0 && c0 < 1.0)) continue;
                /* Youngs normal n = -grad C with 1-2-1 weights on the two
                 * transverse axes (lower axis inner) */
                double n[3];
                for (int dax = 0; dax < 3; dax++) {
                    int t1 = (dax == 0) ? 1 : 0, t2 = (dax == 2) ? 1 : 2;
                    double gsum = 0.0;
                    for (int b2 = -1; b2 <= 1; b2++)
                        for (int b1 = -1; b1 <= 1; b1++) {
                            int qp[3] = {i, j, k}, qm[3] = {i, j, k};
                            qp[dax] += 1;
                            qm[dax] -= 1;
                            qp[t1] += b1;
                            qm[t1] += b1;
                            qp[t2] += b2;
                            qm[t2] += b2;
                            gsum += (w[b1 + 1] * w[b2 + 1]) * (C[nid(&g, qp)] - C[nid(&g, qm)]);
                        }
                    n[dax] = -gsum;
                }
                /* axes by decreasing |n|, ties to the lower axis */
                int ord[3] = {0, 1, 2};
                for (int a2 = 1; a2 < 3; a2++)
                    for (int b2 = a2; b2 > 0 && fabs(n[ord[b2]]) > fabs(n[ord[b2 - 1]]); b2--) {
                        int tmp = ord[b2];
                        ord[b2] = ord[b2 - 1];
                        ord[b2 - 1] = tmp;
                    }
                st[id] = 4;
                for (int oi = 0; oi < 3; oi++) {
                    int dax = ord[oi];
                    int t1 = (dax == 0) ? 1 : 0, t2 = (dax == 2) ? 1 : 2;
                    int below = n[dax] > 0.0; /* phase 1 on the lower side */
                    double eta[3][3];
                    int ok = 1;
                    for (int b2 = -1; b2 <= 1 && ok; b2++)
                        for (int b1 = -1; b1 <= 1 && ok; b1++) {
                            double H = 0.0, lo = 0.0, hi = 0.0;
                            for (int mm = -HFH; mm <= HFH; mm++) {
                                int q[3] = {i, j, k};
                                q[dax] += mm;
                                q[t1] += b1;
                                q[t2] += b2;
                                double cv = C[nid(&g, q)];
                                H += cv;
                                if (mm == -HFH) lo = cv;
                                if (mm == HFH) hi = cv;
                            }
                            if (below ? !(lo == 1.0 && hi == 0.0) : !(lo == 0.0 && hi == 1.0)) ok = 0;
                            eta[b1 + 1][b2 + 1] = below ? H - (HFH + 0.5) : (HFH + 0.5) - H;
                        }
                    if (!ok) continue;
                    double hx = (eta[2][1] - eta[0][1]) * 0.5;
                    double hy = (eta[1][2] - eta[1][0]) * 0.5;
                    double hxx = (eta[2][1] + eta[0][1]) - 2.0 * eta[1][1];
                    double hyy = (eta[1][2] + eta[1][0]) - 2.0 * eta[1][1];
                    double hxy = ((eta[2][2] - eta[2][0]) - (eta[0][2] - eta[0][0])) * 0.25;
                    double num = (1.0 + hy * hy) * hxx + (1.0 + hx * hx) * hyy - 2.0 * hx * hy * hxy;
                    double q2 = 1.0 + hx * hx + hy * hy;
                    double den = q2 * sqrt(q2);
                    double kap = num / den;
                    kh[id] = below ? -kap : kap;
                    st[id] = (uint8_t)(1 + dax);
                    break;
                }
            }
}
