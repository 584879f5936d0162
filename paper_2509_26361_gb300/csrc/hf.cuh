// hf.cuh -- height-function curvature from volume fractions.
//
// The paper computes curvature from the Front2VOF volume fractions with the
// (generalised) height-function method (Sec. 2.6).  This kernel is the standard
// form: for an interface cell (0 < C < 1) the normal n = -grad C is taken from
// the 3x3x3 block with 1-2-1 weights; along the axis of largest |n_d| (ties to
// the lower axis) the heights of a 3x3 stencil of 9-cell columns are summed; a
// column is valid when its end on the reference-phase side is full (C = 1) and
// the other end empty (C = 0).  From the heights eta,
//   kappa h = -sign(n_d) [(1+h_y^2) h_xx + (1+h_x^2) h_yy - 2 h_x h_y h_xy]
//             / (1 + h_x^2 + h_y^2)^(3/2)
// with centred differences; if a column is invalid the next axis by |n| is
// tried, and with none the status is NO_HF (no paraboloid fit).
#pragma once
#include "common.cuh"

namespace ebit {

constexpr int HFH = 4;  // column half-length: 9 cells

struct HFArgs {
    Grid g;
    const double *__restrict__ C;
    double *__restrict__ kh;
    uint8_t *__restrict__ st;
    const int *__restrict__ list;
    const int *__restrict__ count;
    int *__restrict__ iface;        // optional: compacted interface-cell list
    int *__restrict__ iface_count;
};

__device__ __forceinline__ double cval(const HFArgs &a, int x, int y, int z) {
    return __ldg(a.C + lin(a.g, x, y, z));
}

__device__ __noinline__ int hf_cell(const HFArgs &a, int x, int y, int z, double *out) {
    const double w[3] = {1.0, 2.0, 1.0};
    double n[3];
    const int p[3] = {x, y, z};
    for (int d = 0; d < 3; d++) {
        int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        double gsum = 0.0;
        for (int b2 = -1; b2 <= 1; b2++)
            for (int b1 = -1; b1 <= 1; b1++) {
                int qp[3] = {p[0], p[1], p[2]}, qm[3] = {p[0], p[1], p[2]};
                qp[d] += 1;
                qm[d] -= 1;
                qp[t1] += b1;
                qm[t1] += b1;
                qp[t2] += b2;
                qm[t2] += b2;
                gsum += (w[b1 + 1] * w[b2 + 1]) * (cval(a, qp[0], qp[1], qp[2]) - cval(a, qm[0], qm[1], qm[2]));
            }
        n[d] = -gsum;
    }
    int ord[3] = {0, 1, 2};
    for (int i = 1; i < 3; i++)
        for (int j = i; j > 0 && fabs(n[ord[j]]) > fabs(n[ord[j - 1]]); j--) {
            int t = ord[j];
            ord[j] = ord[j - 1];
            ord[j - 1] = t;
        }
    for (int oi = 0; oi < 3; oi++) {
        int d = ord[oi];
        int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        bool below = n[d] > 0.0;
        double eta[3][3];
        bool ok = true;
        for (int b2 = -1; b2 <= 1 && ok; b2++)
            for (int b1 = -1; b1 <= 1 && ok; b1++) {
                double H = 0.0, lo = 0.0, hi = 0.0;
                for (int m = -HFH; m <= HFH; m++) {
                    int q[3] = {p[0], p[1], p[2]};
                    q[d] += m;
                    q[t1] += b1;
                    q[t2] += b2;
                    double cv = cval(a, q[0], q[1], q[2]);
                    H += cv;
                    if (m == -HFH) lo = cv;
                    if (m == HFH) hi = cv;
                }
                if (below ? !(lo == 1.0 && hi == 0.0) : !(lo == 0.0 && hi == 1.0)) ok = false;
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
        *out = below ? -kap : kap;
        return 1 + d;
    }
    *out = 0.0;
    return 4;
}

__global__ void __launch_bounds__(256) hf_kernel(HFArgs a) {
    const int ntl = *a.count;
    for (int li = blockIdx.x; li < ntl; li += gridDim.x) {
        const int tile = a.list[li];
        int o[3];
        tile_origin(a.g, tile, o);
        for (int c = threadIdx.x; c < TILE_CELLS; c += blockDim.x) {
            int x = o[0] + (c & 7), y = o[1] + ((c >> 3) & 7), z = o[2] + (c >> 6);
            if (x >= a.g.n[0] || y >= a.g.n[1] || z >= a.g.n[2]) continue;
            int id = lin(a.g, x, y, z);
            double c0 = __ldg(a.C + id);
            double k = 0.0;
            int st = 0;
            if (c0 > 0.0 && c0 < 1.0) {
                st = hf_cell(a, x, y, z, &k);
                if (a.iface) {
                    int slot = atomicAdd(a.iface_count, 1);
                    a.iface[slot] = id;
                }
            }
            a.kh[id] = k;
            a.st[id] = (uint8_t)st;
        }
    }
}

}  // namespace ebit
