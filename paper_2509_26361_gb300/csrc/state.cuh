// state.cuh -- marker initialisation, state read-back and the active band.
#pragma once
#include "common.cuh"

namespace ebit {

// Marker initialisation (Sec. 3.1): colour = (phi >= 0); on every edge whose end
// colours differ, the marker sits at the linear-interpolation root of phi (or at
// a caller-given offset); saddle faces take the sign of phi at the face centre
// (the mean of the four corners when no face values are given); every other
// face stores its lowest corner's colour.
__global__ void init_kernel(Grid g, const double *__restrict__ phi, const double *__restrict__ phif,
                            const double *__restrict__ sx, uint8_t *__restrict__ cb,
                            double *__restrict__ s0, double *__restrict__ s1, double *__restrict__ s2) {
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    double *sp[3] = {s0, s1, s2};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        int x = (int)(t % g.n[0]);
        int y = (int)((t / g.n[0]) % g.n[1]);
        int z = (int)(t / ((long long)g.n[0] * g.n[1]));
        const int p[3] = {x, y, z};
        const int id = (int)t;
        const double f0 = phi[id];
        const int c0 = f0 >= 0.0;
        int byte = c0;
        for (int a = 0; a < 3; a++) {
            int q[3] = {p[0], p[1], p[2]};
            q[a] += 1;
            int iq = lin3(g, q);
            double f1 = phi[iq];
            int c1 = f1 >= 0.0;
            double v = 0.0;
            if (c0 != c1) {
                double ex = sx ? sx[(long long)a * N + id] : (double)NAN;
                if (ex == ex) v = ex;
                else v = f0 / (f0 - f1);
                if (v < 0.0) v = 0.0;
                if (v > ONE_MINUS) v = ONE_MINUS;
            }
            sp[a][id] = v;
            // face normal to a: corners p, p+e1, p+e2, p+e1+e2 (e1 < e2)
            int e1 = (a == 0) ? 1 : 0, e2 = (a == 2) ? 1 : 2;
            int r1[3] = {p[0], p[1], p[2]}, r2[3] = {p[0], p[1], p[2]}, r3[3] = {p[0], p[1], p[2]};
            r1[e1] += 1;
            r2[e2] += 1;
            r3[e1] += 1;
            r3[e2] += 1;
            int i1 = lin3(g, r1), i2 = lin3(g, r2), i3 = lin3(g, r3);
            int k1 = phi[i1] >= 0.0, k2 = phi[i2] >= 0.0, k3 = phi[i3] >= 0.0;
            int bit = c0;
            if (c0 == k3 && k1 == k2 && c0 != k1) {
                double fc = phif ? phif[(long long)a * N + id]
                                 : 0.25 * ((f0 + phi[i1]) + (phi[i2] + phi[i3]));
                bit = fc >= 0.0;
            }
            byte |= bit << (1 + a);
        }
        cb[id] = (uint8_t)byte;
    }
}

// Read back the offsets with 0 on edges that carry no marker.
__global__ void canonical_s_kernel(Grid g, const uint8_t *__restrict__ cb, const double *__restrict__ s0,
                                   const double *__restrict__ s1, const double *__restrict__ s2,
                                   double *__restrict__ out) {
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const double *sp[3] = {s0, s1, s2};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        int x = (int)(t % g.n[0]);
        int y = (int)((t / g.n[0]) % g.n[1]);
        int z = (int)(t / ((long long)g.n[0] * g.n[1]));
        int c0 = cb[t] & 1;
        int nb[3] = {lin(g, x + 1, y, z), lin(g, x, y + 1, z), lin(g, x, y, z + 1)};
        for (int a = 0; a < 3; a++) out[a * N + t] = ((cb[nb[a]] & 1) != c0) ? sp[a][t] : 0.0;
    }
}

// List of the flagged tiles (no dilation), clearing the flags; zero0 and
// zero1 (may be null) are counters of later launches, cleared as in
// band_kernel.
__global__ void take_flagged_kernel(Grid g, uint8_t *__restrict__ flag, int *__restrict__ list, int *__restrict__ count,
                                    int *zero0, int *zero1) {
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (zero0) *zero0 = 0;
        if (zero1) *zero1 = 0;
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ntiles; t += gridDim.x * blockDim.x) {
        if (flag[t]) {
            flag[t] = 0;
            int slot = atomicAdd(count, 1);
            list[slot] = t;
        }
    }
}

__global__ void iota_kernel(int *list, int n, int *count) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) list[t] = t;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

}  // namespace ebit
