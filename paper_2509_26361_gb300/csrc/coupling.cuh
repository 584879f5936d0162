// coupling.cuh -- the one-fluid coupling terms of the EBIT interface
// (arxiv 2509.26361, Sec. 2.5: Eq. 6 and the surface-tension term).
//
// Eq. 6 with the Heaviside function of the reference phase taken as the
// Front2VOF fraction C: rho = C rho1 + (1 - C) rho2, mu = C mu1 + (1 - C) mu2,
// per cell.  Surface tension as a well-balanced continuum surface force on the
// faces of the MAC grid: on the a-face between cells idx - e_a and idx,
//     f_a = sigma kappa_f (C[idx] - C[idx - e_a]) / h,
// kappa = kappa_h / h on cells whose curvature is valid (height functions
// along x, y or z, or the network), kappa_f the mean of the two cells' values,
// the one valid value, or 0.  One pass over the grid, x fastest: every array
// is read and written once, coalesced; the neighbour values come through L1/L2.
#pragma once
#include "common.cuh"

namespace ebit {

struct CouplingArgs {
    Grid g;
    const double *__restrict__ C;
    const double *__restrict__ kh;
    const uint8_t *__restrict__ st;
    double sigma, rho1, rho2, mu1, mu2, h;
    double *__restrict__ rho;  // may be null
    double *__restrict__ mu;   // may be null
    double *__restrict__ f[3]; // null: no force
};

__device__ __forceinline__ bool curv_valid(uint8_t s) { return s == 1 || s == 2 || s == 3 || s == 5; }

// One block per grid row (y, z) at a time, x across the threads: coalesced
// rows, and the cell coordinates without 64-bit divisions.  The FP64 pipe is
// narrow, so pure cells (C = 0 or 1, bit patterns) take the end values of
// Eq. 6 by selection -- the same values the formula gives there -- and faces
// compare the bit patterns of C; the arithmetic runs at interface cells only.
__global__ void __launch_bounds__(256) coupling_kernel(CouplingArgs a) {
    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const long long nxy = (long long)nx * ny;
    // unaliased copies: the loads of later cells may move ahead of the stores
    const long long *__restrict__ Cb = reinterpret_cast<const long long *>(a.C);
    const double *__restrict__ khp = a.kh;
    const uint8_t *__restrict__ stp = a.st;
    double *__restrict__ rhop = a.rho;
    double *__restrict__ mup = a.mu;
    double *__restrict__ f0 = a.f[0];
    double *__restrict__ f1 = a.f[1];
    double *__restrict__ f2 = a.f[2];
    const double sigma = a.sigma, h = a.h, rho1 = a.rho1, rho2 = a.rho2, mu1 = a.mu1, mu2 = a.mu2;
    for (int row = blockIdx.x; row < ny * nz; row += gridDim.x) {
        const int z = row / ny, y = row - z * ny;
        const long long base = (long long)row * nx;
        // the same row one step back along y and along z (periodic)
        const long long by = base - (long long)y * nx + (long long)(y == 0 ? ny - 1 : y - 1) * nx;
        const long long bz = base - (long long)z * nxy + (long long)(z == 0 ? nz - 1 : z - 1) * nxy;
#pragma unroll 2
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long idx = base + x;
            const long long cbits = __ldg(Cb + idx);
            const double c = __longlong_as_double(cbits);
            const bool c0 = cbits == 0, c1 = cbits == 0x3FF0000000000000LL;
            if (rhop) rhop[idx] = c0 ? rho2 : (c1 ? rho1 : c * rho1 + (1.0 - c) * rho2);
            if (mup) mup[idx] = c0 ? mu2 : (c1 ? mu1 : c * mu1 + (1.0 - c) * mu2);
            if (!f0) continue;
            const long long n0 = base + (x == 0 ? nx - 1 : x - 1), n1 = by + x, n2 = bz + x;
            const long long b0 = __ldg(Cb + n0), b1 = __ldg(Cb + n1), b2 = __ldg(Cb + n2);
            double fd[3] = {0.0, 0.0, 0.0};
            if (b0 != cbits || b1 != cbits || b2 != cbits) {
                const bool ok = curv_valid(__ldg(stp + idx));
                const double k = ok ? __ldg(khp + idx) / h : 0.0;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const long long j = d == 0 ? n0 : (d == 1 ? n1 : n2);
                    const long long nb = d == 0 ? b0 : (d == 1 ? b1 : b2);
                    if (nb == cbits) continue;
                    const bool okn = curv_valid(__ldg(stp + j));
                    const double kn = okn ? __ldg(khp + j) / h : 0.0;
                    const double kf = (ok && okn) ? 0.5 * (k + kn) : (ok ? k : (okn ? kn : 0.0));
                    fd[d] = sigma * kf * (c - __longlong_as_double(nb)) / h;
                }
            }
            f0[idx] = fd[0];
            f1[idx] = fd[1];
            f2[idx] = fd[2];
        }
    }
}

}  // namespace ebit
