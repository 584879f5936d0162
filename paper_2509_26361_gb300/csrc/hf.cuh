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
    const unsigned *__restrict__ prev;  // interface cells of the previous call
    const int *__restrict__ nprev;
    const unsigned *__restrict__ cand;  // candidate cells (all interface cells are among them)
    const int *__restrict__ ncand;
    unsigned *__restrict__ iface;       // interface cells of this call (output list, may be null)
    int *__restrict__ niface;
    int *zero[2];                       // counters of later launches to clear (may be null)
    const int *__restrict__ list;       // tiles, for the full scan
    const int *__restrict__ count;
};

// 0 < C < 1 on the bit pattern (C is never negative; -0 and NaN fail as in IEEE)
__device__ __forceinline__ bool is_interface(double c) {
    long long b = __double_as_longlong(c);
    return b > 0 && b < 0x3FF0000000000000ll;
}

// C at offset (dx, dy, dz) from the cell; WRAP = false uses direct strides (the
// cell is at least HFH+1 cells from every periodic seam)
template <bool WRAP>
struct CAccess {
    const double *__restrict__ C;
    Grid g;
    int x, y, z, id, sy, sz;
    __device__ __forceinline__ double operator()(int dx, int dy, int dz) const {
        if (WRAP) return __ldg(C + lin(g, x + dx, y + dy, z + dz));
        return __ldg(C + id + dx + dy * sy + dz * sz);
    }
};

// heights along axis d on the 3x3 stencil of 9-cell columns; returns false when
// a column's ends are not pure with the reference phase on the expected side.
// The axis is a run-time value so that lanes of a warp with different
// dominant axes share one instruction stream.
template <bool WRAP>
__device__ __forceinline__ bool hf_axis(const CAccess<WRAP> &c, int d, bool below, double *out) {
    const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    int ed[3] = {0, 0, 0}, e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0};
    ed[d] = 1;
    e1[t1] = 1;
    e2[t2] = 1;
    double eta[3][3];
    bool ok = true;
#pragma unroll 1
    for (int b2 = -1; b2 <= 1; b2++)
#pragma unroll
        for (int b1 = -1; b1 <= 1; b1++) {
            const int ox = b1 * e1[0] + b2 * e2[0], oy = b1 * e1[1] + b2 * e2[1], oz = b1 * e1[2] + b2 * e2[2];
            double H = 0.0;
            unsigned long long lo = 0ull, hi = 0ull;
#pragma unroll
            for (int m = -HFH; m <= HFH; m++) {
                double cv = c(ox + m * ed[0], oy + m * ed[1], oz + m * ed[2]);
                H += cv;
                if (m == -HFH) lo = (unsigned long long)__double_as_longlong(cv);
                if (m == HFH) hi = (unsigned long long)__double_as_longlong(cv);
            }
            // pure ends on the bit patterns: == 1.0 is one pattern, == 0.0 two (+0, -0)
            const bool lo1 = lo == 0x3FF0000000000000ull, lo0 = (lo << 1) == 0ull;
            const bool hi1 = hi == 0x3FF0000000000000ull, hi0 = (hi << 1) == 0ull;
            ok = ok && (below ? (lo1 && hi0) : (lo0 && hi1));
            eta[b1 + 1][b2 + 1] = below ? H - (HFH + 0.5) : (HFH + 0.5) - H;
        }
    if (!ok) return false;
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
    return true;
}

// The float at or below c for c in [+0, 1], from the bit pattern (values
// under 2^-126 give 0): an error below one float ulp, at most 2^-24.
__device__ __forceinline__ float trunc_unit_float(double c) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(c);
    const int e = (int)(b >> 52);
    const unsigned f = ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFull);
    return e < 1023 - 126 ? 0.0f : __uint_as_float(f);
}

template <bool WRAP>
__device__ int hf_cell_impl(const CAccess<WRAP> &c, double *out) {
    // the 3x3x3 block once; Youngs sums in the order (b2 outer, b1 inner)
    double blk[3][3][3];
#pragma unroll
    for (int dz = -1; dz <= 1; dz++)
#pragma unroll
        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
            for (int dx = -1; dx <= 1; dx++) blk[dz + 1][dy + 1][dx + 1] = c(dx, dy, dz);
    // The normal decides only the axis order and the side of the reference
    // phase.  A float normal decides them when every |n_d| and every gap
    // between two |n_d| clears the float rounding bound CANON_EPS with margin
    // (then the FP64 sums, within 2e-14 of the exact ones, order and sign them
    // the same); otherwise the FP64 sums below, in the oracle's order.
    // (the bound holds for values in [+0, 1], checked on the bit patterns).
    // The floats are the doubles truncated by integer operations, not rounded
    // by conversion instructions: an input error below 2^-24 instead of 2^-25,
    // which raises the bound from 1.7e-5 to 1.8e-5, still under CANON_EPS.
    float fv[27];
    bool unit = true;
#pragma unroll
    for (int dz = 0; dz < 3; dz++)
#pragma unroll
        for (int dy = 0; dy < 3; dy++)
#pragma unroll
            for (int dx = 0; dx < 3; dx++) {
                unit = unit && (unsigned long long)__double_as_longlong(blk[dz][dy][dx]) <= 0x3FF0000000000000ull;
                fv[dz * 9 + dy * 3 + dx] = trunc_unit_float(blk[dz][dy][dx]);
            }
    float nf[3];
    youngs<float>(fv, nf);
    const float f0 = fabsf(nf[0]), f1 = fabsf(nf[1]), f2 = fabsf(nf[2]);
    if (unit && f0 > CANON_EPS && f1 > CANON_EPS && f2 > CANON_EPS && fabsf(f0 - f1) > 2.0f * CANON_EPS &&
        fabsf(f0 - f2) > 2.0f * CANON_EPS && fabsf(f1 - f2) > 2.0f * CANON_EPS) {
        int o0 = 0, o1 = 1, o2 = 2, tmp;
        const float fa[3] = {f0, f1, f2};
        if (fa[o1] > fa[o0]) { tmp = o0; o0 = o1; o1 = tmp; }
        if (fa[o2] > fa[o1]) {
            tmp = o1; o1 = o2; o2 = tmp;
            if (fa[o1] > fa[o0]) { tmp = o0; o0 = o1; o1 = tmp; }
        }
        const int ord[3] = {o0, o1, o2};
        for (int oi = 0; oi < 3; oi++) {
            const int d = ord[oi];
            if (hf_axis<WRAP>(c, d, nf[d] > 0.0f, out)) return 1 + d;
        }
        *out = 0.0;
        return 4;
    }
    const double w[3] = {1.0, 2.0, 1.0};
    double n[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        double gsum = 0.0;
#pragma unroll
        for (int b2 = -1; b2 <= 1; b2++)
#pragma unroll
            for (int b1 = -1; b1 <= 1; b1++) {
                int op[3] = {0, 0, 0}, om[3] = {0, 0, 0};
                op[d] = 1;
                om[d] = -1;
                op[t1] += b1;
                om[t1] += b1;
                op[t2] += b2;
                om[t2] += b2;
                gsum += (w[b1 + 1] * w[b2 + 1]) *
                        (blk[op[2] + 1][op[1] + 1][op[0] + 1] - blk[om[2] + 1][om[1] + 1][om[0] + 1]);
            }
        n[d] = -gsum;
    }
    int o0 = 0, o1 = 1, o2 = 2, tmp;
    if (fabs(n[o1]) > fabs(n[o0])) { tmp = o0; o0 = o1; o1 = tmp; }
    if (fabs(n[o2]) > fabs(n[o1])) {
        tmp = o1; o1 = o2; o2 = tmp;
        if (fabs(n[o1]) > fabs(n[o0])) { tmp = o0; o0 = o1; o1 = tmp; }
    }
    const int ord[3] = {o0, o1, o2};
    for (int oi = 0; oi < 3; oi++) {
        const int d = ord[oi];
        const bool below = n[d] > 0.0;
        if (hf_axis<WRAP>(c, d, below, out)) return 1 + d;
    }
    *out = 0.0;
    return 4;
}

__device__ __noinline__ int hf_cell(const HFArgs &a, int x, int y, int z, double *out) {
    const int R = HFH + 1;
    const int id = lin(a.g, x, y, z);
    const int sy = a.g.n[0], sz = a.g.n[0] * a.g.n[1];
    if (x >= R && x < a.g.n[0] - R && y >= R && y < a.g.n[1] - R && z >= R && z < a.g.n[2] - R) {
        CAccess<false> c{a.C, a.g, x, y, z, id, sy, sz};
        return hf_cell_impl<false>(c, out);
    }
    CAccess<true> c{a.C, a.g, x, y, z, id, sy, sz};
    return hf_cell_impl<true>(c, out);
}

// Interface-cell pass: entries [0, nprev) reset the previous interface cells
// that are no longer cut (their curvature becomes 0, status NONE); entries of
// the candidate list are computed if 0 < C < 1 and reset otherwise.  Every
// interface cell of the current C is a candidate, so the curvature field is
// complete; one thread per entry, full warps for the FP64 work.  Without
// COMPUTE the interface cells are only listed (the learned curvature writes
// them next).
// 4 blocks of 128 per SM: with the outer column loop kept rolled the kernel
// fits 127 registers without spilling, where the fully unrolled one took 226
// (2 blocks per SM) to keep all 81 column loads in flight
template <bool COMPUTE>
__global__ void __launch_bounds__(128, 4) hf_list_kernel(HFArgs a) {
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (a.zero[0]) *a.zero[0] = 0;
        if (a.zero[1]) *a.zero[1] = 0;
    }
    const int np = *a.nprev, nc = *a.ncand;
    const int total = np + nc;
    const int stride = gridDim.x * blockDim.x;
    const int iters = (total + stride - 1) / stride;
    for (int it = 0; it < iters; it++) {
        const int t = list_item(it);
        bool keep = false;
        int id = 0;
        if (t < total) {
            id = (int)(t < np ? a.prev[t] : a.cand[t - np]);
            bool iface = is_interface(__ldg(a.C + id));
            if (t < np) {
                if (!iface) {
                    a.kh[id] = 0.0;
                    a.st[id] = 0;
                }
            } else if (iface) {
                if (COMPUTE) {
                    const int x = id % a.g.n[0], y = (id / a.g.n[0]) % a.g.n[1], z = id / (a.g.n[0] * a.g.n[1]);
                    double kv = 0.0;
                    int st = hf_cell(a, x, y, z, &kv);
                    a.kh[id] = kv;
                    a.st[id] = (uint8_t)st;
                }
                keep = true;
            } else {
                a.kh[id] = 0.0;
                a.st[id] = 0;
            }
        }
        const unsigned full = 0xffffffffu;
        unsigned m = __ballot_sync(full, keep);
        if (m && a.iface) {
            const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(a.niface, __popc(m));
            base = __shfl_sync(full, base, leader);
            if (keep) a.iface[base + __popc(m & ((1u << lane) - 1u))] = (unsigned)id;
        }
    }
}

// Full scan of the listed tiles (any C): non-interface cells are reset, the
// interface cells are appended to the candidate list for hf_list_kernel.
__global__ void __launch_bounds__(256) hf_scan_kernel(HFArgs a, unsigned *cand, int *ncand) {
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
            bool iface = false;
            int id = 0;
            if (x < a.g.n[0] && y < a.g.n[1] && z < a.g.n[2]) {
                id = lin(a.g, x, y, z);
                iface = is_interface(__ldg(a.C + id));
                if (!iface) {
                    a.kh[id] = 0.0;
                    a.st[id] = 0;
                }
            }
            const unsigned full = 0xffffffffu;
            unsigned m = __ballot_sync(full, iface);
            if (m) {
                const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(ncand, __popc(m));
                base = __shfl_sync(full, base, leader);
                if (iface) cand[base + __popc(m & ((1u << lane) - 1u))] = (unsigned)id;
            }
        }
    }
}

}  // namespace ebit
