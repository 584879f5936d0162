// ebit_noalloc.cu -- ebit_advect_sweep_noalloc: one split advection sweep that
// allocates no device memory.
//
// Some callers cannot allocate device memory: a flow solver that reserves all of
// its device memory at start-up and forbids allocation afterwards; code that runs
// between a memory-pool snapshot and its restore; a real-time loop where a
// cudaMalloc (which may synchronise the device) is not allowed.  For them this
// file provides a context-free variant of the sweep: the caller passes the old
// state, the velocity and the output buffers, and every intermediate array the
// sweep needs (advected marker coordinates, crossing bins, work lists, counters)
// lives in one file-scope device array of fixed size, below.
//
// The scratch array is part of the library image: every GPU that loads the
// library holds it (about 11.3 MB) until the process exits.  Its device address
// is looked up once per device, on the first call made with that device
// current; that first call should therefore come before any stream capture.
// The address stays valid for the life of the device's primary context: a
// process that resets the device (cudaDeviceReset) must not call this entry
// point afterwards, because the cached address would be stale.
// Every call on a device reuses the same array and leaves its contents there;
// the parts that must start at zero are cleared by each call.  Two calls that
// overlap on the GPU (on different streams without ordering, or from different
// host threads) use the same scratch and race: order them.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/ebit.h"
#include "common.cuh"
#include "sweep.cuh"

using namespace ebit;

namespace {

// largest grid the variant accepts: 64^3 cells.  Axes that are not multiples
// of 8 round their tile count up, so the tile parts are sized for the worst
// grid of at most 64^3 cells with every axis >= 8: 9 x 9 x 3236 cells, 2 x 2 x
// 405 = 1620 tiles of 8^3 (a brute-force search over all such grids).
constexpr long long NA_MAX_CELLS = 64LL * 64 * 64;
constexpr int NA_MAX_TILES = 1620;

// byte offsets inside the scratch array (each part 256-byte aligned)
constexpr long long align256(long long x) { return (x + 255) & ~255LL; }
constexpr long long OFF_ADV = 0;
constexpr long long OFF_BIN = align256(OFF_ADV + 3 * NA_MAX_CELLS * 8);
constexpr long long OFF_WORK = align256(OFF_BIN + 3 * NA_MAX_CELLS);
constexpr long long OFF_LIST = align256(OFF_WORK + 4 * NA_MAX_CELLS * 4);
constexpr long long OFF_INTS = align256(OFF_LIST + NA_MAX_TILES * 4);  // all_count, wcount[4]
constexpr long long OFF_CTR = align256(OFF_INTS + 8 * 4);
constexpr long long OFF_TILES = align256(OFF_CTR + C_TOTAL * 8);       // tile_marker (u32), tile_dirty
constexpr long long NA_BYTES = align256(OFF_TILES + 5 * NA_MAX_TILES);

static __device__ __align__(256) unsigned char g_sweep_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[NA_MAX_DEVICES] = {};

// device address of the scratch array on the current device (looked up once)
int scratch_address(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EBIT_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return EBIT_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sweep_scratch) != cudaSuccess || !p) return EBIT_ECUDA;
        g_scratch_ptr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_ptr[dev];
    return EBIT_OK;
}

// tile list 0 .. n-1 and its length
__global__ void na_tiles_kernel(int *list, int n, int *count) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) list[t] = t;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

// offsets of edges without a marker set to 0, in place
__global__ void na_zero_empty_kernel(Grid g, const uint8_t *__restrict__ cb, double *__restrict__ s) {
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % g.n[0]), y = (int)((t / g.n[0]) % g.n[1]), z = (int)(t / ((long long)g.n[0] * g.n[1]));
        const int c0 = cb[t] & 1;
        const int nb[3] = {lin(g, x + 1, y, z), lin(g, x, y + 1, z), lin(g, x, y, z + 1)};
        for (int a = 0; a < 3; a++)
            if ((cb[nb[a]] & 1) == c0) s[a * N + t] = 0.0;
    }
}

template <int D>
void launch_all(const SweepArgs &a, cudaStream_t st, int grid_tiles, int grid_fp64) {
    advect_kernel<D><<<grid_tiles, 256, 0, st>>>(a);
    sweep_kernel<D><<<grid_tiles, 256, 0, st>>>(a);
    fp64_kernel<D><<<grid_fp64, 128, 0, st>>>(a);
}

}  // namespace

extern "C" int ebit_advect_sweep_noalloc(int nx, int ny, int nz, double h, int dir, const uint8_t *cb_in,
                                         const double *s_in, const double *u_face, double dt, uint8_t *cb_out,
                                         double *s_out, void *cuda_stream) {
    if (nx < 8 || ny < 8 || nz < 8) return EBIT_EINVAL;
    const long long N = (long long)nx * ny * nz;
    if (N > NA_MAX_CELLS) return EBIT_EINVAL;  // the scratch array holds at most 64^3 cells
    if (dir < 0 || dir > 2 || !(h > 0.0) || !std::isfinite(h) || !std::isfinite(dt)) return EBIT_EINVAL;
    if (!cb_in || !s_in || !u_face || !cb_out || !s_out) return EBIT_EINVAL;
    unsigned char *base = nullptr;
    int r = scratch_address(&base);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    Grid g;
    g.n[0] = nx;
    g.n[1] = ny;
    g.n[2] = nz;
    grid_tiles(g, 0);
    if (g.ntiles > NA_MAX_TILES) return EBIT_EINVAL;  // cannot happen within 64^3 cells; kept as a guard

    int *list = (int *)(base + OFF_LIST);
    int *ints = (int *)(base + OFF_INTS);
    unsigned long long *ctr = (unsigned long long *)(base + OFF_CTR);

    // zero what must start at zero: list lengths and counters
    if (cudaMemsetAsync(ints, 0, 8 * sizeof(int), st) != cudaSuccess) return EBIT_ECUDA;
    if (cudaMemsetAsync(ctr, 0, C_TOTAL * sizeof(unsigned long long), st) != cudaSuccess) return EBIT_ECUDA;
    // every tile is processed: the list is 0 .. ntiles-1
    na_tiles_kernel<<<(g.ntiles + 255) / 256, 256, 0, st>>>(list, g.ntiles, ints);

    SweepArgs a;
    a.g = g;
    a.cb = cb_in;
    a.cbo = cb_out;  // every tile is processed, so every colour byte is written
    for (int k = 0; k < 3; k++) {
        a.s[k] = s_in + k * N;
        a.so[k] = s_out + k * N;
        a.adv[k] = (double *)(base + OFF_ADV) + k * N;
        a.bin[k] = (int8_t *)(base + OFF_BIN) + k * N;
    }
    for (int k = 0; k < 4; k++) a.work[k] = (unsigned *)(base + OFF_WORK) + k * N;
    a.u = u_face;
    a.lam = dt / h;
    a.list = list;
    a.count = ints;
    a.wcount = ints + 1;
    a.ctr = ctr;
    a.tile_marker = reinterpret_cast<uint32_t *>(base + OFF_TILES);
    a.tile_dirty = base + OFF_TILES + 4 * NA_MAX_TILES;

    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid_tiles = g.ntiles < sms * 4 ? g.ntiles : sms * 4;
    switch (dir) {
    case 0: launch_all<0>(a, st, grid_tiles, sms * 4); break;
    case 1: launch_all<1>(a, st, grid_tiles, sms * 4); break;
    default: launch_all<2>(a, st, grid_tiles, sms * 4); break;
    }
    // offsets of edges without a marker set to 0
    na_zero_empty_kernel<<<(int)((N + 255) / 256), 256, 0, st>>>(g, cb_out, s_out);
    if (cudaGetLastError() != cudaSuccess) return EBIT_ECUDA;
    return EBIT_OK;
}
