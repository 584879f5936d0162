// ebit_batch.cu -- many independent EBIT instances advanced by one launch per
// split sweep (declared in include/ebit.h).
//
// Each instance is a periodic grid of its own size with its own velocity and
// time step; the method is the same as for one context (Sec. 2.1-2.3: split
// marker advection, colour-vertex update, unaligned reconstruction by circle
// fits).  The batch owns one arena of per-sweep state for all instances (two
// colour/offset buffers, advection scratch, FP64 work lists, tile flags,
// counters); every instance also has a context that views its slice of the
// arena, so Front2VOF, curvature, state access and counters work per instance
// through the ordinary entry points' code.
//
// A sweep is one cooperative launch that runs four phases over all instances,
// separated by a grid barrier:
//   band    -- every (instance, tile) whose 3x3x3 tile neighbourhood held a
//              marker is listed; the FP64 list lengths are cleared;
//   advect  -- per listed tile: each marker moved once (velocity interpolated);
//   sweep   -- per listed tile: integer colour/aligned-edge pass, FP64 lists;
//   fp64    -- the FP64 lists of all instances as one index space.
// Data written in one phase and read in a later one is loaded through L2 (not
// the read-only path).  The barrier waits a bounded number of polls; on
// timeout it sets an error flag, every block leaves, and ebit_batch_sync
// reports EBIT_ETIMEOUT.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ebit.h"
#include "common.cuh"
#include "ctx.h"
#include "sweep.cuh"
#include "tc.cuh"

namespace ebit {

constexpr int BATCH_MAX = 1024;      // instances per batch (tile ids keep 20 bits)
constexpr int BATCH_THREADS = 256;
constexpr long long BAR_POLLS = 1LL << 24;  // polls of 64 ns sleep: about a second

struct BatchInst {
    SweepArgs a;  // u, lam, list and count are unused (per-sweep arrays below)
};

struct BatchParams {
    const BatchInst *inst;    // [n], for the current buffer parity
    int n;
    int total_tiles;
    const int *toff;          // [n + 1] first global tile of each instance
    const double *const *u;   // [n] velocity component of the sweep direction
    const double *lam;        // [n] dt / h
    int *band;                // (instance << 20) | tile
    int *nband;
    int *wcount;              // [4 n] FP64 list lengths (all instances)
    unsigned *bar;            // [2] arrivals, generation
    int *err;
};

// Grid-wide barrier of a cooperative launch (all blocks co-resident); gives up
// after max_polls polls, sets the error flag and returns false.
__device__ bool grid_barrier(const BatchParams &p, int *s_ok, long long max_polls = BAR_POLLS) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = p.bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(p.bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(p.bar, 0u);
            __threadfence();
            atomicAdd(p.bar + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g0) {
                if (++it > max_polls) {
                    atomicExch(p.err, 1);
                    ok = 0;
                    break;
                }
                if (it > 64) __nanosleep(64);
            }
        }
        __threadfence();
        if (*(volatile int *)p.err) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ int find_inst(const int *toff, int n, int gt) {
    int lo = 0, hi = n;  // toff[lo] <= gt < toff[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(toff + mid) <= gt) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int D, int SH>
__global__ void __launch_bounds__(BATCH_THREADS, 4) batch_sweep_kernel(BatchParams p) {
    __shared__ uint16_t s_mk[3 * TILE_CELLS];
    __shared__ uint8_t s_c[adv_stage_max()];
    __shared__ uint8_t s_b[stage_n(D, SH)];
    __shared__ int8_t s_bn[stage_n(D, SH)];
    __shared__ int s_n, s_ok;
    __shared__ unsigned s_flag;
    __shared__ int s_pre[4 * BATCH_MAX + 1];
    __shared__ int s_wsum[BATCH_THREADS / 32];
    if (*(volatile int *)p.err) return;
    const int stride = gridDim.x * blockDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;

    // ---- band: tiles near a marker, all instances
    for (int k = gtid; k < 4 * p.n; k += stride) p.wcount[k] = 0;
    {
        const int iters = (p.total_tiles + stride - 1) / stride;
        for (int it = 0; it < iters; it++) {
            const int gt = it * stride + gtid;
            bool on = false;
            int i = 0, t = 0;
            if (gt < p.total_tiles) {
                i = find_inst(p.toff, p.n, gt);
                t = gt - __ldg(p.toff + i);
                const Grid g = p.inst[i].a.g;
                const int tx = t % g.td[0], ty = (t / g.td[0]) % g.td[1], tz = t / (g.td[0] * g.td[1]);
                on = in_band(g, p.inst[i].a.tile_marker, tx, ty, tz);
            }
            const int slot = warp_append(p.nband, on);
            if (slot >= 0) p.band[slot] = (i << 20) | t;
        }
    }
    if (!grid_barrier(p, &s_ok)) return;
    const int nb = __ldcg(p.nband);

    // ---- advect
    for (int li = blockIdx.x; li < nb; li += gridDim.x) {
        const int e = __ldcg(p.band + li);
        const int i = e >> 20;
        advect_tile<D, SH>(p.inst[i].a, p.u[i], p.lam[i], e & 0xFFFFF, s_mk, s_c, &s_n);
    }
    if (!grid_barrier(p, &s_ok)) return;

    // ---- integer band pass
    for (int li = blockIdx.x; li < nb; li += gridDim.x) {
        const int e = __ldcg(p.band + li);
        const int i = e >> 20;
        const SweepArgs &a = p.inst[i].a;
        sweep_tile<D, true, 4, SH>(a, e & 0xFFFFF, s_b, s_bn, &s_flag);
        if (threadIdx.x == 0) atomicAdd(a.ctr + C_TILES, 1ull);
    }
    if (!grid_barrier(p, &s_ok)) return;

    // ---- FP64 lists of every instance as one index space: block-wide prefix
    // sums of the 4 n list lengths
    {
        const int m = 4 * p.n;
        const int per = (m + blockDim.x - 1) / blockDim.x;
        int loc[4 * BATCH_MAX / BATCH_THREADS];
        int sum = 0;
        for (int q = 0; q < per; q++) {
            const int j = threadIdx.x * per + q;
            loc[q] = j < m ? __ldcg(p.wcount + j) : 0;
            sum += loc[q];
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int inc = sum;
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += v;
        }
        if (lane == 31) s_wsum[wid] = inc;
        __syncthreads();
        int base = 0;
        for (int w = 0; w < wid; w++) base += s_wsum[w];
        int run = base + inc - sum;
        for (int q = 0; q < per; q++) {
            const int j = threadIdx.x * per + q;
            if (j < m) s_pre[j] = run;
            run += loc[q];
        }
        if (threadIdx.x == blockDim.x - 1) s_pre[m] = run;
        __syncthreads();
        // marker counts of the unaligned lists (one per entry)
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i < p.n; i += blockDim.x) {
                const int nm = (s_pre[4 * i + 2] - s_pre[4 * i]);
                if (nm) atomicAdd(p.inst[i].a.ctr + C_MARKERS, (unsigned long long)nm);
            }
        const int total = s_pre[m];
        for (int t = gtid; t < total; t += stride) {
            int lo = 0, hi = m;  // s_pre[lo] <= t < s_pre[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_pre[mid] <= t) lo = mid;
                else hi = mid;
            }
            const int i = lo >> 2, kind = lo & 3;
            unsigned ev[C_N] = {0, 0, 0, 0, 0};
            fp64_item<D, true>(p.inst[i].a, kind, t - s_pre[lo], ev);
#pragma unroll
            for (int k = 0; k < C_N; k++)
                if (k != C_MARKERS && ev[k]) atomicAdd(p.inst[i].a.ctr + k, (unsigned long long)ev[k]);
        }
    }
}

// Self-tests of the bounded waits.  Each makes one wait either succeed or wait
// for an event that never comes, with a short poll limit, and records whether
// it returned true; nothing faults and nothing hangs.
//
// Two blocks meet at the grid barrier; with `absent` set, block 1 leaves
// without arriving, so block 0 waits for a generation that never comes.
__global__ void selftest_barrier_kernel(BatchParams p, int absent, long long polls, int *ok_out) {
    __shared__ int s_ok;
    if (absent && blockIdx.x == 1) return;
    const bool ok = grid_barrier(p, &s_ok, polls);
    if (blockIdx.x == 0 && threadIdx.x == 0) *ok_out = ok ? 1 : 0;
}

// An mbarrier expecting one arrival; with `arrive` clear nobody arrives, so
// the wait on its first phase never succeeds.
__global__ void selftest_mbarrier_kernel(int arrive, long long polls, int *ok_out) {
    __shared__ __align__(8) uint64_t mbar;
    const uint32_t mb = tc::smem_u32(&mbar);
    if (threadIdx.x == 0) {
        tc::mbar_init(mb, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
        *ok_out = tc::mbar_wait(mb, 0, polls) ? 1 : 0;
    }
}

}  // namespace ebit

using namespace ebit;

struct ebit_batch {
    DevMem mem;  // the allocator the batch was created with
    int n = 0;
    cudaStream_t stream = nullptr;
    int sms = 1;
    std::vector<ebit_ctx *> inst;
    std::vector<long long> coff;   // first cell of each instance in the arena
    std::vector<int> toff;         // first tile (current tile shape)
    std::vector<int> dims;         // nx, ny, nz of each instance
    std::vector<BatchInst> htab[2];  // host copy of the launch tables
    long long cells = 0;
    int tiles = 0;
    int parity = 0;                // buffer holding the current state
    // arena
    uint8_t *cb[2] = {nullptr, nullptr};
    double *s[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    double *adv[3] = {nullptr, nullptr, nullptr};
    int8_t *bin[3] = {nullptr, nullptr, nullptr};
    unsigned *work[4] = {nullptr, nullptr, nullptr, nullptr};
    int *wcount = nullptr;
    uint32_t *tile_marker = nullptr;
    uint8_t *tile_dirty = nullptr;
    unsigned long long *ctr = nullptr;
    // launch data
    BatchInst *table[2] = {nullptr, nullptr};
    int *d_toff = nullptr;
    double **u[3] = {nullptr, nullptr, nullptr};
    double *lam = nullptr;
    int *band = nullptr, *nband = nullptr;
    unsigned *bar = nullptr;
    int *err = nullptr;
    int have_u[3] = {0, 0, 0};
    int have_dt = 0;
    int occ[N_TILE_SHAPES][3] = {};  // co-resident blocks per SM of each shape's and direction's kernel
    int ctas_per_sm = 1;           // chosen launch shape (autotuned)
    int shape = 0;                 // tile shape (autotuned)
    int tiles_cap = 0;             // tiles the tile tables hold (the largest total over the shapes)
    // CUDA graph of two steps (even: x y z, odd: z y x)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_ok = 0;
    int graph_parity = 0;          // buffer parity the graph was captured from
    std::string graph_note;        // how the graph was made, or why not
    std::string errmsg;
};

namespace {

int bfail(ebit_batch *b, int code, const std::string &m) {
    if (b) b->errmsg = m;
    return code;
}

#define BCU(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return bfail(b, EBIT_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

template <int SH>
const void *sweep_fn_sh(int d) {
    if (d == 0) return (const void *)batch_sweep_kernel<0, SH>;
    if (d == 1) return (const void *)batch_sweep_kernel<1, SH>;
    return (const void *)batch_sweep_kernel<2, SH>;
}

const void *sweep_fn(int d, int sh) {
    static_assert(N_TILE_SHAPES == 3, "one instantiation per tile shape");
    if (sh == 1) return sweep_fn_sh<1>(d);
    if (sh == 2) return sweep_fn_sh<2>(d);
    return sweep_fn_sh<0>(d);
}

// co-resident blocks per SM that every direction's kernel of shape sh allows
int max_ctas(const ebit_batch *b, int sh) { return std::min({b->occ[sh][0], b->occ[sh][1], b->occ[sh][2]}); }

BatchParams sweep_params(const ebit_batch *b, int d, int parity) {
    BatchParams p;
    p.inst = b->table[parity];
    p.n = b->n;
    p.total_tiles = b->tiles;
    p.toff = b->d_toff;
    p.u = b->u[d];
    p.lam = b->lam;
    p.band = b->band;
    p.nband = b->nband;
    p.wcount = b->wcount;
    p.bar = b->bar;
    p.err = b->err;
    return p;
}

int sweep_grid(const ebit_batch *b, int d, int ctas_per_sm) {
    return b->sms * std::max(1, std::min(ctas_per_sm, b->occ[b->shape][d]));
}

// cooperative launch (all blocks co-resident: the grid barrier needs it)
int launch_dir(ebit_batch *b, int d, int ctas_per_sm) {
    BatchParams p = sweep_params(b, d, b->parity);
    BCU(cudaMemsetAsync(b->nband, 0, sizeof(int), b->stream));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sweep_grid(b, d, ctas_per_sm));
    cfg.blockDim = dim3(BATCH_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void *args[] = {&p};
    BCU(cudaLaunchKernelExC(&cfg, sweep_fn(d, b->shape), args));
    return EBIT_OK;
}

// Two steps (x y z, then z y x) as an explicitly built graph: a memset of the
// band count and a cooperative kernel node per sweep.
cudaError_t build_graph(ebit_batch *b, cudaGraph_t *out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    const int ord[6] = {0, 1, 2, 2, 1, 0};
    int par = b->parity;
    cudaGraphNode_t prev = nullptr;
    for (int q = 0; q < 6 && e == cudaSuccess; q++) {
        const int d = ord[q];
        cudaMemsetParams mp = {};
        mp.dst = b->nband;
        mp.value = 0;
        mp.elementSize = sizeof(int);
        mp.width = 1;
        mp.height = 1;
        mp.pitch = 0;
        cudaGraphNode_t mn = nullptr, kn = nullptr;
        e = cudaGraphAddMemsetNode(&mn, g, prev ? &prev : nullptr, prev ? 1 : 0, &mp);
        if (e != cudaSuccess) break;
        BatchParams p = sweep_params(b, d, par);
        void *args[] = {&p};
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void *>(sweep_fn(d, b->shape));
        kp.gridDim = dim3(sweep_grid(b, d, b->ctas_per_sm));
        kp.blockDim = dim3(BATCH_THREADS);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        kp.extra = nullptr;
        e = cudaGraphAddKernelNode(&kn, g, &mn, 1, &kp);
        if (e != cudaSuccess) break;
        cudaLaunchAttributeValue v = {};
        v.cooperative = 1;
        e = cudaGraphKernelNodeSetAttribute(kn, cudaLaunchAttributeCooperative, &v);
        prev = kn;
        par ^= 1;
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    *out = g;
    return cudaSuccess;
}

int sweep_once(ebit_batch *b, int dir, int ctas_per_sm) {
    int r = launch_dir(b, dir, ctas_per_sm);
    if (r) return r;
    b->parity ^= 1;
    for (ebit_ctx *c : b->inst) {
        c->cur = b->parity;
        c->sweeps_since_f2v++;
    }
    return EBIT_OK;
}

void drop_graph(ebit_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->graph_ok = 0;
}

// tiles of instance i with tile shape sh
long long inst_tiles(const ebit_batch *b, int i, int sh) {
    long long nt = 1;
    for (int a = 0; a < 3; a++) nt *= (b->dims[3 * i + a] + tile_edge(sh, a) - 1) / tile_edge(sh, a);
    return nt;
}

// Does tile shape sh fit every instance?  A tile's staged region reaches from
// one node behind its origin to T + 1 nodes past it along an axis with tile
// edge T, and the grid wraps a coordinate by one period at most, so the last
// tile's region must end within two periods: o_max + T + 2 <= 2 n, with
// o_max the origin of the last tile.  (8^3 tiles fit every grid of >= 8 cells.)
bool shape_fits(const ebit_batch *b, int sh) {
    for (int i = 0; i < b->n; i++)
        for (int a = 0; a < 3; a++) {
            const int n = b->dims[3 * i + a], t = tile_edge(sh, a);
            if (t * ((n - 1) / t) + t + 2 > 2 * n) return false;
        }
    return true;
}

// first tile of every instance (and the total, at index n) with tile shape sh
void tile_offsets(const ebit_batch *b, int sh, std::vector<int> &toff) {
    toff.assign(b->n + 1, 0);
    for (int i = 0; i < b->n; i++) toff[i + 1] = toff[i] + (int)inst_tiles(b, i, sh);
}

// Switch the batch to tile shape sh: tile offsets, every instance context
// re-tiled over its new slice of the tile tables (every tile marked for the
// next sweep and Front2VOF), the launch tables rewritten, the graph dropped.
int retile(ebit_batch *b, int sh) {
    if (!shape_fits(b, sh)) return bfail(b, EBIT_EINVAL, "tile shape too large for an instance");
    std::vector<int> toff;
    tile_offsets(b, sh, toff);
    if (toff[b->n] > b->tiles_cap) return bfail(b, EBIT_EINVAL, "retile: tile tables too small");
    std::vector<BatchInst> *tab = b->htab;
    for (int i = 0; i < b->n; i++) {
        ebit_ctx *c = b->inst[i];
        int r = ctx_retile(c, sh, b->tile_marker + toff[i], b->tile_dirty + toff[i]);
        if (r) return bfail(b, r, "retile: " + c->err);
        for (int q = 0; q < 2; q++) {
            tab[q][i].a.g = c->g;
            tab[q][i].a.tile_marker = c->tile_marker;
            tab[q][i].a.tile_dirty = c->tile_dirty;
        }
    }
    for (int q = 0; q < 2; q++)
        BCU(cudaMemcpyAsync(b->table[q], tab[q].data(), b->n * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_toff, toff.data(), (b->n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));  // toff goes out of scope
    b->toff = toff;
    b->tiles = toff[b->n];
    b->shape = sh;
    b->ctas_per_sm = std::min(b->ctas_per_sm, max_ctas(b, sh));
    drop_graph(b);
    return EBIT_OK;
}

}  // namespace

extern "C" {

int ebit_batch_create(int n, const ebit_desc *descs, ebit_batch **out) {
    if (!out) return EBIT_EINVAL;
    *out = nullptr;
    if (n < 1 || n > BATCH_MAX || !descs) return EBIT_EINVAL;
    ebit_batch *b = new ebit_batch();
    b->n = n;
    b->stream = (cudaStream_t)descs[0].cuda_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) {
        delete b;
        return EBIT_ECUDA;
    }
    b->coff.resize(n + 1);
    b->dims.resize(3 * n);
    long long cells = 0;
    long long tiles_cap = 0;
    for (int i = 0; i < n; i++) {
        const ebit_desc &d = descs[i];
        if (d.nx < 8 || d.ny < 8 || d.nz < 8 || !(d.h > 0.0) || d.cuda_stream != descs[0].cuda_stream ||
            (d.flags & EBIT_DESC_DENSE)) {
            delete b;
            return EBIT_EINVAL;
        }
        b->dims[3 * i] = d.nx;
        b->dims[3 * i + 1] = d.ny;
        b->dims[3 * i + 2] = d.nz;
        const long long nc = (long long)d.nx * d.ny * d.nz;
        b->coff[i] = cells;
        cells += (nc + 7) & ~7LL;  // each slice starts on a 32-bit word of the colour bytes
    }
    for (int sh = 0; sh < N_TILE_SHAPES; sh++) {
        long long tiles = 0;
        for (int i = 0; i < n; i++) {
            const long long nt = inst_tiles(b, i, sh);
            if (nt >= (1 << 20)) {  // tile ids keep 20 bits
                delete b;
                return EBIT_EINVAL;
            }
            tiles += nt;
        }
        tiles_cap = std::max(tiles_cap, tiles);
    }
    if (cells >= (1LL << 31) || tiles_cap >= (1LL << 31)) {
        delete b;
        return EBIT_EINVAL;
    }
    b->coff[n] = cells;
    b->cells = cells;
    b->tiles_cap = (int)tiles_cap;
    tile_offsets(b, 0, b->toff);
    const long long tiles = tiles_cap;
    b->tiles = b->toff[n];
    b->mem = current_devmem();
    auto alloc = [&](void **p, size_t bytes) { return dev_alloc(b->mem, p, bytes); };
    bool ok = true;
    for (int q = 0; q < 2 && ok; q++) {
        ok = ok && alloc((void **)&b->cb[q], cells);
        for (int a = 0; a < 3 && ok; a++) ok = ok && alloc((void **)&b->s[q][a], cells * sizeof(double));
    }
    for (int a = 0; a < 3 && ok; a++)
        ok = ok && alloc((void **)&b->adv[a], cells * sizeof(double)) && alloc((void **)&b->bin[a], cells);
    for (int k = 0; k < 4 && ok; k++) ok = ok && alloc((void **)&b->work[k], cells * sizeof(unsigned));
    ok = ok && alloc((void **)&b->wcount, 4 * n * sizeof(int)) && alloc((void **)&b->tile_marker, tiles * sizeof(uint32_t)) &&
         alloc((void **)&b->tile_dirty, tiles) && alloc((void **)&b->ctr, (size_t)n * C_TOTAL * 8) &&
         alloc((void **)&b->table[0], n * sizeof(BatchInst)) && alloc((void **)&b->table[1], n * sizeof(BatchInst)) &&
         alloc((void **)&b->d_toff, (n + 1) * sizeof(int)) && alloc((void **)&b->lam, n * sizeof(double)) &&
         alloc((void **)&b->band, std::max<long long>(tiles, 1) * sizeof(int)) &&
         alloc((void **)&b->nband, sizeof(int)) && alloc((void **)&b->bar, 2 * sizeof(unsigned)) &&
         alloc((void **)&b->err, sizeof(int));
    for (int d = 0; d < 3 && ok; d++) ok = ok && alloc((void **)&b->u[d], n * sizeof(double *));
    if (!ok) {
        cudaGetLastError();
        ebit_batch_destroy(b);
        return EBIT_ENOMEM;
    }
    // instance contexts over the arena slices
    b->inst.assign(n, nullptr);
    std::vector<BatchInst> tab[2];
    tab[0].resize(n);
    tab[1].resize(n);
    for (int i = 0; i < n; i++) {
        const long long c0 = b->coff[i];
        const int t0 = b->toff[i];
        ebit_state_arrays st;
        for (int q = 0; q < 2; q++) {
            st.cb[q] = b->cb[q] + c0;
            for (int a = 0; a < 3; a++) st.s[q][a] = b->s[q][a] + c0;
        }
        for (int a = 0; a < 3; a++) {
            st.adv[a] = b->adv[a] + c0;
            st.bin[a] = b->bin[a] + c0;
        }
        for (int k = 0; k < 4; k++) st.work[k] = b->work[k] + c0;
        st.wcount = b->wcount + 4 * i;
        st.tile_marker = b->tile_marker + t0;
        st.tile_dirty = b->tile_dirty + t0;
        st.ctr = b->ctr + (size_t)i * C_TOTAL;
        int r = ebit_create_view(&descs[i], &st, &b->inst[i]);
        if (r) {
            ebit_batch_destroy(b);
            return r;
        }
        const ebit_ctx *c = b->inst[i];
        for (int q = 0; q < 2; q++) {
            SweepArgs &a = tab[q][i].a;
            std::memset(&a, 0, sizeof(a));
            a.g = c->g;
            a.cb = st.cb[q];
            a.cbo = st.cb[q ^ 1];
            for (int k = 0; k < 3; k++) {
                a.s[k] = st.s[q][k];
                a.so[k] = st.s[q ^ 1][k];
                a.adv[k] = st.adv[k];
                a.bin[k] = st.bin[k];
            }
            for (int k = 0; k < 4; k++) a.work[k] = st.work[k];
            a.wcount = st.wcount;
            a.ctr = st.ctr;
            a.tile_marker = st.tile_marker;
            a.tile_dirty = st.tile_dirty;
        }
    }
    if (cudaMemcpyAsync(b->table[0], tab[0].data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->table[1], tab[1].data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_toff, b->toff.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->err, 0, sizeof(int), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->wcount, 0, 4 * n * sizeof(int), b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        ebit_batch_destroy(b);
        return EBIT_ECUDA;
    }
    for (int sh = 0; sh < N_TILE_SHAPES; sh++)
        for (int d = 0; d < 3; d++) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ[sh][d], sweep_fn(d, sh), BATCH_THREADS, 0);
            b->occ[sh][d] = std::max(1, b->occ[sh][d]);
        }
    b->htab[0] = tab[0];
    b->htab[1] = tab[1];
    b->shape = 0;
    b->ctas_per_sm = max_ctas(b, 0);
    *out = b;
    return EBIT_OK;
}

void ebit_batch_destroy(ebit_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (ebit_ctx *c : b->inst) ebit_destroy(c);
    for (int q = 0; q < 2; q++) {
        dev_free(b->mem, b->cb[q]);
        for (int a = 0; a < 3; a++) dev_free(b->mem, b->s[q][a]);
    }
    for (int a = 0; a < 3; a++) {
        dev_free(b->mem, b->adv[a]);
        dev_free(b->mem, b->bin[a]);
        dev_free(b->mem, b->u[a]);
    }
    for (int k = 0; k < 4; k++) dev_free(b->mem, b->work[k]);
    dev_free(b->mem, b->wcount);
    dev_free(b->mem, b->tile_marker);
    dev_free(b->mem, b->tile_dirty);
    dev_free(b->mem, b->ctr);
    dev_free(b->mem, b->table[0]);
    dev_free(b->mem, b->table[1]);
    dev_free(b->mem, b->d_toff);
    dev_free(b->mem, b->lam);
    dev_free(b->mem, b->band);
    dev_free(b->mem, b->nband);
    dev_free(b->mem, b->bar);
    dev_free(b->mem, b->err);
    delete b;
}

int ebit_batch_size(const ebit_batch *b) { return b ? b->n : 0; }

ebit_ctx *ebit_batch_instance(ebit_batch *b, int i) {
    if (!b || i < 0 || i >= b->n) return nullptr;
    return b->inst[i];
}

int ebit_batch_set_velocity(ebit_batch *b, const double *const *u_faces, const double *dt) {
    if (!b || !u_faces || !dt) return EBIT_EINVAL;
    std::vector<const double *> up[3];
    std::vector<double> lam(b->n);
    for (int i = 0; i < b->n; i++) {
        for (int d = 0; d < 3; d++) {
            if (!u_faces[3 * i + d]) return bfail(b, EBIT_EINVAL, "ebit_batch_set_velocity: null velocity");
            up[d].push_back(u_faces[3 * i + d]);
        }
        if (!std::isfinite(dt[i])) return bfail(b, EBIT_EINVAL, "ebit_batch_set_velocity: non-finite dt");
        lam[i] = dt[i] / b->inst[i]->h;
    }
    for (int d = 0; d < 3; d++)
        BCU(cudaMemcpyAsync(b->u[d], up[d].data(), b->n * sizeof(double *), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->lam, lam.data(), b->n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    b->have_u[0] = b->have_u[1] = b->have_u[2] = 1;
    b->have_dt = 1;
    return EBIT_OK;
}

int ebit_batch_advect_sweep(ebit_batch *b, int dir, const double *const *u_dev, const double *dt) {
    if (!b) return EBIT_EINVAL;
    if (dir < 0 || dir > 2) return bfail(b, EBIT_EINVAL, "ebit_batch_advect_sweep: dir must be 0, 1 or 2");
    if (u_dev) {
        for (int i = 0; i < b->n; i++)
            if (!u_dev[i]) return bfail(b, EBIT_EINVAL, "ebit_batch_advect_sweep: null velocity");
        BCU(cudaMemcpyAsync(b->u[dir], u_dev, b->n * sizeof(double *), cudaMemcpyHostToDevice, b->stream));
        b->have_u[dir] = 1;
    }
    if (dt) {
        std::vector<double> lam(b->n);
        for (int i = 0; i < b->n; i++) {
            if (!std::isfinite(dt[i])) return bfail(b, EBIT_EINVAL, "ebit_batch_advect_sweep: non-finite dt");
            lam[i] = dt[i] / b->inst[i]->h;
        }
        BCU(cudaMemcpyAsync(b->lam, lam.data(), b->n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        BCU(cudaStreamSynchronize(b->stream));  // the host copy of lam goes out of scope
        b->have_dt = 1;
    }
    if (!b->have_u[dir] || !b->have_dt)
        return bfail(b, EBIT_EINVAL, "ebit_batch_advect_sweep: no velocity or time step for this direction");
    return sweep_once(b, dir, b->ctas_per_sm);
}

int ebit_batch_run(ebit_batch *b, int first_step, int steps, int use_graph) {
    if (!b || steps < 0) return EBIT_EINVAL;
    if (!(b->have_u[0] && b->have_u[1] && b->have_u[2] && b->have_dt))
        return bfail(b, EBIT_EINVAL, "ebit_batch_run: no velocity set");
    int n = first_step;
    int left = steps;
    auto one_step = [&](int k) -> int {
        const int ord[2][3] = {{0, 1, 2}, {2, 1, 0}};
        for (int q = 0; q < 3; q++) {
            int r = sweep_once(b, ord[k & 1][q], b->ctas_per_sm);
            if (r) return r;
        }
        return EBIT_OK;
    };
    // leading odd step, so that the graph always starts on an even step
    if (left > 0 && (n & 1)) {
        int r = one_step(n);
        if (r) return r;
        n++;
        left--;
    }
    if (use_graph && left >= 2) {
        if (b->graph_ok && b->graph_parity != b->parity) drop_graph(b);
        if (!b->graph_ok) {
            // two steps from the current parity (a replay restores it): stream
            // capture first, else an explicitly built graph
            drop_graph(b);
            const int par0 = b->parity;
            std::vector<int> since(b->n);
            for (int i = 0; i < b->n; i++) since[i] = b->inst[i]->sweeps_since_f2v;
            std::string why;
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                int r = one_step(0);
                if (r == EBIT_OK) r = one_step(1);
                cudaError_t e = cudaStreamEndCapture(b->stream, &g);
                if (r != EBIT_OK || e != cudaSuccess) {
                    why = "capture: " + (r != EBIT_OK ? b->errmsg : std::string(cudaGetErrorString(e)));
                    if (g) cudaGraphDestroy(g);
                    g = nullptr;
                }
            }
            cudaGetLastError();
            b->parity = par0;
            for (int i = 0; i < b->n; i++) {
                b->inst[i]->cur = par0;
                b->inst[i]->sweeps_since_f2v = since[i];
            }
            int how = 1;
            if (g) {
                cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
                if (e != cudaSuccess) {
                    why += std::string("; instantiate captured: ") + cudaGetErrorString(e);
                    cudaGraphDestroy(g);
                    g = nullptr;
                    b->gexec = nullptr;
                }
            }
            if (!g) {
                how = 2;
                cudaError_t e = build_graph(b, &g);
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
                if (e != cudaSuccess) {
                    why += std::string("; built graph: ") + cudaGetErrorString(e);
                    if (g) cudaGraphDestroy(g);
                    g = nullptr;
                    b->gexec = nullptr;
                }
            }
            cudaGetLastError();
            if (g) {
                b->graph = g;
                b->graph_ok = how;
                b->graph_parity = par0;
            }
            b->graph_note = g ? (how == 1 ? "stream capture" : "explicit graph" + why) : "no graph" + why;
        }
        if (b->graph_ok) {
            while (left >= 2) {
                BCU(cudaGraphLaunch(b->gexec, b->stream));
                for (ebit_ctx *c : b->inst) c->sweeps_since_f2v += 6;
                n += 2;
                left -= 2;
            }
        }
    }
    while (left > 0) {
        int r = one_step(n);
        if (r) return r;
        n++;
        left--;
    }
    return EBIT_OK;
}

int ebit_batch_graph_active(const ebit_batch *b) { return b ? b->graph_ok : 0; }

const char *ebit_batch_graph_note(const ebit_batch *b) { return b ? b->graph_note.c_str() : "null batch"; }

int ebit_batch_sync(ebit_batch *b) {
    if (!b) return EBIT_EINVAL;
    int e = 0;
    BCU(cudaMemcpyAsync(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    if (e) return bfail(b, EBIT_ETIMEOUT, "a grid barrier of the batched sweep gave up");
    return EBIT_OK;
}

int ebit_batch_launch_shape(const ebit_batch *b, int *ctas_per_sm, int *max_ctas_per_sm) {
    if (!b) return EBIT_EINVAL;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    if (max_ctas_per_sm) *max_ctas_per_sm = max_ctas(b, b->shape);
    return EBIT_OK;
}

int ebit_batch_set_launch_shape(ebit_batch *b, int ctas_per_sm) {
    if (!b || ctas_per_sm < 1 || ctas_per_sm > max_ctas(b, b->shape)) return EBIT_EINVAL;
    if (ctas_per_sm != b->ctas_per_sm) drop_graph(b);
    b->ctas_per_sm = ctas_per_sm;
    return EBIT_OK;
}

int ebit_batch_tile_shape(const ebit_batch *b, int *dims) {
    if (!b) return EBIT_EINVAL;
    if (dims)
        for (int a = 0; a < 3; a++) dims[a] = tile_edge(b->shape, a);
    return b->shape;
}

int ebit_batch_set_tile_shape(ebit_batch *b, int shape) {
    if (!b || shape < 0 || shape >= N_TILE_SHAPES) return EBIT_EINVAL;
    if (shape == b->shape) return EBIT_OK;
    BCU(cudaStreamSynchronize(b->stream));
    return retile(b, shape);
}

int ebit_batch_autotune(ebit_batch *b, int sweeps, double *ms_out) {
    if (!b || sweeps < 1) return EBIT_EINVAL;
    if (!(b->have_u[0] && b->have_u[1] && b->have_u[2] && b->have_dt))
        return bfail(b, EBIT_EINVAL, "ebit_batch_autotune: no velocity set");
    static_assert(EBIT_TILE_SHAPES == N_TILE_SHAPES, "tile shapes of the ABI");
    if (ms_out)
        for (int k = 0; k < EBIT_TILE_SHAPES * EBIT_BATCH_MAX_CTAS; k++) ms_out[k] = 0.0;
    BCU(cudaStreamSynchronize(b->stream));
    // trial sweeps run on a copy of the state, which is put back afterwards
    const long long cells = b->cells;
    const int par0 = b->parity, sh0 = b->shape, tiles0 = b->tiles;
    uint8_t *cb_save = nullptr, *td_save = nullptr;
    uint32_t *tm_save = nullptr;
    double *s_save = nullptr;
    unsigned long long *ctr_save = nullptr;
    bool ok = dev_alloc(b->mem, (void **)&cb_save, cells) &&
              dev_alloc(b->mem, (void **)&s_save, 3 * cells * sizeof(double)) &&
              dev_alloc(b->mem, (void **)&tm_save, tiles0 * sizeof(uint32_t)) &&
              dev_alloc(b->mem, (void **)&td_save, tiles0) &&
              dev_alloc(b->mem, (void **)&ctr_save, (size_t)b->n * C_TOTAL * 8);
    auto release = [&]() {
        dev_free(b->mem, cb_save);
        dev_free(b->mem, s_save);
        dev_free(b->mem, tm_save);
        dev_free(b->mem, td_save);
        dev_free(b->mem, ctr_save);
    };
    if (!ok) {
        cudaGetLastError();
        release();
        return bfail(b, EBIT_ENOMEM, "ebit_batch_autotune: no room for the state copy");
    }
    // save: the state, the counters and the tile tables (of the current shape);
    // restore: the state into both buffers and the counters, and the tile
    // tables when the shape is the one they were saved in
    auto copy = [&](bool save, bool tables) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        auto cp = [&](void *dst, const void *src, size_t bytes) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, b->stream);
        };
        if (save) {
            cp(cb_save, b->cb[par0], cells);
            for (int a = 0; a < 3; a++) cp(s_save + a * cells, b->s[par0][a], cells * sizeof(double));
            cp(tm_save, b->tile_marker, tiles0 * sizeof(uint32_t));
            cp(td_save, b->tile_dirty, tiles0);
            cp(ctr_save, b->ctr, (size_t)b->n * C_TOTAL * 8);
        } else {
            for (int q = 0; q < 2; q++) {
                cp(b->cb[q], cb_save, cells);
                for (int a = 0; a < 3; a++) cp(b->s[q][a], s_save + a * cells, cells * sizeof(double));
            }
            if (tables) {
                cp(b->tile_marker, tm_save, tiles0 * sizeof(uint32_t));
                cp(b->tile_dirty, td_save, tiles0);
            }
            cp(b->ctr, ctr_save, (size_t)b->n * C_TOTAL * 8);
        }
        return e;
    };
    auto reset_parity = [&]() {
        b->parity = par0;
        for (int i = 0; i < b->n; i++) b->inst[i]->cur = par0;
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best_sh = sh0, best_c = b->ctas_per_sm;
    double best_ms = 1e300;
    std::vector<int> since(b->n);
    for (int i = 0; i < b->n; i++) since[i] = b->inst[i]->sweeps_since_f2v;
    int r = EBIT_OK;
    if (copy(true, true) != cudaSuccess) r = bfail(b, EBIT_ECUDA, "ebit_batch_autotune: state copy failed");
    for (int sh = 0; sh < N_TILE_SHAPES && r == EBIT_OK; sh++) {
        if (!shape_fits(b, sh)) continue;
        const int maxc = std::min(max_ctas(b, sh), (int)EBIT_BATCH_MAX_CTAS);
        for (int c = 1; c <= maxc && r == EBIT_OK; c++) {
            for (int rep = 0; rep < 2 && r == EBIT_OK; rep++) {  // first pass warms up
                // from the saved state with every tile marked (the re-tiling),
                // one untimed sweep to form the band, then the timed sweeps
                r = retile(b, sh);
                if (r == EBIT_OK && copy(false, false) != cudaSuccess)
                    r = bfail(b, EBIT_ECUDA, "ebit_batch_autotune: state copy failed");
                if (r != EBIT_OK) break;
                reset_parity();
                r = sweep_once(b, 0, c);
                cudaEventRecord(e0, b->stream);
                for (int k = 1; k <= sweeps && r == EBIT_OK; k++) r = sweep_once(b, k % 3, c);
                cudaEventRecord(e1, b->stream);
                if (ebit_batch_sync(b) != EBIT_OK) r = EBIT_ETIMEOUT;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1 && r == EBIT_OK) {
                    if (ms_out) ms_out[sh * EBIT_BATCH_MAX_CTAS + c - 1] = ms;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_sh = sh;
                        best_c = c;
                    }
                }
            }
        }
    }
    // back to the saved state, in the chosen shape; the saved tile tables
    // return with the shape they belong to, any other shape starts with every
    // tile marked (the same results: tiles outside the band are unchanged)
    const int sh_end = r == EBIT_OK ? best_sh : sh0;
    int r2 = retile(b, sh_end);
    if (r2 == EBIT_OK && copy(false, sh_end == sh0) != cudaSuccess)
        r2 = bfail(b, EBIT_ECUDA, "ebit_batch_autotune: restore failed");
    cudaStreamSynchronize(b->stream);
    reset_parity();
    for (int i = 0; i < b->n; i++) b->inst[i]->sweeps_since_f2v = since[i];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    if (r == EBIT_OK) r = r2;
    if (r == EBIT_OK) {
        drop_graph(b);
        b->ctas_per_sm = best_c;
    }
    return r;
}

const char *ebit_batch_last_error(const ebit_batch *b) { return b ? b->errmsg.c_str() : "null batch"; }

int ebit_selftest_bounded_waits(void *cuda_stream, int *report) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *d = nullptr;
    const DevMem mm = current_devmem();
    if (!dev_alloc(mm, (void **)&d, 16 * sizeof(int))) {
        cudaGetLastError();
        return EBIT_ENOMEM;
    }
    // slots: 0..3 results; 4..5 / 8..9 barrier words; 6 / 10 error flags
    int h[16] = {0};
    bool ok = cudaMemsetAsync(d, 0, 16 * sizeof(int), st) == cudaSuccess;
    for (int absent = 0; absent < 2 && ok; absent++) {
        BatchParams p{};
        p.bar = (unsigned *)(d + 4 + 4 * absent);
        p.err = d + 6 + 4 * absent;
        int *out = d + absent;
        long long polls = absent ? 4096 : (1LL << 20);
        void *args[] = {&p, &absent, &polls, &out};
        ok = cudaLaunchCooperativeKernel((const void *)selftest_barrier_kernel, dim3(2), dim3(32), args, 0, st) ==
             cudaSuccess;
    }
    if (ok) {
        selftest_mbarrier_kernel<<<1, 32, 0, st>>>(1, 1 << 20, d + 2);
        selftest_mbarrier_kernel<<<1, 32, 0, st>>>(0, 64, d + 3);
        ok = cudaGetLastError() == cudaSuccess &&
             cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
    }
    // the device still takes work after the waits gave up
    ok = ok && cudaMemsetAsync(d, 0, 16 * sizeof(int), st) == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
    dev_free(mm, d);
    if (!ok) {
        cudaGetLastError();
        return EBIT_ECUDA;
    }
    if (report) {
        const int r[6] = {h[0], h[6], h[1], h[10], h[2], h[3]};
        std::memcpy(report, r, sizeof(r));
    }
    const bool met = h[0] == 1 && h[6] == 0 && h[2] == 1;      // the waits that can succeed did
    const bool gave_up = h[1] == 0 && h[10] == 1 && h[3] == 0; // the others gave up and said so
    return met && gave_up ? EBIT_OK : EBIT_ETIMEOUT;
}

}  // extern "C"
