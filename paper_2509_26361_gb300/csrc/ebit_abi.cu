// ebit_abi.cu -- the C ABI of libebit.so (declared in include/ebit.h).
//
// The context owns a double-buffered EBIT state (colour bytes + three FP64
// offset arrays) and per-tile tables that keep every call on the active band:
// a sweep processes the tiles whose 3x3x3 tile neighbourhood held a marker
// before or after the previous sweep, Front2VOF the tiles swept since its last
// call, curvature the tiles around cells whose volume fraction was rewritten.
// A tile outside the band provably holds no marker and is not changed by the
// call, and both state buffers agree on it, so band processing gives the same
// state as processing every tile (tests compare both against the oracle).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ebit.h"
#include "common.cuh"
#include "ctx.h"
#include "f2v.cuh"
#include "hf.cuh"
#include "mlp.cuh"
#include "state.cuh"
#include "sweep.cuh"
#include "amr.cuh"
#include "coupling.cuh"

using namespace ebit;

namespace {

int fail(ebit_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

#define CU(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(ctx, EBIT_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

int launch_check(ebit_ctx *ctx, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, EBIT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return EBIT_OK;
}

// Launch with programmatic stream serialization: the kernel is launched as
// the previous kernel's blocks exit, and waits (pdl_wait) for that kernel's
// completion before it touches global memory.  Counters that a
// launch appends to are cleared by an earlier kernel of the chain (in its
// zero arguments) instead of by memsets, which would break the overlap.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int launched(ebit_ctx *ctx, cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, EBIT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return launch_check(ctx, what);
}

int mark_all(ebit_ctx *ctx) {
    ctx->sweeps_since_f2v = 1;
    CU(cudaMemsetAsync(ctx->tile_marker, 0xFF, ctx->g.ntiles * sizeof(uint32_t), ctx->stream));
    CU(cudaMemsetAsync(ctx->dirty_set ? ctx->tile_dirty2 : ctx->tile_dirty, 1, ctx->g.ntiles, ctx->stream));
    if (ctx->tile_dirty2)
        CU(cudaMemsetAsync(ctx->dirty_set ? ctx->tile_dirty : ctx->tile_dirty2, 0, ctx->g.ntiles, ctx->stream));
    // the next sweep processes every tile and lists the markers and band anew
    ctx->mk_valid = 0;
    if (ctx->owns_state) {
        CU(cudaMemsetAsync(ctx->band_flag, 0, ctx->g.ntiles * sizeof(uint32_t), ctx->stream));
        CU(cudaMemsetAsync(ctx->band_count, 0, 2 * sizeof(int), ctx->stream));
    }
    ctx->last_C = nullptr;
    ctx->last_kh = nullptr;
    ctx->last_st = nullptr;
    return EBIT_OK;
}

// The main stream waits for everything issued on the side stream so far.
int join_side(ebit_ctx *ctx) {
    if (!ctx->side_pending) return EBIT_OK;
    CU(cudaEventRecord(ctx->ev_side, ctx->side));
    CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_side, 0));
    ctx->side_pending = 0;
    ctx->f2v_pending = 0;
    return EBIT_OK;
}

// The stream for a Front2VOF or curvature call: the side stream (after the
// main stream's work so far) for EBIT_ASYNC, else the main stream (after any
// side-stream work).
int call_stream(ebit_ctx *ctx, int flags, cudaStream_t *st) {
    if (!(flags & EBIT_ASYNC)) {
        *st = ctx->stream;
        return join_side(ctx);
    }
    if (!ctx->owns_state) return fail(ctx, EBIT_EINVAL, "EBIT_ASYNC: not for batch instances");
    if (!ctx->side) {
        CU(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&ctx->ev_main, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&ctx->ev_side, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&ctx->ev_f2v, cudaEventDisableTiming));
    }
    CU(cudaEventRecord(ctx->ev_main, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->side, ctx->ev_main, 0));
    ctx->side_pending = 1;
    *st = ctx->side;
    return EBIT_OK;
}

int copy_other(ebit_ctx *ctx) {
    int o = ctx->cur ^ 1;
    CU(cudaMemcpyAsync(ctx->cb[o], ctx->cb[ctx->cur], ctx->N, cudaMemcpyDeviceToDevice, ctx->stream));
    for (int a = 0; a < 3; a++)
        CU(cudaMemcpyAsync(ctx->s[o][a], ctx->s[ctx->cur][a], ctx->N * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
    return EBIT_OK;
}

int blocks_for(long long n, int threads, int sms) {
    long long b = (n + threads - 1) / threads;
    long long cap = (long long)sms * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// Event pairs around the timed launches; drained into per-kind sums.
int prof_drain(ebit_ctx *ctx) {
    if (ctx->ev_used == 0) return EBIT_OK;
    CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->side) CU(cudaStreamSynchronize(ctx->side));
    for (int i = 0; i < ctx->ev_used; i++) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
        ctx->prof_ms[ctx->ev_kind[i]] += ms;
        ctx->prof_n[ctx->ev_kind[i]] += 1;
    }
    ctx->ev_used = 0;
    return EBIT_OK;
}

struct ProfScope {
    ebit_ctx *ctx;
    int kind;
    bool on;
    cudaStream_t st;
    ProfScope(ebit_ctx *c, int k, cudaStream_t s = nullptr) : ctx(c), kind(k), on(c->prof_on != 0), st(s ? s : c->stream) {
        if (!on) return;
        if (ctx->ev_used * 2 + 2 > (int)ctx->ev.size()) {
            if (prof_drain(ctx) != EBIT_OK) { on = false; return; }
        }
        cudaEventRecord(ctx->ev[2 * ctx->ev_used], st);
    }
    ~ProfScope() {
        if (!on) return;
        cudaEventRecord(ctx->ev[2 * ctx->ev_used + 1], st);
        ctx->ev_kind[ctx->ev_used] = kind;
        ctx->ev_used++;
    }
};

template <int D>
int sweep_launch(ebit_ctx *ctx, const SweepArgs &args, const MarkerLists *ml) {
    {
        ProfScope ps(ctx, EBIT_PROF_ADVECT);
        int r = ml ? launched(ctx, launch_pdl(advect_list_kernel<D, NLISTS>, ctx->grid_advl, 256, 0, ctx->stream,
                                              args, *ml),
                              "advect_list_kernel")
                   : launched(ctx, launch_pdl(advect_kernel<D, NLISTS>, ctx->grid_adv, 256, 0, ctx->stream, args),
                              "advect_kernel");
        if (r) return r;
    }
    {
        ProfScope ps(ctx, EBIT_PROF_SWEEP);
        int r = launched(ctx, launch_pdl(sweep_kernel<D, NLISTS>, ctx->grid_sweep, 256, 0, ctx->stream, args),
                         "sweep_kernel");
        if (r) return r;
    }
    ProfScope ps(ctx, EBIT_PROF_FP64);
    return launched(ctx, launch_pdl(fp64_kernel<D, NLISTS>, ctx->grid_fp64, 128, 0, ctx->stream, args),
                    "fp64_kernel");
}

}  // namespace


static DevMem g_devmem;  // the allocator new objects take (default: cudaMalloc / cudaFree)

DevMem ebit::current_devmem() { return g_devmem; }

int ebit_set_allocator(ebit_alloc_fn alloc, ebit_free_fn free_fn, void *user) {
    if (!alloc != !free_fn) return EBIT_EINVAL;
    g_devmem.alloc = alloc;
    g_devmem.free = free_fn;
    g_devmem.user = alloc ? user : nullptr;
    return EBIT_OK;
}

static int create_ctx(const ebit_desc *desc, const ebit_state_arrays *st, ebit_ctx **out) {
    ebit_ctx *ctx = nullptr;
    if (!desc || !out) return EBIT_EINVAL;
    *out = nullptr;
    if (desc->nx < 8 || desc->ny < 8 || desc->nz < 8) return EBIT_EINVAL;
    if (!(desc->h > 0.0) || !std::isfinite(desc->h)) return EBIT_EINVAL;
    if ((long long)desc->nx * desc->ny * desc->nz >= (1LL << 31)) return EBIT_EINVAL;
    ctx = new ebit_ctx();
    ctx->owns_state = st ? 0 : 1;
    std::memset(&ctx->g, 0, sizeof(ctx->g));
    for (int b = 0; b < 2; b++) {
        ctx->cb[b] = nullptr;
        for (int a = 0; a < 3; a++) ctx->s[b][a] = nullptr;
    }
    for (int a = 0; a < 3; a++) {
        ctx->adv[a] = nullptr;
        ctx->bin[a] = nullptr;
    }
    for (int k = 0; k < NLISTS; k++) ctx->work[k] = ctx->work2[k] = nullptr;
    ctx->wcount2 = ctx->mk_count = ctx->mt_count = ctx->band_list2 = nullptr;
    ctx->mk_al[0] = ctx->mk_al[1] = nullptr;
    ctx->mtiles[0] = ctx->mtiles[1] = nullptr;
    ctx->band_flag = nullptr;
    ctx->tile_dirty2 = nullptr;
    ctx->dirty_set = 0;
    ctx->side = nullptr;
    ctx->ev_main = ctx->ev_side = ctx->ev_f2v = nullptr;
    ctx->side_pending = ctx->f2v_pending = ctx->f2v_buf = 0;
    ctx->mk_par = 0;
    ctx->mk_dir = 0;
    ctx->mk_valid = 0;
    ctx->iface[0] = ctx->iface[1] = nullptr;
    ctx->wcount = ctx->ncut = ctx->niface = ctx->nscan = ctx->zero = nullptr;
    ctx->cut = ctx->scan = nullptr;
    ctx->cur_if = 0;
    ctx->if_slot = 0;
    ctx->band_last = -1;
    ctx->f2v_par = 0;
    ctx->sweeps_since_f2v = 0;
    ctx->mlp = nullptr;
    ctx->own_mlp = nullptr;
    ctx->tile_marker = nullptr;
    ctx->tile_dirty = ctx->tile_cchg = nullptr;
    ctx->band_list = ctx->band_count = ctx->work_list = ctx->work_count = ctx->all_list = ctx->all_count = nullptr;
    ctx->ctr = nullptr;
    ctx->g.n[0] = desc->nx;
    ctx->g.n[1] = desc->ny;
    ctx->g.n[2] = desc->nz;
    grid_tiles(ctx->g, 0);
    ctx->N = (long long)desc->nx * desc->ny * desc->nz;
    ctx->h = desc->h;
    ctx->stream = (cudaStream_t)desc->cuda_stream;
    ctx->dense = (desc->flags & EBIT_DESC_DENSE) ? 1 : 0;
    ctx->cur = 0;
    ctx->scratch = nullptr;
    ctx->amr_flag = ctx->amr_slot = nullptr;
    ctx->amr_ctr = nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    if (ctx->sms <= 0) ctx->sms = 1;
    ctx->mem = current_devmem();
    auto alloc = [&](void **p, size_t bytes) -> bool { return dev_alloc(ctx->mem, p, bytes); };
    bool ok = true;
    int nt = ctx->g.ntiles;
    // a batch instance may be re-tiled with any tile shape (its batch's
    // autotuner): its per-tile arrays hold the largest tile count of them
    ctx->nt_cap = nt;
    for (int sh = 1; st && sh < N_TILE_SHAPES; sh++) {
        Grid t = ctx->g;
        grid_tiles(t, sh);
        ctx->nt_cap = std::max(ctx->nt_cap, t.ntiles);
    }
    const int ntc = ctx->nt_cap;
    if (st) {
        for (int b = 0; b < 2; b++) {
            ctx->cb[b] = st->cb[b];
            for (int a = 0; a < 3; a++) ctx->s[b][a] = st->s[b][a];
        }
        for (int a = 0; a < 3; a++) {
            ctx->adv[a] = st->adv[a];
            ctx->bin[a] = st->bin[a];
        }
        for (int k = 0; k < 4; k++) ctx->work[k] = st->work[k];
        ctx->wcount = st->wcount;
        ctx->tile_marker = st->tile_marker;
        ctx->tile_dirty = st->tile_dirty;
        ctx->ctr = st->ctr;
    } else {
        for (int b = 0; b < 2 && ok; b++) {
            ok = ok && alloc((void **)&ctx->cb[b], (ctx->N + 7) & ~7LL);  // whole 32-bit words
            for (int a = 0; a < 3 && ok; a++) ok = ok && alloc((void **)&ctx->s[b][a], ctx->N * sizeof(double));
        }
        for (int a = 0; a < 3 && ok; a++)
            ok = ok && alloc((void **)&ctx->adv[a], ctx->N * sizeof(double)) && alloc((void **)&ctx->bin[a], ctx->N);
        for (int k = 0; k < NLISTS && ok; k++) ok = ok && alloc((void **)&ctx->work[k], ctx->N * sizeof(unsigned));
        ok = ok && alloc((void **)&ctx->wcount, (NLISTS + 1) * sizeof(int)) && alloc((void **)&ctx->tile_marker, nt * sizeof(uint32_t)) &&
             alloc((void **)&ctx->tile_dirty, nt) && alloc((void **)&ctx->ctr, C_TOTAL * sizeof(unsigned long long));
        for (int k = 0; k < NLISTS && ok; k++) ok = ok && alloc((void **)&ctx->work2[k], ctx->N * sizeof(unsigned));
        for (int q = 0; q < 2 && ok; q++)
            ok = ok && alloc((void **)&ctx->mk_al[q], ctx->N * sizeof(unsigned)) &&
                 alloc((void **)&ctx->mtiles[q], nt * sizeof(int));
        ok = ok && alloc((void **)&ctx->wcount2, (NLISTS + 1) * sizeof(int)) && alloc((void **)&ctx->mk_count, 2 * sizeof(int)) &&
             alloc((void **)&ctx->mt_count, 2 * sizeof(int)) && alloc((void **)&ctx->band_list2, nt * sizeof(int)) &&
             alloc((void **)&ctx->band_flag, nt * sizeof(uint32_t)) && alloc((void **)&ctx->tile_dirty2, nt);
    }
    ok = ok && alloc((void **)&ctx->cut, ctx->N * sizeof(unsigned)) && alloc((void **)&ctx->scan, ctx->N * sizeof(unsigned)) &&
         alloc((void **)&ctx->iface[0], ctx->N * sizeof(unsigned)) &&
         alloc((void **)&ctx->iface[1], ctx->N * sizeof(unsigned)) &&
         alloc((void **)&ctx->ncut, sizeof(int)) && alloc((void **)&ctx->niface, 3 * sizeof(int)) &&
         alloc((void **)&ctx->nscan, sizeof(int)) && alloc((void **)&ctx->zero, sizeof(int));
    ok = ok && alloc((void **)&ctx->tile_cchg, ntc) && alloc((void **)&ctx->band_list, ntc * sizeof(int)) &&
         alloc((void **)&ctx->band_count, 2 * sizeof(int)) && alloc((void **)&ctx->work_list, ntc * sizeof(int)) &&
         alloc((void **)&ctx->work_count, 2 * sizeof(int)) && alloc((void **)&ctx->all_list, ntc * sizeof(int)) &&
         alloc((void **)&ctx->all_count, sizeof(int));
    if (!ok) {
        cudaGetLastError();
        ebit_destroy(ctx);
        return EBIT_ENOMEM;
    }
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_kernel<0, NLISTS>, 256, 0);
    ctx->grid_sweep = std::max(1, std::min(nt, ctx->sms * std::max(occ, 1)));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, advect_kernel<0, NLISTS>, 256, 0);
    ctx->grid_adv = std::max(1, std::min(nt, ctx->sms * std::max(occ, 1)));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, advect_list_kernel<0, NLISTS>, 256, 0);
    ctx->grid_advl = ctx->sms * std::max(occ, 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp64_kernel<0, NLISTS>, 128, 0);
    ctx->grid_fp64 = ctx->sms * std::max(occ, 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f2v_band_kernel, 256, 0);
    ctx->grid_f2v = std::max(1, std::min(ntc, ctx->sms * std::max(occ, 1)));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f2v_list_kernel, 128, 0);
    ctx->grid_f2vl = ctx->sms * std::max(occ, 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hf_scan_kernel, 256, 0);
    ctx->grid_hf = std::max(1, std::min(ntc, ctx->sms * std::max(occ, 1)));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hf_list_kernel<true>, 128, 0);
    ctx->grid_hfl = ctx->sms * std::max(occ, 1);
    cudaMemsetAsync(ctx->wcount, 0, (ctx->owns_state ? NLISTS + 1 : 4) * sizeof(int), ctx->stream);
    if (ctx->owns_state) {
        cudaMemsetAsync(ctx->wcount2, 0, (NLISTS + 1) * sizeof(int), ctx->stream);
        cudaMemsetAsync(ctx->mk_count, 0, 2 * sizeof(int), ctx->stream);
        cudaMemsetAsync(ctx->mt_count, 0, 2 * sizeof(int), ctx->stream);
    }
    cudaMemsetAsync(ctx->ncut, 0, sizeof(int), ctx->stream);
    cudaMemsetAsync(ctx->niface, 0, 3 * sizeof(int), ctx->stream);
    cudaMemsetAsync(ctx->band_count, 0, 2 * sizeof(int), ctx->stream);
    cudaMemsetAsync(ctx->work_count, 0, 2 * sizeof(int), ctx->stream);
    cudaMemsetAsync(ctx->nscan, 0, sizeof(int), ctx->stream);
    cudaMemsetAsync(ctx->zero, 0, sizeof(int), ctx->stream);
    iota_kernel<<<blocks_for(nt, 256, ctx->sms), 256, 0, ctx->stream>>>(ctx->all_list, nt, ctx->all_count);
    if (cudaMemsetAsync(ctx->ctr, 0, C_TOTAL * sizeof(unsigned long long), ctx->stream) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess) {
        ebit_destroy(ctx);
        return EBIT_ECUDA;
    }
    ctx->prof_on = 0;
    ctx->ev_used = 0;
    for (int k = 0; k < EBIT_PROF_KINDS; k++) {
        ctx->prof_ms[k] = 0.0;
        ctx->prof_n[k] = 0;
    }
    mark_all(ctx);
    *out = ctx;
    return EBIT_OK;
}

int ctx_retile(ebit_ctx *ctx, int sh, uint32_t *tile_marker, uint8_t *tile_dirty) {
    if (!ctx || ctx->owns_state || sh < 0 || sh >= N_TILE_SHAPES || !tile_marker || !tile_dirty) return EBIT_EINVAL;
    Grid g = ctx->g;
    grid_tiles(g, sh);
    if (g.ntiles > ctx->nt_cap) return fail(ctx, EBIT_EINVAL, "ctx_retile: more tiles than the context holds");
    ctx->g = g;
    ctx->tile_marker = tile_marker;
    ctx->tile_dirty = tile_dirty;
    ctx->band_last = -1;
    iota_kernel<<<blocks_for(g.ntiles, 256, ctx->sms), 256, 0, ctx->stream>>>(ctx->all_list, g.ntiles, ctx->all_count);
    if (int r = launch_check(ctx, "iota_kernel")) return r;
    return mark_all(ctx);
}

int ebit_create_view(const ebit_desc *desc, const ebit_state_arrays *st, ebit_ctx **out) {
    if (!st) return EBIT_EINVAL;
    return create_ctx(desc, st, out);
}

extern "C" {

int ebit_create(const ebit_desc *desc, ebit_ctx **out) { return create_ctx(desc, nullptr, out); }

void ebit_destroy(ebit_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
        cudaEventDestroy(ctx->ev_main);
        cudaEventDestroy(ctx->ev_side);
        cudaEventDestroy(ctx->ev_f2v);
    }
    if (ctx->own_mlp) ebit_mlp_destroy(ctx->own_mlp);
    if (ctx->owns_state) {
        for (int b = 0; b < 2; b++) {
            dev_free(ctx->mem, ctx->cb[b]);
            for (int a = 0; a < 3; a++) dev_free(ctx->mem, ctx->s[b][a]);
        }
        dev_free(ctx->mem, ctx->tile_marker);
        dev_free(ctx->mem, ctx->tile_dirty);
        dev_free(ctx->mem, ctx->ctr);
        for (int a = 0; a < 3; a++) {
            dev_free(ctx->mem, ctx->adv[a]);
            dev_free(ctx->mem, ctx->bin[a]);
        }
        for (int k = 0; k < NLISTS; k++) {
            dev_free(ctx->mem, ctx->work[k]);
            dev_free(ctx->mem, ctx->work2[k]);
        }
        dev_free(ctx->mem, ctx->wcount);
        dev_free(ctx->mem, ctx->wcount2);
        dev_free(ctx->mem, ctx->mk_al[0]);
        dev_free(ctx->mem, ctx->mk_al[1]);
        dev_free(ctx->mem, ctx->mk_count);
        dev_free(ctx->mem, ctx->mtiles[0]);
        dev_free(ctx->mem, ctx->mtiles[1]);
        dev_free(ctx->mem, ctx->mt_count);
        dev_free(ctx->mem, ctx->band_flag);
        dev_free(ctx->mem, ctx->tile_dirty2);
        dev_free(ctx->mem, ctx->band_list2);
    }
    dev_free(ctx->mem, ctx->tile_cchg);
    dev_free(ctx->mem, ctx->band_list);
    dev_free(ctx->mem, ctx->band_count);
    dev_free(ctx->mem, ctx->work_list);
    dev_free(ctx->mem, ctx->work_count);
    dev_free(ctx->mem, ctx->all_list);
    dev_free(ctx->mem, ctx->all_count);
    dev_free(ctx->mem, ctx->scratch);
    dev_free(ctx->mem, ctx->amr_flag);
    dev_free(ctx->mem, ctx->amr_slot);
    dev_free(ctx->mem, ctx->amr_ctr);
    dev_free(ctx->mem, ctx->cut);
    dev_free(ctx->mem, ctx->scan);
    dev_free(ctx->mem, ctx->iface[0]);
    dev_free(ctx->mem, ctx->iface[1]);
    dev_free(ctx->mem, ctx->ncut);
    dev_free(ctx->mem, ctx->niface);
    dev_free(ctx->mem, ctx->nscan);
    dev_free(ctx->mem, ctx->zero);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    delete ctx;
}

int ebit_init(ebit_ctx *ctx, const double *phi_nodes, const double *phi_faces, const double *s_exact) {
    if (!ctx || !phi_nodes) return fail(ctx, EBIT_EINVAL, "ebit_init: null argument");
    if (int r = join_side(ctx)) return r;
    int c = ctx->cur;
    init_kernel<<<blocks_for(ctx->N, 256, ctx->sms), 256, 0, ctx->stream>>>(
        ctx->g, phi_nodes, phi_faces, s_exact, ctx->cb[c], ctx->s[c][0], ctx->s[c][1], ctx->s[c][2]);
    int r = launch_check(ctx, "init_kernel");
    if (r) return r;
    if ((r = copy_other(ctx))) return r;
    return mark_all(ctx);
}

int ebit_set_state(ebit_ctx *ctx, const uint8_t *cb, const double *s) {
    if (!ctx || !cb || !s) return fail(ctx, EBIT_EINVAL, "ebit_set_state: null argument");
    if (int r = join_side(ctx)) return r;
    int c = ctx->cur;
    CU(cudaMemcpyAsync(ctx->cb[c], cb, ctx->N, cudaMemcpyDefault, ctx->stream));
    for (int a = 0; a < 3; a++)
        CU(cudaMemcpyAsync(ctx->s[c][a], s + a * ctx->N, ctx->N * sizeof(double), cudaMemcpyDefault, ctx->stream));
    int r = copy_other(ctx);
    if (r) return r;
    return mark_all(ctx);
}

// the refinement scratch (per-tile flags and slots, two counters), on first use
static int amr_scratch(ebit_ctx *ctx) {
    if (ctx->amr_flag) return EBIT_OK;
    const size_t nt = (size_t)ctx->nt_cap;
    if (!dev_alloc(ctx->mem, (void **)&ctx->amr_flag, nt * sizeof(int)) ||
        !dev_alloc(ctx->mem, (void **)&ctx->amr_slot, nt * sizeof(int)) ||
        !dev_alloc(ctx->mem, (void **)&ctx->amr_ctr, 2 * sizeof(unsigned long long))) {
        cudaGetLastError();
        dev_free(ctx->mem, ctx->amr_flag);
        dev_free(ctx->mem, ctx->amr_slot);
        dev_free(ctx->mem, ctx->amr_ctr);
        ctx->amr_flag = ctx->amr_slot = nullptr;
        ctx->amr_ctr = nullptr;
        return fail(ctx, EBIT_ENOMEM, "refinement scratch: allocation failed");
    }
    return EBIT_OK;
}

// refine_kernel over the current state: per-tile flags, background colours
// (bg may be ctx scratch when the caller gives none), refined-cell count
static int refine_pass(ebit_ctx *ctx, uint8_t *mask, uint8_t *bg) {
    if (int r = amr_scratch(ctx)) return r;
    CU(cudaMemsetAsync(ctx->amr_ctr, 0, 2 * sizeof(unsigned long long), ctx->stream));
    refine_kernel<<<std::min(ctx->g.ntiles, 4 * ctx->sms), 256, 0, ctx->stream>>>(
        ctx->g, ctx->cb[ctx->cur], mask, ctx->amr_flag, bg ? bg : reinterpret_cast<uint8_t *>(ctx->amr_slot),
        ctx->amr_ctr);
    return launch_check(ctx, "refine_kernel");
}

int ebit_refine_mask(ebit_ctx *ctx, uint8_t *mask, int64_t *count) {
    if (!ctx) return EBIT_EINVAL;
    if (ctx->g.tl[0] != 3 || ctx->g.tl[1] != 3 || ctx->g.tl[2] != 3)
        return fail(ctx, EBIT_EINVAL, "ebit_refine_mask: 8^3 tiles only");
    if (int r = join_side(ctx)) return r;
    if (int r = refine_pass(ctx, mask, nullptr)) return r;
    if (count) {
        unsigned long long n = 0;
        CU(cudaMemcpyAsync(&n, ctx->amr_ctr, sizeof(n), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        *count = (int64_t)n;
    }
    return EBIT_OK;
}

int ebit_pack_bricks(ebit_ctx *ctx, int capacity, int *tiles, uint8_t *cb, double *s, uint8_t *bg, int *nbricks) {
    if (!ctx || !nbricks || capacity < 0) return fail(ctx, EBIT_EINVAL, "ebit_pack_bricks: bad argument");
    if (capacity > 0 && (!tiles || !cb || !s || !bg)) return fail(ctx, EBIT_EINVAL, "ebit_pack_bricks: null array");
    if (ctx->g.tl[0] != 3 || ctx->g.tl[1] != 3 || ctx->g.tl[2] != 3)
        return fail(ctx, EBIT_EINVAL, "ebit_pack_bricks: 8^3 tiles only");
    if (int r = join_side(ctx)) return r;
    if (int r = refine_pass(ctx, nullptr, capacity > 0 ? bg : nullptr)) return r;
    int *nb_dev = reinterpret_cast<int *>(ctx->amr_ctr + 1);
    compact_tiles_kernel<<<1, 1024, 0, ctx->stream>>>(ctx->amr_flag, ctx->g.ntiles, tiles, capacity, nb_dev);
    if (int r = launch_check(ctx, "compact_tiles_kernel")) return r;
    int n = 0;
    CU(cudaMemcpyAsync(&n, nb_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *nbricks = n;
    if (capacity == 0) return EBIT_OK;
    if (n > capacity) return fail(ctx, EBIT_EINVAL, "ebit_pack_bricks: capacity below the brick count");
    if (n > 0) {
        const int c = ctx->cur;
        pack_kernel<<<std::min(n, 8 * ctx->sms), 256, 0, ctx->stream>>>(ctx->g, ctx->cb[c], ctx->s[c][0], ctx->s[c][1],
                                                                        ctx->s[c][2], tiles, n, cb, s);
        if (int r = launch_check(ctx, "pack_kernel")) return r;
    }
    return EBIT_OK;
}

int ebit_unpack_bricks(ebit_ctx *ctx, int nbricks, const int *tiles, const uint8_t *cb, const double *s,
                       const uint8_t *bg) {
    if (!ctx || nbricks < 0 || !bg || (nbricks > 0 && (!tiles || !cb || !s)))
        return fail(ctx, EBIT_EINVAL, "ebit_unpack_bricks: bad argument");
    if (!ctx->owns_state) return fail(ctx, EBIT_EINVAL, "ebit_unpack_bricks: a batch instance's state is the batch's");
    if (int r = join_side(ctx)) return r;
    if (int r = amr_scratch(ctx)) return r;
    int *bad_dev = reinterpret_cast<int *>(ctx->amr_ctr + 1) + 1;
    CU(cudaMemsetAsync(ctx->amr_slot, 0xFF, (size_t)ctx->g.ntiles * sizeof(int), ctx->stream));
    CU(cudaMemsetAsync(bad_dev, 0, sizeof(int), ctx->stream));
    if (nbricks > 0) {
        brick_slots_kernel<<<blocks_for(nbricks, 256, ctx->sms), 256, 0, ctx->stream>>>(tiles, nbricks, ctx->g.ntiles,
                                                                                        ctx->amr_slot, bad_dev);
        if (int r = launch_check(ctx, "brick_slots_kernel")) return r;
    }
    int bad = 0;
    CU(cudaMemcpyAsync(&bad, bad_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (bad) return fail(ctx, EBIT_EINVAL, "ebit_unpack_bricks: tile id out of range");
    const int c = ctx->cur;
    unpack_kernel<<<std::min(ctx->g.ntiles, 8 * ctx->sms), 256, 0, ctx->stream>>>(
        ctx->g, ctx->amr_slot, cb, s, bg, ctx->cb[c], ctx->s[c][0], ctx->s[c][1], ctx->s[c][2]);
    if (int r = launch_check(ctx, "unpack_kernel")) return r;
    if (int r = copy_other(ctx)) return r;
    return mark_all(ctx);
}

int ebit_one_fluid(ebit_ctx *ctx, const double *C, const double *kappa_h, const uint8_t *status, double sigma,
                   double rho1, double rho2, double mu1, double mu2, double *rho, double *mu, double *force) {
    if (!ctx || !C || (force && (!kappa_h || !status))) return fail(ctx, EBIT_EINVAL, "ebit_one_fluid: null argument");
    if (!std::isfinite(sigma) || !std::isfinite(rho1) || !std::isfinite(rho2) || !std::isfinite(mu1) ||
        !std::isfinite(mu2))
        return fail(ctx, EBIT_ENONFINITE, "ebit_one_fluid: non-finite coefficient");
    if (int r = join_side(ctx)) return r;
    CouplingArgs a;
    a.g = ctx->g;
    a.C = C;
    a.kh = kappa_h;
    a.st = status;
    a.sigma = sigma;
    a.rho1 = rho1;
    a.rho2 = rho2;
    a.mu1 = mu1;
    a.mu2 = mu2;
    a.h = ctx->h;
    a.rho = rho;
    a.mu = mu;
    for (int d = 0; d < 3; d++) a.f[d] = force ? force + d * ctx->N : nullptr;
    if (!rho && !mu && !force) return EBIT_OK;
    ProfScope ps(ctx, EBIT_PROF_COUPLING, ctx->stream);
    coupling_kernel<<<std::min(ctx->g.n[1] * ctx->g.n[2], 8 * ctx->sms), 256, 0, ctx->stream>>>(a);
    return launch_check(ctx, "coupling_kernel");
}

int ebit_get_state(ebit_ctx *ctx, uint8_t *cb, double *s) {
    if (!ctx || !cb || !s) return fail(ctx, EBIT_EINVAL, "ebit_get_state: null argument");
    if (int r = join_side(ctx)) return r;
    if (!ctx->scratch && !dev_alloc(ctx->mem, (void **)&ctx->scratch, 3 * ctx->N * sizeof(double))) {
        cudaGetLastError();
        return fail(ctx, EBIT_ENOMEM, "ebit_get_state: no room for the scratch copy");
    }
    int c = ctx->cur;
    canonical_s_kernel<<<blocks_for(ctx->N, 256, ctx->sms), 256, 0, ctx->stream>>>(
        ctx->g, ctx->cb[c], ctx->s[c][0], ctx->s[c][1], ctx->s[c][2], ctx->scratch);
    int r = launch_check(ctx, "canonical_s_kernel");
    if (r) return r;
    CU(cudaMemcpyAsync(cb, ctx->cb[c], ctx->N, cudaMemcpyDefault, ctx->stream));
    CU(cudaMemcpyAsync(s, ctx->scratch, 3 * ctx->N * sizeof(double), cudaMemcpyDefault, ctx->stream));
    return ebit_sync(ctx);
}

int ebit_advect_sweep(ebit_ctx *ctx, int dir, const double *u_face, double dt) {
    if (!ctx) return EBIT_EINVAL;
    if (dir < 0 || dir > 2) return fail(ctx, EBIT_EINVAL, "ebit_advect_sweep: dir must be 0, 1 or 2");
    if (!u_face) return fail(ctx, EBIT_EINVAL, "ebit_advect_sweep: null velocity");
    if (!ctx->owns_state)
        return fail(ctx, EBIT_EINVAL, "ebit_advect_sweep: a batch instance is swept by ebit_batch_advect_sweep");
    if (!std::isfinite(dt)) return fail(ctx, EBIT_ENONFINITE, "ebit_advect_sweep: non-finite dt");
    // Band sweeps alternate between two sets of lists (see ebit_ctx): this
    // sweep reads set rd (the markers to move and the tiles with markers
    // nearby, listed by the previous sweep), builds its band into band list
    // rd from the latter, and writes set wr for the next one.  After a state
    // change, and in dense mode, every tile is processed and the markers are
    // found from the colours of each tile instead.
    // an asynchronous Front2VOF may still read the buffer this sweep writes
    if (ctx->f2v_pending && (ctx->cur ^ 1) == ctx->f2v_buf) {
        CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_f2v, 0));
        ctx->f2v_pending = 0;
    }
    const int rd = ctx->mk_par, wr = rd ^ 1;
    const bool lists = !ctx->dense && ctx->mk_valid;
    const int *list = lists ? (rd ? ctx->band_list2 : ctx->band_list) : ctx->all_list;
    const int *count = lists ? ctx->band_count + rd : ctx->all_count;
    SweepArgs a;
    a.g = ctx->g;
    int c = ctx->cur, o = c ^ 1;
    a.cb = ctx->cb[c];
    a.cbo = ctx->cb[o];
    for (int k = 0; k < 3; k++) {
        a.s[k] = ctx->s[c][k];
        a.so[k] = ctx->s[o][k];
        a.adv[k] = ctx->adv[k];
        a.bin[k] = ctx->bin[k];
    }
    unsigned *const *wk_wr = wr ? ctx->work2 : ctx->work;
    for (int k = 0; k < NLISTS; k++) a.work[k] = wk_wr[k];
    a.wcount = wr ? ctx->wcount2 : ctx->wcount;
    a.tile_next = a.wcount + NLISTS;  // one int after the list lengths
    a.u = u_face;
    a.lam = dt / ctx->h;
    a.list = list;
    a.count = count;
    a.ctr = ctx->ctr;
    a.tile_marker = ctx->tile_marker;
    a.tile_dirty = ctx->dirty_set ? ctx->tile_dirty2 : ctx->tile_dirty;
    if (!ctx->dense) {
        a.mk_out = ctx->mk_al[wr];
        a.mk_out_count = ctx->mk_count + wr;
        a.mt_out = ctx->mtiles[wr];
        a.mt_out_count = ctx->mt_count + wr;
        a.band_flag = lists ? ctx->band_flag : nullptr;
        a.band_next_count = ctx->band_count + wr;
    }
    MarkerLists ml;
    if (lists) {
        // the previous sweep's aligned markers and its unaligned work lists
        const int pd = ctx->mk_dir;
        unsigned *const *wk_rd = rd ? ctx->work2 : ctx->work;
        const int *wc_rd = rd ? ctx->wcount2 : ctx->wcount;
        ml.list[0] = ctx->mk_al[rd];
        ml.count[0] = ctx->mk_count + rd;
        ml.axis[0] = pd;
        ml.list[1] = wk_rd[0];
        ml.count[1] = wc_rd + 0;
        ml.axis[1] = (pd + 1) % 3;
        ml.list[2] = wk_rd[1];
        ml.count[2] = wc_rd + 1;
        ml.axis[2] = (pd + 2) % 3;
        ml.mtiles = ctx->mtiles[rd];
        ml.mtiles_count = ctx->mt_count + rd;
        ml.band = rd ? ctx->band_list2 : ctx->band_list;
        ml.band_count = ctx->band_count + rd;
    }
    int r;
    switch (dir) {
    case 0: r = sweep_launch<0>(ctx, a, lists ? &ml : nullptr); break;
    case 1: r = sweep_launch<1>(ctx, a, lists ? &ml : nullptr); break;
    default: r = sweep_launch<2>(ctx, a, lists ? &ml : nullptr); break;
    }
    if (r) return r;
    ctx->band_last = lists ? rd : -1;
    if (!ctx->dense) {
        ctx->mk_par = wr;
        ctx->mk_dir = dir;
        ctx->mk_valid = 1;
    }
    if (r) return r;
    ctx->cur = o;
    ctx->sweeps_since_f2v++;
    return EBIT_OK;
}

int ebit_front2vof(ebit_ctx *ctx, double *C, int flags) {
    if (!ctx || !C) return fail(ctx, EBIT_EINVAL, "ebit_front2vof: null argument");
    const int *list, *count;
    bool full = (flags & EBIT_FULL) || ctx->dense || C != ctx->last_C;
    // nothing was swept since the last call on this buffer: C is current
    if (!full && ctx->sweeps_since_f2v == 0) return EBIT_OK;
    cudaStream_t st;
    if (int r = call_stream(ctx, flags, &st)) return r;
    // this call consumes the dirty set the sweeps since the last call marked;
    // the next sweeps mark the other one (a batch view has one set)
    uint8_t *dirty = ctx->dirty_set ? ctx->tile_dirty2 : ctx->tile_dirty;
    if (ctx->tile_dirty2) ctx->dirty_set ^= 1;
    if (full) {
        CU(cudaMemsetAsync(ctx->ncut, 0, sizeof(int), st));
        CU(cudaMemsetAsync(dirty, 0, ctx->g.ntiles, st));
        list = ctx->all_list;
        count = ctx->all_count;
    } else {
        // work_count[fp] is 0; the tile-list kernel clears the other slot for
        // the next incremental call, and the cut-cell count (its readers, the
        // previous Front2VOF and curvature, are complete)
        ProfScope ps(ctx, EBIT_PROF_F2V, st);
        const int fp = ctx->f2v_par;
        int r = launched(ctx,
                         launch_pdl(take_flagged_kernel, blocks_for(ctx->g.ntiles, 256, ctx->sms), 256, 0, st,
                                    ctx->g, dirty, ctx->work_list, ctx->work_count + fp,
                                    ctx->work_count + (fp ^ 1), ctx->ncut),
                         "take_flagged_kernel");
        if (r) return r;
        list = ctx->work_list;
        count = ctx->work_count + fp;
        ctx->f2v_par = fp ^ 1;
    }
    F2VArgs a;
    a.g = ctx->g;
    int c = ctx->cur;
    a.cb = ctx->cb[c];
    for (int k = 0; k < 3; k++) a.s[k] = ctx->s[c][k];
    a.C = C;
    a.list = list;
    a.count = count;
    a.cut = ctx->cut;
    a.ncut = ctx->ncut;
    a.bad = ctx->ctr + C_F2V_BAD;
    int r;
    {
        ProfScope ps(ctx, EBIT_PROF_F2V, st);
        r = launched(ctx, launch_pdl(f2v_band_kernel, ctx->grid_f2v, 256, 0, st, a), "f2v_band_kernel");
    }
    if (r) return r;
    {
        ProfScope ps(ctx, EBIT_PROF_F2V, st);
        r = launched(ctx, launch_pdl(f2v_list_kernel, ctx->grid_f2vl, 128, 0, st, a), "f2v_list_kernel");
    }
    if (r) return r;
    if (st != ctx->stream) {
        // the sweep that overwrites state buffer c waits for this event
        CU(cudaEventRecord(ctx->ev_f2v, st));
        ctx->f2v_pending = 1;
        ctx->f2v_buf = c;
    }
    ctx->last_C = C;
    ctx->sweeps_since_f2v = 0;
    return EBIT_OK;
}

int ebit_curvature(ebit_ctx *ctx, const double *C, double *kappa_h, uint8_t *status, int mode, int flags) {
    if (!ctx || !C || !kappa_h || !status) return fail(ctx, EBIT_EINVAL, "ebit_curvature: null argument");
    if (mode != EBIT_CURV_HF && mode != EBIT_CURV_MLP && mode != EBIT_CURV_MLP_HF)
        return fail(ctx, EBIT_EINVAL, "ebit_curvature: unknown mode");
    if (mode != EBIT_CURV_HF && !ctx->mlp) return fail(ctx, EBIT_EINVAL, "ebit_curvature: no network (ebit_set_mlp)");
    bool full = (flags & EBIT_FULL) || ctx->dense || C != ctx->last_C || kappa_h != ctx->last_kh ||
                status != ctx->last_st;
    cudaStream_t st;
    if (int r = call_stream(ctx, flags, &st)) return r;
    const int nw = ctx->cur_if ^ 1;
    // list lengths rotate over three slots: this call appends to slot cs
    // (0, cleared by the previous call), reads the previous call's length in
    // slot cprev, and clears slot cnext (last read by the previous call) for
    // the next call
    const int cs = ctx->if_slot, cnext = (cs + 1) % 3, cprev = (cs + 2) % 3;
    HFArgs a;
    a.g = ctx->g;
    a.C = C;
    a.kh = kappa_h;
    a.st = status;
    a.iface = ctx->iface[nw];
    a.niface = ctx->niface + cs;
    a.list = ctx->all_list;
    a.count = ctx->all_count;
    a.zero[0] = ctx->niface + cnext;
    a.zero[1] = nullptr;
    if (full) {
        // any C: scan every tile, reset non-interface cells, list the interface cells
        ProfScope ps(ctx, EBIT_PROF_SCAN, st);
        CU(cudaMemsetAsync(ctx->nscan, 0, sizeof(int), st));
        int r = launched(ctx, launch_pdl(hf_scan_kernel, ctx->grid_hf, 256, 0, st, a, ctx->scan, ctx->nscan),
                         "hf_scan_kernel");
        if (r) return r;
        a.prev = ctx->iface[ctx->cur_if];
        a.nprev = ctx->zero;
        a.cand = ctx->scan;
        a.ncand = ctx->nscan;
    } else {
        // C is this context's Front2VOF output: its cut cells hold every interface cell
        a.prev = ctx->iface[ctx->cur_if];
        a.nprev = ctx->niface + cprev;
        a.cand = ctx->cut;
        a.ncand = ctx->ncut;
        // the fallback list of the learned pass below starts empty
        if (mode != EBIT_CURV_HF) a.zero[1] = ctx->nscan;
    }
    {
        // height functions on every interface cell (mode HF), or only the list
        ProfScope ps(ctx, EBIT_PROF_HF, st);
        cudaError_t e = (mode == EBIT_CURV_HF)
                            ? launch_pdl(hf_list_kernel<true>, ctx->grid_hfl, 128, 0, st, a)
                            : launch_pdl(hf_list_kernel<false>, ctx->grid_hfl, 128, 0, st, a);
        int r = launched(ctx, e, "hf_list_kernel");
        if (r) return r;
    }
    if (mode != EBIT_CURV_HF) {
        // learned curvature on this call's interface cells (height functions
        // where it falls back, mode MLP_HF)
        MlpArgs m{};
        m.g = ctx->g;
        m.C = C;
        m.cells = reinterpret_cast<const int *>(ctx->iface[nw]);
        m.ncells = ctx->niface + cs;
        m.params = ctx->mlp->p;
        m.w1b = ctx->mlp->w1b;
        m.w2b = ctx->mlp->w2b;
        m.kh = kappa_h;
        m.st = status;
        m.mode = mode;
        m.fb = ctx->scan;  // free again: the listing pass above has consumed it
        m.nfb = ctx->nscan;
        if (full) CU(cudaMemsetAsync(ctx->nscan, 0, sizeof(int), st));
        int r;
        {
            ProfScope pm(ctx, EBIT_PROF_MLP, st);
            m.err = ctx->mlp->err;
            cudaError_t e =
                (ctx->mlp->path == EBIT_MLP_PATH_TCGEN05)
                    ? launch_pdl(mlp_fwd_tc_kernel<true, true>, ctx->sms, TC_THREADS, FWD_TC_SMEM, st, m)
                    : launch_pdl(mlp_fwd_kernel<true, true>, ctx->mlp->fwd_blocks * ctx->sms, 128, FWD_SMEM,
                                 st, m);
            r = launched(ctx, e, "mlp_fwd_kernel");
        }
        if (r) return r;
        if (mode == EBIT_CURV_MLP_HF) {
            // height functions on the cells the learned value left to them
            HFArgs f = a;
            f.prev = ctx->iface[ctx->cur_if];
            f.nprev = ctx->zero;
            f.cand = ctx->scan;
            f.ncand = ctx->nscan;
            f.iface = nullptr;
            f.niface = nullptr;
            f.zero[0] = f.zero[1] = nullptr;
            ProfScope pf(ctx, EBIT_PROF_MLP, st);
            r = launched(ctx, launch_pdl(hf_list_kernel<true>, ctx->grid_hfl, 128, 0, st, f),
                         "hf_list_kernel");
            if (r) return r;
        }
    }
    ctx->cur_if = nw;
    ctx->if_slot = cnext;
    ctx->last_kh = kappa_h;
    ctx->last_st = status;
    return EBIT_OK;
}

int ebit_counters(ebit_ctx *ctx, ebit_counters_t *out) {
    if (!ctx || !out) return fail(ctx, EBIT_EINVAL, "ebit_counters: null argument");
    if (int r = join_side(ctx)) return r;
    unsigned long long h[C_TOTAL];
    CU(cudaMemcpyAsync(h, ctx->ctr, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    out->markers = (int64_t)h[C_MARKERS];
    out->annihilate = (int64_t)h[C_ANNIHILATE];
    out->multi = (int64_t)h[C_MULTI];
    out->inconsistent = (int64_t)h[C_INCONSISTENT] + (int64_t)h[C_F2V_BAD];
    out->cfl = (int64_t)h[C_CFL];
    out->tiles = (int64_t)h[C_TILES];
    out->nonfinite = (int64_t)h[C_NONFINITE];
    if (out->nonfinite) return fail(ctx, EBIT_ENONFINITE, "a marker's displacement was not finite (NaN or infinite velocity)");
    if (out->cfl) return fail(ctx, EBIT_ECFL, "a marker moved a full cell or more in one sweep");
    return out->inconsistent ? EBIT_WINCONSISTENT : EBIT_OK;
}

int ebit_reset_counters(ebit_ctx *ctx) {
    if (!ctx) return EBIT_EINVAL;
    if (int r = join_side(ctx)) return r;
    CU(cudaMemsetAsync(ctx->ctr, 0, C_TOTAL * sizeof(unsigned long long), ctx->stream));
    return EBIT_OK;
}

int ebit_join(ebit_ctx *ctx) {
    if (!ctx) return EBIT_EINVAL;
    return join_side(ctx);
}

int ebit_event_record(ebit_ctx *ctx, void *cuda_event) {
    if (!ctx || !cuda_event) return fail(ctx, EBIT_EINVAL, "ebit_event_record: null argument");
    CU(cudaEventRecord((cudaEvent_t)cuda_event, ctx->side_pending ? ctx->side : ctx->stream));
    return EBIT_OK;
}

int ebit_sync(ebit_ctx *ctx) {
    if (!ctx) return EBIT_EINVAL;
    if (int r = join_side(ctx)) return r;
    unsigned long long h[C_TOTAL];
    CU(cudaMemcpyAsync(h, ctx->ctr, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    // a non-finite velocity is reported before the CFL error it would also trip
    if (h[C_NONFINITE]) return fail(ctx, EBIT_ENONFINITE, "a marker's displacement was not finite (NaN or infinite velocity)");
    if (h[C_CFL]) return fail(ctx, EBIT_ECFL, "a marker moved a full cell or more in one sweep");
    return EBIT_OK;
}

int ebit_band_tiles(ebit_ctx *ctx) {
    if (!ctx) return -1;
    if (ctx->dense || ctx->band_last < 0) return ctx->g.ntiles;
    int n = -1;
    if (cudaMemcpyAsync(&n, ctx->band_count + ctx->band_last, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return -1;
    return n;
}

int ebit_profile(ebit_ctx *ctx, int enable) {
    if (!ctx) return EBIT_EINVAL;
    if (enable && ctx->ev.empty()) {
        ctx->ev.resize(2 * 16384);
        ctx->ev_kind.resize(16384);
        for (auto &e : ctx->ev) CU(cudaEventCreate(&e));
    }
    int r = prof_drain(ctx);
    if (r) return r;
    ctx->prof_on = enable ? 1 : 0;
    for (int k = 0; k < EBIT_PROF_KINDS; k++) {
        ctx->prof_ms[k] = 0.0;
        ctx->prof_n[k] = 0;
    }
    return EBIT_OK;
}

int ebit_profile_read(ebit_ctx *ctx, double *ms, int64_t *launches) {
    if (!ctx || !ms || !launches) return fail(ctx, EBIT_EINVAL, "ebit_profile_read: null argument");
    int r = prof_drain(ctx);
    if (r) return r;
    for (int k = 0; k < EBIT_PROF_KINDS; k++) {
        ms[k] = ctx->prof_ms[k];
        launches[k] = ctx->prof_n[k];
    }
    return EBIT_OK;
}

int ebit_set_mlp(ebit_ctx *ctx, ebit_mlp *mlp) {
    if (!ctx) return EBIT_EINVAL;
    ctx->mlp = mlp;
    return EBIT_OK;
}

int ebit_mlp_load(ebit_ctx *ctx, const void *weights, size_t bytes) {
    if (!ctx || !weights) return fail(ctx, EBIT_EINVAL, "ebit_mlp_load: null argument");
    if (bytes != (size_t)MLP_NP * sizeof(float))
        return fail(ctx, EBIT_EINVAL, "ebit_mlp_load: expected ebit_mlp_nparams() floats");
    if (!ctx->own_mlp) {
        int r = ebit_mlp_create(ctx->stream, &ctx->own_mlp);
        if (r) return fail(ctx, r, "ebit_mlp_load: could not create the network");
    }
    int r = ebit_mlp_set_params(ctx->own_mlp, static_cast<const float *>(weights));
    if (r) return fail(ctx, r, std::string("ebit_mlp_load: ") + ebit_mlp_last_error(ctx->own_mlp));
    ctx->mlp = ctx->own_mlp;
    return EBIT_OK;
}

// ------------------------------------------------------- learned curvature
#define MCU(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) {                                                                           \
            mlp->errmsg = std::string(#call ": ") + cudaGetErrorString(e_);                               \
            return EBIT_ECUDA;                                                                             \
        }                                                                                                  \
    } while (0)

static bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

int ebit_mlp_nparams(void) { return MLP_NP; }

int ebit_mlp_create(void *cuda_stream, ebit_mlp **out) {
    if (!out) return EBIT_EINVAL;
    *out = nullptr;
    ebit_mlp *mlp = new ebit_mlp();
    mlp->stream = (cudaStream_t)cuda_stream;
    mlp->p = mlp->g = mlp->m = mlp->v = mlp->loss = nullptr;
    mlp->w1b = mlp->w2b = nullptr;
    mlp->err = nullptr;
    mlp->step = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&mlp->sms, cudaDevAttrMultiProcessorCount, dev);
    mlp->mem = current_devmem();
    const DevMem &mm = mlp->mem;
    bool ok = dev_alloc(mm, (void **)&mlp->p, MLP_NP * 4) && dev_alloc(mm, (void **)&mlp->g, MLP_NP * 4) &&
              dev_alloc(mm, (void **)&mlp->m, MLP_NP * 4) && dev_alloc(mm, (void **)&mlp->v, MLP_NP * 4) &&
              dev_alloc(mm, (void **)&mlp->w1b, MLP_H * MLP_IN * 2) &&
              dev_alloc(mm, (void **)&mlp->w2b, MLP_H * MLP_H * 2) && dev_alloc(mm, (void **)&mlp->loss, 8) &&
              dev_alloc(mm, (void **)&mlp->err, 4);
    if (!ok) {
        cudaGetLastError();
        ebit_mlp_destroy(mlp);
        return EBIT_ENOMEM;
    }
    if (cudaFuncSetAttribute(mlp_fwd_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(mlp_fwd_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TRAIN_SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(mlp_fwd_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             FWD_TC_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_fwd_tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             FWD_TC_SMEM) != cudaSuccess) {
        cudaGetLastError();
        ebit_mlp_destroy(mlp);
        return EBIT_ECUDA;
    }
    mlp->fwd_blocks = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mlp->fwd_blocks, mlp_fwd_kernel<true, true>, 128, FWD_SMEM);
    mlp->fwd_blocks = std::max(1, mlp->fwd_blocks);
    mlp->fwd_tc_blocks = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mlp->fwd_tc_blocks, mlp_fwd_tc_kernel<true, true>, TC_THREADS,
                                                  FWD_TC_SMEM);
    // a block holds all 512 TMEM columns (one per SM)
    mlp->fwd_tc_blocks = 1;
    mlp->path = EBIT_MLP_PATH_TCGEN05;
    cudaMemsetAsync(mlp->err, 0, sizeof(int), mlp->stream);
    cudaMemsetAsync(mlp->loss, 0, 8, mlp->stream);  // a training step starts from a cleared loss
    cudaMemsetAsync(mlp->p, 0, MLP_NP * 4, mlp->stream);
    cudaMemsetAsync(mlp->g, 0, MLP_NP * 4, mlp->stream);
    cudaMemsetAsync(mlp->m, 0, MLP_NP * 4, mlp->stream);
    cudaMemsetAsync(mlp->v, 0, MLP_NP * 4, mlp->stream);
    if (cudaGetLastError() != cudaSuccess) {
        ebit_mlp_destroy(mlp);
        return EBIT_ECUDA;
    }
    *out = mlp;
    return EBIT_OK;
}

void ebit_mlp_destroy(ebit_mlp *mlp) {
    if (!mlp) return;
    cudaStreamSynchronize(mlp->stream);
    dev_free(mlp->mem, mlp->p);
    dev_free(mlp->mem, mlp->g);
    dev_free(mlp->mem, mlp->m);
    dev_free(mlp->mem, mlp->v);
    dev_free(mlp->mem, mlp->w1b);
    dev_free(mlp->mem, mlp->w2b);
    dev_free(mlp->mem, mlp->loss);
    dev_free(mlp->mem, mlp->err);
    delete mlp;
}

int ebit_mlp_set_params(ebit_mlp *mlp, const float *params) {
    if (!mlp || !params) return EBIT_EINVAL;
    MCU(cudaMemcpyAsync(mlp->p, params, MLP_NP * 4, cudaMemcpyDefault, mlp->stream));
    MCU(cudaMemsetAsync(mlp->g, 0, MLP_NP * 4, mlp->stream));
    MCU(cudaMemsetAsync(mlp->m, 0, MLP_NP * 4, mlp->stream));
    MCU(cudaMemsetAsync(mlp->v, 0, MLP_NP * 4, mlp->stream));
    mlp->step = 0;
    mlp_cast_kernel<<<(MLP_NP + 255) / 256, 256, 0, mlp->stream>>>(mlp->p, mlp->w1b, mlp->w2b);
    MCU(cudaGetLastError());
    return EBIT_OK;
}

int ebit_mlp_get_params(ebit_mlp *mlp, float *params) {
    if (!mlp || !params) return EBIT_EINVAL;
    MCU(cudaMemcpyAsync(params, mlp->p, MLP_NP * 4, cudaMemcpyDefault, mlp->stream));
    MCU(cudaStreamSynchronize(mlp->stream));
    return EBIT_OK;
}

int ebit_selftest_f64_to_f32(const double *in, float *out, int n, void *cuda_stream) {
    if (!in || !out || n < 0) return EBIT_EINVAL;
    if (n == 0) return EBIT_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    f64_to_f32_kernel<<<std::min((n + 255) / 256, 4 * std::max(sms, 1)), 256, 0, (cudaStream_t)cuda_stream>>>(in, out, n);
    return cudaGetLastError() == cudaSuccess ? EBIT_OK : EBIT_ECUDA;
}

int ebit_mlp_gather(ebit_mlp *mlp, const double *C, int nx, int ny, int nz, const int *cells, int m, uint16_t *X,
                    uint8_t *frag) {
    if (!mlp || !C || !cells || !X || m < 0 || nx < 8 || ny < 8 || nz < 8 || !aligned16(X)) return EBIT_EINVAL;
    if (m == 0) return EBIT_OK;
    Grid g{};
    g.n[0] = nx;
    g.n[1] = ny;
    g.n[2] = nz;
    mlp_gather_kernel<<<std::min((m + 127) / 128, 8 * mlp->sms), 128, 0, mlp->stream>>>(
        C, g, cells, m, reinterpret_cast<__nv_bfloat16 *>(X), frag);
    MCU(cudaGetLastError());
    return EBIT_OK;
}

int ebit_mlp_forward(ebit_mlp *mlp, const uint16_t *X, int m, float *y) {
    if (!mlp || !X || !y || m < 0 || !aligned16(X)) return EBIT_EINVAL;
    if (m == 0) return EBIT_OK;
    MlpArgs a{};
    a.X = reinterpret_cast<const __nv_bfloat16 *>(X);
    a.m = m;
    a.ncells = nullptr;
    a.params = mlp->p;
    a.w1b = mlp->w1b;
    a.w2b = mlp->w2b;
    a.y = y;
    const int ntile = (m + 127) / 128;
    a.err = mlp->err;
    if (mlp->path == EBIT_MLP_PATH_TCGEN05)
        mlp_fwd_tc_kernel<false, false><<<std::min((ntile + TC_GROUPS - 1) / TC_GROUPS, mlp->sms), TC_THREADS,
                                          FWD_TC_SMEM, mlp->stream>>>(a);
    else
        mlp_fwd_kernel<false, false><<<std::min(ntile, mlp->fwd_blocks * mlp->sms), 128, FWD_SMEM, mlp->stream>>>(a);
    MCU(cudaGetLastError());
    return EBIT_OK;
}

// mlp->loss[0] is 0 on entry: cleared at creation, by the Adam kernel of each
// training step and at the end of ebit_mlp_gradient
static int mlp_grad_launch(ebit_mlp *mlp, const uint16_t *X, const float *t, const int *idx, int batch) {
    MlpArgs a{};
    a.X = reinterpret_cast<const __nv_bfloat16 *>(X);
    a.t = t;
    a.idx = idx;
    a.batch = batch;
    a.params = mlp->p;
    a.w1b = mlp->w1b;
    a.w2b = mlp->w2b;
    a.grad = mlp->g;
    a.loss = mlp->loss;
    const int ntile = (batch + 127) / 128;
    mlp_train_kernel<<<std::min(ntile, mlp->sms), TRAIN_THREADS, TRAIN_SMEM, mlp->stream>>>(a);
    MCU(cudaGetLastError());
    return EBIT_OK;
}

int ebit_mlp_gradient(ebit_mlp *mlp, const uint16_t *X, const float *t, int batch, float *grad_out) {
    if (!mlp || !X || !t || !grad_out || batch <= 0 || !aligned16(X)) return EBIT_EINVAL;
    MCU(cudaMemsetAsync(mlp->g, 0, MLP_NP * 4, mlp->stream));
    int r = mlp_grad_launch(mlp, X, t, nullptr, batch);
    if (r) return r;
    MCU(cudaMemcpyAsync(grad_out, mlp->g, MLP_NP * 4, cudaMemcpyDefault, mlp->stream));
    MCU(cudaMemsetAsync(mlp->g, 0, MLP_NP * 4, mlp->stream));
    MCU(cudaMemsetAsync(mlp->loss, 0, 4, mlp->stream));
    return EBIT_OK;
}

int ebit_mlp_train_step(ebit_mlp *mlp, const uint16_t *X, const float *t, const int *idx, int batch, float lr,
                        float *loss_out) {
    if (!mlp || !X || !t || batch <= 0 || !(lr > 0.0f) || !aligned16(X)) return EBIT_EINVAL;
    int r = mlp_grad_launch(mlp, X, t, idx, batch);
    if (r) return r;
    mlp->step++;
    const float bc1 = 1.0f - powf(0.9f, (float)mlp->step), bc2 = 1.0f - powf(0.999f, (float)mlp->step);
    // a device loss_out is written by the Adam kernel itself; a host one is
    // copied from the second loss slot after it
    bool dev_out = false;
    if (loss_out) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, loss_out) == cudaSuccess)
            dev_out = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
        cudaGetLastError();
    }
    float *dst = loss_out ? (dev_out ? loss_out : mlp->loss + 1) : nullptr;
    mlp_adam_kernel<<<(MLP_NP + 255) / 256, 256, 0, mlp->stream>>>(mlp->p, mlp->g, mlp->m, mlp->v, mlp->w1b, mlp->w2b,
                                                                  lr, bc1, bc2, mlp->loss, dst);
    MCU(cudaGetLastError());
    if (loss_out && !dev_out) MCU(cudaMemcpyAsync(loss_out, mlp->loss + 1, 4, cudaMemcpyDefault, mlp->stream));
    return EBIT_OK;
}

int ebit_mlp_sync(ebit_mlp *mlp) {
    if (!mlp) return EBIT_EINVAL;
    int e = 0;
    MCU(cudaMemcpyAsync(&e, mlp->err, sizeof(int), cudaMemcpyDeviceToHost, mlp->stream));
    MCU(cudaStreamSynchronize(mlp->stream));
    if (e) {
        mlp->errmsg = e == 2 ? "tensor memory allocation outside the expected range" : "a tensor-core wait gave up";
        return EBIT_ETIMEOUT;
    }
    return EBIT_OK;
}

int ebit_mlp_set_path(ebit_mlp *mlp, int path) {
    if (!mlp || (path != EBIT_MLP_PATH_MMA && path != EBIT_MLP_PATH_TCGEN05)) return EBIT_EINVAL;
    mlp->path = path;
    return EBIT_OK;
}

const char *ebit_mlp_last_error(const ebit_mlp *mlp) { return mlp ? mlp->errmsg.c_str() : "null network"; }

const char *ebit_last_error(const ebit_ctx *ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

}  // extern "C"
