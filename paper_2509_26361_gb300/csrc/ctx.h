// ctx.h -- the library's internal context types, shared by its translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ebit.h"
#include "common.cuh"
#include "devmem.h"

using ebit::Grid;

// work lists of a context's sweep: unaligned edges and saddle faces of the two
// face families, and the annihilation checks of the two families
constexpr int NLISTS = 6;

struct ebit_mlp {
    ebit::DevMem mem;  // the allocator the network was created with
    cudaStream_t stream;
    int sms;
    float *p, *g, *m, *v;      // FP32 parameters, gradient, Adam moments
    __nv_bfloat16 *w1b, *w2b;  // bf16 copies for the tensor cores
    float *loss;               // summed weighted squared error of the last step
    int step;
    int fwd_blocks;            // co-resident forward blocks per SM (warp-level MMA kernel)
    int fwd_tc_blocks;         // the same for the tcgen05 kernel
    int path;                  // EBIT_MLP_PATH_MMA or EBIT_MLP_PATH_TCGEN05
    int *err;                  // set by a tcgen05 kernel whose bounded wait gave up
    std::string errmsg;
};

struct ebit_ctx {
    ebit::DevMem mem;  // the allocator the context was created with
    Grid g;
    int nt_cap;        // tiles the per-tile arrays hold (a batch instance: any tile shape)
    int owns_state;           // 0: cb, s, scratch arrays, tile flags and counters belong to a batch
    long long N;
    double h;
    cudaStream_t stream;
    int dense;
    int sms;
    uint8_t *cb[2];
    double *s[2][3];
    int cur;
    uint32_t *tile_marker;    // per tile: proximity mask of its markers (see near_bits)
    uint8_t *tile_dirty, *tile_cchg;
    // Front2VOF and curvature may run on a side stream (EBIT_ASYNC), overlapping
    // the next sweeps.  The sweeps mark processed tiles in dirty set dirty_set;
    // each Front2VOF call consumes that set and the next sweeps mark the other
    // (tile_dirty2 is set 1; a batch view keeps one set).
    uint8_t *tile_dirty2;
    int dirty_set;
    cudaStream_t side;        // created on the first EBIT_ASYNC call
    cudaEvent_t ev_main, ev_side, ev_f2v;
    int side_pending;         // side-stream work not yet joined into the main stream
    int f2v_pending;          // an async Front2VOF may still read state buffer f2v_buf
    int f2v_buf;
    int *band_list, *band_count;  // band_count[2]: the lengths of band_list and band_list2
    int band_last;                // slot of the last sweep's band list (-1: every tile)
    int *work_list, *work_count;  // work_count[2]: one slot per incremental Front2VOF parity
    int f2v_par;
    int *all_list, *all_count;
    unsigned long long *ctr;  // C_N event counters + Front2VOF inconsistencies
    double *scratch;          // 3N doubles, allocated on first ebit_get_state
    int *amr_flag;            // per tile: holds a refined cell (ebit_refine_mask / ebit_pack_bricks), lazily
    int *amr_slot;            // per tile: its brick in a store being unpacked, or -1, lazily
    unsigned long long *amr_ctr;  // refined cells | brick count, ids out of range (two ints)
    double *adv[3];           // advected marker coordinates of the current sweep (scratch)
    int8_t *bin[3];           // floor(2 adv) (scratch)
    unsigned *work[NLISTS];   // work lists of a sweep (scratch; a batch view has the first 4)
    int *wcount;              // [NLISTS] list lengths ([4] in a batch view), then the band pass's tile counter
    // A context's band sweeps alternate between two sets of lists: a sweep
    // reads set mk_par (the markers and band the previous sweep listed) and
    // writes set mk_par ^ 1.  Set 0 is work/wcount above, set 1 work2/wcount2.
    unsigned *work2[NLISTS];
    int *wcount2;
    unsigned *mk_al[2];       // aligned edges that carry a marker, per set
    int *mk_count;            // [2] their lengths
    int *mtiles[2];           // tiles whose proximity mask is not empty, per set
    int *mt_count;            // [2] their lengths
    int *band_list2;          // the band list of set 1 (set 0: band_list)
    uint32_t *band_flag;      // per tile: in the band list being built or processed
    int mk_par;               // set written by the last sweep
    int mk_dir;               // sweep axis of the last sweep
    int mk_valid;             // the lists of set mk_par describe the current state
    unsigned *cut;            // cells cut by the interface at the last Front2VOF
    int *ncut;
    unsigned *iface[2];       // interface cells of the last two curvature calls
    int *niface;              // [3] list lengths, one slot per curvature call modulo 3
    int cur_if;               // list buffer of the last curvature call
    int if_slot;              // length slot of the next call (0 on entry)
    unsigned *scan;           // interface cells found by a full curvature scan
    int *nscan;
    int *zero;                // a device int that stays 0
    int sweeps_since_f2v;
    ebit_mlp *mlp;            // learned curvature (ebit_set_mlp or ebit_mlp_load)
    ebit_mlp *own_mlp;        // the network ebit_mlp_load made (owned)
    const double *last_C;
    const double *last_kh;
    const uint8_t *last_st;
    int grid_sweep, grid_adv, grid_advl, grid_fp64, grid_f2v, grid_f2vl, grid_hf, grid_hfl;
    // per-kernel CUDA-event timing (ebit_profile)
    int prof_on;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    int ev_used;
    double prof_ms[EBIT_PROF_KINDS];
    long long prof_n[EBIT_PROF_KINDS];
    std::string err;
};


// Per-sweep state arrays that a batch provides for its instances (an
// instance's context then owns only its Front2VOF and curvature scratch).
struct ebit_state_arrays {
    uint8_t *cb[2];
    double *s[2][3];
    double *adv[3];
    int8_t *bin[3];
    unsigned *work[4];
    int *wcount;
    uint32_t *tile_marker;
    uint8_t *tile_dirty;
    unsigned long long *ctr;
};

// A context over batch-owned state arrays (see ebit_create for the rest).
int ebit_create_view(const ebit_desc *desc, const ebit_state_arrays *st, ebit_ctx **out);

// Re-tile a batch instance with tile shape sh (its batch passes the slices of
// its tile tables for that shape): the tile counts, the list of all tiles,
// and every tile marked for the next sweep and Front2VOF.  EBIT_EINVAL if the
// shape needs more tiles than the context's arrays hold.
int ctx_retile(ebit_ctx *ctx, int sh, uint32_t *tile_marker, uint8_t *tile_dirty);
