/*
 * ebit.h -- C ABI of the GB300 EBIT kinematics library (libebit.so).
 *
 * The library advances an interface represented by the 3D Edge-Based Interface
 * Tracking method (arxiv 2509.26361) on a uniform periodic N^3 grid:
 *   - one marker per grid edge, stored as an FP64 offset along the edge;
 *   - a colour-vertex field at the cell corners and face centres that encodes
 *     the marker connectivity (Sec. 2.2, Fig. 7b);
 *   - split advection: each sweep moves the markers along one axis and
 *     rebuilds the unaligned markers by circle fits on the two face families
 *     that contain that axis (Sec. 2.1 Eqs. 1-2, Fig. 1, Fig. 2; Sec. 2.3 Fig. 6);
 *   - Front2VOF volume fractions (Sec. 2.6, Eq. 7) and height-function
 *     curvature from them (Sec. 2.6).
 *
 * Conventions shared by every call.
 *   Grid: nx, ny, nz cells, periodic on every axis, each >= 8.  Node (i,j,k) is
 *     the lowest corner of cell (i,j,k); linear index idx = (k*ny + j)*nx + i.
 *     The a-edge of node idx joins it to the next node along axis a (a = 0,1,2
 *     for x,y,z).  The a-face of node idx is the face normal to a whose lowest
 *     corner is node idx.  A velocity component u_a lives at the centres of the
 *     a-faces (MAC layout).
 *   State (owned by the context, on the device): one colour byte per node --
 *     bit 0 the node colour (1 = reference phase), bit 1+a the colour of the
 *     a-face (stored for saddle faces, i.e. faces with a marker on all four
 *     edges; any other face stores its lowest corner's colour) -- and three
 *     FP64 arrays s[a][idx], the marker offset in [0, 1) of the a-edge of node
 *     idx, in units of that edge.  An edge carries a marker iff the colours of
 *     its two end nodes differ; the offset of an edge without a marker is
 *     unspecified inside the context and reads back as 0.
 *   Pointers: unless stated otherwise every array argument is a DEVICE pointer
 *     (cudaMalloc or torch) of the documented size, borrowed for the duration
 *     of the call and used in stream order on the context's stream.  The
 *     caller keeps ownership.  All arrays are dense, C-contiguous, idx-ordered;
 *     arrays of three families are family-major ([a][idx]).
 *   Errors: every call returns an int status; 0 = EBIT_OK, negative = error,
 *     positive = warning.  No exception, abort or exit crosses the ABI.  A
 *     failed call leaves a message readable with ebit_last_error().  Errors
 *     found on the device (CFL >= 1 at a marker, a device wait that gave up)
 *     are raised by the next call that synchronises (ebit_sync,
 *     ebit_counters, ebit_get_state).
 */
#ifndef EBIT_H
#define EBIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    EBIT_OK = 0,
    EBIT_EINVAL = -1,     /* bad argument: dir, sizes, null pointer, non-finite dt */
    EBIT_ENONFINITE = -2, /* non-finite data where finite data is required */
    EBIT_ECUDA = -3,      /* a CUDA runtime call failed */
    EBIT_ETIMEOUT = -4,   /* a bounded device wait gave up */
    EBIT_ENOMEM = -5,     /* device allocation failed */
    EBIT_ECFL = -6,       /* a marker moved a full cell or more in one sweep */
    EBIT_WINCONSISTENT = 1 /* consistency counters are non-zero (warning) */
};

/* flags for ebit_front2vof / ebit_curvature (EBIT_ASYNC may be OR-ed in) */
enum {
    EBIT_INCREMENTAL = 0, /* recompute only the cells the sweeps may have changed */
    EBIT_FULL = 1,        /* recompute every cell */
    EBIT_ASYNC = 2        /* run on the context's side stream (see ebit_join) */
};

/* curvature modes */
enum {
    EBIT_CURV_HF = 0,     /* height functions only */
    EBIT_CURV_MLP = 1,    /* learned curvature only (needs ebit_mlp_load) */
    EBIT_CURV_MLP_HF = 2  /* learned curvature, height functions where it falls back */
};

/* height-function status codes written by ebit_curvature */
enum {
    EBIT_ST_NONE = 0,     /* not an interface cell (C is 0 or 1); kappa*h = 0 */
    EBIT_ST_HF_X = 1,     /* heights along x */
    EBIT_ST_HF_Y = 2,     /* heights along y */
    EBIT_ST_HF_Z = 3,     /* heights along z */
    EBIT_ST_NO_HF = 4,    /* no consistent 3x3 stencil of 9-cell columns; kappa*h = 0 */
    EBIT_ST_MLP = 5       /* learned curvature */
};

typedef struct ebit_ctx ebit_ctx;

typedef struct {
    int nx, ny, nz;    /* cells per axis, periodic, each >= 8 */
    double h;          /* cell size (> 0); dt/h is the sweep's CFL factor */
    void *cuda_stream; /* cudaStream_t used for every launch; NULL = legacy default stream.
                          The kernels of a sweep, Front2VOF and curvature are launched with
                          programmatic stream serialization: each waits for the preceding
                          kernel on the stream to complete before it touches memory, so
                          stream order holds as for ordinary launches. */
    int flags;         /* EBIT_DESC_DENSE: process every tile on every call (no band) */
} ebit_desc;

enum { EBIT_DESC_DENSE = 1 };

typedef struct {
    int64_t markers;      /* markers present after the last sweep, summed over sweeps */
    int64_t annihilate;   /* edges where an even number (>= 2) of markers met (Fig. 5) */
    int64_t multi;        /* edges where three markers met; the median was kept */
    int64_t inconsistent; /* colour/crossing parity disagreements (never expected) */
    int64_t cfl;          /* marker displacements of a full cell or more (error) */
    int64_t tiles;        /* 512-cell tiles processed by the sweeps (band size, summed) */
    int64_t nonfinite;    /* markers whose displacement was NaN or infinite (error) */
} ebit_counters_t;

/* Device memory.  Every device allocation of the library (the state and
 * tables of a context, a network's parameters, a batch's arrays, and the
 * scratch that ebit_get_state and ebit_batch_autotune take) goes through
 * cudaMalloc / cudaFree, or through the caller's pair installed here: a memory
 * pool, a framework's caching allocator, or a test that refuses the k-th
 * allocation.  This is host-side resource management; no passage of the
 * paper defines it.
 *   alloc(bytes, user)  returns a device pointer on the current device,
 *                       aligned to 256 bytes, or NULL when it cannot allocate.
 *   free_fn(ptr, user)  releases a pointer that alloc returned.
 *   Both NULL restore cudaMalloc / cudaFree.
 * A context, network or batch takes a copy of the pair in force when it is
 * created (ebit_create, ebit_create_view, ebit_mlp_create, ebit_batch_create)
 * and allocates and frees through that copy for its whole life, so a later
 * call changes only objects created after it.  When an allocation fails, the
 * creating call frees what it had allocated through free_fn and returns
 * EBIT_ENOMEM; a later call that needs scratch returns EBIT_ENOMEM and
 * leaves the object usable.  The pair is process-wide: do not call this
 * concurrently with a creating call.
 * Errors: EBIT_EINVAL when exactly one of alloc and free_fn is NULL (the
 * previous pair stays in force). */
typedef void *(*ebit_alloc_fn)(size_t bytes, void *user);
typedef void (*ebit_free_fn)(void *ptr, void *user);
int ebit_set_allocator(ebit_alloc_fn alloc, ebit_free_fn free_fn, void *user);

/* Create a context for one grid: allocates the double-buffered state and the
 * tile tables on the current CUDA device.  *out receives the handle.
 * Errors: EBIT_EINVAL (null, sizes < 8, h <= 0), EBIT_ENOMEM, EBIT_ECUDA. */
int ebit_create(const ebit_desc *desc, ebit_ctx **out);

/* Release every device allocation of the context (synchronises its stream).
 * Accepts NULL. */
void ebit_destroy(ebit_ctx *ctx);

/* Marker initialisation from a level set (Sec. 3.1: colour = (phi >= 0); a
 * marker at the linear-interpolation root of phi on every edge whose end
 * colours differ).
 *   phi_nodes  [N]   phi at the nodes (device).
 *   phi_faces  [3N]  phi at the face centres, family-major; decides the colour
 *                    of saddle faces.  May be NULL: the mean of the four corner
 *                    values is used instead.
 *   s_exact    [3N]  optional offsets that replace the linear root on
 *                    sign-change edges (NaN entries keep the linear root).
 *                    May be NULL.
 * Errors: EBIT_EINVAL (null ctx or phi_nodes), EBIT_ECUDA. */
int ebit_init(ebit_ctx *ctx, const double *phi_nodes, const double *phi_faces, const double *s_exact);

/* Replace the state.  cb [N] colour bytes, s [3N] offsets (offsets of edges
 * without a marker are ignored).  Host or device pointers (copied with
 * cudaMemcpyDefault).  Errors: EBIT_EINVAL, EBIT_ECUDA. */
int ebit_set_state(ebit_ctx *ctx, const uint8_t *cb, const double *s);

/* Read the state: cb [N] and s [3N] (0 on edges without a marker).  Host or
 * device pointers.  Synchronises the stream and raises pending device errors. */
int ebit_get_state(ebit_ctx *ctx, uint8_t *cb, double *s);

/* One split advection sweep along axis dir (0,1,2) (Sec. 2.1 Eq. 2, Fig. 1;
 * Sec. 2.3 Fig. 6): every marker moves by u_dir * dt along dir (explicit Euler
 * with trilinearly interpolated velocity); aligned markers (on dir-edges)
 * land on the edge that holds them, node colours flip where markers cross
 * them (Fig. 4), edges whose end colours became equal lose their markers
 * (topology change, Fig. 5), and the markers of the two unaligned families are
 * rebuilt from the advected polylines of the two face families containing dir
 * by the two-circle fit with the radius-ratio rule (Fig. 2).
 *   u_face [N]  u_dir at the dir-faces (device).  A field of the form
 *               g(t) * u0 may be passed as u0 with dt * g(t).
 *   dt          signed time step (finite); |u| dt / h must stay below 1.
 * Errors: EBIT_EINVAL (dir, null), EBIT_ENONFINITE (dt NaN or infinite),
 * EBIT_ECUDA.  Found on the device and reported by the next ebit_sync or
 * ebit_counters: EBIT_ENONFINITE if the velocity at a marker was NaN or
 * infinite (the marker is left in place), else EBIT_ECFL if a marker moved a
 * full cell (its displacement is clamped). */
int ebit_advect_sweep(ebit_ctx *ctx, int dir, const double *u_face, double dt);

/* Front2VOF volume fractions (Sec. 2.6, Eq. 7): per cell, the face segments
 * given by the colours are chained into closed loops, each loop is fanned
 * into triangles around the centroid of its markers, and the enclosed volume
 * of the reference phase follows from Gauss's theorem.  C [N] (device).
 * flags: EBIT_INCREMENTAL writes only cells that may have changed since the
 * last call on this context with the same C pointer (anything else is taken
 * as a full request); EBIT_FULL writes every cell. */
int ebit_front2vof(ebit_ctx *ctx, double *C, int flags);

/* Curvature kappa*h of every interface cell (0 < C < 1) from the volume
 * fractions C [N]: height functions on a 3x3 stencil of 9-cell columns along
 * the dominant normal axis, other axes as fallback (Sec. 2.6, standard
 * height-function method); mode selects HF, learned, or learned with HF
 * fallback.  kappa_h [N] FP64 and status [N] (EBIT_ST_*) are written (device).
 * flags as for ebit_front2vof (incremental only when C is this context's last
 * Front2VOF output and kappa_h/status are the previous call's buffers). */
int ebit_curvature(ebit_ctx *ctx, const double *C, double *kappa_h, uint8_t *status, int mode,
                   int flags);

/* Copy the event counters accumulated since the last reset (synchronises).
 * Returns EBIT_ENONFINITE or EBIT_ECFL as ebit_sync does, EBIT_WINCONSISTENT
 * if the consistency counters are non-zero, else EBIT_OK. */
int ebit_counters(ebit_ctx *ctx, ebit_counters_t *out);

/* Zero the event counters (stream-ordered). */
int ebit_reset_counters(ebit_ctx *ctx);

/* Wait for the context's stream; returns pending device errors
 * (EBIT_ENONFINITE before EBIT_ECFL, see ebit_advect_sweep) or EBIT_OK.
 * Joins the side stream first (ebit_join). */
int ebit_sync(ebit_ctx *ctx);

/* Asynchronous Front2VOF and curvature.  Not in the paper: its per-step
 * pipeline (advection, then volume fractions, then curvature; Sec. 2.6) is
 * kept, only overlapped.  With EBIT_ASYNC in flags, ebit_front2vof and
 * ebit_curvature run on a side stream the context creates on first use, after
 * the work already issued on the context's stream, and return at once; the
 * next sweeps then run on the context's stream alongside them.  The library
 * orders what depends on them: a sweep that would overwrite the state an
 * asynchronous Front2VOF is reading waits for it (with the two buffers of a
 * split step that is the step's second sweep), the sweeps mark their tiles
 * for the following Front2VOF in a second set of tile flags, and every other
 * call that reads or writes the state, the counters or C (ebit_init,
 * ebit_set_state, ebit_get_state, ebit_counters, ebit_reset_counters,
 * ebit_sync, a call without EBIT_ASYNC) first makes the context's stream
 * wait for the side stream.  Callers that read C, kappa_h or status must do
 * the same: ebit_join makes the context's stream wait for all side-stream
 * work so far (no host synchronisation); ebit_event_record records
 * cuda_event (a cudaEvent_t) where the last Front2VOF/curvature output is
 * complete, so that another stream (a device-to-host copy) can wait for it
 * without holding back the context's stream.  Not for batch instances
 * (EBIT_EINVAL).  Errors: EBIT_EINVAL (null), EBIT_ECUDA. */
int ebit_join(ebit_ctx *ctx);
int ebit_event_record(ebit_ctx *ctx, void *cuda_event);

/* Number of tiles (8x8x8 cells) the last sweep processed; -1 if unknown. */
int ebit_band_tiles(ebit_ctx *ctx);

/* Per-kernel timing.  With profiling on, the library brackets every kernel it
 * launches on the context's stream with a pair of CUDA events and sums the
 * elapsed device time per kind.  Kinds (index into the arrays below): */
enum {
    EBIT_PROF_SWEEP = 0, /* split-sweep reconstruction kernels */
    EBIT_PROF_BAND = 1,  /* (no kernel of its own: each sweep's band pass lists the next sweep's band) */
    EBIT_PROF_F2V = 2,   /* Front2VOF: list of the swept tiles (incremental calls), band and cut-cell kernels */
    EBIT_PROF_HF = 3,    /* height-function kernel (interface-cell list pass) */
    EBIT_PROF_MLP = 4,   /* learned-curvature kernels (with the height-function fallback pass) */
    EBIT_PROF_ADVECT = 5, /* marker advection (velocity interpolation) kernels */
    EBIT_PROF_FP64 = 6,   /* sweep work lists: circle fits and face-centre colours */
    EBIT_PROF_SCAN = 7,   /* full interface-cell scan of ebit_curvature (EBIT_FULL or foreign C) */
    EBIT_PROF_COUPLING = 8, /* one-fluid properties and surface-tension force (ebit_one_fluid) */
    EBIT_PROF_KINDS = 9
};
/* enable != 0 switches timing on and zeroes the sums; 0 switches it off. */
int ebit_profile(ebit_ctx *ctx, int enable);
/* ms[EBIT_PROF_KINDS] total device milliseconds and launches[EBIT_PROF_KINDS]
 * launch counts since the last ebit_profile call (synchronises). */
int ebit_profile_read(ebit_ctx *ctx, double *ms, int64_t *launches);

/* ---------------------------------------------------------------------------
 * Learned curvature.  Not in the paper: a 27 -> 128 -> 128 -> 1 ReLU network
 * maps the canonically oriented 3x3x3 volume-fraction stencil of an interface
 * cell to kappa*h, standing in for the height-function curvature of Sec. 2.6
 * (which stays the fallback).  Canonical orientation: reflect the axes whose
 * Youngs normal component is negative, then order the axes by increasing |n|.
 * Inputs: 64 bf16 per stencil -- the 27 values rounded to float and split into
 * a bf16 head (27 values, 5 zeros) and a bf16 tail (27, 5 zeros).  Tensor-core
 * kernels (warp-level bf16 MMA, FP32 accumulation).  X buffers must start on a
 * 16-byte boundary (EBIT_EINVAL otherwise); every call runs on the network's
 * stream and returns EBIT_EINVAL on null or negative arguments.  Parameters are
 * ebit_mlp_nparams() floats: W1[128][64], b1[128], W2[128][128], b2[128],
 * w3[128], b3.  Loss of training: mean of ((y - t) / max(|t|, 0.05))^2; Adam
 * (0.9, 0.999, 1e-8) on FP32 master weights.
 * ------------------------------------------------------------------------- */
typedef struct ebit_mlp ebit_mlp;

int ebit_mlp_nparams(void);
/* Create a network (parameters zero; set them with ebit_mlp_set_params). */
int ebit_mlp_create(void *cuda_stream, ebit_mlp **out);
void ebit_mlp_destroy(ebit_mlp *mlp);
/* Parameters from / to host or device memory (set resets the Adam state). */
int ebit_mlp_set_params(ebit_mlp *mlp, const float *params);
int ebit_mlp_get_params(ebit_mlp *mlp, float *params);
/* Encoded canonical stencils X [m][64] (bf16 bit patterns, device) of the
 * cells cells[m] (linear ids, device) of the fractions C [nx*ny*nz] (device).
 * frag [m] (device, may be NULL) receives 1 where the 3x3x3 block holds a cell
 * with C > 0 that is not 6-connected to the centre through cells with C > 0. */
int ebit_mlp_gather(ebit_mlp *mlp, const double *C, int nx, int ny, int nz, const int *cells, int m, uint16_t *X,
                    uint8_t *frag);
/* y [m] (device, FP32) = network(X [m][64]). */
int ebit_mlp_forward(ebit_mlp *mlp, const uint16_t *X, int m, float *y);
/* Gradient of the training loss over one batch X [batch][64], t [batch] into
 * grad_out [nparams] (host or device); parameters unchanged. */
int ebit_mlp_gradient(ebit_mlp *mlp, const uint16_t *X, const float *t, int batch, float *grad_out);
/* One Adam step on a batch: rows X[idx[r]], t[idx[r]] for r < batch (idx
 * device int32, or NULL for the first batch rows).  *loss_out (host or device,
 * may be NULL) receives the summed weighted squared error of the batch. */
int ebit_mlp_train_step(ebit_mlp *mlp, const uint16_t *X, const float *t, const int *idx, int batch, float lr,
                        float *loss_out);
/* Wait for the network's stream; EBIT_ECUDA (message in ebit_mlp_last_error)
 * if a launch or copy on it failed, EBIT_ETIMEOUT if a tensor-core wait of the
 * tcgen05 path gave up (the kernel then freed its tensor memory and left). */
int ebit_mlp_sync(ebit_mlp *mlp);
/* Inference path of ebit_mlp_forward and ebit_curvature:
 * EBIT_MLP_PATH_TCGEN05 (default): 5th-generation tensor cores, a persistent
 * block per SM with three pipelines, each issuing tcgen05.mma from shared
 * memory into its tensor-memory columns; EBIT_MLP_PATH_MMA: warp-level BF16
 * MMA (mma.sync m16n8k16), the layer-1 activations in registers.  Both compute
 * the same network in bf16 with FP32 accumulation. */
enum { EBIT_MLP_PATH_MMA = 0, EBIT_MLP_PATH_TCGEN05 = 1 };
int ebit_mlp_set_path(ebit_mlp *mlp, int path);
const char *ebit_mlp_last_error(const ebit_mlp *mlp);
/* Network used by ebit_curvature in modes EBIT_CURV_MLP and EBIT_CURV_MLP_HF
 * (NULL detaches).  EBIT_CURV_MLP writes the learned value (status
 * EBIT_ST_MLP) on every interface cell and computes no height functions.
 * EBIT_CURV_MLP_HF computes height functions only where the learned value
 * leaves the trained range |kappa h| <= 1 or the stencil holds a phase-1
 * fragment (see ebit_mlp_gather); those cells get the height-function value
 * and status. */
int ebit_set_mlp(ebit_ctx *ctx, ebit_mlp *mlp);
/* Parameters (host or device, ebit_mlp_nparams() floats in the order above,
 * bytes = 4 * ebit_mlp_nparams()) into a network the context owns and uses
 * for ebit_curvature (created on first use on the context's stream, freed by
 * ebit_destroy).  EBIT_EINVAL on a size mismatch. */
int ebit_mlp_load(ebit_ctx *ctx, const void *weights, size_t bytes);

/* ---------------------------------------------------------------------------
 * Batches: many independent instances (each a periodic grid with its own size,
 * velocity and time step; the method of ebit_advect_sweep, Sec. 2.1-2.3)
 * advanced together.  One split sweep of every instance is ONE cooperative
 * kernel launch whose phases (band listing, marker advection, integer band
 * pass, FP64 work lists) are separated by a grid barrier; ebit_batch_run
 * replays two whole steps (x-y-z then z-y-x sweeps) as a CUDA graph.
 * Each instance's result equals that of a separate context given the same
 * inputs.  The barrier waits a bounded time; if it gives up, the batch's
 * state is undefined and ebit_batch_sync returns EBIT_ETIMEOUT.
 * ------------------------------------------------------------------------- */
typedef struct ebit_batch ebit_batch;

/* descs[n]: one descriptor per instance (n <= 1024, every edge >= 8 cells, at
 * most 2^20 tiles of 8^3 cells per instance and 2^31 cells in all, the same
 * cuda_stream for all, no EBIT_DESC_DENSE).  EBIT_ECUDA if the device has no
 * cooperative launch. */
int ebit_batch_create(int n, const ebit_desc *descs, ebit_batch **out);
void ebit_batch_destroy(ebit_batch *b);
int ebit_batch_size(const ebit_batch *b);
/* The context of instance i (owned by the batch; NULL if i is out of range):
 * use it for ebit_init, ebit_set_state, ebit_get_state, ebit_front2vof,
 * ebit_curvature and the counters.  ebit_advect_sweep on it returns
 * EBIT_EINVAL: instances are swept through the batch. */
ebit_ctx *ebit_batch_instance(ebit_batch *b, int i);
/* Velocities and time steps for the following sweeps: u_faces[3 i + d] is
 * instance i's u_d on its d-normal faces (device, N_i doubles, read at every
 * sweep, so the caller keeps it alive and may rewrite it between sweeps);
 * dt[i] (host) its time step.  Synchronises. */
int ebit_batch_set_velocity(ebit_batch *b, const double *const *u_faces, const double *dt);
/* One split sweep along dir (0, 1, 2) of every instance.  u_dev (host array
 * of n device pointers: instance i's u_dir on its dir-normal faces) and dt
 * (host array of n time steps) replace the stored velocity of that direction
 * and the stored time steps; either may be NULL to keep what
 * ebit_batch_set_velocity (or an earlier call) stored. */
int ebit_batch_advect_sweep(ebit_batch *b, int dir, const double *const *u_dev, const double *dt);
/* Steps first_step .. first_step + steps - 1 (even steps x-y-z, odd steps
 * z-y-x).  use_graph != 0 replays pairs of steps from a CUDA graph captured on
 * first use (and again after a launch-shape change); where capture is not
 * available the sweeps are launched directly (ebit_batch_graph_active tells). */
int ebit_batch_run(ebit_batch *b, int first_step, int steps, int use_graph);
/* 0: no graph (sweeps launched directly), 1: graph from stream capture,
 * 2: graph built node by node; ebit_batch_graph_note says how or why not. */
int ebit_batch_graph_active(const ebit_batch *b);
const char *ebit_batch_graph_note(const ebit_batch *b);
/* Wait for the batch's stream; EBIT_ETIMEOUT if a grid barrier gave up. */
int ebit_batch_sync(ebit_batch *b);
/* Launch shape: blocks of 256 threads per SM (1 .. max co-resident for the
 * current tile shape). */
int ebit_batch_launch_shape(const ebit_batch *b, int *ctas_per_sm, int *max_ctas_per_sm);
int ebit_batch_set_launch_shape(ebit_batch *b, int ctas_per_sm);
/* Tile shape: the cells per tile edge along x, y, z of the band tiles that the
 * batched sweep works on (512 cells each; every edge at least 4 cells, so the
 * tile proximity rule of the band still reaches only adjacent tiles).  The
 * shape changes how the work is cut and staged, never the result: tiles
 * outside the band are unchanged by a sweep whatever their shape.
 *   EBIT_TILE_8x8x8 (0, the initial shape and that of single contexts),
 *   EBIT_TILE_16x8x4 (1), EBIT_TILE_32x4x4 (2: x-lines).
 * ebit_batch_tile_shape returns the current shape and writes its edges to
 * dims[3] (host, may be NULL).  ebit_batch_set_tile_shape re-tiles every
 * instance (synchronises the stream; every tile is processed by the next
 * sweep and recomputed by the next Front2VOF); EBIT_EINVAL for an unknown
 * shape or one that does not fit an instance.  A shape fits when, along
 * every axis with tile edge T and n cells, T floor((n - 1) / T) + T + 2 <= 2 n
 * (a tile's staged region, which reaches T + 1 nodes past its origin, wraps
 * at most once): edges of 4 and 8 fit every instance, 16 needs n >= 9 and
 * 32 needs n >= 17 along that axis.  The "tiles" counter counts tiles of the
 * shape in use. */
enum { EBIT_TILE_8x8x8 = 0, EBIT_TILE_16x8x4 = 1, EBIT_TILE_32x4x4 = 2, EBIT_TILE_SHAPES = 3 };
enum { EBIT_BATCH_MAX_CTAS = 8 };
int ebit_batch_tile_shape(const ebit_batch *b, int *dims);
int ebit_batch_set_tile_shape(ebit_batch *b, int shape);
/* Autotuner: for every tile shape and every launch shape, starting from a
 * copy of the current state with every tile marked, one untimed sweep forms
 * the band, then `sweeps` sweeps are timed with CUDA events (the second of
 * two passes; the first warms up); shapes that do not fit an instance are
 * skipped.  Keeps the fastest pair and puts the state
 * back (the tile tables too when the shape is unchanged).  ms_out (host, may
 * be NULL) receives EBIT_TILE_SHAPES x EBIT_BATCH_MAX_CTAS doubles, index
 * shape * EBIT_BATCH_MAX_CTAS + ctas_per_sm - 1, 0 where the pair was not
 * run.  Allocates a state copy. */
int ebit_batch_autotune(ebit_batch *b, int sweeps, double *ms_out);
const char *ebit_batch_last_error(const ebit_batch *b);
/* Self-test of the bounded device waits (the grid barrier of the batched
 * sweep and the mbarrier waits of the tensor-core kernels), run on
 * cuda_stream (NULL: the legacy default stream).  Each wait runs twice in a
 * tiny kernel with a short poll limit: once where the awaited event comes
 * (two blocks both reach the barrier; one arrival on the mbarrier), once
 * where it never comes (one block leaves without arriving; nobody arrives),
 * so that the wait must give up.  The second case shows, without any fault
 * or hang, that a wait which runs out returns, sets the error flag the host
 * reads, and leaves the device usable.  report (host, may be NULL) gets six
 * ints: barrier result and error flag when both blocks arrive (1, 0), barrier
 * result and error flag when one is absent (0, 1), mbarrier result with and
 * without the arrival (1, 0).  Returns EBIT_OK when all six are as stated,
 * EBIT_ETIMEOUT otherwise, EBIT_ENOMEM / EBIT_ECUDA if its 64-byte buffer
 * cannot be allocated or a launch or copy fails. */
int ebit_selftest_bounded_waits(void *cuda_stream, int *report);

/* One-fluid coupling terms (Sec. 2.5): what a Navier-Stokes solver in the
 * one-fluid formulation takes from the interface.
 *   rho [N], mu [N] (device, may be NULL): Eq. 6 with the Heaviside function of
 *     the reference phase taken as C: rho = C rho1 + (1 - C) rho2, and mu
 *     likewise, per cell.
 *   force [3N] (device, family-major, may be NULL): the surface-tension term
 *     sigma kappa n delta_S as a well-balanced continuum surface force on the
 *     MAC faces.  force[a][idx], on the a-face of cell idx (between cells
 *     idx - e_a and idx, where u_a lives), is sigma kappa_f (C[idx] -
 *     C[idx - e_a]) / h, with kappa = kappa_h / h on cells whose status is
 *     EBIT_ST_HF_X/Y/Z or EBIT_ST_MLP, and kappa_f the mean of the face's two
 *     cells' values, the one valid value, or 0.  A uniform kappa_f makes the
 *     force the exact discrete gradient of sigma kappa_f C: a pressure of that
 *     form balances it.
 *   C [N] (device) the fractions; kappa_h [N], status [N] (device) the output
 *     of ebit_curvature, needed for force only.
 * Runs on the context's stream after any EBIT_ASYNC work.  EBIT_EINVAL for a
 * null C (or null curvature arrays with force), EBIT_ENONFINITE for a
 * non-finite coefficient. */
int ebit_one_fluid(ebit_ctx *ctx, const double *C, const double *kappa_h, const uint8_t *status, double sigma,
                   double rho1, double rho2, double mu1, double mu2, double *rho, double *mu, double *force);

/* AMR refinement rule and narrow-band brick store (Sec. 2.5).  With one marker
 * per edge, two refinement levels must never share the interface, so every
 * cell within the 3x3x3 block of cells around an interfacial cell is refined
 * to the finest level.  A cell is interfacial when its eight corner colours
 * differ (an edge carries a marker exactly when its end colours differ).
 *
 * ebit_refine_mask: mask [N] (device, caller-owned, may be NULL) receives 1
 *   for every cell that the rule refines and 0 elsewhere (cell idx = its lowest
 *   corner's node idx); count (host, may be NULL) the number of such cells,
 *   which makes the call synchronise.  Reads the current state (after any
 *   EBIT_ASYNC work is joined).
 *
 * ebit_pack_bricks: the narrow-band store of the current state.  The bricks are
 *   the 8x8x8 tiles that hold a refined cell, in ascending tile id (tile id =
 *   (tz * tiles_y + ty) * tiles_x + tx, tiles_a = ceil(n_a / 8)).  Any other
 *   tile holds no interfacial cell: one node colour, no marker, face colours
 *   equal to it.  Outputs, device arrays owned by the caller:
 *     tiles [capacity]              brick k's tile id;
 *     cb    [capacity][512]         brick k's colour bytes, cell c = x + 8 (y + 8 z)
 *                                   in the tile (0 for cells past the grid);
 *     s     [capacity][3][512]      its offsets per edge family, 0 on an edge
 *                                   without a marker;
 *     bg    [tiles]                 bit 0: every tile's origin-node colour
 *                                   (the colour of each tile that is not a brick).
 *   *nbricks (host) receives the brick count.  capacity = 0 (arrays may be
 *   NULL) only counts.  Synchronises.  EBIT_EINVAL when capacity is below the
 *   count (the outputs are then unspecified) or the grid uses tiles other than
 *   8^3 (a batch instance re-tiled by its autotuner).
 *
 * ebit_unpack_bricks: replaces the state with the one a store describes: the
 *   bricks' cells from cb and s, every other tile filled with its bg colour
 *   (colour byte 0x0F or 0x00, offsets 0); each tile at most once.  Like
 *   ebit_set_state, the next sweep and Front2VOF treat every tile.  EBIT_EINVAL
 *   for a tile id out of range (checked on the device; synchronises) or on a
 *   batch instance.  Arrays as for ebit_pack_bricks, borrowed for the call. */
int ebit_refine_mask(ebit_ctx *ctx, uint8_t *mask, int64_t *count);
int ebit_pack_bricks(ebit_ctx *ctx, int capacity, int *tiles, uint8_t *cb, double *s, uint8_t *bg, int *nbricks);
int ebit_unpack_bricks(ebit_ctx *ctx, int nbricks, const int *tiles, const uint8_t *cb, const double *s,
                       const uint8_t *bg);

/* Self-test of the integer double -> float conversion that the learned
 * curvature's gather uses for the C values (no paper passage: GB300's FP64
 * pipe is narrow, so the gather converts from the bit patterns).  out[i] =
 * in[i] rounded to float, nearest-even, exactly as the IEEE conversion for
 * every non-NaN input; a NaN gives a quiet NaN.  in, out: n device values
 * (caller-owned), on cuda_stream.  EBIT_EINVAL for null arrays or n < 0. */
int ebit_selftest_f64_to_f32(const double *in, float *out, int n, void *cuda_stream);

/* One split advection sweep that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- a flow solver that reserves all of its
 * device memory at start-up and forbids allocation afterwards, or a real-time
 * loop in which a cudaMalloc (which may synchronise the device) is not
 * allowed.  It needs no context: the caller passes the old state, the
 * velocity and the output buffers (all DEVICE pointers), and the sweep's
 * intermediate arrays live in one fixed file-scope device array.
 *   nx, ny, nz, h   grid as in ebit_desc; nx*ny*nz must not exceed 64^3 =
 *                   262144 cells (EBIT_EINVAL beyond), each axis >= 8.  The
 *                   tile parts of the scratch hold 1620 tiles of 8^3, the
 *                   most any such grid has (9 x 9 x 3236), so every grid
 *                   within the cell limit is accepted.
 *   dir, u_face, dt as for ebit_advect_sweep.
 *   cb_in [N], s_in [3N]    state before the sweep (colour bytes, offsets).
 *   cb_out [N], s_out [3N]  state after the sweep (offsets 0 on edges without
 *                   a marker); must not overlap the inputs.
 *   cuda_stream     cudaStream_t for every launch (NULL = default stream).
 * Every tile is processed (no active band).  Marker displacements of a full
 * cell or more are clamped and not reported (use ebit_advect_sweep for the
 * event counters).  The scratch array is about 11.3 MB and is held by every
 * GPU that loads the library until the process exits; its address is looked
 * up on the first call made on each device, so make that first call before
 * any stream capture.  The address is kept for the life of the device's
 * primary context: do not call this entry point after a cudaDeviceReset.
 * All calls on a device share it: calls that overlap on the GPU race and must
 * be ordered by the caller.
 * Errors: EBIT_EINVAL (sizes, dir, null pointers, non-finite h or dt),
 * EBIT_ECUDA (a launch or copy failed). */
int ebit_advect_sweep_noalloc(int nx, int ny, int nz, double h, int dir, const uint8_t *cb_in,
                              const double *s_in, const double *u_face, double dt, uint8_t *cb_out,
                              double *s_out, void *cuda_stream);

/* Message of the last failed call on this context (never NULL). */
const char *ebit_last_error(const ebit_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* EBIT_H */
