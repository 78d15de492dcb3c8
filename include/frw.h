/*
 * frw.h -- C ABI of the GB300 floating-random-walk (FRW) capacitance engine with
 * MicroWalk transitions (Huang & Yu, "Efficient FRW Transitions via Stochastic
 * Finite Differences for Handling Non-Stratified Dielectrics").
 *
 * Plain C types only.  Pointers marked "host" point to host memory, "device" to
 * memory of the context's CUDA device.  Every entry point returns an int status
 * (FRW_OK = 0, else one of the FRW_E* codes; frw_strerror gives a message) and
 * never throws.  A context is used by one host thread at a time.
 *
 * Units: lengths in micrometres, permittivities relative, capacitances in fF
 * (the vacuum permittivity 8.8541878128e-3 fF/um is applied inside).
 *
 * Method summary (paper sections):
 *   - Algorithm 1 (FRW): a walk starts on the master's Gaussian surface, makes a
 *     first transition that carries the weight omega, then hops from cube centre
 *     to cube surface until it reaches an electrode k; C_ik accumulates omega.
 *   - Transition cube (Sec. II-A): the largest conductor-free cube centred at the
 *     walk's point, voxelised into an N x N x N lattice with one permittivity per
 *     voxel (Sec. III-A).
 *   - Algorithm 3 (MicroWalk): for a non-stratified cube, a random walk on the
 *     lattice with the jump law of Eq. 6, exact by Theorem 1.
 *   - Sec. III-C (hybrid): stratified cubes take the analytical route (the exact
 *     FD surface Green's function of the layered lattice, Eq. 8, cached by
 *     profile); the first cube uses the special treatment (stratified /
 *     shrink-to-stratified / homogenise).
 */
#ifndef FRW_H
#define FRW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FRW_OK 0
#define FRW_EINVAL 1      /* bad argument or structure (message via frw_last_error) */
#define FRW_ENOMEM 2      /* device allocation failed / admission refused */
#define FRW_ETIMEOUT 3    /* a bounded wait gave up */
#define FRW_EDEVICE 4     /* CUDA error, or a device-side check failed */
#define FRW_ENOTCONV 5    /* walk budget exhausted before the sigma target (results valid) */
#define FRW_ECAPACITY 6   /* a fixed-size table (materials, cache, jobs) is full */
#define FRW_ENOTFOUND 7   /* unknown structure id / ticket */
#define FRW_ECANCELED 8   /* the request was cancelled (frw_cancel) */

/* ---- option values ---- */
#define FRW_FP64_GEOM 0   /* cube sizing, voxel ranges and points in FP64 */
#define FRW_FP32_GEOM 1   /* the same in FP32 with a conservative margin on the cube size */
#define FRW_FIRST_HYBRID 0

/* ---- table kinds of the analytical route (frw_table) ---- */
#define FRW_TAB_SGF 0        /* surface Green's function, layered along table axis t2 */
#define FRW_TAB_FLUX_PAR 1   /* first-cube flux kernel, normal = t2 = layering axis */
#define FRW_TAB_FLUX_PERP 2  /* first-cube flux kernel, normal = t0, layering axis t2 */
#define FRW_TAB_SGF_HOM 3    /* surface Green's function of a homogeneous cube */
#define FRW_TAB_FLUX_HOM 4   /* flux kernel of a homogeneous cube with eps = 1 */

#define FRW_MAX_N 32         /* lattice edge N: even, 2 <= N <= 32 */
#define FRW_MAX_MATERIALS 15 /* distinct permittivities per context */
#define FRW_MAX_CUBE_BLOCKS 14
#define FRW_FDM_MAX_N 24     /* FD transitions: the solve's vectors of N^3 floats in shared memory */

#define FRW_TRANSITION_MICROWALK 0
#define FRW_TRANSITION_FDM 1

typedef struct frw_ctx frw_ctx;

/* Axis-aligned box [lo, hi] (um), lo < hi on every axis. */
typedef struct {
    double lo[3], hi[3];
} frw_box;

/* Dielectric block: box + material index into the structure's eps_r table.
 * Where blocks overlap, the later block in the array wins (the background is
 * below every block); a block is sampled at voxel centres with lo <= x < hi. */
typedef struct {
    double lo[3], hi[3];
    int32_t mat;
    int32_t reserved;
} frw_block;

typedef struct {
    int32_t N;                 /* lattice edge per transition cube (paper: 24) */
    int32_t precision;         /* FRW_FP64_GEOM or FRW_FP32_GEOM */
    uint64_t seed;             /* Philox key material */
    int32_t first_cube_mode;   /* FRW_FIRST_HYBRID */
    int32_t hybrid;            /* 1: stratified cubes take the analytical route; 0: MicroWalk */
    double gauss_offset_frac;  /* Gaussian surface offset = frac * smallest gap (0 < frac < 1) */
    int32_t max_hops;          /* hop cap; a capped walk counts with zero contribution */
    int32_t slots;             /* walks in flight on the device (0: default) */
    int32_t table_capacity;    /* analytical-table cache entries (0: default) */
    int32_t mw_warps_per_cta;  /* stand-alone MicroWalk kernel: warps per CTA, 1..16 (0: 16) */
    int32_t mw_ctas_per_sm;    /* stand-alone MicroWalk kernel: CTAs per SM, 1..32 (0: 2) */
    int32_t geom_threads;      /* ignored (kept for layout) */
    int32_t serve_jobs;        /* serving: job-table entries of one run (0: 4096) */
    int32_t serve_arena_mb;    /* serving: MB of per-walk records of one run, 32 B per walk of
                                  budget; also sizes its batch arenas (0: 4096) */
    int32_t mwe_factor;        /* MicroWalk-E (Sec. III-B, Fig. 3b): a later transition cube that is
                                  not stratified is expanded this many times (the paper: 5) and may
                                  hold conductors, whose voxels absorb the walk; lowered while the
                                  cube lists more than 14 blocks, conductors and exterior slabs,
                                  plain MicroWalk below 2 or above 254 conductors (0 .. 16; 0 or 1:
                                  off, plain FRW-MW) */
    int32_t idle_timeout_ms;   /* a walk-kernel CTA with nothing to do gives up waiting after this
                                  long and ends the run with an error status (0: 10000) */
    int32_t transition;        /* later non-stratified cubes: FRW_TRANSITION_MICROWALK (Algorithm 3,
                                  FRW-MW) or FRW_TRANSITION_FDM (Algorithm 2, FRW-FDM: the cube's
                                  FD system is solved and its SGF sampled; the paper's comparator;
                                  N <= FRW_FDM_MAX_N, no MicroWalk-E) */
    int32_t reserved;
} frw_options;

/* One extraction: a row of the capacitance matrix for one master conductor. */
typedef struct {
    uint64_t walk_budget;      /* maximum number of walks */
    double sigma_target;       /* stop when stderr/|C| <= target on C_ii and on the
                                  largest |C_ij| (j != i, ground excluded); 0 = budget only */
    uint64_t request_id;       /* RNG stream of this request (with the context seed) */
    uint64_t batch;            /* walks per convergence check (0: 16384) */
    uint64_t walk_begin;       /* first walk id (0 normally; resume / sharding offset) */
} frw_extract_params;

typedef struct {
    uint64_t walks;            /* walks counted in the estimate */
    uint64_t hops;             /* transitions, first one included */
    uint64_t micro_steps;      /* MicroWalk lattice steps */
    uint64_t truncated;        /* walks that hit max_hops */
    uint64_t branch[3];        /* first cube: stratified / shrunk to stratified / homogenised */
    uint64_t strat_hops;       /* later hops through the analytical route, layered cube */
    uint64_t hom_hops;         /* ... homogeneous cube */
    uint64_t mw_hops;          /* later hops through MicroWalk */
    uint64_t tables_built;     /* analytical tables filled on the device during the call */
    uint64_t rounds;           /* epochs of the persistent walk kernel (largest over its CTAs) */
    double seconds;            /* wall time of the call */
    double geom_ms;            /* walk-kernel time in its geometry phase: kernel_ms x that phase's
                                  share of the CTAs' busy cycles */
    double fill_ms;            /* ... in its table-fill phase */
    double mw_ms;              /* ... in its MicroWalk phase */
    uint64_t launches;         /* kernels launched by the call (memsets not counted) */
    uint64_t mw_jobs;          /* MicroWalk transitions */
    uint64_t walks_issued;     /* walk ids started (>= walks: a sigma-target run stops mid-flight) */
    double kernel_ms;          /* device time of the walk kernel (CUDA events on the launch stream) */
    double reduce_ms;          /* walk-kernel time in its batch-reduction phase (as geom_ms) */
    uint64_t stage_bytes;      /* bytes of the structure's geometry that each walk-kernel CTA copied into
                                  shared memory and read from there (0: read from global memory) */
} frw_stats;

/* Fill *opt with defaults (N = 24, FP64 geometry, hybrid on, offset 0.5,
 * max_hops = 100000, seed 0). */
void frw_default_options(frw_options *opt);

/* Create a context on CUDA device `device`.  Allocates the device working set
 * (walk slots, queues, table cache) and computes the homogeneous tables on the
 * device.  *out owns all device memory until frw_destroy. */
int frw_create(frw_ctx **out, int device, const frw_options *opt);
void frw_destroy(frw_ctx *ctx);

/* Launch subsequent work on this CUDA stream (cudaStream_t as void*; NULL =
 * the context's own stream). */
int frw_set_stream(frw_ctx *ctx, void *cuda_stream);

/* Load a structure (Algorithm 1 input): grounded domain box, n_cond disjoint
 * conductor boxes inside it, permittivity table eps_r[n_mat] (> 0), background
 * material, dielectric blocks.  All inputs are host pointers, copied; the caller
 * keeps ownership.  The index of the max-cube query (Sec. II-A: a uniform grid
 * whose cells list the conductor boxes that can be nearest) is built on the
 * device; with the environment variable FRW_INDEX_HOST=1 the host's cores build
 * the same lists.  The call returns when the structure is ready.  Returns
 * FRW_EINVAL for overlapping/outside conductors, bad material ids or
 * non-positive permittivities, FRW_ECAPACITY if the context would exceed
 * FRW_MAX_MATERIALS distinct permittivities. */
int frw_load_structure(frw_ctx *ctx, const frw_box *domain, const frw_box *conductors,
                       int32_t n_cond, const double *eps_r, int32_t n_mat, int32_t background_mat,
                       const frw_block *blocks, int32_t n_blocks, int32_t *structure_id);
/* A structure whose conductors are unions of boxes (Sec. "next" of this library:
 * the paper's conductors are single boxes).  Box i (host array boxes[n_boxes])
 * belongs to conductor box_conductor[i], 0 <= id < n_cond, and every conductor has
 * at least one box.  Boxes of one conductor may touch or overlap; boxes of
 * different conductors must be apart (positive L-infinity gap); every box lies
 * strictly inside the domain.  The distance to a conductor is the smallest over
 * its boxes; a walk that reaches any box is absorbed by its conductor.  Only
 * conductors of exactly one box can be masters (extraction of another returns
 * FRW_EINVAL: the Gaussian surface of Algorithm 1 is the master's box grown by a
 * margin), and the full matrix needs every conductor to be one.  At most 65535
 * boxes.  Otherwise as frw_load_structure. */
int frw_load_structure_boxes(frw_ctx *ctx, const frw_box *domain, const frw_box *boxes,
                             const int32_t *box_conductor, int32_t n_boxes, int32_t n_cond,
                             const double *eps_r, int32_t n_mat, int32_t background_mat,
                             const frw_block *blocks, int32_t n_blocks, int32_t *structure_id);
int frw_unload_structure(frw_ctx *ctx, int32_t structure_id);

/* A structure in full (one descriptor for every input of Algorithm 1 this library
 * takes): the domain box; grounded_walls (must be 1: the domain walls are the
 * ground electrode, index n_cond of every row -- Algorithm 1 ends a walk on an
 * electrode and the FD lattice of Eq. 4-6 has Dirichlet panels only, so no other
 * wall condition is offered); conductor boxes with their conductor ids
 * (box_conductor may be NULL: box i is conductor i, n_boxes = n_cond) as for
 * frw_load_structure_boxes; the permittivity table and background material; an
 * optional permittivity voxel map; dielectric blocks.
 * Voxel map (Sec. III-A: permittivity constant in each voxel): voxel_mat (host,
 * may be NULL) holds vox_dims[0] * vox_dims[1] * vox_dims[2] material ids, x
 * slowest and z fastest (cell (i, j, k) at (i * ny + j) * nz + k), of the cells of
 * a uniform grid over the domain: cell i on axis a spans [e_a(i), e_a(i + 1)) with
 * e_a(i) = lo_a + ((hi_a - lo_a) * i) / n_a and e_a(n_a) = hi_a.  An id below n_mat
 * gives the cell that material; FRW_VOXEL_NONE leaves it to the background.
 * Priority: a dielectric block (later blocks first) wins over the voxel map,
 * which wins over the background.  The map is loaded as boxes: maximal runs of
 * one material along z, runs with equal extent and material merged across
 * consecutive y, then rectangles merged across consecutive x, the boxes ordered
 * by their first cell (x, then y, then z) and placed below the blocks.  At most
 * 2^24 cells and 65535 boxes and blocks together (FRW_ECAPACITY beyond).
 * Otherwise as frw_load_structure. */
#define FRW_VOXEL_NONE 255
typedef struct {
    frw_box domain;
    int32_t grounded_walls;
    int32_t n_boxes, n_cond;
    int32_t n_mat, background_mat;
    int32_t n_blocks;
    int32_t vox_dims[3];
    int32_t reserved;
    const frw_box *boxes;
    const int32_t *box_conductor;
    const double *eps_r;
    const frw_block *blocks;
    const uint8_t *voxel_mat;
} frw_structure;
int frw_load_structure_ex(frw_ctx *ctx, const frw_structure *desc, int32_t *structure_id);

/* Capacitance row of `master` (Algorithm 1 output).  C_row and stderr_row are host
 * arrays of n_cond + 1 doubles (last entry = grounded walls).  stats may be NULL.
 * Returns FRW_ENOTCONV (results still filled) when the budget ran out before the
 * sigma target.  Results are bit-reproducible for a given (seed, request_id). */
int frw_extract(frw_ctx *ctx, int32_t structure_id, int32_t master,
                const frw_extract_params *params, double *C_row, double *stderr_row,
                frw_stats *stats);

/* Like frw_extract, but returns the estimator's exact sums instead of the row, for
 * combining shards of one extraction run on several GPUs (disjoint walk-id ranges
 * through params->walk_begin; sigma_target must be 0).  sums (host, 4 (n_cond + 1)
 * uint64): [2k, 2k+1] = S1_k = sum of omega over walks ending at k, as a two's
 * complement int128 (low word first) in units of 2^-64 fF; [2(n_cond+1) + 2k, +1]
 * = S2_k = sum of omega^2 in units of 2^-40 fF^2.  *n_walks = walks counted.
 * Integer sums add exactly, so the combined shards give bit-for-bit the row of a
 * single run over the union of the ranges: C_k = S1_k / n, and the standard error
 * sqrt((S2_k - S1_k^2 / n) / (n (n - 1))), each sum converted to double first. */
int frw_extract_sums(frw_ctx *ctx, int32_t structure_id, int32_t master, const frw_extract_params *params,
                     uint64_t *sums, uint64_t *n_walks, frw_stats *stats);

/* The exact sums of frw_extract_sums batch by batch (for a sigma-target extraction
 * shared by several processes, Sec. IV's stop rule evaluated on the combined
 * batches): walks params->walk_begin .. walk_begin + walk_budget - 1 in batches of
 * params->batch walks (0: 16384); walk_begin must be a multiple of the batch size
 * (FRW_EINVAL otherwise) so that batches line up across processes; sigma_target
 * must be 0.  n_b = ceil(walk_budget / batch) batches.  Host outputs: sums[b * 4
 * (n_cond + 1) + i] = word i of batch b in frw_extract_sums' layout; n_in_batch[b]
 * = walks counted in batch b (the batch size, less for a final partial batch). */
int frw_extract_batch_sums(frw_ctx *ctx, int32_t structure_id, int32_t master, const frw_extract_params *params,
                           uint64_t *sums, uint64_t *n_in_batch, frw_stats *stats);

/* Several extractions (possibly different structures, masters, budgets and
 * targets) interleaved in one engine run.  C_rows / stderr_rows are host arrays
 * holding each job's n_cond + 1 entries back to back in job order; stats (may be
 * NULL) has n_jobs entries. */
typedef struct {
    int32_t structure_id;
    int32_t master;
    uint64_t walk_budget;
    double sigma_target;
    uint64_t request_id;
    uint64_t batch;
} frw_job;

int frw_extract_batch(frw_ctx *ctx, const frw_job *jobs, int32_t n_jobs, double *C_rows,
                      double *stderr_rows, frw_stats *stats);

/* Full capacitance matrix of a structure (every conductor as master, in one run;
 * master i runs as request params->request_id + i with the other parameters of
 * params, walk_begin ignored).  C and stderr (host, n_cond x (n_cond + 1), row i
 * = frw_extract's row of master i, last column = grounded walls); C_sym (host,
 * n_cond x n_cond, may be NULL) = the symmetrised matrix, (C_ij + C_ji) / 2 off
 * the diagonal, C_ii on it (the reciprocity C_ij = C_ji holds in expectation).
 * stats: n_cond entries or NULL.  FRW_ENOTCONV if some row missed its target. */
int frw_extract_matrix(frw_ctx *ctx, int32_t structure_id, const frw_extract_params *params, double *C,
                       double *stderr_rows, double *C_sym, frw_stats *stats);

/* Batching with a captured launch (the paper has no counterpart).  A plan lays a
 * fixed set of jobs out once, in a job table, arenas and record pool of its own,
 * and captures its whole launch sequence (arena reset, job publication from
 * pinned host staging, the persistent walk kernel) in a CUDA graph.  Each
 * frw_plan_run replays the graph with request ids shifted by request_offset
 * (job i runs as request jobs[i].request_id + request_offset) and returns the
 * rows as frw_extract_batch does (same layout, same results for the same ids).
 * A plan keeps its device memory until frw_plan_destroy; destroy plans before
 * their context. */
typedef struct frw_plan frw_plan;
int frw_plan_create(frw_ctx *ctx, const frw_job *jobs, int32_t n_jobs, frw_plan **out);
int frw_plan_run(frw_plan *plan, uint64_t request_offset, double *C_rows, double *stderr_rows,
                 frw_stats *stats);
void frw_plan_destroy(frw_plan *plan);

/* Launch settings of the walk kernel and of the stand-alone MicroWalk kernel.
 * No setting changes any result (walks are keyed by their ids and accumulated
 * exactly); they change only speed. */
typedef struct {
    int32_t pool_per_cta;      /* walk slots per CTA of the walk kernel (256 .. 4096, multiple of 256;
                                  at most the context's pool) */
    int32_t hops_per_epoch;    /* analytical hops one walk may take per epoch (1 .. 64) */
    int32_t suspend_lanes;     /* a MicroWalk warp of the walk kernel with at most this many lanes
                                  still walking may park them until the next epoch (0 .. 32) */
    int32_t mw_warps_per_cta;  /* stand-alone MicroWalk kernel: warps per CTA (1 .. 16) */
    int32_t mw_ctas_per_sm;    /* ... CTAs per SM (1 .. 32) */
    int32_t suspend_min_steps; /* ... once each of them has made this many steps in the epoch (4 .. 4096) */
    int32_t geo_warps;         /* 0: the walk kernel alternates geometry and MicroWalk phases with all its
                                  warps; 1 .. 13: it runs this many warps per CTA on geometry and the
                                  others on MicroWalk at the same time (the pool then at most 2048) */
    int32_t unstaged;          /* 0: when every job of a closed run or plan uses one structure, each CTA of
                                  the phased walk kernel copies that structure's conductor boxes, dielectric
                                  blocks and slab masks into shared memory (the groups that fit without
                                  lowering the kernel's CTAs per SM) and sizes cubes from the copy;
                                  1: the geometry is read from global memory only */
    double walks_per_s;        /* frw_autotune: measured with the chosen walk-kernel settings */
    double mw_steps_per_s;     /* frw_autotune: measured with the chosen MicroWalk shape */
} frw_tuning;

int frw_get_tuning(frw_ctx *ctx, frw_tuning *out);
int frw_set_tuning(frw_ctx *ctx, const frw_tuning *t);   /* FRW_EINVAL outside the ranges above */

/* Autotuner: runs the sample jobs in budget mode (each capped at sample_walks
 * walks) once per candidate walk-kernel setting (slots per CTA in {1024, 2048,
 * 3072, 4096, the context's pool} up to the context's pool x ten combinations of
 * analytical hops per epoch (1-4), suspension lanes (16 or 32) and suspension
 * progress guard (32-256): (1, 32, 128), (1, 32, 64), (1, 32, 256), (1, 16, 128),
 * (1, 32, 32), (2, 32, 128), (2, 32, 64), (2, 32, 256), (3, 32, 128), (4, 32, 64))
 * and keeps the fastest; the context starts with 1 hop per epoch, 32 lanes and a
 * guard of 128 steps;
 * then times the stand-alone MicroWalk kernel on 512 random cubes of the
 * context's N (2-6 blocks of up to four of its registered materials, 4096
 * samples each) for each shape (warps per CTA x
 * CTAs per SM in {8x2, 8x4, 16x1, 16x2, 16x3}) and keeps the fastest.  The
 * chosen settings apply to later calls; *out (may be NULL) receives them. */
int frw_autotune(frw_ctx *ctx, const frw_job *sample, int32_t n_sample, uint64_t sample_walks,
                 frw_tuning *out);

/* Serving (the paper has no counterpart: a deployment form of Algorithm 1's
 * extraction).  frw_submit queues one extraction and returns at once with a
 * ticket; a scheduler thread of the context admits queued requests, in arrival
 * order, into the running persistent walk kernel whenever the run's job table and
 * arenas have room for the request's walk budget (admission by memory: 32 B of
 * records per walk of budget plus its batch accumulators).  Admitted requests'
 * walks interleave on the device with those of earlier requests, and each request
 * completes as soon as its own stop rule holds.  A request that can never fit the
 * serving arena (options serve_arena_mb / serve_jobs) completes with FRW_ENOMEM.
 * Results are identical to frw_extract of the same job (same seed and request_id),
 * whatever else is running.  frw_submit, frw_poll and frw_wait may be called from
 * any host thread.  While a serving run is on the device, frw_extract*,
 * frw_walk_records and frw_unload_structure wait for it to end (it ends after
 * 0.5 s without requests).
 *   frw_submit: job as in frw_extract_batch; *ticket receives the request's id.
 *   frw_poll:   *done = 1 once the request has completed (FRW_ENOTFOUND for an
 *               unknown or already collected ticket).
 *   frw_wait:   blocks until completion (timeout_s < 0: no limit; FRW_ETIMEOUT if
 *               the limit passes first, the ticket stays valid), then fills C_row /
 *               stderr_row (n_cond + 1 doubles each, host) and stats (may be NULL;
 *               stats->seconds = time from submission to completion) and releases
 *               the ticket.  Returns the request's status (FRW_OK, FRW_ENOTCONV with
 *               results filled, or an error). */
int frw_submit(frw_ctx *ctx, const frw_job *job, uint64_t *ticket);
/* Cancel a submitted request: a queued one is never admitted; a running one has
 * its walks dropped and its job closed by the kernel at its next epoch.  The
 * ticket then completes with FRW_ECANCELED (frw_wait still collects it).
 * FRW_ENOTFOUND for an unknown or collected ticket; a request that has already
 * completed keeps its result (FRW_OK returned, nothing changed). */
int frw_cancel(frw_ctx *ctx, uint64_t ticket);

/* Counters of the serving loop since the context was created. */
typedef struct {
    uint64_t submitted, completed, cancelled, refused;   /* refused: could never fit (FRW_ENOMEM) */
    uint64_t runs;                /* open runs of the walk kernel started */
    uint64_t runs_failed;         /* runs that ended with a device error status (e.g. the idle limit
                                     of idle_timeout_ms ran out); the next request starts a new run */
    uint32_t last_status;         /* device status flags of the last failed run (0: none) */
    uint32_t reserved;
} frw_serve_info;
int frw_get_serve_info(frw_ctx *ctx, frw_serve_info *out);
int frw_poll(frw_ctx *ctx, uint64_t ticket, int32_t *done);
int frw_wait(frw_ctx *ctx, uint64_t ticket, double timeout_s, double *C_row, double *stderr_row,
             frw_stats *stats);

/* Per-walk records of walks walk_begin .. walk_begin + n_walks - 1 (host arrays of
 * n_walks entries each; any may be NULL): weight omega, electrode reached
 * (n_cond = ground, -1 = capped), hop count, MicroWalk steps, first-cube branch. */
int frw_walk_records(frw_ctx *ctx, int32_t structure_id, int32_t master, uint64_t request_id,
                     uint64_t walk_begin, uint64_t n_walks, double *omega, int32_t *electrode,
                     uint32_t *hops, uint64_t *micro_steps, int32_t *branch);

/* MicroWalk alone (Algorithm 3) on n_cubes lattice cubes of edge N given as
 * integer voxel ranges; samples_per_cube walks from the centre of each.
 * d_cubes (device): n_cubes records of 64 int32: [0] background material,
 * [1] block count 0 <= K <= 8, [2 + 7b .. 8 + 7b] block b = (i0, i1, j0, j1, k0, k1,
 * mat) with 0 <= lo < hi <= N; later blocks win.  Material ids index eps_r (host)
 * and must be below n_mat.  Sample s of cube c is walk id c * samples_per_cube + s.
 * Outputs (device): d_exit[walk] = (x+1) | (y+1) << 8 | (z+1) << 16 of the exit node
 * (one coordinate is -1 or N), d_steps[walk] = number of steps.  Either output may
 * be NULL.  The records are checked on the device: a malformed one (K, a range or
 * a material id out of bounds) makes the call return FRW_EINVAL, its samples are
 * written as exit 0 and 0 steps, and the other cubes' samples are still valid. */
int frw_microwalk_cubes(frw_ctx *ctx, int32_t N, int32_t n_cubes, const int32_t *d_cubes,
                        const double *eps_r, int32_t n_mat, uint64_t samples_per_cube,
                        uint64_t request_id, uint32_t *d_exit, uint32_t *d_steps);

/* Allocation-free variant of frw_microwalk_cubes (the paper has no counterpart:
 * this is a deployment convenience).  Some callers cannot allocate device memory:
 * a host application that owns all device memory through its own allocator, or a
 * loop with a fixed device-memory budget that must not pay the device-wide
 * synchronisation that cudaMalloc / cudaFree imply.  This entry point allocates
 * nothing and needs no context: it runs on the current CUDA device and on
 * `cuda_stream` (cudaStream_t as void*, NULL = the default stream), takes the same
 * inputs and writes the same outputs as frw_microwalk_cubes (bit-identical for the
 * same seed and request id), and keeps its scratch -- the job counter, an error
 * word and the 16 x 16 jump-weight table, 1.25 KB in all -- in one fixed
 * file-scope device array of 2 KB that every GPU loading the library holds until
 * the process exits.
 *   - The first call on a device looks up that array's device address (once per
 *     device) and keeps it for the life of the process; after cudaDeviceReset the
 *     kept address is stale, so do not use this entry point on a device that has
 *     been reset in the same process.
 *   - Every call shares the array: it zeroes the counter and error word and writes
 *     the weight table before its launch, so calls in sequence are independent, but
 *     calls that overlap on the GPU (other streams, other host threads) race.
 *   - Limits: 2 <= N <= 32 even, at most 15 materials (n_mat > 15 returns
 *     FRW_ECAPACITY: the weight table has 15 rows), permittivities positive and
 *     finite, records as for frw_microwalk_cubes (at most 8 blocks, material ids
 *     below n_mat; a malformed record returns FRW_EINVAL).
 *   - Every call copies its error word back and synchronises `cuda_stream`, so it
 *     blocks the calling thread until the launch has finished and cannot be
 *     recorded into a CUDA graph.  FRW_EDEVICE if the kernel's step cap was hit or
 *     a CUDA call failed. */
int frw_microwalk_cubes_noalloc(int32_t N, int32_t n_cubes, const int32_t *d_cubes, const double *eps_r,
                                int32_t n_mat, uint64_t seed, uint64_t samples_per_cube, uint64_t request_id,
                                uint32_t *d_exit, uint32_t *d_steps, void *cuda_stream);

/* FD-based transition (Algorithm 2) on n_cubes lattice cubes given as for
 * frw_microwalk_cubes (records of 64 int32, at most 8 blocks; N = the context's N,
 * N <= FRW_FDM_MAX_N): per cube, the discrete SGF P = e_c^T A_II^{-1} A_IB of Eq. 8
 * with the unquantised alpha of Eq. 6 and e_c averaging the 8 central nodes, from a
 * mixed-precision solve of the symmetric FD system (FP32 conjugate gradients
 * refined in FP64 until the FP64 residual is at most 1e-12 of ||e_c||_2), then one
 * boundary node sampled with the word d_u[c]: the first panel, in natural face
 * order (face 2a + side, then the other two axes in increasing order), whose
 * threshold min(floor(2^32 cum / total), 2^32 - 1) exceeds the word.
 * Device inputs: d_cubes; d_u (n_cubes words; NULL: 0xffffffff for every cube).
 * Device outputs, each may be NULL: d_P[c * 6N^2 + m] = P of panel m (not
 * normalised: the sum is 1 up to the solve's residual); d_exit[c] = the sampled
 * boundary node, packed as by frw_microwalk_cubes; d_iters[c] = inner conjugate-
 * gradient iterations | (refinement passes << 24).  FRW_EDEVICE if a solve did not
 * reach its tolerance.  Blocks the calling thread until done. */
int frw_fdm_cubes(frw_ctx *ctx, int32_t N, int32_t n_cubes, const int32_t *d_cubes, const double *eps_r,
                  int32_t n_mat, const uint32_t *d_u, double *d_P, uint32_t *d_exit, uint32_t *d_iters);

/* One analytical table computed on the device (Eq. 8 for SGF kinds; the
 * first-cube flux kernel for FLUX kinds) for the context's N: profile[N] = material
 * ids (into eps_r) of the layers along table axis t2 (ignored for HOM kinds).
 * Host outputs: thr[6N^2] sampling thresholds in canonical panel order,
 * neg[6N^2] sign flags (flux kinds), *total = sum of |values| (flux) or of P (SGF),
 * values[6N^2] (may be NULL) the raw panel values. */
int frw_table(frw_ctx *ctx, int32_t kind, const int32_t *profile, const double *eps_r,
              int32_t n_mat, uint32_t *thr, uint8_t *neg, double *total, double *values);

/* Message for a status code, and the detail of the context's last error. */
const char *frw_strerror(int code);
const char *frw_last_error(frw_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FRW_H */
