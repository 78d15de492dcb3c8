// frw_internal.h -- device data layout shared by the kernels (frw_kernels.cu) and
// the host runtime (frw_runtime.cu).  Not part of the public ABI (include/frw.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace frw {

constexpr int MAXN = 32;                 // lattice edge limit (mask rows, byte coords)
constexpr int KMAX = 14;                 // blocks per transition cube (mask bits 1..14)
constexpr int BOUNDARY = 15;             // material id of absorbing boundary nodes
constexpr int NMAT = 16;                 // material slots (15 real + boundary)
constexpr double EPS0 = 8.8541878128e-3; // fF / um
constexpr int FDM_MAX_N = 24;            // FD transitions: p and r of N^3 floats in shared memory
constexpr int GUIDE = 2048;              // guide-table buckets of the inverse-CDF sampler (2^11)

// analytical table kinds (same numbering as the ABI's FRW_TAB_*)
enum : uint32_t { TAB_SGF = 0, TAB_FLUX_PAR = 1, TAB_FLUX_PERP = 2, TAB_SGF_HOM = 3, TAB_FLUX_HOM = 4 };
// table cache entry states
enum : uint32_t { TE_EMPTY = 0, TE_CLAIMED = 1, TE_REQUESTED = 2, TE_READY = 3 };
// walk slot states
enum : uint32_t { ST_IDLE = 0, ST_FRESH = 1, ST_FIRST = 2, ST_HOP = 3, ST_MW = 4, ST_MWDONE = 5 };
// device error flags (status word 1)
enum : uint32_t {
    ERR_MWQ_OVERFLOW = 1u, ERR_CACHE_FULL = 2u, ERR_FILL = 4u, ERR_SHRINK = 8u, ERR_ACC_RANGE = 16u,
    ERR_MW_STEPS = 32u, ERR_IDLE_TIMEOUT = 64u, ERR_REDUCE_QUEUE = 128u,
    ERR_CHECK = 256u,             // a bounds check of the debug build (-DFRW_CHECKS) failed
    ERR_FDM = 512u,               // an FD transition solve did not reach its tolerance
    ERR_INPUT = 1024u             // a caller-given cube record is malformed (block count, range, material id)
};
// status words
enum { STAT_ACTIVE = 0, STAT_ERR = 1, STAT_BUILT = 2, STAT_MWJOBS = 3, STAT_EPOCHS = 4, STAT_SUSPENDED = 5,
       STAT_PROGRESS = 6,   // epochs in which some walk-kernel CTA had work (its idle CTAs wait while it moves)
       STAT_STAGED = 7,     // walk-kernel CTAs that read the structure geometry from their shared-memory copy
       STAT_WORDS = 8 };
// host control words read by the running walk kernel
enum { CTRL_OPEN = 0, CTRL_ABORT = 1, CTRL_WORDS = 4 };

// cube classes
enum : int { CUBE_HOM = 0, CUBE_STRAT = 1, CUBE_NONSTRAT = 2, CUBE_OVERFLOW = 3 };

// fixed-point scales of the exact 128-bit accumulators
constexpr double ACC_S1_SCALE = 18446744073709551616.0;   // 2^64
constexpr double ACC_S2_SCALE = 1099511627776.0;          // 2^40

// One loaded structure.  Coordinates SoA: x[a * n + i].  Material ids are the
// context's global ids.
struct DevStructure {
    int n_c, n_b, bg;      // conductor boxes, dielectric blocks, background material
    int n_cond;            // conductors (a conductor is the union of its boxes); the walls are n_cond
    double dom_lo[3], dom_hi[3];
    float dom_lo_f[3], dom_hi_f[3];
    double tau;            // absorption distance, FP64 mode
    float tau_f;           // absorption distance, FP32 mode
    float margin_f;        // FP32 cube-size safety margin
    const double *c_lo, *c_hi;
    const float *c_lo_f, *c_hi_f;
    const double *b_lo, *b_hi;
    const float *b_lo_f, *b_hi_f;
    const uint8_t *b_mat;
    const int32_t *box_cond;   // conductor of each box (boxes sorted by conductor)
    // index built at load time:
    //  - uniform grid; each cell lists (ascending) every conductor that can be the
    //    nearest electrode of some point of the cell (exact nearest query);
    //  - per axis, slab prefix masks: L[a][s] = blocks with lo below the upper edge
    //    of slab s, H[a][s] = blocks with hi above its lower edge, so that
    //    L[a][slab(c+R)] & H[a][slab(c-R)] over the three axes is a superset of the
    //    blocks meeting the cube [c-R, c+R], enumerated in priority order.
    int gdim[3];
    int sl_S, sl_words;
    int pad2;
    double g_org[3], g_inv[3];
    float g_org_f[3], g_inv_f[3];
    double sl_org[3], sl_inv[3];
    float sl_org_f[3], sl_inv_f[3];
    const uint32_t *g_off;     // [cells + 1]
    const uint16_t *g_ids;
    const uint32_t *sl_L;      // [3][S][words]
    const uint32_t *sl_H;      // [3][S][words]
};

// The structure as the geometry code reads it, in one precision: the fields of
// DevStructure for that precision.  Built on the host at load time and kept in
// device memory per structure, so that walk threads reference one shared copy
// (read through L1, the same line for every thread of a structure) instead of
// each holding its own.
template <typename T> struct SView {
    int n_c, n_b, bg, n_cond;   // boxes, blocks, background, conductors
    const int32_t *bcond;       // conductor of each box
    T dlo[3], dhi[3];
    T tau, margin;
    const T *clo, *chi, *blo, *bhi;
    const uint8_t *bmat;
    int gdim[3], sl_S, sl_words;
    T g_org[3], g_inv[3], sl_org[3], sl_inv[3];
    const uint32_t *g_off;
    const uint16_t *g_ids;
    const uint32_t *sl_L, *sl_H;
};

template <typename T> __host__ __device__ inline SView<T> sview(const DevStructure &S);
template <> __host__ __device__ inline SView<double> sview<double>(const DevStructure &S)
{
    SView<double> v;
    v.n_c = S.n_c; v.n_b = S.n_b; v.bg = S.bg; v.n_cond = S.n_cond; v.bcond = S.box_cond;
    for (int a = 0; a < 3; a++) { v.dlo[a] = S.dom_lo[a]; v.dhi[a] = S.dom_hi[a]; }
    v.tau = S.tau; v.margin = 0.0;
    v.clo = S.c_lo; v.chi = S.c_hi; v.blo = S.b_lo; v.bhi = S.b_hi; v.bmat = S.b_mat;
    for (int a = 0; a < 3; a++) {
        v.gdim[a] = S.gdim[a]; v.g_org[a] = S.g_org[a]; v.g_inv[a] = S.g_inv[a];
        v.sl_org[a] = S.sl_org[a]; v.sl_inv[a] = S.sl_inv[a];
    }
    v.sl_S = S.sl_S; v.sl_words = S.sl_words;
    v.g_off = S.g_off; v.g_ids = S.g_ids; v.sl_L = S.sl_L; v.sl_H = S.sl_H;
    return v;
}
template <> __host__ __device__ inline SView<float> sview<float>(const DevStructure &S)
{
    SView<float> v;
    v.n_c = S.n_c; v.n_b = S.n_b; v.bg = S.bg; v.n_cond = S.n_cond; v.bcond = S.box_cond;
    for (int a = 0; a < 3; a++) { v.dlo[a] = S.dom_lo_f[a]; v.dhi[a] = S.dom_hi_f[a]; }
    v.tau = S.tau_f; v.margin = S.margin_f;
    v.clo = S.c_lo_f; v.chi = S.c_hi_f; v.blo = S.b_lo_f; v.bhi = S.b_hi_f; v.bmat = S.b_mat;
    for (int a = 0; a < 3; a++) {
        v.gdim[a] = S.gdim[a]; v.g_org[a] = S.g_org_f[a]; v.g_inv[a] = S.g_inv_f[a];
        v.sl_org[a] = S.sl_org_f[a]; v.sl_inv[a] = S.sl_inv_f[a];
    }
    v.sl_S = S.sl_S; v.sl_words = S.sl_words;
    v.g_off = S.g_off; v.g_ids = S.g_ids; v.sl_L = S.sl_L; v.sl_H = S.sl_H;
    return v;
}

// One extraction job (request x master).
// 256-byte aligned: the host publishes jobs into a running kernel, and no cache
// line of a job may be shared with another job's.
struct alignas(256) DevJob {
    int sid;               // index into the structure table
    int master;
    int n_c;
    int record;            // write per-walk records
    uint32_t key0, key1;   // Philox key
    double g_lo[3], g_hi[3];
    double cum[6];         // cumulative face areas of the Gaussian surface
    double area;
    uint64_t walk_begin;   // walk ids walk_begin .. walk_begin + walk_count - 1
    uint64_t walk_count;
    uint64_t batch;        // walks per accumulator batch
    uint64_t acc_base;     // u64 offset of batch 0 in the accumulator pool
    uint32_t acc_stride;   // u64 words per batch
    uint32_t pad;
    uint64_t rec_base;     // offset of walk 0 in the record arrays
    uint64_t batch_base;   // index of batch 0 in the run's batch arrays
    double sigma;          // relative standard-error target (0: budget only)
};

// Device-side state of a job (followed in walk-id order): its completed batches
// are folded, in order, into its running sums; the job is decided when its stop
// rule holds or its budget is used up.
struct JobState {
    unsigned long long prefix;     // complete batches folded so far
    unsigned long long used;       // walks in the estimate once decided
    uint32_t decided;              // 1: converged, 2: budget exhausted, 3: cancelled
    uint32_t lock;                 // held by the thread folding batches
    uint32_t pending;              // set by a thread that found the lock held
    uint32_t pad;
};

// job-table control words (device memory)
enum {
    JC_PUBLISHED = 0,   // jobs 0 .. published-1 are visible to the kernel (host-written)
    JC_DECIDED = 1,     // number of decided jobs (device counter)
    JC_LOW = 2,         // every job below this index is decided (device, monotone)
    JC_WORDS = 4
};

// per-batch accumulator block (u64 words):
//   [0, 2(nc+1))            S1 as (lo, hi) int128 pairs, fixed point 2^-64
//   [2(nc+1), 4(nc+1))      S2 as (lo, hi) pairs, fixed point 2^-40
//   +0 done, +1 hops, +2 steps, +3 strat, +4 hom, +5 mw, +6..8 branches, +9 truncated
constexpr int ACC_EXTRA = 10;
__host__ __device__ inline uint32_t acc_stride_for(int nc) { return 4u * (uint32_t)(nc + 1) + ACC_EXTRA; }

// MicroWalk job: one non-stratified transition cube handed from the geometry
// kernel to the MicroWalk kernel.  rng[b] = (i0 | i1<<8 | j0<<16 | j1<<24,
// k0 | k1<<8 | mat<<16) for the cube's blocks in priority order.
struct alignas(16) MWJob {
    uint32_t slot, hop, walk_lo, walk_hi;
    uint32_t start, K, mm_lo, mm_hi;   // start node packed x|y<<8|z<<16; material nibble map
    uint32_t key0, key1, pad0, pad1;
    uint2 rng[KMAX];
};

struct SlotArrays {
    uint32_t *state, *job, *hop, *exitnode, *cnt_sh, *cnt_mw;
    int32_t *branch;
    uint64_t *walk, *steps;
    double *pos;      // [3][NS]
    double *cube;     // [4][NS]  c0, c1, c2, R of the cube handed to MicroWalk
    double *omega;
};

// Per-walk records (one entry per walk id of every job of a run).  k starts at
// REC_PENDING and is written last, when the walk finishes.
constexpr int32_t REC_PENDING = (int32_t)0x80808080;
struct RecArrays {
    double *omega;
    int32_t *k;
    uint32_t *hops;
    uint32_t *steps;
    uint32_t *cnt_sh;   // strat hops (low 16) | homogeneous hops (high 16)
    uint32_t *cnt_mw;
    int32_t *branch;
};

struct TableCache {
    uint32_t cap;          // power of two
    uint32_t P;            // panels per table = 6 N^2
    uint32_t P32;          // sign words per table
    uint32_t *keys;        // [cap][5]
    uint32_t *state;       // [cap]
    uint32_t *thr;         // [cap + 2][P]; entries cap, cap+1 = homogeneous SGF / flux
    uint32_t *sgn;         // [cap + 2][P32]
    uint16_t *guide;       // [cap + 2][GUIDE]: first panel whose threshold exceeds each bucket start
    double *ktot;          // [cap + 2]
    uint32_t *fillq;       // [cap]
    uint32_t *fillq_count, *fillq_head;
};

// Constants of the separable solve (host-computed, see fill kernel):
// u[(p-1)*N + i] = DST-II basis, lam[p-1], a[p-1], d[p-1].
struct FillConsts {
    const double *u, *lam, *a, *d;
};

struct EngineView {
    int N;
    int hybrid;
    int max_hops;
    int fp32;
    uint32_t NS;           // slots = grid x pool
    uint32_t pool;         // slots per CTA of the walk kernel (multiple of its block size)
    int n_jobs;            // job-table capacity
    int max_nc;            // largest conductor count a job of this run may have (reduction scratch)
    SlotArrays s;
    const DevStructure *structs;
    const void *view_f, *view_d;     // per structure: SView<float>[] and SView<double>[]
    const DevJob *jobs;
    unsigned long long *job_next;    // next walk offset per job (claimed by compare-and-swap)
    unsigned long long *job_limit;   // issue limit per job (<= walk_count), written by the host
    int *job_cancel;                 // 1: the stop rule holds; 2: cancelled by the host (walks dropped)
    JobState *jstate;                // per job
    uint32_t *jctl;                  // JC_WORDS job-table control words
    uint32_t *batch_job;             // job of each batch
    unsigned long long *jsum;        // per job: running prefix sums, acc_stride words each
    unsigned long long *jsum_off;    // per job: offset of its running sums
    unsigned long long *acc;         // batch accumulator blocks
    uint32_t *batch_done;            // finished walks per batch
    uint32_t *batch_ready;           // 1 once the batch block is written
    uint32_t *rq, *rq_count, *rq_head;   // queue of completed batches awaiting reduction
    uint32_t rq_cap;
    RecArrays rec;
    uint64_t rec_cap, acc_cap, jsum_cap;   // record, accumulator and running-sum capacities (bounds checks)
    MWJob *mwq;                      // one MicroWalk job record per slot
    TableCache tc;
    const uint32_t *W;     // [16][16] quantised alpha of Eq. 6 by global material (row: centre)
    int wtab_lanes;        // 1: every material id of the context is below 7 (the per-lane table copies)
    const double *eps;     // [16]
    FillConsts fc;
    double *fill_scratch;  // per walk-kernel CTA: fill_stride doubles of table-fill scratch
    size_t fill_stride;
    uint32_t *status;      // STAT_WORDS
    uint32_t *ctrl;        // CTRL_WORDS (host -> device)
    unsigned long long *cycles;   // [5] CTA cycles: geometry busy, fill, reduce, MicroWalk busy, total
    double idle_timeout_s; // idle wait limit of the walk kernel
    int hops_per_epoch;    // analytical hops one walk may take per epoch (tunable, >= 1)
    int mwe;               // MicroWalk-E expansion factor (0 or 1: plain MicroWalk)
    int transition;        // non-stratified transitions: 0 MicroWalk, 1 FD solve (FRW-FDM)
    unsigned char *fdm_scratch;   // FRW-FDM: per walk-kernel CTA, fdm_cube_scratch_bytes(N)
    int geo_warps;         // 0: phased walk kernel; else warps per CTA on geometry (warp-specialised kernel)
    int stage_sid;         // structure whose geometry every CTA copies into shared memory (-1: none)
    uint32_t stage_flags;  // STAGE_* groups copied
    uint32_t stage_off;    // byte offset of the copy in the walk kernel's dynamic shared memory
    uint32_t stage_bytes;  // its size (dynamic shared memory = stage_off + stage_bytes)
    int suspend_lanes;     // a MicroWalk warp with at most this many lanes left may suspend them
    uint32_t suspend_min_steps;   // ... once each has made this many steps in the epoch
};

// Shared-memory copy of one structure's geometry in the walk kernel (the max-cube
// query of Sec. II-A and the cube classification read it): groups of arrays in
// this order, each group 16-byte aligned; T = float or double (tsize bytes).
constexpr uint32_t STAGE_BOXES = 1u;    // conductor boxes: clo[3 n_c], chi[3 n_c]
constexpr uint32_t STAGE_BLOCKS = 2u;   // dielectric blocks: blo[3 n_b], bhi[3 n_b], then bmat[n_b]
constexpr uint32_t STAGE_SLABS = 4u;    // slab masks: sl_L[3 S w], sl_H[3 S w]
__host__ __device__ inline uint32_t stage_round16(uint32_t b) { return (b + 15u) & ~15u; }
__host__ __device__ inline uint32_t stage_group_bytes(uint32_t grp, int n_c, int n_b, int sl_S, int sl_words,
                                                      int tsize)
{
    if (grp == STAGE_BOXES) return stage_round16(6u * (uint32_t)n_c * (uint32_t)tsize);
    if (grp == STAGE_BLOCKS)
        return n_b > 0 ? stage_round16(6u * (uint32_t)n_b * (uint32_t)tsize) + stage_round16((uint32_t)n_b) : 0u;
    return stage_round16(2u * 3u * (uint32_t)sl_S * (uint32_t)sl_words * 4u);
}

// ---- launchers (frw_kernels.cu) ----
struct LaunchShape {
    int geom_threads;
    int mw_warps;
    int mw_ctas_per_sm;
    int fill_ctas;
    int sms;
};

// the persistent walk kernel: runs every job of the view to completion
// (prepare_walk sets its shared-memory limit; call it before launching, and
// outside any stream capture)
cudaError_t prepare_walk(const EngineView &E);
cudaError_t launch_walk(const EngineView &E, const LaunchShape &L, cudaStream_t st);
size_t walk_smem_bytes(int N, int max_nc, int transition);
size_t walk_fill_scratch_doubles(int N);
int walk_pool_slots();
int walk_geo_warps_max();
int walk_ctas_per_sm(int N, int fp32, int mwe, int transition);
// dynamic shared memory a walk-kernel CTA may add for the geometry copy without
// lowering the kernel's CTAs per SM below ctas_per_sm (0: no copy for this view)
uint32_t walk_stage_cap(const EngineView &E, int ctas_per_sm);
// FD transitions (Algorithm 2) of stand-alone cubes, one CTA per cube at a time;
// scratch = grid x fdm_cube_scratch_bytes(N)
size_t fdm_cube_scratch_bytes(int N);
cudaError_t launch_fdm_cubes(int N, const int32_t *d_cubes, uint32_t n_cubes, const uint8_t *map, const double *eps,
                             const uint32_t *d_u, double *d_P, uint32_t *d_exit, uint32_t *d_iters,
                             unsigned char *scratch, int grid, uint32_t *d_err, cudaStream_t st);
// fill one table with an explicit key into entry `entry` of the cache arrays
cudaError_t launch_fill_one(const EngineView &E, uint32_t kind, const uint32_t prof[4],
                            uint32_t entry, double *values_out, cudaStream_t st);
size_t fill_smem_bytes(int N);
size_t mw_smem_bytes(int N, int warps);
cudaError_t launch_mw_cubes(int N, const int32_t *d_cubes, uint64_t n_cubes, uint64_t spc,
                            uint32_t key0, uint32_t key1, int n_mat, int n_global_mat,
                            const uint8_t *matmap_local_to_global,
                            const uint32_t *W, uint32_t *d_exit, uint32_t *d_steps,
                            unsigned long long *d_head, uint32_t *d_err, const LaunchShape &L,
                            cudaStream_t st);
cudaError_t set_kernel_attributes(int N, int mw_warps, int max_nc);
// uniform-grid candidate lists of one structure (frw_kernels.cu, k_grid_lists):
// pass 0 writes the counts and turns them into offsets off[0 .. cells] (off has
// cells + 1 entries; off[cells] = the list total), pass 1 writes ids[off[c] ..)
struct GridBuild {
    int gdim[3];
    int n_box;
    double dlo[3], dhi[3];   // domain
    double w[3];             // cell edge per axis (extent / gdim)
    double tol;              // list tolerance (covers FP32 rounding of device distances)
    const double *clo, *chi; // device boxes, SoA [a * n_box + k]
};
cudaError_t launch_grid_lists(const GridBuild &G, uint32_t *off, uint16_t *ids, int pass, cudaStream_t st);

}  // namespace frw
