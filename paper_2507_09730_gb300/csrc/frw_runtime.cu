// frw_runtime.cu -- host side of the C ABI in include/frw.h: context, material
// registry, structure loading and validation, runs of the persistent walk kernel
// (closed runs for frw_extract*, open runs fed by the serving loop).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "frw.h"
#include "frw_internal.h"

using namespace frw;

namespace {

struct HostStructure {
    int n_c = 0, n_b = 0;             // conductors, dielectric blocks
    int n_box = 0;                    // conductor boxes (sorted by conductor)
    int mat_need = 0;                 // 1 + the largest global material id it uses
    std::vector<double> c_lo, c_hi;   // n_box x 3 (AoS, host copy for Gaussian set-up)
    std::vector<int32_t> box_cond;    // conductor of each box
    std::vector<int32_t> master_box;  // per conductor: its box if it has exactly one, else -1
    double dom_lo[3], dom_hi[3];
    std::vector<void *> dev;          // device allocations of this structure
    DevStructure d;
    bool live = false;
};

// Job table and arenas of the persistent walk kernel (device), owned by the
// context and grown on demand between runs.
struct RunBufs {
    uint32_t jcap = 0;
    uint64_t bcap = 0, acap = 0, scap = 0;
    DevJob *jobs = nullptr;
    unsigned long long *next = nullptr, *limit = nullptr, *jsum = nullptr, *jsoff = nullptr, *acc = nullptr;
    int *cancel = nullptr;
    JobState *js = nullptr;
    uint32_t *done = nullptr, *ready = nullptr, *bjob = nullptr, *rq = nullptr, *rqc = nullptr, *jctl = nullptr;
    std::vector<void *> allocs;
};

struct Server;

}  // namespace

struct frw_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    frw_options opt;
    LaunchShape shape;
    std::string last_error;
    // materials (global ids)
    std::vector<double> eps;
    uint32_t W[16][16];
    // device memory
    std::vector<void *> allocs;
    uint32_t NS = 0;
    SlotArrays slots;
    MWJob *mwq = nullptr;               // one MicroWalk job record per slot
    TableCache tc;
    uint32_t *status = nullptr;
    uint32_t *d_W = nullptr;
    double *d_eps = nullptr;
    FillConsts fc;
    double *fc_buf = nullptr;
    DevStructure *d_structs = nullptr;
    SView<float> *d_view_f = nullptr;    // per structure, built at load
    SView<double> *d_view_d = nullptr;
    int struct_cap = 0;
    std::vector<HostStructure> structs;
    uint32_t *h_status = nullptr;       // pinned
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t aux = nullptr;                // control / monitoring copies during a run
    uint32_t *ctrl = nullptr;                  // device control words
    unsigned long long *cycles = nullptr;      // phase cycle counters
    int grid = 0;                              // walk-kernel CTAs
    double *fill_scratch = nullptr;            // per CTA table-fill scratch
    unsigned char *fdm_scratch = nullptr;      // FRW-FDM: per CTA FD-solve scratch
    RecArrays rec;                      // per-walk records (grown on demand)
    uint64_t rec_cap = 0;
    std::vector<void *> rec_allocs;
    RunBufs rb;                         // job table and arenas
    std::mutex engine_mu;               // held for the whole of a run (closed or serving)
    std::mutex struct_mu;               // guards the host structure table against the serving thread
    Server *srv = nullptr;              // serving loop (started by the first frw_submit)
    frw_tuning tune;                    // walk-kernel settings (defaults or frw_autotune)
};

static const char *kErr[] = {"ok",
                             "invalid argument",
                             "out of device memory / admission refused",
                             "timeout",
                             "device error",
                             "walk budget exhausted before the sigma target",
                             "capacity exceeded",
                             "not found",
                             "cancelled"};

static int fail(frw_ctx *c, int code, const std::string &msg)
{
    if (c) c->last_error = msg;
    return code;
}

static int cuda_fail(frw_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? FRW_ENOMEM : FRW_EDEVICE, m);
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

template <typename T> static int dalloc(frw_ctx *ctx, T **p, size_t count, std::vector<void *> &owner)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    owner.push_back(q);
    *p = (T *)q;
    return FRW_OK;
}

// ---------------------------------------------------------------------------
// quantised alpha of Eq. 6: W[v][i] = round(eps_i / (eps_i + eps_v) * 2^24), boundary 2^24
static void rebuild_w(frw_ctx *ctx)
{
    for (int a = 0; a < 16; a++)
        for (int b = 0; b < 16; b++) ctx->W[a][b] = 0;
    const int n = (int)ctx->eps.size();
    for (int v = 0; v < n; v++) {
        for (int i = 0; i < n; i++) {
            const double al = ctx->eps[i] / (ctx->eps[i] + ctx->eps[v]);
            ctx->W[v][i] = (uint32_t)std::floor(al * 16777216.0 + 0.5);
        }
        ctx->W[v][BOUNDARY] = 16777216u;
    }
}

// map a local permittivity table onto global material ids (exact equality merges)
static int register_materials(frw_ctx *ctx, const double *eps_r, int n_mat, std::vector<uint8_t> &map)
{
    map.assign(16, 0);
    std::vector<double> add = ctx->eps;
    for (int i = 0; i < n_mat; i++) {
        if (!(eps_r[i] > 0.0) || !std::isfinite(eps_r[i]))
            return fail(ctx, FRW_EINVAL, "permittivity must be positive and finite");
        int g = -1;
        for (size_t j = 0; j < add.size(); j++)
            if (add[j] == eps_r[i]) g = (int)j;
        if (g < 0) {
            if ((int)add.size() >= FRW_MAX_MATERIALS)
                return fail(ctx, FRW_ECAPACITY, "more than 15 distinct permittivities in one context");
            add.push_back(eps_r[i]);
            g = (int)add.size() - 1;
        }
        map[i] = (uint8_t)g;
    }
    if (add.size() != ctx->eps.size()) {
        ctx->eps = add;
        rebuild_w(ctx);
        double e16[16] = {0};
        for (size_t j = 0; j < ctx->eps.size(); j++) e16[j] = ctx->eps[j];
        CK(cudaMemcpyAsync(ctx->d_eps, e16, sizeof(e16), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_W, ctx->W, sizeof(ctx->W), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return FRW_OK;
}

static EngineView make_view(frw_ctx *ctx)
{
    EngineView E;
    memset(&E, 0, sizeof(E));
    E.N = ctx->opt.N;
    E.hybrid = ctx->opt.hybrid;
    E.max_hops = ctx->opt.max_hops;
    E.fp32 = ctx->opt.precision == FRW_FP32_GEOM;
    E.NS = ctx->NS;
    E.pool = ctx->grid ? ctx->NS / ctx->grid : ctx->NS;
    E.s = ctx->slots;
    E.structs = ctx->d_structs;
    E.view_f = ctx->d_view_f;
    E.view_d = ctx->d_view_d;
    E.mwq = ctx->mwq;
    E.tc = ctx->tc;
    E.W = ctx->d_W;
    E.wtab_lanes = ctx->eps.size() <= 7 ? 1 : 0;
    E.eps = ctx->d_eps;
    E.fc = ctx->fc;
    E.status = ctx->status;
    E.fill_scratch = ctx->fill_scratch;
    E.fill_stride = walk_fill_scratch_doubles(ctx->opt.N);
    E.ctrl = ctx->ctrl;
    E.cycles = ctx->cycles;
    E.idle_timeout_s = ctx->opt.idle_timeout_ms > 0 ? 1e-3 * ctx->opt.idle_timeout_ms : 10.0;
    E.hops_per_epoch = ctx->tune.hops_per_epoch;
    E.mwe = ctx->opt.mwe_factor;
    E.transition = ctx->opt.transition;
    E.fdm_scratch = ctx->fdm_scratch;
    E.suspend_lanes = ctx->tune.suspend_lanes;
    E.suspend_min_steps = (uint32_t)ctx->tune.suspend_min_steps;
    E.geo_warps = ctx->opt.transition == FRW_TRANSITION_FDM ? 0 : ctx->tune.geo_warps;
    E.stage_sid = -1;   // no geometry copy unless choose_stage picks one
    return E;
}


// ---------------------------------------------------------------------------
extern "C" void frw_default_options(frw_options *o)
{
    memset(o, 0, sizeof(*o));
    o->N = 24;
    o->precision = FRW_FP64_GEOM;
    o->seed = 0;
    o->first_cube_mode = FRW_FIRST_HYBRID;
    o->hybrid = 1;
    o->gauss_offset_frac = 0.5;
    o->max_hops = 100000;
}

extern "C" const char *frw_strerror(int code)
{
    if (code < 0 || code > 8) return "unknown status";
    return kErr[code];
}

extern "C" const char *frw_last_error(frw_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

extern "C" int frw_set_stream(frw_ctx *ctx, void *s)
{
    if (!ctx) return FRW_EINVAL;
    ctx->stream = s ? (cudaStream_t)s : ctx->own_stream;
    return FRW_OK;
}

static void stop_server(frw_ctx *ctx);

extern "C" void frw_destroy(frw_ctx *ctx)
{
    if (!ctx) return;
    stop_server(ctx);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &s : ctx->structs)
        for (void *p : s.dev) cudaFree(p);
    for (void *p : ctx->allocs) cudaFree(p);
    for (void *p : ctx->rec_allocs) cudaFree(p);
    for (void *p : ctx->rb.allocs) cudaFree(p);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    delete ctx;
}

static int check_status(frw_ctx *ctx, cudaStream_t st = nullptr)
{
    if (!st) st = ctx->stream;
    CK(cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(uint32_t) * STAT_WORDS, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const uint32_t e = ctx->h_status[STAT_ERR];
    if (e) {
        char buf[256];
        snprintf(buf, sizeof buf, "device check failed (flags 0x%x: %s%s%s%s%s%s%s%s%s%s%s)", e,
                 (e & ERR_MWQ_OVERFLOW) ? "queue overflow " : "", (e & ERR_CACHE_FULL) ? "table cache full " : "",
                 (e & ERR_FILL) ? "table fill check " : "", (e & ERR_SHRINK) ? "cube shrink limit " : "",
                 (e & ERR_ACC_RANGE) ? "accumulator range " : "", (e & ERR_MW_STEPS) ? "MicroWalk step cap " : "",
                 (e & ERR_IDLE_TIMEOUT) ? "idle limit " : "", (e & ERR_REDUCE_QUEUE) ? "reduction queue " : "",
                 (e & ERR_CHECK) ? "bounds check " : "", (e & ERR_FDM) ? "FD solve tolerance " : "",
                 (e & ERR_INPUT) ? "malformed cube record" : "");
        return fail(ctx, (e & ERR_INPUT) ? FRW_EINVAL : (e & ERR_CACHE_FULL) ? FRW_ECAPACITY : FRW_EDEVICE, buf);
    }
    return FRW_OK;
}

extern "C" int frw_create(frw_ctx **out, int device, const frw_options *opt_in)
{
    if (!out) return FRW_EINVAL;
    *out = nullptr;
    frw_options opt;
    if (opt_in) opt = *opt_in;
    else frw_default_options(&opt);
    if (opt.N < 2 || opt.N > FRW_MAX_N || (opt.N & 1)) return FRW_EINVAL;
    if (opt.precision != FRW_FP64_GEOM && opt.precision != FRW_FP32_GEOM) return FRW_EINVAL;
    if (!(opt.gauss_offset_frac > 0.0 && opt.gauss_offset_frac < 1.0)) return FRW_EINVAL;
    if (opt.max_hops <= 0) return FRW_EINVAL;
    if (opt.mw_warps_per_cta < 0 || opt.mw_warps_per_cta > 16 || opt.mw_ctas_per_sm < 0 || opt.mw_ctas_per_sm > 32)
        return FRW_EINVAL;
    if (opt.mwe_factor < 0 || opt.mwe_factor > 16 || opt.idle_timeout_ms < 0) return FRW_EINVAL;
    if (opt.transition != FRW_TRANSITION_MICROWALK && opt.transition != FRW_TRANSITION_FDM) return FRW_EINVAL;
    if (opt.transition == FRW_TRANSITION_FDM && (opt.N > FDM_MAX_N || opt.mwe_factor > 1)) return FRW_EINVAL;
    frw_ctx *ctx = new frw_ctx();
    ctx->opt = opt;
    ctx->device = device;
    cudaError_t ce = cudaSetDevice(device);
    if (ce != cudaSuccess) {
        int r = cuda_fail(ctx, ce, "cudaSetDevice");
        delete ctx;
        return r;
    }
    int rc = FRW_OK;
    auto bail = [&](int code) {
        frw_destroy(ctx);
        return code;
    };
    if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(FRW_EDEVICE);
    if (cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) != cudaSuccess) return bail(FRW_EDEVICE);
    ctx->stream = ctx->own_stream;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    ctx->shape.sms = sms > 0 ? sms : 1;
    ctx->shape.geom_threads = opt.geom_threads > 0 ? opt.geom_threads : 128;
    ctx->shape.mw_warps = opt.mw_warps_per_cta > 0 ? opt.mw_warps_per_cta : 16;
    ctx->shape.mw_ctas_per_sm = opt.mw_ctas_per_sm > 0 ? opt.mw_ctas_per_sm : 2;
    ctx->shape.fill_ctas = ctx->shape.sms;
    const int N = opt.N;
    // walk kernel: CTAs resident at once (as many per SM as fit), each with a pool of slots
    ctx->grid = walk_ctas_per_sm(N, opt.precision == FRW_FP32_GEOM, opt.mwe_factor, opt.transition) * ctx->shape.sms;
    {
        // FRW-FDM: one slot per thread by default (a CTA solves its cubes one at a time)
        const uint64_t dflt = opt.transition == FRW_TRANSITION_FDM ? 256ull * ctx->grid : (1ull << 20);
        uint64_t want = opt.slots > 0 ? (uint64_t)opt.slots : dflt;
        uint64_t pool = (want + ctx->grid - 1) / ctx->grid;
        pool = ((pool + 255) / 256) * 256;
        if (pool < 256) pool = 256;
        if (pool > (uint64_t)walk_pool_slots()) pool = walk_pool_slots();
        ctx->NS = (uint32_t)(pool * ctx->grid);
    }
    ctx->tune.pool_per_cta = (int32_t)(ctx->NS / ctx->grid);
    ctx->tune.hops_per_epoch = 1;
    ctx->tune.suspend_lanes = 32;
    ctx->tune.suspend_min_steps = 128;
    ctx->tune.geo_warps = 0;
    ctx->tune.unstaged = 0;
    ctx->tune.mw_warps_per_cta = ctx->shape.mw_warps;
    ctx->tune.mw_ctas_per_sm = ctx->shape.mw_ctas_per_sm;
    ctx->tune.walks_per_s = 0.0;
    ctx->tune.mw_steps_per_s = 0.0;
    uint32_t cap = opt.table_capacity > 0 ? (uint32_t)opt.table_capacity : (N <= 16 ? (1u << 16) : (1u << 14));
    uint32_t c2 = 1;
    while (c2 < cap) c2 <<= 1;
    cap = c2;
    auto &A = ctx->allocs;
    const uint32_t NS = ctx->NS;
    SlotArrays &S = ctx->slots;
    if ((rc = dalloc(ctx, &S.state, NS, A)) || (rc = dalloc(ctx, &S.job, NS, A)) || (rc = dalloc(ctx, &S.hop, NS, A)) ||
        (rc = dalloc(ctx, &S.exitnode, NS, A)) || (rc = dalloc(ctx, &S.cnt_sh, NS, A)) ||
        (rc = dalloc(ctx, &S.cnt_mw, NS, A)) || (rc = dalloc(ctx, &S.branch, NS, A)) ||
        (rc = dalloc(ctx, &S.walk, NS, A)) || (rc = dalloc(ctx, &S.steps, NS, A)) ||
        (rc = dalloc(ctx, &S.pos, 3 * (size_t)NS, A)) || (rc = dalloc(ctx, &S.cube, 4 * (size_t)NS, A)) ||
        (rc = dalloc(ctx, &S.omega, NS, A)) || (rc = dalloc(ctx, &ctx->mwq, NS, A)) ||
        (rc = dalloc(ctx, &ctx->status, STAT_WORDS, A)) ||
        (rc = dalloc(ctx, &ctx->d_W, 256, A)) || (rc = dalloc(ctx, &ctx->d_eps, 16, A)) ||
        (rc = dalloc(ctx, &ctx->ctrl, CTRL_WORDS, A)) || (rc = dalloc(ctx, &ctx->cycles, 8, A)) ||
        (rc = dalloc(ctx, &ctx->fill_scratch, (size_t)ctx->grid * walk_fill_scratch_doubles(N), A)))
        return bail(rc);
    if (opt.transition == FRW_TRANSITION_FDM &&
        (rc = dalloc(ctx, &ctx->fdm_scratch, (size_t)ctx->grid * fdm_cube_scratch_bytes(N), A)))
        return bail(rc);
    TableCache &T = ctx->tc;
    T.cap = cap;
    T.P = 6u * N * N;
    T.P32 = (T.P + 31) / 32;
    if ((rc = dalloc(ctx, &T.keys, 5 * (size_t)cap, A)) || (rc = dalloc(ctx, &T.state, cap, A)) ||
        (rc = dalloc(ctx, &T.thr, (size_t)(cap + 2) * T.P, A)) ||
        (rc = dalloc(ctx, &T.sgn, (size_t)(cap + 2) * T.P32, A)) || (rc = dalloc(ctx, &T.ktot, cap + 2, A)) ||
        (rc = dalloc(ctx, &T.guide, (size_t)(cap + 2) * GUIDE, A)) ||
        (rc = dalloc(ctx, &T.fillq, cap, A)) || (rc = dalloc(ctx, &T.fillq_count, 2, A)))
        return bail(rc);
    T.fillq_head = T.fillq_count + 1;
    // separable-solve constants: DST-II basis, eigenvalues, centre projections
    {
        std::vector<double> h((size_t)N * N + 3 * N);
        const double pi = 3.14159265358979323846;
        for (int p = 1; p <= N; p++) {
            for (int i = 0; i < N; i++) {
                double v;
                if (p < N) v = std::sqrt(2.0 / N) * std::sin(pi * p * (i + 0.5) / N);
                else v = ((i & 1) ? -1.0 : 1.0) / std::sqrt((double)N);
                h[(size_t)(p - 1) * N + i] = v;
            }
            const double s = std::sin(pi * p / (2.0 * N));
            h[(size_t)N * N + p - 1] = 4.0 * s * s;
            const double u0 = h[(size_t)(p - 1) * N + N / 2 - 1], u1 = h[(size_t)(p - 1) * N + N / 2];
            h[(size_t)N * N + N + p - 1] = 0.5 * (u0 + u1);
            h[(size_t)N * N + 2 * N + p - 1] = u1 - u0;
        }
        if ((rc = dalloc(ctx, &ctx->fc_buf, h.size(), A))) return bail(rc);
        if (cudaMemcpy(ctx->fc_buf, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(FRW_EDEVICE);
        ctx->fc.u = ctx->fc_buf;
        ctx->fc.lam = ctx->fc_buf + (size_t)N * N;
        ctx->fc.a = ctx->fc_buf + (size_t)N * N + N;
        ctx->fc.d = ctx->fc_buf + (size_t)N * N + 2 * N;
    }
    ctx->struct_cap = 256;
    if ((rc = dalloc(ctx, &ctx->d_structs, ctx->struct_cap, A)) || (rc = dalloc(ctx, &ctx->d_view_f, ctx->struct_cap, A)) ||
        (rc = dalloc(ctx, &ctx->d_view_d, ctx->struct_cap, A)))
        return bail(rc);
    if (cudaMallocHost(&ctx->h_status, sizeof(uint32_t) * STAT_WORDS) != cudaSuccess) return bail(FRW_ENOMEM);
    for (auto &e : ctx->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(FRW_EDEVICE);
    cudaError_t e2 = set_kernel_attributes(N, ctx->shape.mw_warps, 0);
    if (e2 != cudaSuccess) return bail(cuda_fail(ctx, e2, "cudaFuncSetAttribute"));
    cudaMemsetAsync(T.state, 0, sizeof(uint32_t) * cap, ctx->stream);
    cudaMemsetAsync(T.fillq_count, 0, sizeof(uint32_t) * 2, ctx->stream);
    cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t) * STAT_WORDS, ctx->stream);
    cudaMemsetAsync(ctx->d_W, 0, sizeof(uint32_t) * 256, ctx->stream);
    cudaMemsetAsync(ctx->d_eps, 0, sizeof(double) * 16, ctx->stream);
    // homogeneous tables (independent of the permittivity): SGF at entry cap, flux at cap + 1
    EngineView E = make_view(ctx);
    const uint32_t zero[4] = {0, 0, 0, 0};
    if (launch_fill_one(E, TAB_SGF_HOM, zero, cap, nullptr, ctx->stream) != cudaSuccess ||
        launch_fill_one(E, TAB_FLUX_HOM, zero, cap + 1, nullptr, ctx->stream) != cudaSuccess)
        return bail(cuda_fail(ctx, cudaGetLastError(), "homogeneous table fill"));
    rc = check_status(ctx);
    if (rc) return bail(rc);
    *out = ctx;
    return FRW_OK;
}

// ---------------------------------------------------------------------------
static bool box_ok(const frw_box &b)
{
    for (int a = 0; a < 3; a++)
        if (!(b.lo[a] < b.hi[a]) || !std::isfinite(b.lo[a]) || !std::isfinite(b.hi[a])) return false;
    return true;
}

static double box_gap(const double *lo1, const double *hi1, const double *lo2, const double *hi2)
{
    double d = 0.0;
    for (int a = 0; a < 3; a++) {
        const double t1 = lo2[a] - hi1[a], t2 = lo1[a] - hi2[a];
        if (t1 > d) d = t1;
        if (t2 > d) d = t2;
    }
    return d;
}

static float ulpf(float x)
{
    return std::nextafter(x, INFINITY) - x;
}

// ---------------------------------------------------------------------------
// Structure index (a0).  Nearest-conductor grid: for each cell (grown by 2 % of
// its width to absorb rounding of the device's cell computation), keep every
// conductor whose smallest possible distance to the cell does not exceed an upper
// bound on the nearest-electrode distance anywhere in the cell.  Block slabs:
// prefix masks per axis (see DevStructure).
struct IndexHost {
    int gdim[3];
    double g_org[3], g_inv[3];
    std::vector<uint32_t> g_off;
    std::vector<uint16_t> g_ids;
    int S, words;
    double sl_org[3], sl_inv[3];
    std::vector<uint32_t> L, H;
};

// Index of one structure: the uniform grid's dimensions (and, with host_lists,
// its candidate lists, built on the host's cores; otherwise the device builds the
// lists, k_grid_lists) and the slab masks of the dielectric blocks.
static void build_index(const frw_box &dom, const frw_box *cond, int nc, const frw_block *blk, int nb, IndexHost &X,
                        bool host_lists)
{
    double ext[3], vol = 1.0, edge = 0.0;
    for (int a = 0; a < 3; a++) {
        ext[a] = dom.hi[a] - dom.lo[a];
        vol *= ext[a];
        edge = std::max(edge, ext[a]);
    }
    const double target = std::min(262144.0, std::max(4096.0, 4194304.0 / std::max(1, nc)));
    const double h = std::cbrt(vol / target);
    for (int a = 0; a < 3; a++) {
        X.gdim[a] = (int)std::min(512.0, std::max(1.0, std::ceil(ext[a] / h)));
        X.g_org[a] = dom.lo[a];
        X.g_inv[a] = X.gdim[a] / ext[a];
    }
    const size_t cells = (size_t)X.gdim[0] * X.gdim[1] * X.gdim[2];
    X.g_off.clear();
    X.g_ids.clear();
    if (host_lists) {
    X.g_off.assign(cells + 1, 0);
    // candidate lists of the x-slabs [i0, i1) of cells (independent), in cell order
    auto slab = [&](int i0, int i1, std::vector<uint32_t> &count, std::vector<uint16_t> &ids) {
        std::vector<double> dmin(nc);
        for (int i = i0; i < i1; i++)
            for (int j = 0; j < X.gdim[1]; j++)
                for (int k = 0; k < X.gdim[2]; k++) {
                    const int ii[3] = {i, j, k};
                    double lo[3], hi[3];
                    for (int a = 0; a < 3; a++) {
                        const double w = ext[a] / X.gdim[a];
                        lo[a] = dom.lo[a] + ii[a] * w - 0.02 * w;
                        hi[a] = dom.lo[a] + (ii[a] + 1) * w + 0.02 * w;
                    }
                    // upper bound on the nearest-electrode distance over the cell
                    double U = INFINITY;
                    for (int a = 0; a < 3; a++) U = std::min(U, std::min(hi[a] - dom.lo[a], dom.hi[a] - lo[a]));
                    for (int c = 0; c < nc; c++) {
                        double dmax = 0.0, dm = 0.0;
                        for (int a = 0; a < 3; a++) {
                            dmax = std::max(dmax, std::max(cond[c].lo[a] - lo[a], hi[a] - cond[c].hi[a]));
                            dm = std::max(dm, std::max(cond[c].lo[a] - hi[a], lo[a] - cond[c].hi[a]));
                        }
                        dmin[c] = dm;
                        U = std::min(U, dmax);
                    }
                    const double tol = 1e-6 * edge;   // covers FP32 rounding of device distances
                    uint32_t n = 0;
                    for (int c = 0; c < nc; c++)
                        if (dmin[c] <= U + tol) {
                            ids.push_back((uint16_t)c);
                            n++;
                        }
                    count.push_back(n);
                }
    };
    // the slabs run on the host's cores (the index is the same for any split)
    const int nth = (int)std::max(1u, std::min(32u, std::min((unsigned)X.gdim[0], std::thread::hardware_concurrency())));
    std::vector<std::vector<uint32_t>> counts(nth);
    std::vector<std::vector<uint16_t>> idl(nth);
    {
        std::vector<std::thread> th;
        int started = 0;
        try {
            for (; started < nth; started++) {
                const int t = started;
                const int i0 = (int)((int64_t)X.gdim[0] * t / nth), i1 = (int)((int64_t)X.gdim[0] * (t + 1) / nth);
                th.emplace_back([&, t, i0, i1]() { slab(i0, i1, counts[t], idl[t]); });
            }
        } catch (...) {   // no thread to be had: the remaining slabs on this thread
        }
        for (int t = started; t < nth; t++)
            slab((int)((int64_t)X.gdim[0] * t / nth), (int)((int64_t)X.gdim[0] * (t + 1) / nth), counts[t], idl[t]);
        for (auto &x : th) x.join();
    }
    size_t cell = 0;
    for (int t = 0; t < nth; t++) {
        size_t p = 0;
        for (uint32_t n : counts[t]) {
            X.g_ids.insert(X.g_ids.end(), idl[t].begin() + p, idl[t].begin() + p + n);
            p += n;
            X.g_off[++cell] = (uint32_t)X.g_ids.size();
        }
    }
    }
    // slabs
    X.S = 256;
    X.words = std::max(1, (nb + 31) / 32);
    X.L.assign((size_t)3 * X.S * X.words, 0u);
    X.H.assign((size_t)3 * X.S * X.words, 0u);
    for (int a = 0; a < 3; a++) {
        const double w = ext[a] / X.S, m = w / 64.0 + 1e-9 * edge;
        X.sl_org[a] = dom.lo[a];
        X.sl_inv[a] = X.S / ext[a];
        for (int s2 = 0; s2 < X.S; s2++) {
            const double top = (s2 == X.S - 1) ? INFINITY : dom.lo[a] + (s2 + 1) * w + m;
            const double bot = (s2 == 0) ? -INFINITY : dom.lo[a] + s2 * w - m;
            uint32_t *Lw = &X.L[((size_t)a * X.S + s2) * X.words];
            uint32_t *Hw = &X.H[((size_t)a * X.S + s2) * X.words];
            for (int b = 0; b < nb; b++) {
                if (blk[b].lo[a] <= top) Lw[b >> 5] |= 1u << (b & 31);
                if (blk[b].hi[a] >= bot) Hw[b >> 5] |= 1u << (b & 31);
            }
        }
    }
}

// Load a structure whose conductors are unions of boxes: box i of `in_boxes`
// belongs to conductor in_cond[i] (in_cond null: box i is conductor i).  The
// boxes are stored sorted by conductor, so that the nearest-electrode scan's
// lowest box index on ties is the lowest conductor index.
static int load_structure(frw_ctx *ctx, const frw_box *domain, const frw_box *in_boxes, const int32_t *in_cond,
                          int32_t n_box, int32_t n_cond, const double *eps_r, int32_t n_mat, int32_t background_mat,
                          const frw_block *blocks, int32_t n_blocks, int32_t *structure_id)
{
    if (!ctx || !domain || !in_boxes || !eps_r || !structure_id) return FRW_EINVAL;
    if (n_cond < 1 || n_box < n_cond || n_box > 65535 || n_mat < 1 || n_blocks < 0 || (n_blocks > 0 && !blocks))
        return fail(ctx, FRW_EINVAL, "need at least one conductor, a box per conductor and one material");
    if (background_mat < 0 || background_mat >= n_mat) return fail(ctx, FRW_EINVAL, "background material out of range");
    if (!box_ok(*domain)) return fail(ctx, FRW_EINVAL, "degenerate domain");
    std::vector<int32_t> perm(n_box), bc(n_box), per_cond(n_cond, 0);
    for (int i = 0; i < n_box; i++) {
        perm[i] = i;
        bc[i] = in_cond ? in_cond[i] : i;
        if (bc[i] < 0 || bc[i] >= n_cond) return fail(ctx, FRW_EINVAL, "box conductor index out of range");
        per_cond[bc[i]]++;
    }
    for (int k = 0; k < n_cond; k++)
        if (per_cond[k] == 0) return fail(ctx, FRW_EINVAL, "a conductor has no box");
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return bc[a] < bc[b]; });
    std::vector<frw_box> boxv(n_box);
    std::vector<int32_t> box_cond(n_box);
    for (int i = 0; i < n_box; i++) {
        boxv[i] = in_boxes[perm[i]];
        box_cond[i] = bc[perm[i]];
    }
    const frw_box *conductors = boxv.data();
    for (int k = 0; k < n_box; k++) {
        if (!box_ok(conductors[k])) return fail(ctx, FRW_EINVAL, "degenerate conductor box");
        for (int a = 0; a < 3; a++)
            if (!(conductors[k].lo[a] > domain->lo[a] && conductors[k].hi[a] < domain->hi[a]))
                return fail(ctx, FRW_EINVAL, "conductor not strictly inside the domain");
    }
    // boxes of one conductor may touch or overlap; those of different conductors may not
    for (int k = 0; k < n_box; k++)
        for (int l = k + 1; l < n_box; l++)
            if (box_cond[k] != box_cond[l] &&
                !(box_gap(conductors[k].lo, conductors[k].hi, conductors[l].lo, conductors[l].hi) > 0.0))
                return fail(ctx, FRW_EINVAL, "conductors touch or overlap");
    for (int b = 0; b < n_blocks; b++) {
        if (!box_ok({{blocks[b].lo[0], blocks[b].lo[1], blocks[b].lo[2]}, {blocks[b].hi[0], blocks[b].hi[1], blocks[b].hi[2]}}))
            return fail(ctx, FRW_EINVAL, "degenerate dielectric block");
        if (blocks[b].mat < 0 || blocks[b].mat >= n_mat) return fail(ctx, FRW_EINVAL, "block material out of range");
    }
    std::lock_guard<std::mutex> lk(ctx->struct_mu);
    std::vector<uint8_t> map;
    int rc = register_materials(ctx, eps_r, n_mat, map);
    if (rc) return rc;
    int mat_need = 0;
    for (int i = 0; i < n_mat; i++) mat_need = std::max(mat_need, (int)map[i] + 1);
    // slot in the structure table
    int sid = -1;
    for (size_t i = 0; i < ctx->structs.size(); i++)
        if (!ctx->structs[i].live) sid = (int)i;
    if (sid < 0) {
        if ((int)ctx->structs.size() >= ctx->struct_cap) return fail(ctx, FRW_ECAPACITY, "too many structures");
        ctx->structs.emplace_back();
        sid = (int)ctx->structs.size() - 1;
    }
    HostStructure &H = ctx->structs[sid];
    H = HostStructure();
    H.n_c = n_cond;
    H.n_box = n_box;
    H.mat_need = mat_need;
    H.n_b = n_blocks;
    H.box_cond = box_cond;
    H.master_box.assign(n_cond, -1);
    for (int k = 0; k < n_box; k++)
        if (per_cond[box_cond[k]] == 1) H.master_box[box_cond[k]] = k;
    H.c_lo.resize(3 * (size_t)n_box);
    H.c_hi.resize(3 * (size_t)n_box);
    for (int k = 0; k < n_box; k++)
        for (int a = 0; a < 3; a++) {
            H.c_lo[3 * k + a] = conductors[k].lo[a];
            H.c_hi[3 * k + a] = conductors[k].hi[a];
        }
    DevStructure &D = H.d;
    memset(&D, 0, sizeof(D));
    D.n_c = n_box;
    D.n_cond = n_cond;
    D.n_b = n_blocks;
    D.bg = map[background_mat];
    double edge = 0.0, maxabs = 0.0;
    for (int a = 0; a < 3; a++) {
        D.dom_lo[a] = H.dom_lo[a] = domain->lo[a];
        D.dom_hi[a] = H.dom_hi[a] = domain->hi[a];
        D.dom_lo_f[a] = (float)domain->lo[a];
        D.dom_hi_f[a] = (float)domain->hi[a];
        edge = std::max(edge, domain->hi[a] - domain->lo[a]);
        maxabs = std::max(maxabs, std::max(std::fabs(domain->lo[a]), std::fabs(domain->hi[a])));
    }
    D.tau = 1e-9 * edge;
    const float m = 8.0f * ulpf((float)maxabs);
    D.margin_f = m;
    D.tau_f = std::max((float)(1e-9 * edge), 2.0f * m);
    // SoA device copies
    std::vector<double> clo(3 * (size_t)n_box), chi(3 * (size_t)n_box);
    std::vector<float> clof(3 * (size_t)n_box), chif(3 * (size_t)n_box);
    for (int k = 0; k < n_box; k++)
        for (int a = 0; a < 3; a++) {
            clo[(size_t)a * n_box + k] = conductors[k].lo[a];
            chi[(size_t)a * n_box + k] = conductors[k].hi[a];
            clof[(size_t)a * n_box + k] = (float)conductors[k].lo[a];
            chif[(size_t)a * n_box + k] = (float)conductors[k].hi[a];
        }
    std::vector<double> blo(3 * (size_t)n_blocks), bhi(3 * (size_t)n_blocks);
    std::vector<float> blof(3 * (size_t)n_blocks), bhif(3 * (size_t)n_blocks);
    std::vector<uint8_t> bm((size_t)n_blocks);
    for (int b = 0; b < n_blocks; b++) {
        for (int a = 0; a < 3; a++) {
            blo[(size_t)a * n_blocks + b] = blocks[b].lo[a];
            bhi[(size_t)a * n_blocks + b] = blocks[b].hi[a];
            blof[(size_t)a * n_blocks + b] = (float)blocks[b].lo[a];
            bhif[(size_t)a * n_blocks + b] = (float)blocks[b].hi[a];
        }
        bm[b] = map[blocks[b].mat];
    }
    auto up = [&](auto **dst, const auto &src) -> int {
        using E = typename std::remove_reference<decltype(src)>::type::value_type;
        E *p = nullptr;
        int r = dalloc(ctx, &p, src.size(), H.dev);
        if (r) return r;
        if (!src.empty()) {
            cudaError_t e = cudaMemcpyAsync(p, src.data(), src.size() * sizeof(E), cudaMemcpyHostToDevice, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "structure upload");
        }
        *dst = p;
        return FRW_OK;
    };
    IndexHost X;
    // FRW_INDEX_HOST=1: the grid's candidate lists built on the host (the same lists)
    const char *ih = std::getenv("FRW_INDEX_HOST");
    const bool host_lists = ih && ih[0] == '1';
    build_index(*domain, conductors, n_box, blocks, n_blocks, X, host_lists);
    for (int a = 0; a < 3; a++) {
        D.gdim[a] = X.gdim[a];
        D.g_org[a] = X.g_org[a];
        D.g_inv[a] = X.g_inv[a];
        D.g_org_f[a] = (float)X.g_org[a];
        D.g_inv_f[a] = (float)X.g_inv[a];
        D.sl_org[a] = X.sl_org[a];
        D.sl_inv[a] = X.sl_inv[a];
        D.sl_org_f[a] = (float)X.sl_org[a];
        D.sl_inv_f[a] = (float)X.sl_inv[a];
    }
    D.sl_S = X.S;
    D.sl_words = X.words;
    if ((host_lists && ((rc = up((uint32_t **)&D.g_off, X.g_off)) || (rc = up((uint16_t **)&D.g_ids, X.g_ids)))) ||
        (rc = up((uint32_t **)&D.sl_L, X.L)) || (rc = up((uint32_t **)&D.sl_H, X.H)) ||
        (rc = up((double **)&D.c_lo, clo)) || (rc = up((double **)&D.c_hi, chi)) ||
        (rc = up((float **)&D.c_lo_f, clof)) || (rc = up((float **)&D.c_hi_f, chif)) ||
        (rc = up((double **)&D.b_lo, blo)) || (rc = up((double **)&D.b_hi, bhi)) ||
        (rc = up((float **)&D.b_lo_f, blof)) || (rc = up((float **)&D.b_hi_f, bhif)) ||
        (rc = up((uint8_t **)&D.b_mat, bm)) || (rc = up((int32_t **)&D.box_cond, box_cond))) {
        for (void *p : H.dev) cudaFree(p);
        H.dev.clear();
        return rc;
    }
    if (!host_lists) {
        // the grid's candidate lists on the device: counts, offsets, then the lists
        GridBuild G;
        for (int a = 0; a < 3; a++) {
            G.gdim[a] = X.gdim[a];
            G.dlo[a] = domain->lo[a];
            G.dhi[a] = domain->hi[a];
            G.w[a] = (domain->hi[a] - domain->lo[a]) / X.gdim[a];
        }
        G.n_box = n_box;
        G.tol = 1e-6 * edge;
        G.clo = D.c_lo;
        G.chi = D.c_hi;
        const size_t cells = (size_t)X.gdim[0] * X.gdim[1] * X.gdim[2];
        uint32_t *off = nullptr, total = 0;
        uint16_t *ids = nullptr;
        cudaError_t e = cudaSuccess;
        if ((rc = dalloc(ctx, &off, cells + 1, H.dev)) == FRW_OK) {
            e = launch_grid_lists(G, off, nullptr, 0, ctx->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&total, off + cells, sizeof(total), cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e == cudaSuccess && (rc = dalloc(ctx, &ids, total, H.dev)) == FRW_OK)
                e = launch_grid_lists(G, off, ids, 1, ctx->stream);
        }
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "grid index build");
        if (rc) {
            for (void *p : H.dev) cudaFree(p);
            H.dev.clear();
            return rc;
        }
        D.g_off = off;
        D.g_ids = ids;
    }
    const SView<float> vf = sview<float>(D);
    const SView<double> vd = sview<double>(D);
    CK(cudaMemcpyAsync(ctx->d_structs + sid, &D, sizeof(DevStructure), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_view_f + sid, &vf, sizeof(vf), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_view_d + sid, &vd, sizeof(vd), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    H.live = true;
    *structure_id = sid;
    return FRW_OK;
}

extern "C" int frw_load_structure(frw_ctx *ctx, const frw_box *domain, const frw_box *conductors, int32_t n_cond,
                                  const double *eps_r, int32_t n_mat, int32_t background_mat,
                                  const frw_block *blocks, int32_t n_blocks, int32_t *structure_id)
{
    return load_structure(ctx, domain, conductors, nullptr, n_cond, n_cond, eps_r, n_mat, background_mat, blocks,
                          n_blocks, structure_id);
}

extern "C" int frw_load_structure_boxes(frw_ctx *ctx, const frw_box *domain, const frw_box *boxes,
                                        const int32_t *box_conductor, int32_t n_boxes, int32_t n_cond,
                                        const double *eps_r, int32_t n_mat, int32_t background_mat,
                                        const frw_block *blocks, int32_t n_blocks, int32_t *structure_id)
{
    if (!box_conductor) return FRW_EINVAL;
    return load_structure(ctx, domain, boxes, box_conductor, n_boxes, n_cond, eps_r, n_mat, background_mat, blocks,
                          n_blocks, structure_id);
}

// Boxes of a permittivity voxel map over the domain (the frw_structure rule): runs
// of one material along z, merged across y where extent and material agree, then
// across x; ordered by first cell.  Cells of FRW_VOXEL_NONE produce no box.
static int voxel_boxes(frw_ctx *ctx, const frw_box &dom, const uint8_t *vm, const int32_t dims[3], int32_t n_mat,
                       std::vector<frw_block> &out)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    if (nx < 1 || ny < 1 || nz < 1) return fail(ctx, FRW_EINVAL, "voxel map dimensions must be positive");
    if (nx * ny * nz > (int64_t)1 << 24) return fail(ctx, FRW_ECAPACITY, "voxel map larger than 2^24 cells");
    for (int64_t c = 0; c < nx * ny * nz; c++)
        if (vm[c] != FRW_VOXEL_NONE && (int)vm[c] >= n_mat) return fail(ctx, FRW_EINVAL, "voxel material out of range");
    struct Rect { int64_t j0, j1, k0, k1; int m; };
    struct Box { int64_t i0, i1, j0, j1, k0, k1; int m; };
    std::vector<Box> boxes;
    std::map<std::tuple<int64_t, int64_t, int64_t, int64_t, int>, size_t> open_x;   // -> index in boxes
    for (int64_t i = 0; i < nx; i++) {
        std::vector<Rect> rects;
        std::map<std::tuple<int64_t, int64_t, int>, size_t> open_y;                    // -> index in rects
        for (int64_t j = 0; j < ny; j++) {
            const uint8_t *col = vm + (i * ny + j) * nz;
            for (int64_t k = 0; k < nz;) {
                const int m = col[k];
                int64_t k1 = k + 1;
                while (k1 < nz && col[k1] == m) k1++;
                if (m != FRW_VOXEL_NONE) {
                    auto key = std::make_tuple(k, k1, m);
                    auto it = open_y.find(key);
                    if (it != open_y.end() && rects[it->second].j1 == j) rects[it->second].j1 = j + 1;
                    else {
                        open_y[key] = rects.size();
                        rects.push_back({j, j + 1, k, k1, m});
                    }
                }
                k = k1;
            }
        }
        for (const Rect &r : rects) {
            auto key = std::make_tuple(r.j0, r.j1, r.k0, r.k1, r.m);
            auto it = open_x.find(key);
            if (it != open_x.end() && boxes[it->second].i1 == i) boxes[it->second].i1 = i + 1;
            else {
                open_x[key] = boxes.size();
                boxes.push_back({i, i + 1, r.j0, r.j1, r.k0, r.k1, r.m});
            }
        }
    }
    std::sort(boxes.begin(), boxes.end(), [](const Box &a, const Box &b) {
        return std::make_tuple(a.i0, a.j0, a.k0) < std::make_tuple(b.i0, b.j0, b.k0);
    });
    auto edge = [&](int a, int64_t i, int64_t n) {
        return i == n ? dom.hi[a] : dom.lo[a] + ((dom.hi[a] - dom.lo[a]) * (double)i) / (double)n;
    };
    out.clear();
    out.reserve(boxes.size());
    for (const Box &b : boxes) {
        frw_block q;
        q.lo[0] = edge(0, b.i0, nx); q.hi[0] = edge(0, b.i1, nx);
        q.lo[1] = edge(1, b.j0, ny); q.hi[1] = edge(1, b.j1, ny);
        q.lo[2] = edge(2, b.k0, nz); q.hi[2] = edge(2, b.k1, nz);
        q.mat = b.m;
        out.push_back(q);
    }
    return FRW_OK;
}

extern "C" int frw_load_structure_ex(frw_ctx *ctx, const frw_structure *d, int32_t *structure_id)
{
    if (!ctx || !d || !structure_id) return FRW_EINVAL;
    if (d->grounded_walls != 1)
        return fail(ctx, FRW_EINVAL, "the domain walls must be grounded (grounded_walls = 1)");
    if (d->n_blocks < 0 || (d->n_blocks > 0 && !d->blocks)) return fail(ctx, FRW_EINVAL, "bad block list");
    if (!d->box_conductor && d->n_boxes != d->n_cond)
        return fail(ctx, FRW_EINVAL, "without box_conductor every conductor is one box (n_boxes = n_cond)");
    std::vector<frw_block> all;
    if (d->voxel_mat) {
        if (!box_ok(d->domain)) return fail(ctx, FRW_EINVAL, "degenerate domain");
        int rc = voxel_boxes(ctx, d->domain, d->voxel_mat, d->vox_dims, d->n_mat, all);
        if (rc) return rc;
    }
    if ((int64_t)all.size() + d->n_blocks > 65535)
        return fail(ctx, FRW_ECAPACITY, "more than 65535 dielectric boxes (voxel map and blocks)");
    for (int b = 0; b < d->n_blocks; b++) all.push_back(d->blocks[b]);
    return load_structure(ctx, &d->domain, d->boxes, d->box_conductor, d->n_boxes, d->n_cond, d->eps_r, d->n_mat,
                          d->background_mat, all.empty() ? nullptr : all.data(), (int32_t)all.size(), structure_id);
}

extern "C" int frw_unload_structure(frw_ctx *ctx, int32_t sid)
{
    if (!ctx) return FRW_EINVAL;
    std::lock_guard<std::mutex> engine(ctx->engine_mu);   // no run on the device meanwhile
    std::lock_guard<std::mutex> lk(ctx->struct_mu);
    if (sid < 0 || sid >= (int)ctx->structs.size() || !ctx->structs[sid].live) return FRW_ENOTFOUND;
    cudaStreamSynchronize(ctx->stream);
    for (void *p : ctx->structs[sid].dev) cudaFree(p);
    ctx->structs[sid] = HostStructure();
    return FRW_OK;
}

// ---------------------------------------------------------------------------
// Gaussian surface of a master (reading: box grown by frac x the smallest
// L-infinity gap to another conductor or a wall; point uniform by area).
static void gauss_setup(const HostStructure &H, int master, double frac, DevJob &J)
{
    const int mb = H.master_box[master];   // single box (checked when the job was accepted)
    const double *lo = &H.c_lo[3 * (size_t)mb], *hi = &H.c_hi[3 * (size_t)mb];
    double gap = INFINITY;
    for (int k = 0; k < H.n_box; k++) {
        if (H.box_cond[k] == master) continue;
        const double d = box_gap(lo, hi, &H.c_lo[3 * (size_t)k], &H.c_hi[3 * (size_t)k]);
        if (d < gap) gap = d;
    }
    for (int a = 0; a < 3; a++) {
        double t = lo[a] - H.dom_lo[a];
        if (t < gap) gap = t;
        t = H.dom_hi[a] - hi[a];
        if (t < gap) gap = t;
    }
    const double dg = frac * gap;
    for (int a = 0; a < 3; a++) {
        J.g_lo[a] = lo[a] - dg;
        J.g_hi[a] = hi[a] + dg;
    }
    const double ex = J.g_hi[0] - J.g_lo[0], ey = J.g_hi[1] - J.g_lo[1], ez = J.g_hi[2] - J.g_lo[2];
    const double fa[6] = {ey * ez, ey * ez, ex * ez, ex * ez, ex * ey, ex * ey};
    double acc = 0.0;
    for (int f = 0; f < 6; f++) {
        acc += fa[f];
        J.cum[f] = acc;
    }
    J.area = acc;
}

typedef __int128 i128;

static i128 rd128(const unsigned long long *p)
{
    const unsigned __int128 u = ((unsigned __int128)p[1] << 64) | (unsigned __int128)p[0];
    return (i128)u;
}

struct JobRun {
    frw_job desc;
    uint64_t walk_begin = 0;         // first walk id (resume / shard offset)
    DevJob d;
    uint64_t n_batches = 0;
    uint64_t sum_off = 0;            // u64 offset of the job's running sums
    uint64_t first_limit = 0;        // issue limit at publication
    bool converged = false;
    std::vector<i128> S1, S2;        // exact sums of the estimate
    uint64_t walks = 0;
    uint64_t issued = 0;
    uint64_t ex[ACC_EXTRA] = {0};
};

static int ensure_records(frw_ctx *ctx, uint64_t n)
{
    if (n <= ctx->rec_cap) return FRW_OK;
    if (n * 32ull > (64ull << 30)) return fail(ctx, FRW_ENOMEM, "walk budget too large for the record pool (64 GB)");
    for (void *p : ctx->rec_allocs) cudaFree(p);
    ctx->rec_allocs.clear();
    ctx->rec_cap = 0;
    RecArrays &R = ctx->rec;
    int rc;
    if ((rc = dalloc(ctx, &R.omega, n, ctx->rec_allocs)) || (rc = dalloc(ctx, &R.k, n, ctx->rec_allocs)) ||
        (rc = dalloc(ctx, &R.hops, n, ctx->rec_allocs)) || (rc = dalloc(ctx, &R.steps, n, ctx->rec_allocs)) ||
        (rc = dalloc(ctx, &R.cnt_sh, n, ctx->rec_allocs)) || (rc = dalloc(ctx, &R.cnt_mw, n, ctx->rec_allocs)) ||
        (rc = dalloc(ctx, &R.branch, n, ctx->rec_allocs)))
        return rc;
    ctx->rec_cap = n;
    return FRW_OK;
}

// job table and arenas, grown (never while a run is on the device) to at least the
// given capacities
static int grow_runbufs(frw_ctx *ctx, RunBufs &B, uint32_t jcap, uint64_t bcap, uint64_t acap, uint64_t scap)
{
    if (jcap <= B.jcap && bcap <= B.bcap && acap <= B.acap && scap <= B.scap) return FRW_OK;
    jcap = std::max(jcap, B.jcap);
    bcap = std::max(bcap, B.bcap);
    acap = std::max(acap, B.acap);
    scap = std::max(scap, B.scap);
    for (void *p : B.allocs) cudaFree(p);
    B = RunBufs();
    int rc;
    if ((rc = dalloc(ctx, &B.jobs, jcap, B.allocs)) || (rc = dalloc(ctx, &B.next, jcap, B.allocs)) ||
        (rc = dalloc(ctx, &B.limit, jcap, B.allocs)) || (rc = dalloc(ctx, &B.cancel, jcap, B.allocs)) ||
        (rc = dalloc(ctx, &B.js, jcap, B.allocs)) || (rc = dalloc(ctx, &B.jsoff, jcap, B.allocs)) ||
        (rc = dalloc(ctx, &B.jsum, scap, B.allocs)) || (rc = dalloc(ctx, &B.acc, acap, B.allocs)) ||
        (rc = dalloc(ctx, &B.done, bcap, B.allocs)) || (rc = dalloc(ctx, &B.ready, bcap, B.allocs)) ||
        (rc = dalloc(ctx, &B.bjob, bcap, B.allocs)) || (rc = dalloc(ctx, &B.rq, bcap, B.allocs)) ||
        (rc = dalloc(ctx, &B.rqc, 2, B.allocs)) || (rc = dalloc(ctx, &B.jctl, JC_WORDS, B.allocs))) {
        for (void *p : B.allocs) cudaFree(p);
        B = RunBufs();
        return rc;
    }
    B.jcap = jcap;
    B.bcap = bcap;
    B.acap = acap;
    B.scap = scap;
    return FRW_OK;
}

static int ensure_runbufs(frw_ctx *ctx, uint32_t jcap, uint64_t bcap, uint64_t acap, uint64_t scap)
{
    return grow_runbufs(ctx, ctx->rb, jcap, bcap, acap, scap);
}

// Bump allocation of a run's arenas.
struct Arena {
    uint32_t jobs = 0;
    uint64_t walks = 0, batches = 0, acc = 0, sums = 0;
};

// words of a job's running sums, rounded to whole 128-byte lines (no line is
// shared between jobs)
static uint64_t sum_words(int n_c) { return (acc_stride_for(n_c) + 15u) / 16u * 16u; }

// Fill a job's descriptor and place it at the arena's current ends.
static void place_job(frw_ctx *ctx, JobRun &j, Arena &A)
{
    const HostStructure &H = ctx->structs[j.desc.structure_id];
    DevJob &d = j.d;
    memset(&d, 0, sizeof(d));
    d.sid = j.desc.structure_id;
    d.master = j.desc.master;
    d.n_c = H.n_c;
    d.key0 = (uint32_t)ctx->opt.seed;
    d.key1 = (uint32_t)(ctx->opt.seed >> 32) ^ (uint32_t)j.desc.request_id;
    gauss_setup(H, j.desc.master, ctx->opt.gauss_offset_frac, d);
    d.walk_count = j.desc.walk_budget;
    d.walk_begin = j.walk_begin;
    d.batch = j.desc.batch ? j.desc.batch : 16384;
    d.acc_stride = acc_stride_for(H.n_c);
    d.sigma = j.desc.sigma_target;
    j.n_batches = (d.walk_count + d.batch - 1) / d.batch;
    d.acc_base = A.acc;
    d.rec_base = A.walks;
    d.batch_base = A.batches;
    j.sum_off = A.sums;
    A.acc += j.n_batches * d.acc_stride;
    A.walks += d.walk_count;
    A.batches += j.n_batches;
    A.sums += sum_words(H.n_c);
    A.jobs++;
    j.S1.assign(H.n_c + 1, 0);
    j.S2.assign(H.n_c + 1, 0);
}

// Zero a run's job table and arenas up to the given sizes (stream order).
static cudaError_t zero_run(RunBufs &B, int32_t *rec_k, uint32_t jobs, const Arena &A, cudaStream_t st)
{
    const uint64_t nb = std::max<uint64_t>(A.batches, 1);
    cudaError_t e;
    if ((e = cudaMemsetAsync(B.next, 0, sizeof(unsigned long long) * std::max<uint32_t>(jobs, 1), st)) ||
        (e = cudaMemsetAsync(B.cancel, 0, sizeof(int) * std::max<uint32_t>(jobs, 1), st)) ||
        (e = cudaMemsetAsync(B.js, 0, sizeof(JobState) * std::max<uint32_t>(jobs, 1), st)) ||
        (e = cudaMemsetAsync(B.jsum, 0, sizeof(unsigned long long) * std::max<uint64_t>(A.sums, 1), st)) ||
        (e = cudaMemsetAsync(B.acc, 0, sizeof(unsigned long long) * std::max<uint64_t>(A.acc, 1), st)) ||
        (e = cudaMemsetAsync(B.done, 0, sizeof(uint32_t) * nb, st)) ||
        (e = cudaMemsetAsync(B.ready, 0, sizeof(uint32_t) * nb, st)) ||
        (e = cudaMemsetAsync(B.rq, 0xff, sizeof(uint32_t) * nb, st)) ||
        (e = cudaMemsetAsync(B.rqc, 0, sizeof(uint32_t) * 2, st)) ||
        (e = cudaMemsetAsync(B.jctl, 0, sizeof(uint32_t) * JC_WORDS, st)) ||
        (e = cudaMemsetAsync(rec_k, 0x80, sizeof(int32_t) * std::max<uint64_t>(A.walks, 1), st)))
        return e;
    return cudaSuccess;
}

// Host image of jobs [j0, j0 + n) of a run's table.
struct PublishStage {
    std::vector<DevJob> d;
    std::vector<unsigned long long> lim, off;
    std::vector<uint32_t> bjob;
    uint64_t b0 = 0;
    uint32_t pub = 0;
};

static void stage_jobs(JobRun *const *jobs, uint32_t j0, uint32_t n, PublishStage &P)
{
    P.d.resize(n);
    P.lim.resize(n);
    P.off.resize(n);
    P.bjob.clear();
    P.b0 = n ? jobs[0]->d.batch_base : 0;
    for (uint32_t i = 0; i < n; i++) {
        const JobRun &j = *jobs[i];
        P.d[i] = j.d;
        P.lim[i] = j.first_limit;
        P.off[i] = j.sum_off;
        for (uint64_t b = 0; b < j.n_batches; b++) P.bjob.push_back(j0 + i);
    }
    P.pub = j0 + n;
}

// Write jobs [j0, j0 + n) into the table and then publish them: the kernel sees a
// job only once the published count covers it (copies in stream order).  The
// host buffers must stay valid until the stream has run the copies.
static cudaError_t publish_copies(RunBufs &B, uint32_t j0, uint32_t n, const DevJob *d, const unsigned long long *lim,
                                  const unsigned long long *off, uint64_t b0, const uint32_t *bjob, uint64_t nb,
                                  const uint32_t *pub, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(B.jobs + j0, d, sizeof(DevJob) * n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(B.limit + j0, lim, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(B.jsoff + j0, off, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, st)))
        return e;
    if (nb && (e = cudaMemcpyAsync(B.bjob + b0, bjob, sizeof(uint32_t) * nb, cudaMemcpyHostToDevice, st))) return e;
    return cudaMemcpyAsync(B.jctl + JC_PUBLISHED, pub, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
}

static cudaError_t publish_jobs(RunBufs &B, JobRun *const *jobs, uint32_t j0, uint32_t n, PublishStage &P,
                                cudaStream_t st)
{
    stage_jobs(jobs, j0, n, P);
    return publish_copies(B, j0, n, P.d.data(), P.lim.data(), P.off.data(), P.b0, P.bjob.data(), P.bjob.size(),
                          &P.pub, st);
}

// Read a decided job's sums and counters back (stream order) and fill its result.
static void take_result(JobRun &j, const JobState &S, const unsigned long long *sum, unsigned long long issued)
{
    const int nc1 = j.d.n_c + 1;
    for (int k = 0; k < nc1; k++) {
        j.S1[k] = rd128(sum + 2 * k);
        j.S2[k] = rd128(sum + 2 * nc1 + 2 * k);
    }
    for (int x = 0; x < ACC_EXTRA; x++) j.ex[x] = sum[4 * nc1 + x];
    j.walks = S.used;
    j.converged = S.decided == 1u;
    j.issued = issued;
}

static void fill_stats(frw_stats &s, const JobRun &j)
{
    memset(&s, 0, sizeof(s));
    s.walks = j.walks;
    s.hops = j.ex[1];
    s.micro_steps = j.ex[2];
    s.strat_hops = j.ex[3];
    s.hom_hops = j.ex[4];
    s.mw_hops = j.ex[5];
    s.branch[0] = j.ex[6];
    s.branch[1] = j.ex[7];
    s.branch[2] = j.ex[8];
    s.truncated = j.ex[9];
    s.mw_jobs = j.ex[5];
    s.walks_issued = j.issued;
}

// first issue limit of a sigma job: 1/div of its share of the slot pool, at least
// 4 batches; the device then steers the limit to the need predicted from the
// completed prefix.  Closed runs (throughput) take the whole share (div 1).  The
// serving loop (latency) takes an eighth: the stop rule reads a prefix of walk
// ids, and walks issued together finish together, so a request that needs few
// walks would otherwise wait for a whole pool of them.
static uint64_t first_wave(const JobRun &j, uint64_t slots, int n_sigma, uint64_t div)
{
    if (!(j.desc.sigma_target > 0.0)) return j.d.walk_count;
    const uint64_t b = j.d.batch;
    uint64_t first = std::max<uint64_t>(4 * b, slots / (div * (uint64_t)std::max(1, n_sigma)));
    first = (first + b - 1) / b * b;
    return std::min<uint64_t>(first, j.d.walk_count);
}

// Wall-clock limit of one run (seconds; environment FRW_RUN_TIMEOUT_S, default 3600).
static double run_timeout_s()
{
    const char *v = std::getenv("FRW_RUN_TIMEOUT_S");
    const double t = v ? std::atof(v) : 0.0;
    return t > 0.0 ? t : 3600.0;
}

// The geometry copy of a closed run or plan: when every job uses one structure,
// the groups of its geometry (boxes, blocks, slab masks, in that order) that fit
// the dynamic shared memory a CTA can add at the launched CTAs per SM.
static void choose_stage(frw_ctx *ctx, EngineView &E, const std::vector<JobRun *> &live)
{
    E.stage_sid = -1;
    E.stage_flags = 0;
    E.stage_bytes = 0;
    E.stage_off = 0;
    if (ctx->tune.unstaged || live.empty()) return;
    const int sid = live[0]->desc.structure_id;
    for (const JobRun *j : live)
        if (j->desc.structure_id != sid) return;
    const uint32_t cap = walk_stage_cap(E, ctx->grid / std::max(1, ctx->shape.sms));
    const DevStructure &d = ctx->structs[sid].d;
    const int ts = E.fp32 ? 4 : 8;
    uint32_t used = 0, fl = 0;
    for (uint32_t g = STAGE_BOXES; g <= STAGE_SLABS; g <<= 1) {
        const uint32_t b = stage_group_bytes(g, d.n_c, d.n_b, d.sl_S, d.sl_words, ts);
        if (b > 0 && used + b <= cap) {
            used += b;
            fl |= g;
        }
    }
    if (!fl) return;
    E.stage_sid = sid;
    E.stage_flags = fl;
    E.stage_bytes = used;
    E.stage_off = stage_round16((uint32_t)walk_smem_bytes(E.N, E.max_nc, E.transition));
}

static EngineView run_view(frw_ctx *ctx, RunBufs &B, const RecArrays &rec, uint64_t rec_cap, uint32_t jcap,
                           int max_nc, uint32_t pool, uint64_t batches)
{
    EngineView E = make_view(ctx);
    E.n_jobs = (int)jcap;
    E.max_nc = max_nc;
    E.jobs = B.jobs;
    E.job_next = B.next;
    E.job_limit = B.limit;
    E.job_cancel = B.cancel;
    E.jstate = B.js;
    E.jctl = B.jctl;
    E.batch_job = B.bjob;
    E.jsum = B.jsum;
    E.jsum_off = B.jsoff;
    E.acc = B.acc;
    E.batch_done = B.done;
    E.batch_ready = B.ready;
    E.rq = B.rq;
    E.rq_count = B.rqc;
    E.rq_head = B.rqc + 1;
    E.rq_cap = (uint32_t)std::max<uint64_t>(batches, 1);
    E.rec = rec;
    E.rec_cap = rec_cap;
    E.acc_cap = B.acap;
    E.jsum_cap = B.scap;
    E.pool = pool;
    E.NS = pool * (uint32_t)ctx->grid;
    return E;
}

// slots per CTA for a run of `walks` walks: the tuned pool, fewer for small runs
static uint32_t run_pool_for(frw_ctx *ctx, uint64_t walks)
{
    const uint32_t pool0 = ctx->grid ? ctx->NS / ctx->grid : ctx->NS;
    const uint32_t tuned = std::min<uint32_t>(pool0, (uint32_t)ctx->tune.pool_per_cta);
    const uint64_t per = std::max<uint64_t>(256, ((walks / ctx->grid + 255) / 256) * 256);
    return (uint32_t)std::min<uint64_t>(tuned, per);
}

// Run a set of jobs to completion: one launch of the persistent walk kernel with
// every job published before it starts.  The kernel applies each job's stop rule
// and folds its batches; the host reads the decided sums back.  The caller holds
// the engine lock.
// acc_out (optional): the run's batch accumulator arena, copied back after the run
// (per batch: S1 and S2 as int128 pairs, then the ACC_EXTRA counters)
static int run_jobs(frw_ctx *ctx, std::vector<JobRun> &jobs, frw_stats *stats_out,
                    std::vector<unsigned long long> *acc_out = nullptr)
{
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<JobRun *> live;
    for (auto &j : jobs) {
        const HostStructure &H = ctx->structs[j.desc.structure_id];
        j.S1.assign(H.n_c + 1, 0);
        j.S2.assign(H.n_c + 1, 0);
        j.d.n_c = H.n_c;
        if (j.desc.walk_budget) live.push_back(&j);
    }
    if (stats_out)
        for (size_t i = 0; i < jobs.size(); i++) memset(&stats_out[i], 0, sizeof(frw_stats));
    if (live.empty()) return FRW_OK;
    const uint32_t nj = (uint32_t)live.size();
    Arena A;
    int max_nc = 1;
    for (JobRun *j : live) {
        place_job(ctx, *j, A);
        max_nc = std::max(max_nc, j->d.n_c);
    }
    if (A.batches >= 0xffffffffull) return fail(ctx, FRW_EINVAL, "too many batches");
    int rc = ensure_records(ctx, A.walks);
    if (rc) return rc;
    if ((rc = ensure_runbufs(ctx, nj, A.batches, A.acc, A.sums))) return rc;
    const uint32_t run_pool = run_pool_for(ctx, A.walks);
    const uint64_t run_slots = (uint64_t)run_pool * ctx->grid;
    int n_sigma = 0;
    for (JobRun *j : live) n_sigma += j->desc.sigma_target > 0.0 ? 1 : 0;
    for (JobRun *j : live) j->first_limit = first_wave(*j, run_slots, n_sigma, 1);
    cudaStream_t st = ctx->stream, ax = ctx->aux;
    PublishStage P;
    const uint32_t ctrl0[CTRL_WORDS] = {0u, 0u, 0u, 0u};
    CK(zero_run(ctx->rb, ctx->rec.k, nj, A, st));
    CK(cudaMemcpyAsync(ctx->ctrl, ctrl0, sizeof(ctrl0), cudaMemcpyHostToDevice, st));
    CK(publish_jobs(ctx->rb, live.data(), 0, nj, P, st));
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t) * STAT_WORDS, st));
    CK(cudaMemsetAsync(ctx->cycles, 0, sizeof(unsigned long long) * 8, st));
    EngineView E = run_view(ctx, ctx->rb, ctx->rec, ctx->rec_cap, nj, max_nc, run_pool, A.batches);
    choose_stage(ctx, E, live);
    CK(prepare_walk(E));
    CK(cudaEventRecord(ctx->ev[0], st));
    CK(launch_walk(E, ctx->shape, st));
    CK(cudaEventRecord(ctx->ev[1], st));
    // wait for the kernel (which applies the stop rules itself) under a wall-clock guard
    const double limit_s = run_timeout_s();
    bool timed_out = false;
    while (cudaEventQuery(ctx->ev[1]) == cudaErrorNotReady) {
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit_s) {
            static const uint32_t abort1 = 1;   // the kernel stops at its next epoch boundary
            CK(cudaMemcpyAsync(ctx->ctrl + CTRL_ABORT, &abort1, sizeof(uint32_t), cudaMemcpyHostToDevice, ax));
            CK(cudaStreamSynchronize(ax));
            timed_out = true;
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    CK(cudaStreamSynchronize(st));
    rc = check_status(ctx);
    if (rc) return rc;
    if (timed_out) return fail(ctx, FRW_ETIMEOUT, "run exceeded its wall-clock limit (FRW_RUN_TIMEOUT_S)");
    std::vector<JobState> hjs(nj);
    std::vector<unsigned long long> hsum(A.sums), hnext(nj);
    CK(cudaMemcpy(hjs.data(), ctx->rb.js, sizeof(JobState) * nj, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hsum.data(), ctx->rb.jsum, sizeof(unsigned long long) * A.sums, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hnext.data(), ctx->rb.next, sizeof(unsigned long long) * nj, cudaMemcpyDeviceToHost));
    for (uint32_t i = 0; i < nj; i++) {
        if (hjs[i].decided == 0u) return fail(ctx, FRW_EDEVICE, "a job was not decided when the kernel ended");
        take_result(*live[i], hjs[i], hsum.data() + live[i]->sum_off, hnext[i]);
    }
    if (acc_out) {
        acc_out->assign(A.acc, 0ull);
        CK(cudaMemcpy(acc_out->data(), ctx->rb.acc, sizeof(unsigned long long) * A.acc, cudaMemcpyDeviceToHost));
    }
    float kms = 0.f;
    cudaEventElapsedTime(&kms, ctx->ev[0], ctx->ev[1]);
    unsigned long long cyc[5] = {0, 0, 0, 0, 0};
    CK(cudaMemcpy(cyc, ctx->cycles, sizeof(cyc), cudaMemcpyDeviceToHost));
    const double ctot = (double)cyc[4];   // phases overlap: busy shares of the kernel's CTA time
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats_out) {
        for (size_t i = 0; i < jobs.size(); i++) {
            frw_stats &s = stats_out[i];
            fill_stats(s, jobs[i]);
            s.tables_built = ctx->h_status[STAT_BUILT];
            s.rounds = ctx->h_status[STAT_EPOCHS];
            s.seconds = secs;
            s.geom_ms = ctot > 0 ? kms * (double)cyc[0] / ctot : 0.0;
            s.fill_ms = ctot > 0 ? kms * (double)cyc[1] / ctot : 0.0;
            s.reduce_ms = ctot > 0 ? kms * (double)cyc[2] / ctot : 0.0;
            s.mw_ms = ctot > 0 ? kms * (double)cyc[3] / ctot : 0.0;
            s.launches = 1;
            s.kernel_ms = kms;
            s.stage_bytes = ctx->h_status[STAT_STAGED] ? E.stage_bytes : 0;
        }
    }
    return FRW_OK;
}

static void row_from(const JobRun &j, double *C, double *se)
{
    const int nc1 = j.d.n_c + 1;
    const double n = (double)j.walks;
    for (int k = 0; k < nc1; k++) {
        const double s1 = (double)j.S1[k] / ACC_S1_SCALE, s2 = (double)j.S2[k] / ACC_S2_SCALE;
        if (C) C[k] = n > 0 ? s1 / n : 0.0;
        if (se) {
            const double v = n > 1 ? (s2 - s1 * s1 / n) / (n * (n - 1.0)) : 0.0;
            se[k] = std::sqrt(v > 0 ? v : 0);
        }
    }
}

static int check_job(frw_ctx *ctx, const frw_job &j)
{
    if (j.structure_id < 0 || j.structure_id >= (int)ctx->structs.size() || !ctx->structs[j.structure_id].live)
        return fail(ctx, FRW_ENOTFOUND, "unknown structure id");
    if (j.master < 0 || j.master >= ctx->structs[j.structure_id].n_c) return fail(ctx, FRW_EINVAL, "master out of range");
    if (ctx->structs[j.structure_id].master_box[j.master] < 0)
        return fail(ctx, FRW_EINVAL, "the master has several boxes (its Gaussian surface is defined for one box)");
    if (!(j.sigma_target >= 0.0)) return fail(ctx, FRW_EINVAL, "negative sigma target");
    return FRW_OK;
}

extern "C" int frw_extract_batch(frw_ctx *ctx, const frw_job *jobs, int32_t n_jobs, double *C_rows,
                                 double *stderr_rows, frw_stats *stats)
{
    if (!ctx || (n_jobs > 0 && !jobs) || n_jobs < 0) return FRW_EINVAL;
    if (n_jobs == 0) return FRW_OK;
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<JobRun> runs(n_jobs);
    for (int i = 0; i < n_jobs; i++) {
        int rc = check_job(ctx, jobs[i]);
        if (rc) return rc;
        runs[i].desc = jobs[i];
    }
    std::vector<frw_stats> st(n_jobs);
    int rc = run_jobs(ctx, runs, st.data());
    if (rc) return rc;
    bool notconv = false;
    size_t off = 0;
    for (int i = 0; i < n_jobs; i++) {
        const int nc1 = runs[i].d.n_c + 1;
        row_from(runs[i], C_rows ? C_rows + off : nullptr, stderr_rows ? stderr_rows + off : nullptr);
        off += nc1;
        if (stats) stats[i] = st[i];
        if (jobs[i].sigma_target > 0.0 && !runs[i].converged) notconv = true;
    }
    return notconv ? FRW_ENOTCONV : FRW_OK;
}

extern "C" int frw_extract_matrix(frw_ctx *ctx, int32_t sid, const frw_extract_params *p, double *C, double *se,
                                  double *C_sym, frw_stats *stats)
{
    if (!ctx || !p || !C) return FRW_EINVAL;
    int n = 0;
    {
        std::lock_guard<std::mutex> ls(ctx->struct_mu);
        if (sid < 0 || sid >= (int)ctx->structs.size() || !ctx->structs[sid].live) return FRW_ENOTFOUND;
        n = ctx->structs[sid].n_c;
    }
    std::vector<frw_job> jobs(n);
    for (int i = 0; i < n; i++) {
        jobs[i].structure_id = sid;
        jobs[i].master = i;
        jobs[i].walk_budget = p->walk_budget;
        jobs[i].sigma_target = p->sigma_target;
        jobs[i].request_id = p->request_id + (uint64_t)i;
        jobs[i].batch = p->batch;
    }
    std::vector<double> se_local;
    if (!se) {
        se_local.resize((size_t)n * (n + 1));
        se = se_local.data();
    }
    const int rc = frw_extract_batch(ctx, jobs.data(), n, C, se, stats);
    if (rc != FRW_OK && rc != FRW_ENOTCONV) return rc;
    if (C_sym)
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                C_sym[(size_t)i * n + j] =
                    i == j ? C[(size_t)i * (n + 1) + i]
                           : 0.5 * (C[(size_t)i * (n + 1) + j] + C[(size_t)j * (n + 1) + i]);
    return rc;
}

extern "C" int frw_extract(frw_ctx *ctx, int32_t sid, int32_t master, const frw_extract_params *p, double *C_row,
                           double *stderr_row, frw_stats *stats)
{
    if (!ctx || !p) return FRW_EINVAL;
    frw_job j;
    j.structure_id = sid;
    j.master = master;
    j.walk_budget = p->walk_budget;
    j.sigma_target = p->sigma_target;
    j.request_id = p->request_id;
    j.batch = p->batch;
    if (p->walk_begin == 0) return frw_extract_batch(ctx, &j, 1, C_row, stderr_row, stats);
    // shard / resume: walk ids start at walk_begin (batches and the stop rule count from there)
    int rc = check_job(ctx, j);
    if (rc) return rc;
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<JobRun> runs(1);
    runs[0].desc = j;
    runs[0].walk_begin = p->walk_begin;
    frw_stats st;
    rc = run_jobs(ctx, runs, &st);
    if (rc) return rc;
    row_from(runs[0], C_row, stderr_row);
    if (stats) *stats = st;
    return (j.sigma_target > 0.0 && !runs[0].converged) ? FRW_ENOTCONV : FRW_OK;
}

extern "C" int frw_extract_sums(frw_ctx *ctx, int32_t sid, int32_t master, const frw_extract_params *p,
                                uint64_t *sums, uint64_t *n_walks, frw_stats *stats)
{
    if (!ctx || !p || !sums || !n_walks) return FRW_EINVAL;
    if (p->sigma_target != 0.0) return fail(ctx, FRW_EINVAL, "shards run in budget mode (sigma_target = 0)");
    frw_job j;
    j.structure_id = sid;
    j.master = master;
    j.walk_budget = p->walk_budget;
    j.sigma_target = 0.0;
    j.request_id = p->request_id;
    j.batch = p->batch;
    int rc = check_job(ctx, j);
    if (rc) return rc;
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<JobRun> runs(1);
    runs[0].desc = j;
    runs[0].walk_begin = p->walk_begin;
    frw_stats st;
    rc = run_jobs(ctx, runs, &st);
    if (rc) return rc;
    const int nc1 = runs[0].d.n_c + 1;
    for (int k = 0; k < nc1; k++) {
        const unsigned __int128 a = (unsigned __int128)runs[0].S1[k], b = (unsigned __int128)runs[0].S2[k];
        sums[2 * k] = (uint64_t)a;
        sums[2 * k + 1] = (uint64_t)(a >> 64);
        sums[2 * nc1 + 2 * k] = (uint64_t)b;
        sums[2 * nc1 + 2 * k + 1] = (uint64_t)(b >> 64);
    }
    *n_walks = runs[0].walks;
    if (stats) *stats = st;
    return FRW_OK;
}

extern "C" int frw_extract_batch_sums(frw_ctx *ctx, int32_t sid, int32_t master, const frw_extract_params *p,
                                      uint64_t *sums, uint64_t *n_in_batch, frw_stats *stats)
{
    if (!ctx || !p || !sums || !n_in_batch) return FRW_EINVAL;
    if (p->sigma_target != 0.0) return fail(ctx, FRW_EINVAL, "batch sums are taken in budget mode (sigma_target = 0)");
    frw_job j;
    j.structure_id = sid;
    j.master = master;
    j.walk_budget = p->walk_budget;
    j.sigma_target = 0.0;
    j.request_id = p->request_id;
    j.batch = p->batch;
    int rc = check_job(ctx, j);
    if (rc) return rc;
    const uint64_t B = p->batch ? p->batch : 16384;
    if (p->walk_begin % B) return fail(ctx, FRW_EINVAL, "walk_begin must be a multiple of the batch size");
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<JobRun> runs(1);
    runs[0].desc = j;
    runs[0].walk_begin = p->walk_begin;
    frw_stats st;
    std::vector<unsigned long long> acc;
    rc = run_jobs(ctx, runs, &st, &acc);
    if (rc) return rc;
    const JobRun &r = runs[0];
    const int nc1 = r.d.n_c + 1;
    for (uint64_t b = 0; b < r.n_batches; b++) {
        const unsigned long long *blk = acc.data() + r.d.acc_base + b * r.d.acc_stride;
        for (int w = 0; w < 4 * nc1; w++) sums[b * 4 * nc1 + w] = blk[w];
        n_in_batch[b] = blk[4 * nc1];
    }
    if (stats) *stats = st;
    return FRW_OK;
}

extern "C" int frw_walk_records(frw_ctx *ctx, int32_t sid, int32_t master, uint64_t request_id, uint64_t walk_begin,
                                uint64_t n_walks, double *omega, int32_t *electrode, uint32_t *hops,
                                uint64_t *micro_steps, int32_t *branch)
{
    if (!ctx) return FRW_EINVAL;
    frw_job j;
    j.structure_id = sid;
    j.master = master;
    j.walk_budget = n_walks;
    j.sigma_target = 0.0;
    j.request_id = request_id;
    j.batch = 0;
    int rc = check_job(ctx, j);
    if (rc) return rc;
    if (n_walks == 0) return FRW_OK;
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<JobRun> runs(1);
    runs[0].desc = j;
    runs[0].walk_begin = walk_begin;
    frw_stats st;
    rc = run_jobs(ctx, runs, &st);
    if (rc) return rc;
    // records of job 0 start at index 0 of the record pool
    const RecArrays &R = ctx->rec;
    cudaStream_t s = ctx->stream;
    std::vector<uint32_t> st32(micro_steps ? n_walks : 0);
    if (omega) CK(cudaMemcpyAsync(omega, R.omega, sizeof(double) * n_walks, cudaMemcpyDeviceToHost, s));
    if (electrode) CK(cudaMemcpyAsync(electrode, R.k, sizeof(int32_t) * n_walks, cudaMemcpyDeviceToHost, s));
    if (hops) CK(cudaMemcpyAsync(hops, R.hops, sizeof(uint32_t) * n_walks, cudaMemcpyDeviceToHost, s));
    if (micro_steps) CK(cudaMemcpyAsync(st32.data(), R.steps, sizeof(uint32_t) * n_walks, cudaMemcpyDeviceToHost, s));
    if (branch) CK(cudaMemcpyAsync(branch, R.branch, sizeof(int32_t) * n_walks, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (micro_steps)
        for (uint64_t i = 0; i < n_walks; i++) micro_steps[i] = st32[i];
    return FRW_OK;
}

// ---------------------------------------------------------------------------
extern "C" int frw_microwalk_cubes(frw_ctx *ctx, int32_t N, int32_t n_cubes, const int32_t *d_cubes,
                                   const double *eps_r, int32_t n_mat, uint64_t samples_per_cube, uint64_t request_id,
                                   uint32_t *d_exit, uint32_t *d_steps)
{
    if (!ctx || (n_cubes > 0 && !d_cubes) || !eps_r || n_mat < 1 || n_mat > FRW_MAX_MATERIALS) return FRW_EINVAL;
    if (N != ctx->opt.N) return fail(ctx, FRW_EINVAL, "cube lattice edge must equal the context's N");
    if (n_cubes <= 0 || samples_per_cube == 0) return FRW_OK;
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<uint8_t> map;
    int rc;
    {
        std::lock_guard<std::mutex> ls(ctx->struct_mu);
        rc = register_materials(ctx, eps_r, n_mat, map);
    }
    if (rc) return rc;
    std::vector<void *> tmp;
    unsigned long long *d_head = nullptr;
    if ((rc = dalloc(ctx, &d_head, 1, tmp))) return rc;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(d_head, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t) * STAT_WORDS, st);
    const uint32_t key0 = (uint32_t)ctx->opt.seed, key1 = (uint32_t)(ctx->opt.seed >> 32) ^ (uint32_t)request_id;
    if (e == cudaSuccess)
        e = launch_mw_cubes(N, d_cubes, (uint64_t)n_cubes, samples_per_cube, key0, key1, n_mat, (int)ctx->eps.size(),
                            map.data(), ctx->d_W, d_exit,
                            d_steps, d_head, ctx->status + STAT_ERR, ctx->shape, st);
    if (e != cudaSuccess) {
        for (void *p : tmp) cudaFree(p);
        return cuda_fail(ctx, e, "MicroWalk cube launch");
    }
    rc = check_status(ctx);
    for (void *p : tmp) cudaFree(p);
    return rc;
}

extern "C" int frw_fdm_cubes(frw_ctx *ctx, int32_t N, int32_t n_cubes, const int32_t *d_cubes, const double *eps_r,
                             int32_t n_mat, const uint32_t *d_u, double *d_P, uint32_t *d_exit, uint32_t *d_iters)
{
    if (!ctx || (n_cubes > 0 && !d_cubes) || !eps_r || n_mat < 1 || n_mat > FRW_MAX_MATERIALS) return FRW_EINVAL;
    if (N != ctx->opt.N) return fail(ctx, FRW_EINVAL, "cube lattice edge must equal the context's N");
    if (N > FDM_MAX_N) return fail(ctx, FRW_EINVAL, "FD transitions need N <= FRW_FDM_MAX_N");
    if (n_cubes <= 0) return FRW_OK;
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<uint8_t> map;
    int rc;
    {
        std::lock_guard<std::mutex> ls(ctx->struct_mu);
        rc = register_materials(ctx, eps_r, n_mat, map);
    }
    if (rc) return rc;
    const int grid = std::min(n_cubes, ctx->shape.sms);
    std::vector<void *> tmp;
    unsigned char *scratch = nullptr;
    if ((rc = dalloc(ctx, &scratch, (size_t)grid * fdm_cube_scratch_bytes(N), tmp))) return rc;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t) * STAT_WORDS, st);
    if (e == cudaSuccess)
        e = launch_fdm_cubes(N, d_cubes, (uint32_t)n_cubes, map.data(), ctx->d_eps, d_u, d_P, d_exit, d_iters, scratch,
                             grid, ctx->status + STAT_ERR, st);
    if (e != cudaSuccess) {
        for (void *p : tmp) cudaFree(p);
        return cuda_fail(ctx, e, "FD transition launch");
    }
    rc = check_status(ctx);
    for (void *p : tmp) cudaFree(p);
    return rc;
}

extern "C" int frw_table(frw_ctx *ctx, int32_t kind, const int32_t *profile, const double *eps_r, int32_t n_mat,
                         uint32_t *thr, uint8_t *neg, double *total, double *values)
{
    if (!ctx || kind < 0 || kind > 4) return FRW_EINVAL;
    const int N = ctx->opt.N;
    const bool hom = (kind == TAB_SGF_HOM || kind == TAB_FLUX_HOM);
    uint32_t prof[4] = {0, 0, 0, 0};
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    if (!hom) {
        if (!profile || !eps_r || n_mat < 1) return FRW_EINVAL;
        std::vector<uint8_t> map;
        int rc;
        {
            std::lock_guard<std::mutex> ls(ctx->struct_mu);
            rc = register_materials(ctx, eps_r, n_mat, map);
        }
        if (rc) return rc;
        for (int i = 0; i < N; i++) {
            if (profile[i] < 0 || profile[i] >= n_mat) return fail(ctx, FRW_EINVAL, "profile material out of range");
            prof[i >> 3] |= (uint32_t)map[profile[i]] << (4 * (i & 7));
        }
    }
    std::vector<void *> tmp;
    const size_t P = 6 * (size_t)N * N, P32 = (P + 31) / 32;
    uint32_t *d_thr = nullptr, *d_sgn = nullptr;
    double *d_k = nullptr, *d_v = nullptr;
    int rc;
    if ((rc = dalloc(ctx, &d_thr, P, tmp)) || (rc = dalloc(ctx, &d_sgn, P32, tmp)) || (rc = dalloc(ctx, &d_k, 1, tmp)) ||
        (rc = dalloc(ctx, &d_v, P, tmp))) {
        for (void *p : tmp) cudaFree(p);
        return rc;
    }
    EngineView E = make_view(ctx);
    E.tc.thr = d_thr;
    E.tc.sgn = d_sgn;
    E.tc.ktot = d_k;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t) * STAT_WORDS, st);
    if (e == cudaSuccess) e = launch_fill_one(E, (uint32_t)kind, prof, 0, d_v, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::vector<uint32_t> hs(P32);
    if (e == cudaSuccess && thr) e = cudaMemcpy(thr, d_thr, sizeof(uint32_t) * P, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hs.data(), d_sgn, sizeof(uint32_t) * P32, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && total) e = cudaMemcpy(total, d_k, sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && values) e = cudaMemcpy(values, d_v, sizeof(double) * P, cudaMemcpyDeviceToHost);
    for (void *p : tmp) cudaFree(p);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "table fill");
    if (neg)
        for (size_t n = 0; n < P; n++) neg[n] = (hs[n >> 5] >> (n & 31)) & 1u;
    return FRW_OK;
}

// ---------------------------------------------------------------------------
// Serving.  Requests submitted from any host thread queue in arrival order; a
// scheduler thread admits them into an open run of the persistent walk kernel as
// long as the run's job table and arenas have room (admission by memory).  Their
// walks interleave on the device with the walks of earlier requests, and each
// request completes as soon as its own stop rule holds (the host polls the job
// states through copies on a second stream while the kernel runs).  A run closes
// when a request needs more room than is left, or after a quiet spell; the next
// request starts a new run.
namespace {

struct Ticket {
    JobRun run;
    std::chrono::steady_clock::time_point t_submit, t_done;
    int state = 0;            // 0 queued, 1 on the device, 2 done
    int rc = FRW_OK;
    uint32_t index = 0;       // job-table index in its run (state 1)
};

struct ServeRun {
    bool active = false, closing = false;
    Arena A;                  // arena ends (bump allocation)
    uint32_t jcap = 0;
    uint64_t wcap = 0, bcap = 0, acap = 0, scap = 0;
    int max_nc = 1, n_mat = 0;
    uint32_t pool = 0;
    uint64_t slots = 0;
    std::vector<uint64_t> ids;          // ticket of each published job
    std::vector<char> finished;
    uint32_t lo = 0;                    // every job below is finished
    std::chrono::steady_clock::time_point t_start, t_quiet;
    PublishStage P;
};

struct Server {
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool quit = false;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
    cudaStream_t st = nullptr;          // run set-up and the kernel
    cudaStream_t poll = nullptr;        // publications, job-state copies and control words while it runs
    cudaEvent_t ev_end = nullptr;
    JobState *h_js = nullptr;           // pinned
    unsigned long long *h_buf = nullptr;   // pinned: one job's sums + its issued count
    size_t h_js_cap = 0, h_buf_cap = 0;
    ServeRun R;
    frw_serve_info info = {};       // counters (under mu)
};

}  // namespace

static double serve_quiet_s() { return 0.5; }   // an idle open run closes after this long

// admission verdict for one request: 0 fits now, 1 fits a new run, 2 never fits
static int serve_fits(frw_ctx *ctx, const ServeRun &R, const Ticket &t, int *why)
{
    const frw_job &j = t.run.desc;
    if (j.structure_id < 0 || j.structure_id >= (int)ctx->structs.size() || !ctx->structs[j.structure_id].live) {
        *why = FRW_ENOTFOUND;
        return 2;
    }
    const HostStructure &H = ctx->structs[j.structure_id];
    const uint64_t batch = j.batch ? j.batch : 16384;
    const uint64_t nb = (j.walk_budget + batch - 1) / batch;
    const uint64_t aw = nb * acc_stride_for(H.n_c), sw = sum_words(H.n_c);
    if (j.walk_budget > R.wcap || nb > R.bcap || aw > R.acap || sw > R.scap) {
        *why = FRW_ENOMEM;
        return 2;
    }
    if (H.n_c > R.max_nc || H.mat_need > R.n_mat) return 1;   // the run's kernel was set up without it
    if (R.A.jobs >= R.jcap || R.A.walks + j.walk_budget > R.wcap || R.A.batches + nb > R.bcap ||
        R.A.acc + aw > R.acap || R.A.sums + sw > R.scap)
        return 1;
    return 0;
}

static int serve_start_run(frw_ctx *ctx, Server &S)
{
    ServeRun &R = S.R;
    ctx->engine_mu.lock();
    R = ServeRun();
    {
        std::lock_guard<std::mutex> lk(ctx->struct_mu);
        for (const auto &H : ctx->structs)
            if (H.live) R.max_nc = std::max(R.max_nc, H.n_c);
        R.n_mat = (int)ctx->eps.size();
    }
    const int64_t mb = ctx->opt.serve_arena_mb > 0 ? ctx->opt.serve_arena_mb : 4096;
    R.jcap = ctx->opt.serve_jobs > 0 ? (uint32_t)ctx->opt.serve_jobs : 4096u;
    R.wcap = ((uint64_t)mb << 20) / 32;                 // 32 bytes of records per walk
    R.bcap = R.wcap / 1024 + R.jcap;                    // batches of >= 1024 walks, one partial per job
    R.acap = R.bcap * acc_stride_for(R.max_nc);
    R.scap = (uint64_t)R.jcap * sum_words(R.max_nc);
    int rc;
    if ((rc = ensure_records(ctx, R.wcap)) || (rc = ensure_runbufs(ctx, R.jcap, R.bcap, R.acap, R.scap))) {
        ctx->engine_mu.unlock();
        return rc;
    }
    if (S.h_js_cap < R.jcap) {
        if (S.h_js) cudaFreeHost(S.h_js);
        S.h_js = nullptr;
        if (cudaMallocHost(&S.h_js, sizeof(JobState) * R.jcap) != cudaSuccess) {
            ctx->engine_mu.unlock();
            return fail(ctx, FRW_ENOMEM, "pinned job-state buffer");
        }
        S.h_js_cap = R.jcap;
    }
    const size_t hb = sum_words(R.max_nc) + 1;
    if (S.h_buf_cap < hb) {
        if (S.h_buf) cudaFreeHost(S.h_buf);
        S.h_buf = nullptr;
        if (cudaMallocHost(&S.h_buf, sizeof(unsigned long long) * hb) != cudaSuccess) {
            ctx->engine_mu.unlock();
            return fail(ctx, FRW_ENOMEM, "pinned result buffer");
        }
        S.h_buf_cap = hb;
    }
    R.pool = run_pool_for(ctx, ~0ull >> 8);
    R.slots = (uint64_t)R.pool * ctx->grid;
    Arena full;
    full.jobs = R.jcap;
    full.walks = R.wcap;
    full.batches = R.bcap;
    full.acc = R.acap;
    full.sums = R.scap;
    static const uint32_t ctrl_open[CTRL_WORDS] = {1u, 0u, 0u, 0u};
    cudaError_t e = zero_run(ctx->rb, ctx->rec.k, R.jcap, full, S.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->ctrl, ctrl_open, sizeof(ctrl_open), cudaMemcpyHostToDevice, S.st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t) * STAT_WORDS, S.st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->cycles, 0, sizeof(unsigned long long) * 8, S.st);
    // the set-up is complete before the kernel starts and before any publication
    // (publications and polls go through the second stream while the kernel runs)
    if (e == cudaSuccess) e = cudaStreamSynchronize(S.st);
    const EngineView E = run_view(ctx, ctx->rb, ctx->rec, ctx->rec_cap, R.jcap, R.max_nc, R.pool, R.bcap);
    if (e == cudaSuccess) e = prepare_walk(E);
    if (e == cudaSuccess) e = launch_walk(E, ctx->shape, S.st);
    if (e == cudaSuccess) e = cudaEventRecord(S.ev_end, S.st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(S.st);
        ctx->engine_mu.unlock();
        return cuda_fail(ctx, e, "serving run start");
    }
    R.active = true;
    R.t_start = R.t_quiet = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.info.runs++;
    }
    return FRW_OK;
}

static void serve_complete(Server &S, Ticket &t, int rc)
{
    t.rc = rc;
    t.state = 2;
    if (rc == FRW_ECANCELED) S.info.cancelled++;
    else if (rc == FRW_ENOMEM) S.info.refused++;
    else S.info.completed++;
    t.t_done = std::chrono::steady_clock::now();
    S.cv_done.notify_all();
}

// copy the states of the run's unfinished jobs; finish every decided one
static int serve_poll(frw_ctx *ctx, Server &S)
{
    ServeRun &R = S.R;
    const uint32_t pub = (uint32_t)R.ids.size();
    if (pub <= R.lo) return FRW_OK;
    const uint32_t n = pub - R.lo;
    CK(cudaMemcpyAsync(S.h_js + R.lo, ctx->rb.js + R.lo, sizeof(JobState) * n, cudaMemcpyDeviceToHost, S.poll));
    CK(cudaStreamSynchronize(S.poll));
    for (uint32_t i = R.lo; i < pub; i++) {
        if (R.finished[i] || S.h_js[i].decided == 0u) continue;
        // decided: the job's sums and state are final; read them again, in full
        Ticket *tp;
        {
            std::lock_guard<std::mutex> lk(S.mu);
            tp = S.tickets[R.ids[i]].get();
        }
        JobRun &j = tp->run;
        if (S.h_js[i].decided == 3u) {   // cancelled: no result
            R.finished[i] = 1;
            std::lock_guard<std::mutex> lk(S.mu);
            serve_complete(S, *tp, FRW_ECANCELED);
            continue;
        }
        const uint32_t words = acc_stride_for(j.d.n_c);
        CK(cudaMemcpyAsync(S.h_js + i, ctx->rb.js + i, sizeof(JobState), cudaMemcpyDeviceToHost, S.poll));
        CK(cudaMemcpyAsync(S.h_buf, ctx->rb.jsum + j.sum_off, sizeof(unsigned long long) * words,
                           cudaMemcpyDeviceToHost, S.poll));
        CK(cudaMemcpyAsync(S.h_buf + words, ctx->rb.next + i, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           S.poll));
        CK(cudaStreamSynchronize(S.poll));
        take_result(j, S.h_js[i], S.h_buf, S.h_buf[words]);
        R.finished[i] = 1;
        std::lock_guard<std::mutex> lk(S.mu);
        serve_complete(S, *tp, j.desc.sigma_target > 0.0 && !j.converged ? FRW_ENOTCONV : FRW_OK);
    }
    while (R.lo < pub && R.finished[R.lo]) R.lo++;
    return FRW_OK;
}

static void serve_end_run(frw_ctx *ctx, Server &S, int rc_run)
{
    ServeRun &R = S.R;
    cudaStreamSynchronize(S.st);
    int rc = rc_run ? rc_run : check_status(ctx, S.st);
    if (rc) {
        std::lock_guard<std::mutex> lk(S.mu);
        S.info.runs_failed++;
        S.info.last_status = ctx->h_status[STAT_ERR];
    }
    if (!rc) rc = serve_poll(ctx, S);
    {
        std::lock_guard<std::mutex> lk(S.mu);
        for (size_t i = 0; i < R.ids.size(); i++)
            if (!R.finished[i]) serve_complete(S, *S.tickets[R.ids[i]], rc ? rc : FRW_EDEVICE);
    }
    R.active = false;
    R.closing = false;
    ctx->engine_mu.unlock();
}

static void serve_loop(frw_ctx *ctx)
{
    Server &S = *ctx->srv;
    cudaSetDevice(ctx->device);
    static const uint32_t closed = 0u;
    for (;;) {
        ServeRun &R = S.R;
        if (!R.active) {
            {
                std::unique_lock<std::mutex> lk(S.mu);
                S.cv_work.wait(lk, [&] { return S.quit || !S.queue.empty(); });
                if (S.queue.empty()) break;   // quit with nothing queued
            }
            const int rc = serve_start_run(ctx, S);
            if (rc) {
                std::lock_guard<std::mutex> lk(S.mu);
                while (!S.queue.empty()) {
                    serve_complete(S, *S.tickets[S.queue.front()], rc);
                    S.queue.pop_front();
                }
                continue;
            }
        }
        // admission, in arrival order
        std::vector<JobRun *> adm;
        bool want_close = false;
        {
            std::lock_guard<std::mutex> lk(S.mu);
            std::lock_guard<std::mutex> ls(ctx->struct_mu);
            while (!R.closing && !S.queue.empty()) {
                Ticket &t = *S.tickets[S.queue.front()];
                if (t.run.desc.walk_budget == 0) {   // nothing to run: an all-zero row
                    const int nc = t.run.desc.structure_id >= 0 && t.run.desc.structure_id < (int)ctx->structs.size()
                                       ? ctx->structs[t.run.desc.structure_id].n_c : 0;
                    t.run.d.n_c = nc;
                    t.run.S1.assign(nc + 1, 0);
                    t.run.S2.assign(nc + 1, 0);
                    serve_complete(S, t, FRW_OK);
                    S.queue.pop_front();
                    continue;
                }
                int why = FRW_OK;
                const int v = serve_fits(ctx, R, t, &why);
                if (v == 2) {
                    serve_complete(S, t, why);
                    S.queue.pop_front();
                    continue;
                }
                if (v == 1) {
                    want_close = true;
                    break;
                }
                place_job(ctx, t.run, R.A);
                t.state = 1;
                t.index = (uint32_t)R.ids.size();
                adm.push_back(&t.run);
                R.ids.push_back(S.queue.front());
                R.finished.push_back(0);
                S.queue.pop_front();
            }
        }
        int rc = FRW_OK;
        if (!adm.empty()) {
            int n_sigma = 0;
            for (size_t i = R.lo; i < R.ids.size(); i++) n_sigma += R.finished[i] ? 0 : 1;
            for (JobRun *j : adm) j->first_limit = first_wave(*j, R.slots, n_sigma, 8);
            const uint32_t j0 = (uint32_t)(R.ids.size() - adm.size());
            cudaError_t e = publish_jobs(ctx->rb, adm.data(), j0, (uint32_t)adm.size(), R.P, S.poll);
            if (e == cudaSuccess) e = cudaStreamSynchronize(S.poll);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "serving publication");
            R.t_quiet = std::chrono::steady_clock::now();
        }
        if (!rc) rc = serve_poll(ctx, S);
        const auto now = std::chrono::steady_clock::now();
        const bool all_done = R.lo == (uint32_t)R.ids.size();
        if (!all_done) R.t_quiet = now;
        bool quit_now;
        {
            std::lock_guard<std::mutex> lk(S.mu);
            quit_now = S.quit && S.queue.empty();
        }
        const bool quiet = all_done && std::chrono::duration<double>(now - R.t_quiet).count() > serve_quiet_s();
        const bool overdue = std::chrono::duration<double>(now - R.t_start).count() > run_timeout_s();
        if (!R.closing && (rc || want_close || quiet || quit_now || overdue)) {
            if (overdue) {
                static const uint32_t abort1 = 1;
                cudaMemcpyAsync(ctx->ctrl + CTRL_ABORT, &abort1, sizeof(uint32_t), cudaMemcpyHostToDevice, S.poll);
                if (!rc) rc = fail(ctx, FRW_ETIMEOUT, "serving run exceeded its wall-clock limit (FRW_RUN_TIMEOUT_S)");
            }
            cudaMemcpyAsync(ctx->ctrl + CTRL_OPEN, &closed, sizeof(uint32_t), cudaMemcpyHostToDevice, S.poll);
            cudaStreamSynchronize(S.poll);
            R.closing = true;
        }
        // the run ends once closed and drained, or when its kernel ended on its own
        // (a device error, e.g. the idle limit): the next request starts a new run
        if (cudaEventQuery(S.ev_end) != cudaErrorNotReady) {
            serve_end_run(ctx, S, rc);
            continue;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(30));
    }
}

static int start_server(frw_ctx *ctx)
{
    if (ctx->srv) return FRW_OK;
    std::unique_ptr<Server> S(new Server());
    if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->poll, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->ev_end, cudaEventDisableTiming) != cudaSuccess)
        return fail(ctx, FRW_EDEVICE, "serving streams");
    ctx->srv = S.release();
    ctx->srv->th = std::thread(serve_loop, ctx);
    return FRW_OK;
}

static void stop_server(frw_ctx *ctx)
{
    Server *S = ctx->srv;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->quit = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    if (S->h_js) cudaFreeHost(S->h_js);
    if (S->h_buf) cudaFreeHost(S->h_buf);
    if (S->ev_end) cudaEventDestroy(S->ev_end);
    if (S->st) cudaStreamDestroy(S->st);
    if (S->poll) cudaStreamDestroy(S->poll);
    delete S;
    ctx->srv = nullptr;
}

extern "C" int frw_submit(frw_ctx *ctx, const frw_job *job, uint64_t *ticket)
{
    if (!ctx || !job || !ticket) return FRW_EINVAL;
    {
        std::lock_guard<std::mutex> ls(ctx->struct_mu);
        const int rc = check_job(ctx, *job);
        if (rc) return rc;
    }
    if (!ctx->srv) {
        const int rc = start_server(ctx);
        if (rc) return rc;
    }
    Server &S = *ctx->srv;
    std::unique_ptr<Ticket> t(new Ticket());
    t->run.desc = *job;
    t->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        const uint64_t id = S.next_ticket++;
        S.tickets[id] = std::move(t);
        S.queue.push_back(id);
        S.info.submitted++;
        *ticket = id;
    }
    S.cv_work.notify_all();
    return FRW_OK;
}

extern "C" int frw_get_serve_info(frw_ctx *ctx, frw_serve_info *out)
{
    if (!ctx || !out) return FRW_EINVAL;
    memset(out, 0, sizeof(*out));
    if (!ctx->srv) return FRW_OK;
    std::lock_guard<std::mutex> lk(ctx->srv->mu);
    *out = ctx->srv->info;
    return FRW_OK;
}

extern "C" int frw_cancel(frw_ctx *ctx, uint64_t ticket)
{
    if (!ctx) return FRW_EINVAL;
    if (!ctx->srv) return FRW_ENOTFOUND;
    Server &S = *ctx->srv;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end()) return FRW_ENOTFOUND;
    Ticket &t = *it->second;
    if (t.state == 0) {
        for (auto q = S.queue.begin(); q != S.queue.end(); ++q)
            if (*q == ticket) {
                S.queue.erase(q);
                break;
            }
        serve_complete(S, t, FRW_ECANCELED);
    } else if (t.state == 1) {
        // the kernel drops the job's walks and closes the job at its next epoch; the
        // copy completes before the lock is released, hence before the run can end
        static const int two = 2;
        CK(cudaMemcpyAsync(ctx->rb.cancel + t.index, &two, sizeof(int), cudaMemcpyHostToDevice, S.poll));
        CK(cudaStreamSynchronize(S.poll));
    }
    return FRW_OK;
}

extern "C" int frw_poll(frw_ctx *ctx, uint64_t ticket, int32_t *done)
{
    if (!ctx || !done) return FRW_EINVAL;
    if (!ctx->srv) return FRW_ENOTFOUND;
    Server &S = *ctx->srv;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end()) return FRW_ENOTFOUND;
    *done = it->second->state == 2 ? 1 : 0;
    return FRW_OK;
}

extern "C" int frw_wait(frw_ctx *ctx, uint64_t ticket, double timeout_s, double *C_row, double *stderr_row,
                        frw_stats *stats)
{
    if (!ctx) return FRW_EINVAL;
    if (!ctx->srv) return FRW_ENOTFOUND;
    Server &S = *ctx->srv;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end()) return FRW_ENOTFOUND;
    Ticket *t = it->second.get();
    const auto pred = [&] { return t->state == 2; };
    if (timeout_s < 0) S.cv_done.wait(lk, pred);
    else if (!S.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return FRW_ETIMEOUT;
    const int rc = t->rc;
    if (rc == FRW_OK || rc == FRW_ENOTCONV) {
        row_from(t->run, C_row, stderr_row);
        if (stats) {
            fill_stats(*stats, t->run);
            stats->seconds = std::chrono::duration<double>(t->t_done - t->t_submit).count();
            stats->launches = 0;
        }
    }
    S.tickets.erase(it);
    return rc;
}

// ---------------------------------------------------------------------------
// Launch settings and the autotuner.
static int tuning_ok(frw_ctx *ctx, const frw_tuning &t)
{
    const int pool0 = (int)(ctx->NS / ctx->grid);
    return t.pool_per_cta >= 256 && t.pool_per_cta <= pool0 && t.pool_per_cta % 256 == 0 && t.hops_per_epoch >= 1 &&
           t.hops_per_epoch <= 64 && t.suspend_lanes >= 0 && t.suspend_lanes <= 32 && t.suspend_min_steps >= 4 &&
           t.suspend_min_steps <= 4096 && t.mw_warps_per_cta >= 1 &&
           t.mw_warps_per_cta <= 16 && t.mw_ctas_per_sm >= 1 && t.mw_ctas_per_sm <= 32 && t.geo_warps >= 0 &&
           t.geo_warps <= walk_geo_warps_max() && (t.unstaged == 0 || t.unstaged == 1);
}

static int apply_tuning(frw_ctx *ctx, const frw_tuning &t)
{
    if (!tuning_ok(ctx, t)) return fail(ctx, FRW_EINVAL, "tuning outside its ranges");
    const cudaError_t e = set_kernel_attributes(ctx->opt.N, t.mw_warps_per_cta, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    ctx->tune = t;
    ctx->shape.mw_warps = t.mw_warps_per_cta;
    ctx->shape.mw_ctas_per_sm = t.mw_ctas_per_sm;
    return FRW_OK;
}

extern "C" int frw_get_tuning(frw_ctx *ctx, frw_tuning *out)
{
    if (!ctx || !out) return FRW_EINVAL;
    *out = ctx->tune;
    return FRW_OK;
}

extern "C" int frw_set_tuning(frw_ctx *ctx, const frw_tuning *t)
{
    if (!ctx || !t) return FRW_EINVAL;
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    CK(cudaSetDevice(ctx->device));
    return apply_tuning(ctx, *t);
}

// random cube records for timing the MicroWalk kernel (64 int32 words each, the
// frw_microwalk_cubes layout): background and 2-6 blocks with voxel ranges
// uniform in [0, N] and materials 0 .. n_mat-1 (a plain 64-bit LCG)
static void tune_cubes(int N, int n_cubes, int n_mat, std::vector<int32_t> &rec)
{
    rec.assign((size_t)n_cubes * 64, 0);
    uint64_t x = 0x9e3779b97f4a7c15ull;
    auto next = [&](uint32_t m) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        return (uint32_t)((x >> 33) % m);
    };
    for (int c = 0; c < n_cubes; c++) {
        int32_t *r = &rec[(size_t)c * 64];
        r[0] = (int32_t)next((uint32_t)n_mat);
        const int K = 2 + (int)next(5);
        r[1] = K;
        for (int b = 0; b < K; b++) {
            for (int a = 0; a < 3; a++) {
                int lo = (int)next((uint32_t)N), hi = (int)next((uint32_t)N);
                if (lo > hi) std::swap(lo, hi);
                r[2 + 7 * b + 2 * a] = lo;
                r[3 + 7 * b + 2 * a] = hi + 1;
            }
            r[8 + 7 * b] = (int32_t)next((uint32_t)n_mat);
        }
    }
}

extern "C" int frw_autotune(frw_ctx *ctx, const frw_job *sample, int32_t n_sample, uint64_t sample_walks,
                            frw_tuning *out)
{
    if (!ctx || (n_sample > 0 && !sample) || n_sample < 0) return FRW_EINVAL;
    CK(cudaSetDevice(ctx->device));
    frw_tuning best = ctx->tune;
    // walk kernel: slots per CTA x analytical hops per epoch on the sample jobs (budget mode)
    if (n_sample > 0 && sample_walks > 0) {
        std::vector<frw_job> jobs(sample, sample + n_sample);
        for (auto &j : jobs) {
            int rc = check_job(ctx, j);
            if (rc) return rc;
            j.sigma_target = 0.0;
            j.walk_budget = std::min<uint64_t>(j.walk_budget ? j.walk_budget : sample_walks, sample_walks);
        }
        const int pool0 = (int)(ctx->NS / ctx->grid);
        // candidate pools: 1024 .. 4096 up to the context's own, and the context's own, once each
        std::vector<int> pools;
        for (int pool : {1024, 2048, 3072, 4096})
            if (pool < pool0) pools.push_back(pool);
        pools.push_back(pool0);
        double best_rate = 0.0;
        for (int rep = 0; rep < 2; rep++) {           // the first pass also warms the table cache
            for (int pool : pools) {
                // (hops per epoch, suspension lanes, suspension progress guard)
                static const int cand[][3] = {{1, 32, 128}, {1, 32, 64}, {1, 32, 256}, {1, 16, 128}, {1, 32, 32},
                                              {2, 32, 128}, {2, 32, 64}, {2, 32, 256}, {3, 32, 128}, {4, 32, 64}};
                for (const auto &c : cand) {
                    frw_tuning t = ctx->tune;
                    t.pool_per_cta = pool;
                    t.hops_per_epoch = c[0];
                    t.suspend_lanes = c[1];
                    t.suspend_min_steps = c[2];
                    std::vector<JobRun> runs(jobs.size());
                    for (size_t i = 0; i < jobs.size(); i++) runs[i].desc = jobs[i];
                    std::vector<frw_stats> st(jobs.size());
                    std::lock_guard<std::mutex> engine(ctx->engine_mu);
                    const frw_tuning keep = ctx->tune;
                    ctx->tune = t;
                    const int rc = run_jobs(ctx, runs, st.data());
                    ctx->tune = keep;
                    if (rc) return rc;
                    uint64_t walks = 0;
                    for (auto &r : runs) walks += r.walks;
                    const double rate = st[0].kernel_ms > 0 ? walks / (st[0].kernel_ms * 1e-3) : 0.0;
                    if (rep == 1 && rate > best_rate) {
                        best_rate = rate;
                        best.pool_per_cta = pool;
                        best.hops_per_epoch = t.hops_per_epoch;
                        best.suspend_lanes = t.suspend_lanes;
                        best.suspend_min_steps = t.suspend_min_steps;
                        best.walks_per_s = rate;
                    }
                }
            }
        }
    }
    // stand-alone MicroWalk kernel: warps per CTA x CTAs per SM on random cubes of the context's N
    {
        const int N = ctx->opt.N, n_cubes = 512;
        const uint64_t spc = 4096;
        std::vector<int32_t> rec;
        std::vector<uint8_t> map;
        int rc = FRW_OK, n_mat = 0;
        {
            // the context's own materials when it has some (registers nothing new)
            std::lock_guard<std::mutex> ls(ctx->struct_mu);
            n_mat = std::min<int>(4, (int)ctx->eps.size());
            if (n_mat >= 2) {
                map.assign(16, 0);
                for (int i = 0; i < n_mat; i++) map[i] = (uint8_t)i;
            } else {
                const double eps4[4] = {2.5, 3.9, 7.0, 25.0};
                n_mat = 4;
                rc = register_materials(ctx, eps4, 4, map);
            }
        }
        if (rc) return rc;
        tune_cubes(N, n_cubes, n_mat, rec);
        std::vector<void *> tmp;
        int32_t *d_cubes = nullptr;
        uint32_t *d_exit = nullptr, *d_steps = nullptr;
        unsigned long long *d_head = nullptr;
        auto cleanup = [&]() {
            for (void *p : tmp) cudaFree(p);
        };
        if ((rc = dalloc(ctx, &d_cubes, rec.size(), tmp)) || (rc = dalloc(ctx, &d_exit, n_cubes * spc, tmp)) ||
            (rc = dalloc(ctx, &d_steps, n_cubes * spc, tmp)) || (rc = dalloc(ctx, &d_head, 1, tmp))) {
            cleanup();
            return rc;
        }
        std::lock_guard<std::mutex> engine(ctx->engine_mu);
        cudaStream_t st = ctx->stream;
        cudaError_t e = cudaMemcpyAsync(d_cubes, rec.data(), sizeof(int32_t) * rec.size(), cudaMemcpyHostToDevice, st);
        double best_mw = 0.0;
        const int shapes[5][2] = {{8, 2}, {8, 4}, {16, 1}, {16, 2}, {16, 3}};
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
            for (const auto &sh : shapes) {
                LaunchShape L = ctx->shape;
                L.mw_warps = sh[0];
                L.mw_ctas_per_sm = sh[1];
                if ((e = set_kernel_attributes(N, sh[0], 0)) != cudaSuccess) break;
                if ((e = cudaMemsetAsync(d_head, 0, sizeof(unsigned long long), st)) != cudaSuccess) break;
                if ((e = cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t) * STAT_WORDS, st)) != cudaSuccess) break;
                if ((e = cudaEventRecord(ctx->ev[2], st)) != cudaSuccess) break;
                e = launch_mw_cubes(N, d_cubes, (uint64_t)n_cubes, spc, 1u, 2u, 4, (int)ctx->eps.size(), map.data(),
                                    ctx->d_W, d_exit, d_steps,
                                    d_head, ctx->status + STAT_ERR, L, st);
                if (e != cudaSuccess) break;
                if ((e = cudaEventRecord(ctx->ev[3], st)) != cudaSuccess) break;
                if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
                if (rep == 1 && ms > 0.f) {
                    std::vector<uint32_t> steps(n_cubes * spc);
                    if ((e = cudaMemcpy(steps.data(), d_steps, sizeof(uint32_t) * steps.size(),
                                        cudaMemcpyDeviceToHost)) != cudaSuccess)
                        break;
                    double tot = 0.0;
                    for (uint32_t v : steps) tot += v;
                    const double rate = tot / (ms * 1e-3);
                    if (rate > best_mw) {
                        best_mw = rate;
                        best.mw_warps_per_cta = sh[0];
                        best.mw_ctas_per_sm = sh[1];
                        best.mw_steps_per_s = rate;
                    }
                }
            }
        }
        cleanup();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "MicroWalk autotune");
        if ((rc = check_status(ctx))) return rc;
        if ((rc = apply_tuning(ctx, best))) return rc;
    }
    if (out) *out = ctx->tune;
    return FRW_OK;
}

// ---------------------------------------------------------------------------
// Plans: a fixed job set with its launch sequence captured in a CUDA graph.
struct frw_plan {
    frw_ctx *ctx = nullptr;
    std::vector<JobRun> jobs;
    std::vector<JobRun *> live;
    std::vector<uint64_t> base_request;   // request id of each job before the offset
    Arena A;
    int max_nc = 1;
    uint32_t pool = 0;
    uint32_t stage_bytes = 0;   // the walk kernel's geometry copy per CTA (0: none)
    RunBufs rb;
    RecArrays rec;
    std::vector<void *> allocs;
    // pinned staging, read by the graph's copy nodes
    DevJob *h_jobs = nullptr;
    unsigned long long *h_lim = nullptr, *h_off = nullptr;
    uint32_t *h_bjob = nullptr, *h_words = nullptr;   // h_words: [0] published count, [1..4] control words
    uint64_t nbjob = 0;
    JobState *h_js = nullptr;
    unsigned long long *h_sum = nullptr, *h_next = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

extern "C" void frw_plan_destroy(frw_plan *P)
{
    if (!P) return;
    cudaSetDevice(P->ctx->device);
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->ev0) cudaEventDestroy(P->ev0);
    if (P->ev1) cudaEventDestroy(P->ev1);
    for (void *p : P->allocs) cudaFree(p);
    for (void *p : P->rb.allocs) cudaFree(p);
    for (void *p : {(void *)P->h_jobs, (void *)P->h_lim, (void *)P->h_off, (void *)P->h_bjob, (void *)P->h_words,
                    (void *)P->h_js, (void *)P->h_sum, (void *)P->h_next})
        if (p) cudaFreeHost(p);
    delete P;
}

template <typename T> static bool pinned(T **p, size_t n)
{
    return cudaMallocHost((void **)p, sizeof(T) * std::max<size_t>(n, 1)) == cudaSuccess;
}

extern "C" int frw_plan_create(frw_ctx *ctx, const frw_job *jobs, int32_t n_jobs, frw_plan **out)
{
    if (!ctx || !out || n_jobs < 1 || !jobs) return FRW_EINVAL;
    *out = nullptr;
    CK(cudaSetDevice(ctx->device));
    std::unique_ptr<frw_plan, void (*)(frw_plan *)> P(new frw_plan(), frw_plan_destroy);
    P->ctx = ctx;
    P->jobs.resize(n_jobs);
    {
        std::lock_guard<std::mutex> ls(ctx->struct_mu);
        for (int i = 0; i < n_jobs; i++) {
            int rc = check_job(ctx, jobs[i]);
            if (rc) return rc;
            P->jobs[i].desc = jobs[i];
            P->base_request.push_back(jobs[i].request_id);
            const HostStructure &H = ctx->structs[jobs[i].structure_id];
            P->jobs[i].d.n_c = H.n_c;
            P->jobs[i].S1.assign(H.n_c + 1, 0);
            P->jobs[i].S2.assign(H.n_c + 1, 0);
            if (jobs[i].walk_budget) {
                place_job(ctx, P->jobs[i], P->A);
                P->live.push_back(&P->jobs[i]);
                P->max_nc = std::max(P->max_nc, H.n_c);
            }
        }
    }
    const uint32_t nj = (uint32_t)P->live.size();
    if (nj == 0) {
        *out = P.release();
        return FRW_OK;
    }
    if (P->A.batches >= 0xffffffffull) return fail(ctx, FRW_EINVAL, "too many batches");
    if (P->A.walks * 32ull > (64ull << 30)) return fail(ctx, FRW_ENOMEM, "plan's walk budget too large (64 GB of records)");
    int rc;
    RecArrays &R = P->rec;
    const uint64_t nw = P->A.walks;
    if ((rc = grow_runbufs(ctx, P->rb, nj, P->A.batches, P->A.acc, P->A.sums)) ||
        (rc = dalloc(ctx, &R.omega, nw, P->allocs)) || (rc = dalloc(ctx, &R.k, nw, P->allocs)) ||
        (rc = dalloc(ctx, &R.hops, nw, P->allocs)) || (rc = dalloc(ctx, &R.steps, nw, P->allocs)) ||
        (rc = dalloc(ctx, &R.cnt_sh, nw, P->allocs)) || (rc = dalloc(ctx, &R.cnt_mw, nw, P->allocs)) ||
        (rc = dalloc(ctx, &R.branch, nw, P->allocs)))
        return rc;
    P->pool = run_pool_for(ctx, P->A.walks);
    int n_sigma = 0;
    for (JobRun *j : P->live) n_sigma += j->desc.sigma_target > 0.0 ? 1 : 0;
    for (JobRun *j : P->live) j->first_limit = first_wave(*j, (uint64_t)P->pool * ctx->grid, n_sigma, 1);
    PublishStage S;
    stage_jobs(P->live.data(), 0, nj, S);
    P->nbjob = S.bjob.size();
    if (!pinned(&P->h_jobs, nj) || !pinned(&P->h_lim, nj) || !pinned(&P->h_off, nj) || !pinned(&P->h_bjob, P->nbjob) ||
        !pinned(&P->h_words, 1 + CTRL_WORDS) || !pinned(&P->h_js, nj) || !pinned(&P->h_sum, P->A.sums) ||
        !pinned(&P->h_next, nj))
        return fail(ctx, FRW_ENOMEM, "pinned plan staging");
    memcpy(P->h_jobs, S.d.data(), sizeof(DevJob) * nj);
    memcpy(P->h_lim, S.lim.data(), sizeof(unsigned long long) * nj);
    memcpy(P->h_off, S.off.data(), sizeof(unsigned long long) * nj);
    if (P->nbjob) memcpy(P->h_bjob, S.bjob.data(), sizeof(uint32_t) * P->nbjob);
    P->h_words[0] = nj;
    for (int w = 0; w < CTRL_WORDS; w++) P->h_words[1 + w] = 0u;
    CK(cudaEventCreate(&P->ev0));
    CK(cudaEventCreate(&P->ev1));
    // capture: reset, publication, the walk kernel
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    EngineView E = run_view(ctx, P->rb, P->rec, P->A.walks, nj, P->max_nc, P->pool, P->A.batches);
    choose_stage(ctx, E, P->live);
    P->stage_bytes = E.stage_sid >= 0 ? E.stage_bytes : 0;
    CK(prepare_walk(E));
    cudaStream_t st = ctx->stream;
    CK(cudaStreamSynchronize(st));
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = zero_run(P->rb, P->rec.k, nj, P->A, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->ctrl, P->h_words + 1, sizeof(uint32_t) * CTRL_WORDS, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = publish_copies(P->rb, 0, nj, P->h_jobs, P->h_lim, P->h_off, S.b0, P->h_bjob, P->nbjob, P->h_words, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t) * STAT_WORDS, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->cycles, 0, sizeof(unsigned long long) * 8, st);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev0, st);
    if (e == cudaSuccess) e = launch_walk(E, ctx->shape, st);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev1, st);
    const cudaError_t e2 = cudaStreamEndCapture(st, &P->graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plan capture");
    *out = P.release();
    return FRW_OK;
}

extern "C" int frw_plan_run(frw_plan *P, uint64_t request_offset, double *C_rows, double *stderr_rows,
                            frw_stats *stats)
{
    if (!P) return FRW_EINVAL;
    frw_ctx *ctx = P->ctx;
    CK(cudaSetDevice(ctx->device));
    const uint32_t nj = (uint32_t)P->live.size();
    std::lock_guard<std::mutex> engine(ctx->engine_mu);
    const auto t0 = std::chrono::steady_clock::now();
    for (size_t i = 0; i < P->jobs.size(); i++) {
        JobRun &j = P->jobs[i];
        j.desc.request_id = P->base_request[i] + request_offset;
        j.d.key1 = (uint32_t)(ctx->opt.seed >> 32) ^ (uint32_t)j.desc.request_id;
        std::fill(j.S1.begin(), j.S1.end(), 0);
        std::fill(j.S2.begin(), j.S2.end(), 0);
        j.walks = j.issued = 0;
        for (auto &x : j.ex) x = 0;
        j.converged = false;
    }
    for (uint32_t i = 0; i < nj; i++) P->h_jobs[i].key1 = P->live[i]->d.key1;
    cudaStream_t st = ctx->stream;
    if (nj) {
        CK(cudaEventRecord(ctx->ev[0], st));
        CK(cudaGraphLaunch(P->exec, st));
        CK(cudaEventRecord(ctx->ev[1], st));
        const double limit_s = run_timeout_s();
        bool timed_out = false;
        while (cudaEventQuery(ctx->ev[1]) == cudaErrorNotReady) {
            if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit_s) {
                static const uint32_t abort1 = 1;
                CK(cudaMemcpyAsync(ctx->ctrl + CTRL_ABORT, &abort1, sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->aux));
                CK(cudaStreamSynchronize(ctx->aux));
                timed_out = true;
                break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        CK(cudaStreamSynchronize(st));
        int rc = check_status(ctx);
        if (rc) return rc;
        if (timed_out) return fail(ctx, FRW_ETIMEOUT, "run exceeded its wall-clock limit (FRW_RUN_TIMEOUT_S)");
        CK(cudaMemcpyAsync(P->h_js, P->rb.js, sizeof(JobState) * nj, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(P->h_sum, P->rb.jsum, sizeof(unsigned long long) * P->A.sums, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(P->h_next, P->rb.next, sizeof(unsigned long long) * nj, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (uint32_t i = 0; i < nj; i++) {
            if (P->h_js[i].decided == 0u) return fail(ctx, FRW_EDEVICE, "a job was not decided when the kernel ended");
            take_result(*P->live[i], P->h_js[i], P->h_sum + P->live[i]->sum_off, P->h_next[i]);
        }
    }
    float kms = 0.f;   // the whole replay: arena reset, publication and the walk kernel
    if (nj) cudaEventElapsedTime(&kms, ctx->ev[0], ctx->ev[1]);
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool notconv = false;
    size_t off = 0;
    for (size_t i = 0; i < P->jobs.size(); i++) {
        const JobRun &j = P->jobs[i];
        row_from(j, C_rows ? C_rows + off : nullptr, stderr_rows ? stderr_rows + off : nullptr);
        off += j.d.n_c + 1;
        if (stats) {
            fill_stats(stats[i], j);
            stats[i].seconds = secs;
            stats[i].kernel_ms = kms;
            stats[i].launches = nj ? 1 : 0;
            stats[i].rounds = ctx->h_status[STAT_EPOCHS];
            stats[i].tables_built = ctx->h_status[STAT_BUILT];
            stats[i].stage_bytes = ctx->h_status[STAT_STAGED] ? P->stage_bytes : 0;
        }
        if (j.desc.sigma_target > 0.0 && !j.converged) notconv = true;
    }
    return notconv ? FRW_ENOTCONV : FRW_OK;
}
