/*
 * frw_oracle.c -- plain, slow, single-threaded FP64 reference of the FRW +
 * MicroWalk capacitance method (Huang & Yu, "Efficient FRW Transitions via
 * Stochastic Finite Differences for Handling Non-Stratified Dielectrics").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA path is checked
 * against.  Only the test-suite, the smoke check and the bench's CPU-baseline
 * leg may load it; the library never does.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * Everything is done the obvious way:
 *   - the cube's permittivity lattice is built explicitly, one point query per
 *     voxel centre;
 *   - MicroWalk (Algorithm 3) walks that explicit lattice;
 *   - the discrete surface Green's function P = e_c^T A_II^{-1} A_IB (Eq. 8) and
 *     the first-cube flux kernel are obtained from a plain conjugate-gradient
 *     solve of the symmetric form of the finite-difference system (Eq. 4-7) on
 *     the explicit lattice, in the cube's own axes;
 *   - the FRW driver (Algorithm 1) runs walks one after the other.
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add, no fast-math) so
 * that every floating-point operation is the IEEE operation written here.
 *
 * Readings where the paper is silent (all shared, by definition, with the CUDA
 * path, whose code is written separately):
 *   R1 even-N centre: the walk starts on one of the 8 central nodes, chosen by
 *      3 random bits; e_c is the average of their indicators.
 *   R2 voxel material = material at the voxel centre, half-open box test
 *      lo <= x < hi, later blocks win; centre x_i = (c - R) + (i + 0.5) * h with
 *      h = (2 R) / N.
 *   R3 transition cube = largest conductor-free cube (L-infinity distance to the
 *      nearest conductor box or grounded wall).  A cube that lists more than
 *      ORC_KMAX = 14 dielectric blocks (after the rules of cube_classify) is
 *      halved, R -> R / 2, until it lists at most 14.  Any conductor-free cube
 *      centred at the walk's point is a valid transition domain (Sec. II-A: the
 *      potential at the centre is the surface integral over any such cube), so
 *      the estimator stays unbiased; only the walk's path changes.  The limit is
 *      the lattice encoding of the GPU path (a 4-bit slot per listed block), not
 *      a rule of the paper.
 *   R4 jump law: alpha of Eq. 6 quantised to W = floor(alpha * 2^24 + 0.5); a step
 *      draws one 32-bit word u and takes the first k with (u * S) >> 32 < prefix_k
 *      (S = sum of the six W, order -x,+x,-y,+y,-z,+z).
 *   R5 analytical route = the exact FD surface Green's function of the stratified
 *      lattice (the same distribution MicroWalk samples, Theorem 1), sampled by
 *      32-bit thresholds T_n = min(floor(2^32 cum_n), 2^32 - 1) in a canonical
 *      panel order tied to the stratification axis.
 *   R6 first cube: flux kernel F (discrete eps * d(phi)/dn at the centre, Gauss's
 *      law on the lattice) with branches B1 stratified, B2 shrink to stratified,
 *      B3 homogenise to the volume-mean permittivity.
 *   R7 Gaussian surface = master box grown by gauss_frac * (smallest L-infinity gap
 *      to another conductor or wall), point uniform by area.
 *   R8 MicroWalk-E (Sec. III-B, Fig. 3b; optional, factor f > 1): a later cube
 *      that is not stratified is expanded to half-size f * R (R = the half-size of
 *      the conductor-free cube just classified).  A voxel whose centre lies
 *      outside the domain is a node of the grounded walls; one whose centre lies in
 *      conductor k (half-open test) is a node of k, whatever block covers it.
 *      Such a neighbour has alpha = 1 (like a boundary panel, Scheme B); stepping
 *      onto it absorbs the walk at that conductor.  The expanded cube lists its
 *      dielectric blocks (rule of cube_classify) plus every conductor and every
 *      exterior slab (x < lo or x >= hi on one axis) holding a voxel centre; if
 *      that is more than ORC_KMAX objects, or its dielectric list overflows, f is
 *      lowered by one, down to 2, and otherwise plain MicroWalk runs on the R
 *      cube.  Structures of more than 254 conductors use plain MicroWalk.  An exit
 *      panel that lies in a conductor or outside the domain is absorbed by the
 *      next hop's distance test.
 *   R9 FRW-FDM (Algorithm 2; optional): a later cube that is not stratified
 *      takes the FD-based transition instead of MicroWalk: P of Eq. 8 with the
 *      unquantised alpha of Eq. 6, thresholds as in R5 over the panels in natural
 *      face order (face 2a + side, then the other two axes in increasing order),
 *      one panel sampled with the hop's first word (the word MicroWalk uses for
 *      its start node).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BOUNDARY 15        /* material id used for boundary (absorbing) nodes */
#define ORC_KMAX 14            /* at most 14 blocks in a transition cube (R3 shrink rule) */
#define ORC_MAXMAT 15
#define EPS0_FF_PER_UM 8.8541878128e-3

enum { CUBE_HOM = 0, CUBE_STRAT = 1, CUBE_NONSTRAT = 2, CUBE_OVERFLOW = 3 };
enum { KIND_SGF = 0, KIND_FLUX_PAR = 1, KIND_FLUX_PERP = 2, KIND_SGF_HOM = 3, KIND_FLUX_HOM = 4 };
enum { BR_STRAT = 0, BR_SHRINK = 1, BR_HOMOG = 2, BR_EXACT = 3 };

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11: 10 rounds of the 4x32 Philox S-box (two 32x32->64 products
 * with multipliers 0xD2511F53 and 0xCD9E8D57), key bumped by the Weyl constants
 * 0x9E3779B9 / 0xBB67AE85 between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Random words of a walk: key = (seed_lo, seed_hi ^ request_lo); counter =
 * (walk_lo, walk_hi, hop, sub).  sub 0 = the hop's own draws; sub 1 + t/4 holds
 * MicroWalk step t in word t mod 4 (hop 0 uses sub 1 for its second block). */
static void walk_block(const uint32_t key[2], uint64_t walk, uint32_t hop, uint32_t sub,
                       uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)walk, (uint32_t)(walk >> 32), hop, sub};
    orc_philox4x32_10(ctr, key, out);
}

static double u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------- */
typedef struct {
    double dom_lo[3], dom_hi[3];
    int n_c;                     /* conductor boxes */
    const double *c_lo, *c_hi;   /* n_c x 3 */
    const int32_t *c_id;         /* conductor of each box (NULL: box k is conductor k) */
    int n_cond;                  /* conductors; the grounded walls are conductor n_cond */
    int n_b;
    const double *b_lo, *b_hi;   /* n_b x 3 */
    const int32_t *b_mat;
    int n_mat;
    const double *eps;
    int bg;
} orc_structure;

typedef struct {
    int N;
    uint64_t seed, request_id;
    int hybrid;            /* 1: stratified hops take the analytical route */
    int first_mode;        /* 0: branches B1-B3; 1: exact FD flux kernel per walk */
    double gauss_frac;     /* Gaussian-surface offset as a fraction of the smallest gap */
    int max_hops;
    int mwe;               /* MicroWalk-E expansion factor (R8); 0 or 1: off */
    int transition;        /* non-stratified cubes: 0 MicroWalk (Algorithm 3), 1 FD solve (Algorithm 2) */
} orc_options;

/* Quantised alpha of Eq. 6 (reading R4): W[v][i] for an interior neighbour i of v,
 * W[v][BOUNDARY] = 2^24 (alpha = 1). */
static void make_w_table(const double *eps, int n_mat, uint32_t W[16][16])
{
    for (int a = 0; a < 16; a++)
        for (int b = 0; b < 16; b++) W[a][b] = 0;
    for (int v = 0; v < n_mat; v++) {
        for (int i = 0; i < n_mat; i++) {
            double alpha = eps[i] / (eps[i] + eps[v]);
            W[v][i] = (uint32_t)floor(alpha * 16777216.0 + 0.5);
        }
        W[v][ORC_BOUNDARY] = 16777216u;
    }
}

void orc_w_table(const double *eps, int n_mat, uint32_t *W256)
{
    uint32_t W[16][16];
    make_w_table(eps, n_mat, W);
    memcpy(W256, W, sizeof(W));
}

/* ------------------------------------------------------------------------- */
/* Geometry (reading R3). */
static double linf_to_box(const double p[3], const double *lo, const double *hi)
{
    double d = 0.0;
    for (int a = 0; a < 3; a++) {
        double t1 = lo[a] - p[a];
        double t2 = p[a] - hi[a];
        if (t1 > d) d = t1;
        if (t2 > d) d = t2;
    }
    return d;
}

static int cond_of(const orc_structure *S, int k) { return S->c_id ? S->c_id[k] : k; }

/* Distance to the nearest electrode (a conductor is the union of its boxes);
 * *who = conductor index, or n_cond for the walls (ties go to the conductor with
 * the lowest index, then to the walls). */
static double nearest_electrode(const orc_structure *S, const double p[3], int *who)
{
    double best = INFINITY;
    int kb = -1;
    for (int k = 0; k < S->n_c; k++) {
        double d = linf_to_box(p, S->c_lo + 3 * k, S->c_hi + 3 * k);
        if (d < best || (d == best && kb >= 0 && cond_of(S, k) < cond_of(S, kb))) { best = d; kb = k; }
    }
    double dw = INFINITY;
    for (int a = 0; a < 3; a++) {
        double t = p[a] - S->dom_lo[a];
        if (t < dw) dw = t;
        t = S->dom_hi[a] - p[a];
        if (t < dw) dw = t;
    }
    if (best <= dw) { *who = cond_of(S, kb); return best; }
    *who = S->n_cond;
    return dw;
}

static int material_at(const orc_structure *S, const double p[3])
{
    for (int b = S->n_b - 1; b >= 0; b--) {
        const double *lo = S->b_lo + 3 * b, *hi = S->b_hi + 3 * b;
        if (lo[0] <= p[0] && p[0] < hi[0] && lo[1] <= p[1] && p[1] < hi[1] &&
            lo[2] <= p[2] && p[2] < hi[2])
            return S->b_mat[b];
    }
    return S->bg;
}

/* Voxel centre along one axis (reading R2). */
static double vcentre(double base, double h, int i)
{
    return base + ((double)i + 0.5) * h;
}

/* ------------------------------------------------------------------------- */
/* The transition cube centred at c with half-size R, classified by the
 * stratification rule shared with the CUDA path:
 *   - a block takes part iff some voxel centre lies inside it;
 *   - a block that covers every voxel resets the list and becomes the background;
 *   - more than ORC_KMAX remaining blocks -> OVERFLOW (the caller halves R);
 *   - no remaining block -> homogeneous;
 *   - every remaining block spans all voxels on the same two axes (a layer
 *     normal to axis a) -> stratified along a;
 *   - otherwise non-stratified. */
typedef struct {
    int kind, axis, bg;
    int nlist;
    int list[ORC_KMAX];
    int N;
    double c[3], R, h, base[3];
} cube_t;

static void cube_setup(cube_t *q, const double c[3], double R, int N)
{
    q->N = N;
    q->R = R;
    q->h = (2.0 * R) / (double)N;
    for (int a = 0; a < 3; a++) {
        q->c[a] = c[a];
        q->base[a] = c[a] - R;
    }
}

/* Voxel index range [i0, i1) of block b on axis a, by scanning every centre. */
static void block_range(const orc_structure *S, const cube_t *q, int b, int a, int *i0, int *i1)
{
    double lo = S->b_lo[3 * b + a], hi = S->b_hi[3 * b + a];
    int first = q->N, last = -1;
    for (int i = 0; i < q->N; i++) {
        double x = vcentre(q->base[a], q->h, i);
        if (lo <= x && x < hi) {
            if (i < first) first = i;
            last = i;
        }
    }
    *i0 = first;
    *i1 = last + 1;
}

static void cube_classify(const orc_structure *S, cube_t *q)
{
    int N = q->N;
    q->bg = S->bg;
    q->nlist = 0;
    int overflow = 0;
    int span_axis[ORC_KMAX + 1] = {0};
    int tmp_list[4096];
    int ntmp = 0;
    for (int b = 0; b < S->n_b; b++) {
        int r[6], empty = 0, full = 1;
        for (int a = 0; a < 3; a++) {
            block_range(S, q, b, a, &r[2 * a], &r[2 * a + 1]);
            if (r[2 * a] >= r[2 * a + 1]) empty = 1;
            if (!(r[2 * a] == 0 && r[2 * a + 1] == N)) full = 0;
        }
        if (empty) continue;
        if (full) {
            ntmp = 0;
            q->bg = S->b_mat[b];
            continue;
        }
        if (ntmp < 4096) tmp_list[ntmp++] = b;
        else overflow = 1;
    }
    if (ntmp > ORC_KMAX) overflow = 1;
    if (overflow) { q->kind = CUBE_OVERFLOW; return; }
    q->nlist = ntmp;
    for (int t = 0; t < ntmp; t++) q->list[t] = tmp_list[t];
    if (ntmp == 0) { q->kind = CUBE_HOM; q->axis = 2; return; }
    /* layer axis of each listed block: the axis whose two companions are full */
    for (int t = 0; t < ntmp; t++) {
        int b = q->list[t], ax = -1;
        int r[6];
        for (int a = 0; a < 3; a++) block_range(S, q, b, a, &r[2 * a], &r[2 * a + 1]);
        for (int a = 0; a < 3; a++) {
            int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
            if (r[2 * o1] == 0 && r[2 * o1 + 1] == N && r[2 * o2] == 0 && r[2 * o2 + 1] == N) ax = a;
        }
        span_axis[t] = ax;
    }
    int ax0 = span_axis[0];
    int same = ax0 >= 0;
    for (int t = 1; t < ntmp; t++)
        if (span_axis[t] != ax0) same = 0;
    if (same) { q->kind = CUBE_STRAT; q->axis = ax0; }
    else q->kind = CUBE_NONSTRAT;
}

/* Explicit lattice: material id of every voxel, index (i*N + j)*N + k. */
static void cube_lattice(const orc_structure *S, const cube_t *q, uint8_t *lat)
{
    int N = q->N;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                double p[3] = {vcentre(q->base[0], q->h, i), vcentre(q->base[1], q->h, j),
                               vcentre(q->base[2], q->h, k)};
                lat[(i * N + j) * N + k] = (uint8_t)material_at(S, p);
            }
}

/* ------------------------------------------------------------------------- */
/* MicroWalk, Algorithm 3, on an explicit lattice (readings R1, R4).
 * Returns the exit node (one coordinate is -1 or N) and the number of steps. */
static void microwalk(int N, const uint8_t *lat, const uint32_t W[16][16], const uint32_t key[2],
                      uint64_t walk, uint32_t hop, uint32_t start_word, int node[3], uint64_t *steps)
{
    uint32_t s = start_word >> 29;
    int x[3] = {N / 2 - 1 + (int)(s & 1u), N / 2 - 1 + (int)((s >> 1) & 1u),
                N / 2 - 1 + (int)((s >> 2) & 1u)};
    uint32_t blk[4] = {0, 0, 0, 0};
    uint64_t t = 0;
    for (;;) {
        if ((t & 3u) == 0) walk_block(key, walk, hop, (uint32_t)(1u + (uint32_t)(t >> 2)), blk);
        uint32_t u = blk[t & 3u];
        int mv = lat[(x[0] * N + x[1]) * N + x[2]];
        uint32_t prefix[6], acc = 0;
        for (int k = 0; k < 6; k++) {
            int a = k >> 1, d = (k & 1) ? 1 : -1;
            int y[3] = {x[0], x[1], x[2]};
            y[a] += d;
            int mk;
            if (y[a] < 0 || y[a] >= N) mk = ORC_BOUNDARY;
            else mk = lat[(y[0] * N + y[1]) * N + y[2]];
            acc += W[mv][mk];
            prefix[k] = acc;
        }
        uint32_t r = (uint32_t)(((uint64_t)u * (uint64_t)acc) >> 32);
        int k = 0;
        while (k < 5 && !(r < prefix[k])) k++;
        x[k >> 1] += (k & 1) ? 1 : -1;
        t++;
        if (x[k >> 1] < 0 || x[k >> 1] >= N) break;
    }
    node[0] = x[0]; node[1] = x[1]; node[2] = x[2];
    *steps = t;
}

/* ------------------------------------------------------------------------- */
/* MicroWalk-E (reading R8). */
static int in_box(const double p[3], const double *lo, const double *hi)
{
    return lo[0] <= p[0] && p[0] < hi[0] && lo[1] <= p[1] && p[1] < hi[1] && lo[2] <= p[2] && p[2] < hi[2];
}

/* conductor absorbing at point p: n_cond outside the domain, k inside a box of
 * conductor k, -1 in the dielectric */
static int conductor_at(const orc_structure *S, const double p[3])
{
    if (!in_box(p, S->dom_lo, S->dom_hi)) return S->n_cond;
    for (int k = 0; k < S->n_c; k++)
        if (in_box(p, S->c_lo + 3 * k, S->c_hi + 3 * k)) return cond_of(S, k);
    return -1;
}

/* explicit lattice of an expanded cube: material ids and conductor ids (-1: none) */
static void cube_lattice_e(const orc_structure *S, const cube_t *q, uint8_t *lat, int16_t *cond)
{
    int N = q->N;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                double p[3] = {vcentre(q->base[0], q->h, i), vcentre(q->base[1], q->h, j),
                               vcentre(q->base[2], q->h, k)};
                int v = (i * N + j) * N + k;
                cond[v] = (int16_t)conductor_at(S, p);
                lat[v] = (uint8_t)material_at(S, p);
            }
}

/* conductor boxes and exterior slabs holding a voxel centre of the cube */
static int mwe_extra(const orc_structure *S, const cube_t *q)
{
    int N = q->N, n = 0;
    for (int k = 0; k < S->n_c; k++) {
        int hit = 1;
        for (int a = 0; a < 3 && hit; a++) {
            double lo = S->c_lo[3 * k + a], hi = S->c_hi[3 * k + a];
            int any = 0;
            for (int i = 0; i < N; i++) {
                double x = vcentre(q->base[a], q->h, i);
                if (lo <= x && x < hi) any = 1;
            }
            hit = any;
        }
        n += hit;
    }
    for (int a = 0; a < 3; a++) {
        if (vcentre(q->base[a], q->h, 0) < S->dom_lo[a]) n++;
        if (vcentre(q->base[a], q->h, N - 1) >= S->dom_hi[a]) n++;
    }
    return n;
}

/* MicroWalk on an expanded lattice: conductor neighbours have alpha = 1; the walk
 * ends on leaving the lattice (returns -1, exit node) or on stepping onto a
 * conductor node (returns that conductor). */
static int microwalk_e(int N, const uint8_t *lat, const int16_t *cond, const uint32_t W[16][16],
                       const uint32_t key[2], uint64_t walk, uint32_t hop, uint32_t start_word, int node[3],
                       uint64_t *steps)
{
    uint32_t s = start_word >> 29;
    int x[3] = {N / 2 - 1 + (int)(s & 1u), N / 2 - 1 + (int)((s >> 1) & 1u),
                N / 2 - 1 + (int)((s >> 2) & 1u)};
    uint32_t blk[4] = {0, 0, 0, 0};
    uint64_t t = 0;
    int absorbed = -1;
    for (;;) {
        if ((t & 3u) == 0) walk_block(key, walk, hop, (uint32_t)(1u + (uint32_t)(t >> 2)), blk);
        uint32_t u = blk[t & 3u];
        int mv = lat[(x[0] * N + x[1]) * N + x[2]];
        uint32_t prefix[6], acc = 0;
        for (int k = 0; k < 6; k++) {
            int a = k >> 1, d = (k & 1) ? 1 : -1;
            int y[3] = {x[0], x[1], x[2]};
            y[a] += d;
            int mk;
            if (y[a] < 0 || y[a] >= N) mk = ORC_BOUNDARY;
            else {
                int v = (y[0] * N + y[1]) * N + y[2];
                mk = cond[v] >= 0 ? ORC_BOUNDARY : lat[v];
            }
            acc += W[mv][mk];
            prefix[k] = acc;
        }
        uint32_t r = (uint32_t)(((uint64_t)u * (uint64_t)acc) >> 32);
        int k = 0;
        while (k < 5 && !(r < prefix[k])) k++;
        x[k >> 1] += (k & 1) ? 1 : -1;
        t++;
        if (x[k >> 1] < 0 || x[k >> 1] >= N) break;
        int c = cond[(x[0] * N + x[1]) * N + x[2]];
        if (c >= 0) {
            absorbed = c;
            break;
        }
    }
    node[0] = x[0]; node[1] = x[1]; node[2] = x[2];
    *steps = t;
    return absorbed;
}

/* Stand-alone MicroWalk-E for tests: material ids and conductor ids per voxel.
 * Returns the conductor reached, or -1 with node_out on the boundary. */
int orc_microwalk_e(int N, const uint8_t *lat, const int16_t *cond, const double *eps, int n_mat, uint64_t seed,
                    uint64_t request, uint64_t walk, uint32_t hop, int32_t *node_out, uint64_t *steps)
{
    uint32_t W[16][16];
    make_w_table(eps, n_mat, W);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)request};
    uint32_t b0[4];
    walk_block(key, walk, hop, 0, b0);
    int node[3];
    int c = microwalk_e(N, lat, cond, W, key, walk, hop, b0[0], node, steps);
    node_out[0] = node[0]; node_out[1] = node[1]; node_out[2] = node[2];
    return c;
}

/* Stand-alone MicroWalk for tests: lattice given as material ids. */
void orc_microwalk(int N, const uint8_t *lat, const double *eps, int n_mat, uint64_t seed,
                   uint64_t request, uint64_t walk, uint32_t hop, int32_t *node_out, uint64_t *steps)
{
    uint32_t W[16][16];
    make_w_table(eps, n_mat, W);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)request};
    uint32_t b0[4];
    walk_block(key, walk, hop, 0, b0);
    int node[3];
    microwalk(N, lat, W, key, walk, hop, b0[0], node, steps);
    node_out[0] = node[0]; node_out[1] = node[1]; node_out[2] = node[2];
}

/* Lattice of a cube given as integer voxel ranges (later blocks win). */
void orc_lattice_from_ranges(int N, int bg, int nblk, const int32_t *ranges, const int32_t *mat,
                             uint8_t *lat)
{
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                int m = bg;
                for (int b = 0; b < nblk; b++) {
                    const int32_t *r = ranges + 6 * b;
                    if (r[0] <= i && i < r[1] && r[2] <= j && j < r[3] && r[4] <= k && k < r[5]) m = mat[b];
                }
                lat[(i * N + j) * N + k] = (uint8_t)m;
            }
}

/* ------------------------------------------------------------------------- */
/* Finite-difference system of Eq. 4-7, symmetric form.  Multiplying row v of
 * Eq. 6 by eps_v gives S = diag(eps) * L with
 *   S_vi = -eps_v eps_i / (eps_v + eps_i)   (interior neighbour i),
 *   S_vv = sum_i eps_v eps_i / (eps_v + eps_i) + (number of boundary neighbours) * eps_v,
 * symmetric positive definite; A_II^{-1} A_IB = S_II^{-1} S_IB with S_IB = eps_v on
 * each boundary link.  Plain Jacobi-preconditioned conjugate gradients. */
static double coup(double ev, double ei) { return ev * ei / (ev + ei); }

static void s_apply(int N, const double *e, const double *y, double *out)
{
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                int v = (i * N + j) * N + k;
                double ev = e[v], acc = 0.0;
                int nb[3] = {i, j, k};
                for (int a = 0; a < 3; a++)
                    for (int d = -1; d <= 1; d += 2) {
                        int z[3] = {nb[0], nb[1], nb[2]};
                        z[a] += d;
                        if (z[a] < 0 || z[a] >= N) {
                            acc += ev * y[v];
                        } else {
                            int w = (z[0] * N + z[1]) * N + z[2];
                            double c = coup(ev, e[w]);
                            acc += c * (y[v] - y[w]);
                        }
                    }
                out[v] = acc;
            }
}

static void s_diag(int N, const double *e, double *dg)
{
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                int v = (i * N + j) * N + k;
                double acc = 0.0;
                int nb[3] = {i, j, k};
                for (int a = 0; a < 3; a++)
                    for (int d = -1; d <= 1; d += 2) {
                        int z[3] = {nb[0], nb[1], nb[2]};
                        z[a] += d;
                        if (z[a] < 0 || z[a] >= N) acc += e[v];
                        else acc += coup(e[v], e[(z[0] * N + z[1]) * N + z[2]]);
                    }
                dg[v] = acc;
            }
}

/* Solve S y = b; returns the number of iterations (negative if not converged). */
int orc_fd_solve(int N, const double *e, const double *b, double *y)
{
    int n = N * N * N;
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
    double *dg = malloc(sizeof(double) * n);
    s_diag(N, e, dg);
    double bn = 0.0;
    for (int v = 0; v < n; v++) {
        y[v] = 0.0;
        r[v] = b[v];
        z[v] = r[v] / dg[v];
        p[v] = z[v];
        bn += b[v] * b[v];
    }
    bn = sqrt(bn);
    double rz = 0.0;
    for (int v = 0; v < n; v++) rz += r[v] * z[v];
    int it, maxit = 4 * n + 100, conv = 0;
    for (it = 0; it < maxit; it++) {
        s_apply(N, e, p, q);
        double pq = 0.0;
        for (int v = 0; v < n; v++) pq += p[v] * q[v];
        if (pq == 0.0) { conv = 1; break; }
        double alpha = rz / pq;
        double rn = 0.0;
        for (int v = 0; v < n; v++) {
            y[v] += alpha * p[v];
            r[v] -= alpha * q[v];
            rn += r[v] * r[v];
        }
        if (sqrt(rn) <= 1e-15 * bn) { conv = 1; it++; break; }
        double rz2 = 0.0;
        for (int v = 0; v < n; v++) {
            z[v] = r[v] / dg[v];
            rz2 += r[v] * z[v];
        }
        double beta = rz2 / rz;
        rz = rz2;
        for (int v = 0; v < n; v++) p[v] = z[v] + beta * p[v];
    }
    free(r); free(z); free(p); free(q); free(dg);
    return conv ? it : -it;
}

/* Panel values V[f][u][v] from an interior solution y: V = eps_v * y_v at the
 * interior node adjacent to each boundary panel.  Faces f = 2a + side (side 0 =
 * low end of axis a); (u, v) = coordinates on the other two axes in increasing
 * axis order.  Index f*N*N + u*N + v. */
static void panels_from_y(int N, const double *e, const double *y, double *V)
{
    for (int f = 0; f < 6; f++) {
        int a = f >> 1, side = f & 1;
        int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
        for (int u = 0; u < N; u++)
            for (int w = 0; w < N; w++) {
                int x[3];
                x[a] = side ? N - 1 : 0;
                x[o1] = u;
                x[o2] = w;
                int v = (x[0] * N + x[1]) * N + x[2];
                V[(f * N + u) * N + w] = e[v] * y[v];
            }
    }
}

/* Discrete SGF P = e_c^T A_II^{-1} A_IB (Eq. 8) with e_c averaging the 8 central
 * nodes (R1).  eps lattice in natural order; P in the face order above. */
int orc_sgf(int N, const double *e, double *P)
{
    int n = N * N * N;
    double *b = calloc(n, sizeof(double)), *y = malloc(sizeof(double) * n);
    for (int i = N / 2 - 1; i <= N / 2; i++)
        for (int j = N / 2 - 1; j <= N / 2; j++)
            for (int k = N / 2 - 1; k <= N / 2; k++) b[(i * N + j) * N + k] = 0.125;
    int it = orc_fd_solve(N, e, b, y);
    panels_from_y(N, e, y, P);
    free(b); free(y);
    return it;
}

/* Expected MicroWalk length, Eq. 11: E(tau) = e_c^T A_II^{-1} 1.  With
 * A_II = D^{-1} L_II (D = row sums of alpha) and L = diag(eps)^{-1} S this is
 * y^T (eps .* rowsum(alpha)) with S y = e_c. */
double orc_expected_steps(int N, const double *e)
{
    int n = N * N * N;
    double *b = calloc(n, sizeof(double)), *y = malloc(sizeof(double) * n);
    for (int i = N / 2 - 1; i <= N / 2; i++)
        for (int j = N / 2 - 1; j <= N / 2; j++)
            for (int k = N / 2 - 1; k <= N / 2; k++) b[(i * N + j) * N + k] = 0.125;
    orc_fd_solve(N, e, b, y);
    double acc = 0.0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                int v = (i * N + j) * N + k;
                double rs = 0.0;
                int nb[3] = {i, j, k};
                for (int a = 0; a < 3; a++)
                    for (int d = -1; d <= 1; d += 2) {
                        int z[3] = {nb[0], nb[1], nb[2]};
                        z[a] += d;
                        if (z[a] < 0 || z[a] >= N) rs += 1.0;
                        else {
                            double ei = e[(z[0] * N + z[1]) * N + z[2]];
                            rs += ei / (ei + e[v]);
                        }
                    }
                acc += y[v] * e[v] * rs;
            }
    free(b); free(y);
    return acc;
}

/* First-cube flux kernel along +axis n (reading R6): the discrete normal flux at
 * the cube centre, averaged over the 4 node pairs straddling the centre plane,
 * each pair (v-, v+) weighted by the harmonic coupling 2 eps- eps+ / (eps- + eps+):
 *   F~ = sum_pairs w/4 (e_{v+} - e_{v-})^T A_II^{-1} A_IB   (times 1/h for F).
 * Returned per panel in the face order above (the 1/h factor is left out). */
int orc_flux(int N, const double *e, int n_axis, double *F)
{
    int n = N * N * N;
    double *b = calloc(n, sizeof(double)), *y = malloc(sizeof(double) * n);
    int c0 = N / 2 - 1, c1 = N / 2;
    int o1 = (n_axis + 1) % 3, o2 = (n_axis + 2) % 3;
    for (int s = c0; s <= c1; s++)
        for (int t = c0; t <= c1; t++) {
            int xm[3], xp[3];
            xm[n_axis] = c0; xp[n_axis] = c1;
            xm[o1] = xp[o1] = s;
            xm[o2] = xp[o2] = t;
            int vm = (xm[0] * N + xm[1]) * N + xm[2], vp = (xp[0] * N + xp[1]) * N + xp[2];
            double w = 2.0 * e[vm] * e[vp] / (e[vm] + e[vp]);
            b[vp] += 0.25 * w;
            b[vm] -= 0.25 * w;
        }
    int it = orc_fd_solve(N, e, b, y);
    panels_from_y(N, e, y, F);
    free(b); free(y);
    return it;
}

/* ------------------------------------------------------------------------- */
/* Canonical panel order of the sampling tables (reading R5).  A table frame maps
 * table axes (t0, t1, t2) to cube axes fr[0..2].  Table panel n = f*N^2 + u*N + v,
 * f = 2*ta + side over table axes, (u, v) on the other two table axes in
 * increasing table-axis order.  Returns the cube-frame face index into V. */
static int canon_to_natural(int N, const int fr[3], int n)
{
    int f = n / (N * N), rem = n % (N * N);
    int u = rem / N, w = rem % N;
    int ta = f >> 1, side = f & 1;
    int t1 = ta == 0 ? 1 : 0, t2 = ta == 2 ? 1 : 2;
    int q[3];            /* cube-frame node coordinates, -1 / N on the face axis */
    q[fr[ta]] = side ? N : -1;
    q[fr[t1]] = u;
    q[fr[t2]] = w;
    int a = fr[ta];
    int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
    return ((2 * a + side) * N + q[o1]) * N + q[o2];
}

static void frame_of(int kind, int strat_axis, int normal_axis, int fr[3])
{
    if (kind == KIND_SGF_HOM) { fr[0] = 0; fr[1] = 1; fr[2] = 2; return; }
    if (kind == KIND_FLUX_PERP) {
        fr[0] = normal_axis;
        fr[2] = strat_axis;
        fr[1] = 3 - normal_axis - strat_axis;
        return;
    }
    int a = (kind == KIND_FLUX_HOM) ? normal_axis : strat_axis;
    fr[2] = a;
    fr[0] = (a + 1) % 3;
    fr[1] = (a + 2) % 3;
}

typedef struct table_s {
    int kind, axis, naxis;
    uint8_t prof[64];
    int N;
    uint32_t *thr;      /* 6N^2 thresholds */
    uint8_t *neg;       /* flux sign per panel (1 = negative) */
    double ktot;        /* sum |F~| (flux tables) */
    struct table_s *next;
} table_t;

#define TAB_BUCKETS 65536
typedef struct {
    table_t *bucket[TAB_BUCKETS];
    int count;
} tcache_t;

static uint32_t tab_hash(int kind, int axis, int naxis, const uint8_t *prof, int N)
{
    uint32_t h = 2166136261u;
    h = (h ^ (uint32_t)kind) * 16777619u;
    h = (h ^ (uint32_t)axis) * 16777619u;
    h = (h ^ (uint32_t)naxis) * 16777619u;
    for (int i = 0; i < N; i++) h = (h ^ prof[i]) * 16777619u;
    return h & (TAB_BUCKETS - 1);
}

/* Thresholds T_n = min(floor(2^32 cum_n / total), 2^32 - 1), cum over the
 * canonical order (reading R5). */
static void build_thresholds(int N, const double *val_canon, double total, uint32_t *thr)
{
    int P = 6 * N * N;
    double cum = 0.0;
    for (int n = 0; n < P; n++) {
        cum += val_canon[n];
        double t = floor((cum / total) * 4294967296.0);
        if (t > 4294967295.0) t = 4294967295.0;
        if (t < 0.0) t = 0.0;
        thr[n] = (uint32_t)t;
    }
}

/* Table for a homogeneous or stratified cube.  kind SGF/SGF_HOM: P of Eq. 8;
 * kind FLUX_*: first-cube flux kernel for eps = 1 (HOM) or the profile. */
static table_t *table_get(tcache_t *tc, int N, int kind, int axis, int naxis, const uint8_t *prof,
                          const double *eps)
{
    uint8_t key_prof[64];
    memset(key_prof, 0, sizeof(key_prof));
    int hom = (kind == KIND_SGF_HOM || kind == KIND_FLUX_HOM);
    if (!hom) memcpy(key_prof, prof, (size_t)N);
    uint32_t h = tab_hash(kind, axis, naxis, key_prof, N);
    for (table_t *t = tc->bucket[h]; t; t = t->next)
        if (t->kind == kind && t->axis == axis && t->naxis == naxis && t->N == N &&
            memcmp(t->prof, key_prof, (size_t)N) == 0)
            return t;
    table_t *t = calloc(1, sizeof(table_t));
    t->kind = kind; t->axis = axis; t->naxis = naxis; t->N = N;
    memcpy(t->prof, key_prof, sizeof(key_prof));
    int n = N * N * N, P = 6 * N * N;
    double *e = malloc(sizeof(double) * n), *V = malloc(sizeof(double) * P);
    double *vc = malloc(sizeof(double) * P);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                int x[3] = {i, j, k};
                e[(i * N + j) * N + k] = hom ? 1.0 : eps[prof[x[axis]]];
            }
    if (kind == KIND_SGF || kind == KIND_SGF_HOM) orc_sgf(N, e, V);
    else orc_flux(N, e, naxis, V);
    int fr[3];
    frame_of(kind, axis, naxis, fr);
    for (int m = 0; m < P; m++) vc[m] = V[canon_to_natural(N, fr, m)];
    t->thr = malloc(sizeof(uint32_t) * P);
    t->neg = malloc((size_t)P);
    if (kind == KIND_SGF || kind == KIND_SGF_HOM) {
        double tot = 0.0;
        for (int m = 0; m < P; m++) tot += vc[m];
        build_thresholds(N, vc, tot, t->thr);
        memset(t->neg, 0, (size_t)P);
        t->ktot = tot;
    } else {
        double *ab = malloc(sizeof(double) * P), tot = 0.0;
        for (int m = 0; m < P; m++) {
            ab[m] = fabs(vc[m]);
            t->neg[m] = vc[m] < 0.0;
            tot += ab[m];
        }
        build_thresholds(N, ab, tot, t->thr);
        t->ktot = tot;
        free(ab);
    }
    free(e); free(V); free(vc);
    t->next = tc->bucket[h];
    tc->bucket[h] = t;
    tc->count++;
    return t;
}

static void tcache_free(tcache_t *tc)
{
    for (int b = 0; b < TAB_BUCKETS; b++) {
        table_t *t = tc->bucket[b];
        while (t) {
            table_t *nx = t->next;
            free(t->thr); free(t->neg); free(t);
            t = nx;
        }
        tc->bucket[b] = NULL;
    }
    tc->count = 0;
}

/* First n (linear scan) with u < T_n; the last panel takes the rest. */
static int sample_panel(int N, const uint32_t *thr, uint32_t u)
{
    int P = 6 * N * N;
    for (int n = 0; n < P - 1; n++)
        if (u < thr[n]) return n;
    return P - 1;
}

/* Table panel n in frame fr -> cube-frame node coordinates (one is -1 or N). */
static void panel_node(int N, const int fr[3], int n, int q[3])
{
    int f = n / (N * N), rem = n % (N * N);
    int u = rem / N, w = rem % N;
    int ta = f >> 1, side = f & 1;
    int t1 = ta == 0 ? 1 : 0, t2 = ta == 2 ? 1 : 2;
    q[fr[ta]] = side ? N : -1;
    q[fr[t1]] = u;
    q[fr[t2]] = w;
}

/* Boundary node -> point on the cube surface. */
static void node_point(const cube_t *q, const int node[3], double p[3])
{
    for (int a = 0; a < 3; a++) {
        if (node[a] < 0) p[a] = q->c[a] - q->R;
        else if (node[a] >= q->N) p[a] = q->c[a] + q->R;
        else p[a] = vcentre(q->base[a], q->h, node[a]);
    }
}

/* Material profile along the stratification axis, read off point queries on the
 * cube's central line. */
static void strat_profile(const orc_structure *S, const cube_t *q, uint8_t *prof)
{
    int a = q->axis;
    for (int i = 0; i < q->N; i++) {
        double p[3] = {vcentre(q->base[0], q->h, q->N / 2), vcentre(q->base[1], q->h, q->N / 2),
                       vcentre(q->base[2], q->h, q->N / 2)};
        p[a] = vcentre(q->base[a], q->h, i);
        prof[i] = (uint8_t)material_at(S, p);
    }
    if (q->kind == CUBE_HOM)
        for (int i = 0; i < q->N; i++) prof[i] = (uint8_t)q->bg;
}

/* ------------------------------------------------------------------------- */
/* One FRW walk, Algorithm 1. */
typedef struct {
    double omega;
    int32_t k;            /* conductor reached, n_c = ground, -1 = truncated */
    uint32_t hops;
    uint64_t steps;       /* MicroWalk steps */
    int32_t branch;       /* first-cube branch */
    uint32_t n_strat, n_hom, n_mw;
    uint32_t n_mwe;       /* MicroWalk transitions on expanded cubes (R8) */
    uint32_t n_halved;    /* cube halvings of the R3 overflow rule */
} walk_rec;

typedef struct {
    double glo[3], ghi[3], cum[6], area;
} gauss_t;

/* Gaussian surface of master i (reading R7). */
static void gauss_setup(const orc_structure *S, int master, double frac, gauss_t *g)
{
    int mb = 0;                       /* the master's (single) box */
    while (mb < S->n_c && cond_of(S, mb) != master) mb++;
    const double *lo = S->c_lo + 3 * mb, *hi = S->c_hi + 3 * mb;
    double gap = INFINITY;
    for (int k = 0; k < S->n_c; k++) {
        if (cond_of(S, k) == master) continue;
        const double *l2 = S->c_lo + 3 * k, *h2 = S->c_hi + 3 * k;
        double d = 0.0;
        for (int a = 0; a < 3; a++) {
            double t1 = l2[a] - hi[a], t2 = lo[a] - h2[a];
            if (t1 > d) d = t1;
            if (t2 > d) d = t2;
        }
        if (d < gap) gap = d;
    }
    for (int a = 0; a < 3; a++) {
        double t = lo[a] - S->dom_lo[a];
        if (t < gap) gap = t;
        t = S->dom_hi[a] - hi[a];
        if (t < gap) gap = t;
    }
    double dg = frac * gap;
    for (int a = 0; a < 3; a++) {
        g->glo[a] = lo[a] - dg;
        g->ghi[a] = hi[a] + dg;
    }
    double ex = g->ghi[0] - g->glo[0], ey = g->ghi[1] - g->glo[1], ez = g->ghi[2] - g->glo[2];
    double fa[6] = {ey * ez, ey * ez, ex * ez, ex * ez, ex * ey, ex * ey};
    double acc = 0.0;
    for (int f = 0; f < 6; f++) {
        acc += fa[f];
        g->cum[f] = acc;
    }
    g->area = acc;
}

/* Volume-mean permittivity of the explicit lattice (branch B3). */
static double lattice_mean_eps(int N, const uint8_t *lat, const double *eps)
{
    double acc = 0.0;
    int n = N * N * N;
    for (int v = 0; v < n; v++) acc += eps[lat[v]];
    return acc / (double)n;
}

typedef struct {
    const orc_structure *S;
    const orc_options *o;
    uint32_t W[16][16];
    uint32_t key[2];
    gauss_t g;
    double tau;
    tcache_t *tc;
    uint8_t *lat;
    int16_t *cond;
    double *fe, *fp;       /* FD transitions: voxel eps, panel probabilities */
    uint32_t *fthr;        /* FD transitions: cumulative thresholds */
} walker_t;

/* FD-based transition of Algorithm 2 on a voxel lattice: the discrete SGF P of
 * Eq. 8 for the voxel permittivities e (direct CG solve of the symmetric FD
 * system, e_c averaging the 8 central nodes as for MicroWalk), thresholds over the
 * panels in natural face order (face 2a + side, then the other two axes in
 * increasing order), then one boundary node per word u.  fp (6N^2 doubles) and
 * thr (6N^2 words) are work space. */
static void fdm_sample(int N, const double *e, double *fp, uint32_t *thr, int n, const uint32_t *u,
                       int32_t *nodes)
{
    int P = 6 * N * N;
    if (orc_sgf(N, e, fp) < 0) {
        fprintf(stderr, "oracle: FD transition solve did not converge\n");
        abort();
    }
    double tot = 0.0;
    for (int m = 0; m < P; m++) tot += fp[m];
    build_thresholds(N, fp, tot, thr);
    const int natural[3] = {0, 1, 2};
    for (int i = 0; i < n; i++) {
        int q[3];
        panel_node(N, natural, sample_panel(N, thr, u[i]), q);
        for (int a = 0; a < 3; a++) nodes[3 * i + a] = q[a];
    }
}

/* FD transition of the walk (FRW-FDM) on the cube q with the hop's first word u. */
static void fdm_transition(walker_t *wk, const cube_t *q, uint32_t u, int node[3])
{
    const orc_structure *S = wk->S;
    int N = wk->o->N, n3 = N * N * N;
    cube_lattice(S, q, wk->lat);
    for (int v = 0; v < n3; v++) wk->fe[v] = S->eps[wk->lat[v]];
    int32_t nd[3];
    fdm_sample(N, wk->fe, wk->fp, wk->fthr, 1, &u, nd);
    for (int a = 0; a < 3; a++) node[a] = nd[a];
}

/* For tests: n FD transitions of one lattice (material ids, eps per id), one per
 * word of u; boundary nodes (one coordinate -1 or N) into nodes[3n]. */
void orc_fdm_transitions(int N, const uint8_t *lat, const double *eps, int n, const uint32_t *u, int32_t *nodes)
{
    int n3 = N * N * N, P = 6 * N * N;
    double *e = malloc(sizeof(double) * n3), *fp = malloc(sizeof(double) * P);
    uint32_t *thr = malloc(sizeof(uint32_t) * P);
    for (int v = 0; v < n3; v++) e[v] = eps[lat[v]];
    fdm_sample(N, e, fp, thr, n, u, nodes);
    free(e); free(fp); free(thr);
}

static void do_walk(walker_t *wk, uint64_t walk, walk_rec *rec)
{
    const orc_structure *S = wk->S;
    const orc_options *o = wk->o;
    int N = o->N;
    memset(rec, 0, sizeof(*rec));
    rec->k = -1;
    /* --- hop 0: Gaussian-surface point, first transition (R6, R7) --- */
    uint32_t b0[4], b1[4];
    walk_block(wk->key, walk, 0, 0, b0);
    walk_block(wk->key, walk, 0, 1, b1);
    double uf = u53(b0[0], b0[1]), ua = u53(b0[2], b0[3]), ub = u53(b1[0], b1[1]);
    double tt = uf * wk->g.area;
    int f = 0;
    while (f < 5 && !(tt < wk->g.cum[f])) f++;
    int na = f >> 1, side = f & 1;
    int o1 = na == 0 ? 1 : 0, o2 = na == 2 ? 1 : 2;
    double r[3];
    r[na] = side ? wk->g.ghi[na] : wk->g.glo[na];
    r[o1] = wk->g.glo[o1] + ua * (wk->g.ghi[o1] - wk->g.glo[o1]);
    r[o2] = wk->g.glo[o2] + ub * (wk->g.ghi[o2] - wk->g.glo[o2]);
    double orient = side ? 1.0 : -1.0;
    int who;
    double R0 = nearest_electrode(S, r, &who);
    cube_t q;
    cube_setup(&q, r, R0, N);
    cube_classify(S, &q);
    while (q.kind == CUBE_OVERFLOW) {
        cube_setup(&q, r, q.R * 0.5, N);
        cube_classify(S, &q);
        rec->n_halved++;
    }
    table_t *tab = NULL;
    double keff;
    int fr[3];
    uint8_t prof[64];
    if (o->first_mode == 1) {
        /* exact FD flux kernel of this very cube (no table, no branches) */
        cube_lattice(S, &q, wk->lat);
        int n3 = N * N * N, P = 6 * N * N;
        double *e = malloc(sizeof(double) * n3), *F = malloc(sizeof(double) * P);
        double *ab = malloc(sizeof(double) * P);
        for (int v = 0; v < n3; v++) e[v] = S->eps[wk->lat[v]];
        orc_flux(N, e, na, F);
        double tot = 0.0;
        uint32_t *thr = malloc(sizeof(uint32_t) * P);
        for (int m = 0; m < P; m++) { ab[m] = fabs(F[m]); tot += ab[m]; }
        build_thresholds(N, ab, tot, thr);
        int m = sample_panel(N, thr, b1[2]);
        double sg = F[m] < 0.0 ? -1.0 : 1.0;
        int fa = m / (N * N), rem = m % (N * N), ax = fa >> 1;
        int p1 = ax == 0 ? 1 : 0, p2 = ax == 2 ? 1 : 2;
        int node[3];
        node[ax] = (fa & 1) ? N : -1;
        node[p1] = rem / N;
        node[p2] = rem % N;
        rec->omega = ((-wk->g.area * EPS0_FF_PER_UM) * tot) / q.h * sg * orient;
        rec->branch = BR_EXACT;
        node_point(&q, node, r);
        free(e); free(F); free(ab); free(thr);
    } else {
        int br = BR_STRAT;
        cube_t q2 = q;
        if (q.kind == CUBE_NONSTRAT) {
            br = BR_HOMOG;
            for (int m = 1; m <= N / 4; m++) {
                cube_t qs;
                cube_setup(&qs, r, (q.R * (double)(N - 2 * m)) / (double)N, N);
                cube_classify(S, &qs);
                if (qs.kind == CUBE_HOM || qs.kind == CUBE_STRAT) { q2 = qs; br = BR_SHRINK; break; }
            }
        }
        rec->branch = br;
        if (br == BR_HOMOG) {
            cube_lattice(S, &q, wk->lat);
            double em = lattice_mean_eps(N, wk->lat, S->eps);
            tab = table_get(wk->tc, N, KIND_FLUX_HOM, 0, na, NULL, S->eps);
            keff = em * tab->ktot;
            frame_of(KIND_FLUX_HOM, 0, na, fr);
        } else {
            q = q2;
            if (q.kind == CUBE_HOM) {
                tab = table_get(wk->tc, N, KIND_FLUX_HOM, 0, na, NULL, S->eps);
                keff = S->eps[q.bg] * tab->ktot;
                frame_of(KIND_FLUX_HOM, 0, na, fr);
            } else {
                strat_profile(S, &q, prof);
                int kind = (q.axis == na) ? KIND_FLUX_PAR : KIND_FLUX_PERP;
                tab = table_get(wk->tc, N, kind, q.axis, na, prof, S->eps);
                keff = tab->ktot;
                frame_of(kind, q.axis, na, fr);
            }
        }
        int m = sample_panel(N, tab->thr, b1[2]);
        double sg = tab->neg[m] ? -1.0 : 1.0;
        int node[3];
        panel_node(N, fr, m, node);
        rec->omega = ((-wk->g.area * EPS0_FF_PER_UM) * keff) / q.h * sg * orient;
        node_point(&q, node, r);
    }
    uint32_t hop = 1;
    /* --- transitions until a conductor (or the grounded walls) is reached --- */
    for (;;) {
        double d = nearest_electrode(S, r, &who);
        if (d <= wk->tau) {
            rec->k = who;
            rec->hops = hop;
            return;
        }
        if ((int)hop >= o->max_hops) {
            rec->k = -1;
            rec->hops = hop;
            return;
        }
        cube_setup(&q, r, d, N);
        cube_classify(S, &q);
        while (q.kind == CUBE_OVERFLOW) {
            cube_setup(&q, r, q.R * 0.5, N);
            cube_classify(S, &q);
            rec->n_halved++;
        }
        uint32_t hb[4];
        walk_block(wk->key, walk, hop, 0, hb);
        int node[3];
        if (o->hybrid && q.kind == CUBE_HOM) {
            tab = table_get(wk->tc, N, KIND_SGF_HOM, 2, 0, NULL, S->eps);
            frame_of(KIND_SGF_HOM, 2, 0, fr);
            panel_node(N, fr, sample_panel(N, tab->thr, hb[0]), node);
            rec->n_hom++;
        } else if (o->hybrid && q.kind == CUBE_STRAT) {
            strat_profile(S, &q, prof);
            tab = table_get(wk->tc, N, KIND_SGF, q.axis, 0, prof, S->eps);
            frame_of(KIND_SGF, q.axis, 0, fr);
            panel_node(N, fr, sample_panel(N, tab->thr, hb[0]), node);
            rec->n_strat++;
        } else {
            uint64_t st;
            int done = 0;
            if (o->mwe > 1 && S->n_cond <= 254) {
                for (int f = o->mwe; f >= 2 && !done; f--) {
                    cube_t qe;
                    cube_setup(&qe, r, q.R * (double)f, N);
                    cube_classify(S, &qe);
                    if (qe.kind == CUBE_OVERFLOW || qe.nlist + mwe_extra(S, &qe) > ORC_KMAX) continue;
                    cube_lattice_e(S, &qe, wk->lat, wk->cond);
                    int kabs = microwalk_e(N, wk->lat, wk->cond, wk->W, wk->key, walk, hop, hb[0], node, &st);
                    rec->steps += st;
                    rec->n_mw++;
                    rec->n_mwe++;
                    if (kabs >= 0) {
                        rec->k = kabs;
                        rec->hops = hop + 1;
                        return;
                    }
                    q = qe;
                    done = 1;
                }
            }
            if (!done && o->transition == 1) {
                fdm_transition(wk, &q, hb[0], node);
                rec->n_mw++;
                done = 1;
            }
            if (!done) {
                cube_lattice(S, &q, wk->lat);
                microwalk(N, wk->lat, wk->W, wk->key, walk, hop, hb[0], node, &st);
                rec->steps += st;
                rec->n_mw++;
            }
        }
        node_point(&q, node, r);
        hop++;
    }
}

/* ------------------------------------------------------------------------- */
/* Driver (Algorithm 1 + stop rule): walks walk_begin .. walk_begin+n-1 in order.
 * If sigma_target > 0, after every `batch` walks the relative standard error of
 * C_ii and of the largest |C_ij| (j != i, ground excluded) is checked and the run
 * stops at the first batch boundary where both are <= sigma_target.
 * Conductor k is the union of the boxes with c_id == k (c_id NULL: box k is
 * conductor k); the master must be a single box (its Gaussian surface, R7).
 * Outputs: S1, S2 (n_cond + 1 each, last = ground), per-walk records (optional),
 * the number of walks used.  Returns the number of distinct tables built. */
int orc_frw_run(const double *dom_lo, const double *dom_hi, int n_c, const double *c_lo,
                const double *c_hi, const int32_t *c_id, int n_cond, int n_b, const double *b_lo, const double *b_hi,
                const int32_t *b_mat, int n_mat, const double *eps, int bg,
                int N, uint64_t seed, uint64_t request, int hybrid, int first_mode,
                double gauss_frac, int max_hops, int mwe, int transition, int master, uint64_t walk_begin,
                uint64_t n_walks,
                double sigma_target, uint64_t batch,
                double *S1, double *S2, uint64_t *n_used,
                double *rec_omega, int32_t *rec_k, uint32_t *rec_hops, uint64_t *rec_steps,
                int32_t *rec_branch,
                uint64_t *stats /* 11: hops, steps, strat, hom, mw, branch 0..2, truncated, mwe, halvings */)
{
    orc_structure S = {{dom_lo[0], dom_lo[1], dom_lo[2]}, {dom_hi[0], dom_hi[1], dom_hi[2]},
                       n_c, c_lo, c_hi, c_id, c_id ? n_cond : n_c, n_b, b_lo, b_hi, b_mat, n_mat, eps, bg};
    orc_options o = {N, seed, request, hybrid, first_mode, gauss_frac, max_hops, mwe, transition};
    walker_t wk;
    wk.S = &S;
    wk.o = &o;
    make_w_table(eps, n_mat, wk.W);
    wk.key[0] = (uint32_t)seed;
    wk.key[1] = (uint32_t)(seed >> 32) ^ (uint32_t)request;
    gauss_setup(&S, master, gauss_frac, &wk.g);
    double edge = 0.0;
    for (int a = 0; a < 3; a++)
        if (dom_hi[a] - dom_lo[a] > edge) edge = dom_hi[a] - dom_lo[a];
    wk.tau = 1e-9 * edge;
    wk.tc = calloc(1, sizeof(tcache_t));
    wk.lat = malloc((size_t)N * N * N);
    wk.cond = malloc(sizeof(int16_t) * (size_t)N * N * N);
    wk.fe = malloc(sizeof(double) * (size_t)N * N * N);
    wk.fp = malloc(sizeof(double) * 6 * (size_t)N * N);
    wk.fthr = malloc(sizeof(uint32_t) * 6 * (size_t)N * N);
    for (int k = 0; k <= S.n_cond; k++) { S1[k] = 0.0; S2[k] = 0.0; }
    for (int s = 0; s < 11; s++) stats[s] = 0;
    uint64_t used = 0;
    for (uint64_t w = 0; w < n_walks; w++) {
        walk_rec rec;
        do_walk(&wk, walk_begin + w, &rec);
        if (rec.k >= 0) {
            S1[rec.k] += rec.omega;
            S2[rec.k] += rec.omega * rec.omega;
        } else {
            stats[8]++;
        }
        if (rec_omega) rec_omega[w] = rec.omega;
        if (rec_k) rec_k[w] = rec.k;
        if (rec_hops) rec_hops[w] = rec.hops;
        if (rec_steps) rec_steps[w] = rec.steps;
        if (rec_branch) rec_branch[w] = rec.branch;
        stats[0] += rec.hops;
        stats[1] += rec.steps;
        stats[2] += rec.n_strat;
        stats[3] += rec.n_hom;
        stats[4] += rec.n_mw;
        stats[9] += rec.n_mwe;
        stats[10] += rec.n_halved;
        if (rec.branch >= 0 && rec.branch <= 2) stats[5 + rec.branch]++;
        used = w + 1;
        if (sigma_target > 0.0 && batch > 0 && used % batch == 0 && used >= 2) {
            double n = (double)used;
            int ok = 1;
            double ci = S1[master] / n;
            double vi = (S2[master] - S1[master] * S1[master] / n) / (n * (n - 1.0));
            if (!(ci != 0.0 && sqrt(vi > 0 ? vi : 0) <= sigma_target * fabs(ci))) ok = 0;
            int jb = -1;
            double cb = 0.0;
            for (int j = 0; j < S.n_cond; j++) {
                if (j == master) continue;
                double cj = fabs(S1[j] / n);
                if (jb < 0 || cj > cb) { jb = j; cb = cj; }
            }
            if (jb >= 0) {
                double cj = S1[jb] / n;
                double vj = (S2[jb] - S1[jb] * S1[jb] / n) / (n * (n - 1.0));
                if (!(cj != 0.0 && sqrt(vj > 0 ? vj : 0) <= sigma_target * fabs(cj))) ok = 0;
            }
            if (ok) break;
        }
    }
    *n_used = used;
    int ntab = wk.tc->count;
    tcache_free(wk.tc);
    free(wk.tc);
    free(wk.lat);
    free(wk.cond);
    free(wk.fe);
    free(wk.fp);
    free(wk.fthr);
    return ntab;
}

/* Canonical-order table for tests: kind, strat axis, normal axis, profile of
 * material ids (ignored for HOM kinds).  Outputs thresholds, signs and the total. */
void orc_table(int N, int kind, int axis, int naxis, const uint8_t *prof, const double *eps,
               uint32_t *thr, uint8_t *neg, double *ktot)
{
    tcache_t *tc = calloc(1, sizeof(tcache_t));
    table_t *t = table_get(tc, N, kind, axis, naxis, prof, eps);
    memcpy(thr, t->thr, sizeof(uint32_t) * 6 * N * N);
    memcpy(neg, t->neg, (size_t)(6 * N * N));
    *ktot = t->ktot;
    tcache_free(tc);
    free(tc);
}

/* Canonical panel n -> cube-frame boundary node, for tests. */
void orc_panel_node(int N, int kind, int axis, int naxis, int n, int32_t *node)
{
    int fr[3], q[3];
    frame_of(kind, axis, naxis, fr);
    panel_node(N, fr, n, q);
    node[0] = q[0]; node[1] = q[1]; node[2] = q[2];
}

/* Many independent MicroWalks from the centre of one explicit lattice (walk ids
 * walk0 .. walk0+n-1, hop 0), for the Theorem 1 / Eq. 11 tests. */
void orc_microwalk_many(int N, const uint8_t *lat, const double *eps, int n_mat, uint64_t seed,
                        uint64_t request, uint64_t walk0, uint64_t n, int32_t *nodes, uint64_t *steps)
{
    uint32_t W[16][16];
    make_w_table(eps, n_mat, W);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)request};
    for (uint64_t w = 0; w < n; w++) {
        uint32_t b0[4];
        walk_block(key, walk0 + w, 0, 0, b0);
        int node[3];
        microwalk(N, lat, W, key, walk0 + w, 0, b0[0], node, &steps[w]);
        nodes[3 * w] = node[0]; nodes[3 * w + 1] = node[1]; nodes[3 * w + 2] = node[2];
    }
}

/* n MicroWalk-E walks (walk ids walk0 .. walk0+n-1, the given hop) for tests:
 * conductor reached (or -1) and exit node of each. */
void orc_microwalk_e_many(int N, const uint8_t *lat, const int16_t *cond, const double *eps, int n_mat, uint64_t seed,
                          uint64_t request, uint64_t walk0, uint64_t n, uint32_t hop, int32_t *cond_out,
                          int32_t *nodes_out, uint64_t *steps_out)
{
    for (uint64_t w = 0; w < n; w++)
        cond_out[w] = orc_microwalk_e(N, lat, cond, eps, n_mat, seed, request, walk0 + w, hop, nodes_out + 3 * w,
                                      steps_out + w);
}
