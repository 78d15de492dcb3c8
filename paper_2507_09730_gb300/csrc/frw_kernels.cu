// frw_kernels.cu -- sm_103a kernels of the FRW + MicroWalk engine.
//
//   k_walk      the persistent walk kernel: every CTA owns a pool of walk slots and
//               cycles through geometry (walk issue, first transition, cube sizing,
//               hybrid dispatch, analytical route), table fill, batch reduction and
//               MicroWalk (Algorithm 3) phases, with no global barrier;
//   k_fill_one  one analytical table for an explicit key (context set-up, frw_table);
//   k_mw        the MicroWalk loop over stand-alone cubes (frw_microwalk_cubes).
// No CTA waits for another CTA; the only wait is the bounded idle wait of k_walk
// for host control words.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cooperative_groups.h>
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "frw_internal.h"

namespace frw {

namespace cg = cooperative_groups;
#define FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 Philox bijection,
// multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
// Functions that run once per walk, per batch or per epoch, or that would be
// inlined in several places, stay out of line: the persistent walk kernel's hot
// loops then fit the instruction cache.
#define FRW_OUTLINE __noinline__
// the max-cube query and the cube classification as calls (one copy each) or
// inlined at their call sites: the query inlined measured 2 % faster on the
// interconnect workload (budget mode, 3 x 2^20 walks: 33.2 against 34.0 ms), the
// classification inlined 3 % slower
#ifndef FRW_NEAREST_CALL
#define FRW_NEAREST_CALL __forceinline__
#endif
#ifndef FRW_CLASSIFY_CALL
#define FRW_CLASSIFY_CALL FRW_OUTLINE
#endif

// Bounds checks of the debug build (-DFRW_CHECKS): a failed check sets ERR_CHECK
// (the run then ends with an error status) and the guarded access is skipped.
#ifdef FRW_CHECKS
#define FRW_CHECKED(E, cond) ((cond) ? true : (atomicOr(&(E).status[STAT_ERR], ERR_CHECK), false))
#else
#define FRW_CHECKED(E, cond) true
#endif

// Per-slot walk state, MicroWalk job records and result records are each touched
// once per hop and never reused from L1: they go through L2 only (ld/st .cg), so
// that L1 keeps the structure data and sampling tables the geometry work reads
// again and again.
template <class V> __device__ __forceinline__ V ldcg(const V *p) { return __ldcg(p); }
template <class V> __device__ __forceinline__ void stcg(V *p, V v) { __stcg(p, v); }

__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// 53-bit uniform in [0, 1) from two words.
__device__ __forceinline__ double u53(uint32_t a, uint32_t b)
{
    return __dmul_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0), (double)(b >> 6)),
                     1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// Geometry arithmetic with explicit IEEE rounding (no contraction into FMA), so
// that FP64 decisions reproduce a plain host evaluation of the same expressions.
template <typename T> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};

template <typename T> __device__ __forceinline__ const SView<T> &structure_view(const EngineView &E, int sid);
template <> __device__ __forceinline__ const SView<float> &structure_view<float>(const EngineView &E, int sid)
{
    return static_cast<const SView<float> *>(E.view_f)[sid];
}
template <> __device__ __forceinline__ const SView<double> &structure_view<double>(const EngineView &E, int sid)
{
    return static_cast<const SView<double> *>(E.view_d)[sid];
}

// cell / slab index of a coordinate (clamped; the host built the index with
// margins that absorb the rounding of this computation)
template <typename T> __device__ __forceinline__ int cell_of(T x, T org, T inv, int n)
{
    const T f = (x - org) * inv;
    int i = (f > T(0)) ? (int)f : 0;
    return i < n ? i : n - 1;
}

// Loads of the structure arrays that the walk kernel may copy into shared memory
// (conductor boxes, dielectric blocks, slab masks): generic loads, which serve a
// pointer into shared memory and one into global memory alike.  With
// FRW_STAGE_GEOM=0 nothing is copied and the arrays are read through the
// read-only data path.
#ifndef FRW_STAGE_GEOM
#define FRW_STAGE_GEOM 1
#endif
template <class V> __device__ __forceinline__ V gload(const V *p)
{
#if FRW_STAGE_GEOM
    return *p;
#else
    return __ldg(p);
#endif
}

// L-infinity distance to the nearest electrode (conductor box or grounded wall);
// who = conductor of the nearest box (lowest index on ties: boxes are sorted by
// conductor) or n_cond for the walls.  The grid cell of p lists, in ascending
// order, every box that can be nearest (or tie) anywhere in the cell, so the
// result equals the scan over all boxes.
template <typename T>
__device__ FRW_NEAREST_CALL T nearest_electrode(const SView<T> &S, const T p[3], int &who)
{
    typedef Ar<T> A;
    T best = A::inf();
    int kb = -1;
    const int n = S.n_c;
    const int cx = cell_of(p[0], S.g_org[0], S.g_inv[0], S.gdim[0]);
    const int cy = cell_of(p[1], S.g_org[1], S.g_inv[1], S.gdim[1]);
    const int cz = cell_of(p[2], S.g_org[2], S.g_inv[2], S.gdim[2]);
    const int cell = (cx * S.gdim[1] + cy) * S.gdim[2] + cz;
    const uint32_t i0 = __ldg(&S.g_off[cell]), i1 = __ldg(&S.g_off[cell + 1]);
    for (uint32_t i = i0; i < i1; i++) {
        const int k = (int)__ldg(&S.g_ids[i]);
        T d = T(0);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const T t1 = A::sub(gload(&S.clo[a * n + k]), p[a]);
            const T t2 = A::sub(p[a], gload(&S.chi[a * n + k]));
            if (t1 > d) d = t1;
            if (t2 > d) d = t2;
        }
        if (d < best) { best = d; kb = k; }
    }
    T dw = A::inf();
#pragma unroll
    for (int a = 0; a < 3; a++) {
        T t = A::sub(p[a], S.dlo[a]);
        if (t < dw) dw = t;
        t = A::sub(S.dhi[a], p[a]);
        if (t < dw) dw = t;
    }
    if (best <= dw) { who = __ldg(&S.bcond[kb]); return best; }
    who = S.n_cond;
    return dw;
}

// Voxel centre i of an axis: (c - R) + (i + 0.5) h.
template <typename T> __device__ __forceinline__ T vcentre(T base, T h, int i)
{
    return Ar<T>::add(base, Ar<T>::mul(T(i) + T(0.5), h));
}

// Smallest i in [0, N] with centre_i >= v (centres are non-decreasing in i).
template <typename T> __device__ int first_ge(T base, T h, T invh, int N, T v)
{
    T e = (v - base) * invh - T(0.5);
    int i;
    if (!(e > T(0))) i = 0;
    else if (e >= T(N)) i = N;
    else i = (int)ceil(e);
    while (i > 0 && vcentre(base, h, i - 1) >= v) i--;
    while (i < N && vcentre(base, h, i) < v) i++;
    return i;
}

struct CubeInfo {
    int kind, axis, bg, K;
    uint32_t prof[4];         // layer materials along the layering axis (nibbles)
    uint2 rng[KMAX];          // packed voxel ranges + material of the listed blocks
};

__device__ __forceinline__ int rng_lo(const uint2 r, int a) { return (a == 2) ? (int)(r.y & 255u) : (int)((r.x >> (16 * a)) & 255u); }
__device__ __forceinline__ int rng_hi(const uint2 r, int a) { return (a == 2) ? (int)((r.y >> 8) & 255u) : (int)((r.x >> (16 * a + 8)) & 255u); }
__device__ __forceinline__ int rng_mat(const uint2 r) { return (int)((r.y >> 16) & 255u); }

// Transition cube of half-size R centred at c: which blocks take part (some voxel
// centre inside), list reset by a block covering every voxel, and the class:
// homogeneous, layered along one axis, non-stratified, or too many blocks.
template <typename T>
__device__ FRW_CLASSIFY_CALL void classify_cube(const SView<T> &S, const T c[3], T R, int N, CubeInfo &q)
{
    typedef Ar<T> A;
    const T h = A::div(A::mul(T(2), R), T(N));
    const T invh = T(1) / h;
    T base[3], xmax[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        base[a] = A::sub(c[a], R);
        xmax[a] = vcentre(base[a], h, N - 1);
    }
    int count = 0;
    int bg = S.bg;
    const int nb = S.n_b;
    const int SS = S.sl_S, nw = S.sl_words;
    const T *blo = S.blo, *bhi = S.bhi;   // generic: shared or global memory
    const uint8_t *bmat = S.bmat;
    const uint32_t *Lx = S.sl_L + (size_t)(0 * SS + cell_of(A::add(c[0], R), S.sl_org[0], S.sl_inv[0], SS)) * nw;
    const uint32_t *Hx = S.sl_H + (size_t)(0 * SS + cell_of(A::sub(c[0], R), S.sl_org[0], S.sl_inv[0], SS)) * nw;
    const uint32_t *Ly = S.sl_L + (size_t)(1 * SS + cell_of(A::add(c[1], R), S.sl_org[1], S.sl_inv[1], SS)) * nw;
    const uint32_t *Hy = S.sl_H + (size_t)(1 * SS + cell_of(A::sub(c[1], R), S.sl_org[1], S.sl_inv[1], SS)) * nw;
    const uint32_t *Lz = S.sl_L + (size_t)(2 * SS + cell_of(A::add(c[2], R), S.sl_org[2], S.sl_inv[2], SS)) * nw;
    const uint32_t *Hz = S.sl_H + (size_t)(2 * SS + cell_of(A::sub(c[2], R), S.sl_org[2], S.sl_inv[2], SS)) * nw;
    for (int wd = 0; wd < nw; wd++) {
      uint32_t cand = gload(&Lx[wd]) & gload(&Hx[wd]) & gload(&Ly[wd]) & gload(&Hy[wd]) & gload(&Lz[wd]) &
                      gload(&Hz[wd]);
      while (cand) {
        const int b = 32 * wd + __ffs(cand) - 1;
        cand &= cand - 1u;
        T lo[3], hi[3];
        bool rej = false;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            lo[a] = gload(&blo[a * nb + b]);
            hi[a] = gload(&bhi[a * nb + b]);
            rej |= !(hi[a] > base[a]) || (lo[a] > xmax[a]);
        }
        if (rej) continue;
        int r0[3], r1[3];
        bool empty = false, full = true;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            r0[a] = first_ge(base[a], h, invh, N, lo[a]);
            r1[a] = first_ge(base[a], h, invh, N, hi[a]);
            empty |= r0[a] >= r1[a];
            full &= (r0[a] == 0) && (r1[a] == N);
        }
        if (empty) continue;
        const int m = gload(&bmat[b]);
        if (full) { count = 0; bg = m; continue; }
        if (count < KMAX)
            q.rng[count] = make_uint2((uint32_t)r0[0] | ((uint32_t)r1[0] << 8) | ((uint32_t)r0[1] << 16) |
                                          ((uint32_t)r1[1] << 24),
                                      (uint32_t)r0[2] | ((uint32_t)r1[2] << 8) | ((uint32_t)m << 16));
        count++;
      }
    }
    q.bg = bg;
    q.K = count;
    q.axis = 2;
    if (count > KMAX) { q.kind = CUBE_OVERFLOW; return; }
    if (count == 0) {
        q.kind = CUBE_HOM;
        return;
    }
    int ax0 = -2;
    bool same = true;
    for (int t = 0; t < count; t++) {
        const uint2 r = q.rng[t];
        int ax = -1;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
            if (rng_lo(r, o1) == 0 && rng_hi(r, o1) == N && rng_lo(r, o2) == 0 && rng_hi(r, o2) == N) ax = a;
        }
        if (t == 0) ax0 = ax;
        else if (ax != ax0) same = false;
    }
    if (!(same && ax0 >= 0)) { q.kind = CUBE_NONSTRAT; return; }
    q.kind = CUBE_STRAT;
    q.axis = ax0;
    // layer profile along ax0 (later blocks win)
    uint32_t pf[4];
    const uint32_t bgn = (uint32_t)bg * 0x11111111u;
    pf[0] = pf[1] = pf[2] = pf[3] = bgn;
    for (int t = 0; t < count; t++) {
        const uint2 r = q.rng[t];
        const uint32_t m = (uint32_t)rng_mat(r);
        for (int cc = rng_lo(r, ax0); cc < rng_hi(r, ax0); cc++) {
            const int w = cc >> 3, sh = 4 * (cc & 7);
            pf[w] = (pf[w] & ~(15u << sh)) | (m << sh);
        }
    }
    // entries beyond N stay 0 so that keys are canonical
    for (int cc = N; cc < 32; cc++) {
        const int w = cc >> 3, sh = 4 * (cc & 7);
        pf[w] &= ~(15u << sh);
    }
    q.prof[0] = pf[0]; q.prof[1] = pf[1]; q.prof[2] = pf[2]; q.prof[3] = pf[3];
}

// MicroWalk-E cube of half-size R (expanded, may hold conductors): the dielectric
// blocks as classify_cube lists them, then every conductor and every exterior
// slab of the domain (centres with x < lo or x >= hi on one axis) that holds a
// voxel centre, listed after the blocks so that they win, as objects of material
// BOUNDARY (alpha = 1) with their conductor id (n_cond: the walls) in the top byte
// of rng.y (one object per conductor box).  False when the dielectric list
// overflows or more than KMAX objects.
template <typename T>
__device__ FRW_OUTLINE bool classify_cube_e(const SView<T> &S, const T c[3], T R, int N, CubeInfo &q)
{
    typedef Ar<T> A;
    classify_cube(S, c, R, N, q);
    if (q.kind == CUBE_OVERFLOW) return false;
    const T h = A::div(A::mul(T(2), R), T(N));
    const T invh = T(1) / h;
    T base[3], xmax[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        base[a] = A::sub(c[a], R);
        xmax[a] = vcentre(base[a], h, N - 1);
    }
    int count = q.K;
    const int n = S.n_c;
    const uint32_t cmat = (uint32_t)BOUNDARY << 16;
    for (int k = 0; k < n; k++) {
        T lo[3], hi[3];
        bool rej = false;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            lo[a] = gload(&S.clo[a * n + k]);
            hi[a] = gload(&S.chi[a * n + k]);
            rej |= !(hi[a] > base[a]) || (lo[a] > xmax[a]);
        }
        if (rej) continue;
        int r0[3], r1[3];
        bool empty = false;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            r0[a] = first_ge(base[a], h, invh, N, lo[a]);
            r1[a] = first_ge(base[a], h, invh, N, hi[a]);
            empty |= r0[a] >= r1[a];
        }
        if (empty) continue;
        if (count >= KMAX) return false;
        q.rng[count++] = make_uint2((uint32_t)r0[0] | ((uint32_t)r1[0] << 8) | ((uint32_t)r0[1] << 16) |
                                        ((uint32_t)r1[1] << 24),
                                    (uint32_t)r0[2] | ((uint32_t)r1[2] << 8) | cmat |
                                        ((uint32_t)__ldg(&S.bcond[k]) << 24));
    }
    for (int a = 0; a < 3; a++) {
        const int i1 = first_ge(base[a], h, invh, N, S.dlo[a]);   // centres below the domain: [0, i1)
        const int i0 = first_ge(base[a], h, invh, N, S.dhi[a]);   // centres at or above its top: [i0, N)
        for (int side = 0; side < 2; side++) {
            const int lo_a = side ? i0 : 0, hi_a = side ? N : i1;
            if (lo_a >= hi_a) continue;
            if (count >= KMAX) return false;
            int r0[3] = {0, 0, 0}, r1[3] = {N, N, N};
            r0[a] = lo_a;
            r1[a] = hi_a;
            q.rng[count++] = make_uint2((uint32_t)r0[0] | ((uint32_t)r1[0] << 8) | ((uint32_t)r0[1] << 16) |
                                            ((uint32_t)r1[1] << 24),
                                        (uint32_t)r0[2] | ((uint32_t)r1[2] << 8) | cmat |
                                            ((uint32_t)S.n_cond << 24));
        }
    }
    q.K = count;
    q.kind = CUBE_NONSTRAT;
    return true;
}

// Volume-mean permittivity of the cube's lattice: constant-mask runs per axis,
// material of each run triple by the last listed block containing it.
__device__ FRW_OUTLINE double mean_eps(const CubeInfo &q, int N, const double *eps)
{
    int cut[3][2 * KMAX + 2];
    int ncut[3];
    for (int a = 0; a < 3; a++) {
        int n = 0;
        cut[a][n++] = 0;
        cut[a][n++] = N;
        for (int t = 0; t < q.K; t++) {
            const int l = rng_lo(q.rng[t], a), h = rng_hi(q.rng[t], a);
            cut[a][n++] = l;
            cut[a][n++] = h;
        }
        // insertion sort + unique
        for (int i = 1; i < n; i++) {
            int v = cut[a][i], j = i - 1;
            while (j >= 0 && cut[a][j] > v) { cut[a][j + 1] = cut[a][j]; j--; }
            cut[a][j + 1] = v;
        }
        int m = 0;
        for (int i = 0; i < n; i++)
            if (m == 0 || cut[a][i] != cut[a][m - 1]) cut[a][m++] = cut[a][i];
        ncut[a] = m;
    }
    double count[NMAT];
    for (int m = 0; m < NMAT; m++) count[m] = 0.0;
    for (int ix = 0; ix + 1 < ncut[0]; ix++)
        for (int iy = 0; iy + 1 < ncut[1]; iy++)
            for (int iz = 0; iz + 1 < ncut[2]; iz++) {
                const int x = cut[0][ix], y = cut[1][iy], z = cut[2][iz];
                int mat = q.bg;
                for (int t = 0; t < q.K; t++) {
                    const uint2 r = q.rng[t];
                    if (rng_lo(r, 0) <= x && x < rng_hi(r, 0) && rng_lo(r, 1) <= y && y < rng_hi(r, 1) &&
                        rng_lo(r, 2) <= z && z < rng_hi(r, 2))
                        mat = rng_mat(r);
                }
                count[mat] += (double)((cut[0][ix + 1] - x) * (cut[1][iy + 1] - y) * (cut[2][iz + 1] - z));
            }
    double acc = 0.0;
    for (int m = 0; m < NMAT; m++) acc += count[m] * eps[m];
    return acc / (double)(N * N * N);
}

// ---------------------------------------------------------------------------
// Analytical-table cache: open addressing on (kind, profile); compute-if-absent
// by a later fill launch.  Returns the entry when ready, -1 to retry next round,
// -2 when the probe window is full.
__device__ __forceinline__ uint32_t hash5(uint32_t k, const uint32_t p[4])
{
    uint32_t h = 0x9747b28cu ^ (k * 0x85ebca6bu);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint32_t x = p[i] * 0xcc9e2d51u;
        x = (x << 15) | (x >> 17);
        h ^= x * 0x1b873593u;
        h = ((h << 13) | (h >> 19)) * 5u + 0xe6546b64u;
    }
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// CTA-local list of cache entries claimed during the geometry phase; the CTA
// fills them itself in its fill phase.
struct FillList {
    uint32_t *list;
    uint32_t *count;
    uint32_t cap;
};

__device__ int table_lookup(const TableCache &tc, uint32_t kind, const uint32_t prof[4], const FillList &fl)
{
    const uint32_t h = hash5(kind, prof);
    for (uint32_t probe = 0; probe < 64; probe++) {
        const uint32_t e = (h + probe) & (tc.cap - 1);
        uint32_t st = cuda::atomic_ref<uint32_t, cuda::thread_scope_device>(tc.state[e]).load(
            cuda::memory_order_acquire);
        if (st == TE_EMPTY) {
            // claim only if this CTA has room to fill the entry in this epoch
            const uint32_t li = atomicAdd(fl.count, 1u);
            if (li >= fl.cap) return -1;
            const uint32_t old = atomicCAS(&tc.state[e], TE_EMPTY, TE_CLAIMED);
            if (old == TE_EMPTY) {
                uint32_t *k = tc.keys + 5 * e;
                k[0] = kind; k[1] = prof[0]; k[2] = prof[1]; k[3] = prof[2]; k[4] = prof[3];
                __threadfence();
                atomicExch(&tc.state[e], TE_REQUESTED);
                fl.list[li] = e;
                return -1;
            }
            fl.list[li] = 0xffffffffu;   // slot taken by another claimant: nothing to fill
            st = old;
        }
        if (st == TE_CLAIMED) return -1;
        const volatile uint32_t *k = tc.keys + 5 * e;
        if (k[0] == kind && k[1] == prof[0] && k[2] == prof[1] && k[3] == prof[2] && k[4] == prof[3])
            return (st == TE_READY) ? (int)e : -1;
    }
    return -2;
}

// smallest n in [0, P-1] with u < thr[n] (thr[P-1] counts as 2^32).  The guide
// table gives, for the bucket of u (its top 11 bits), the first panel whose
// threshold exceeds the bucket's start; no earlier panel can be the answer, so a
// short forward scan from there returns exactly the inverse-CDF sample.
__device__ __forceinline__ int sample_guided(const uint32_t *__restrict__ thr, const uint16_t *__restrict__ guide,
                                             int P, uint32_t u)
{
    int n = __ldg(&guide[u >> 21]);
    while (n < P - 1 && !(u < __ldg(&thr[n]))) n++;
    return n;
}

__device__ __forceinline__ int sample_thr(const uint32_t *__restrict__ thr, int P, uint32_t u)
{
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (u < __ldg(&thr[mid])) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Table frames: table axes (t0, t1, t2) -> cube axes.
__device__ __forceinline__ void frame_sgf(int a, int fr[3]) { fr[0] = (a + 1) % 3; fr[1] = (a + 2) % 3; fr[2] = a; }
__device__ __forceinline__ void frame_perp(int n, int a, int fr[3]) { fr[0] = n; fr[1] = 3 - n - a; fr[2] = a; }

// canonical table panel n -> boundary node in cube coordinates (-1 / N on the face axis)
__device__ __forceinline__ void panel_node(int N, const int fr[3], int n, int q[3])
{
    const int NN = N * N;
    const int f = n / NN, rem = n - f * NN;
    const int u = rem / N, w = rem - u * N;
    const int ta = f >> 1, side = f & 1;
    const int t1 = ta == 0 ? 1 : 0, t2 = ta == 2 ? 1 : 2;
    q[fr[ta]] = side ? N : -1;
    q[fr[t1]] = u;
    q[fr[t2]] = w;
}

template <typename T>
__device__ __forceinline__ void node_point(const T c[3], T R, int N, const int node[3], T p[3])
{
    typedef Ar<T> A;
    const T h = A::div(A::mul(T(2), R), T(N));
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (node[a] < 0) p[a] = A::sub(c[a], R);
        else if (node[a] >= N) p[a] = A::add(c[a], R);
        else p[a] = vcentre(A::sub(c[a], R), h, node[a]);
    }
}

// ---------------------------------------------------------------------------
// Walk slot bookkeeping
struct WalkState {
    uint32_t job, hop, cnt_sh, cnt_mw;
    int32_t branch;
    uint64_t walk, steps;
    double omega;
};

// A finished walk writes its record (electrode k last, with release order) and
// counts itself in its batch; the group of lanes that completes a batch queues
// it for reduction.
__device__ FRW_OUTLINE void finish_walk(const EngineView &E, const DevJob &J, const WalkState &w, int k)
{
    const uint64_t rel = w.walk - J.walk_begin;
    const uint64_t r = J.rec_base + rel;
    if (!FRW_CHECKED(E, rel < J.walk_count && r < E.rec_cap && J.batch_base + rel / J.batch < E.rq_cap)) return;
    stcg(&E.rec.omega[r], w.omega);
    stcg(&E.rec.hops[r], w.hop);
    stcg(&E.rec.steps[r], (uint32_t)w.steps);
    stcg(&E.rec.cnt_sh[r], w.cnt_sh);
    stcg(&E.rec.cnt_mw[r], w.cnt_mw);
    stcg(&E.rec.branch[r], w.branch);
    cuda::atomic_ref<int32_t, cuda::thread_scope_device>(E.rec.k[r]).store(k, cuda::memory_order_release);
    const uint64_t bi = rel / J.batch;
    const uint64_t g = J.batch_base + bi;
    const uint32_t bsz = (uint32_t)min(J.batch, J.walk_count - bi * J.batch);
    cg::coalesced_group grp = cg::coalesced_threads();
    cg::coalesced_group same = cg::labeled_partition(grp, (unsigned long long)g);
    if (same.thread_rank() == 0) {
        const uint32_t old = atomicAdd(&E.batch_done[g], (uint32_t)same.size());
        if (old + (uint32_t)same.size() == bsz) {
            const uint32_t qi = atomicAdd(E.rq_count, 1u);
            if (qi < E.rq_cap) E.rq[qi] = (uint32_t)g;
            else atomicOr(&E.status[STAT_ERR], ERR_REDUCE_QUEUE);
        }
    }
}

// First transition (hop 0): point on the Gaussian surface, first cube with the
// special treatment, weight omega (Algorithm 1; flux reading of FirstTransition).
// Returns false when a table is not ready yet (retry next round, same draws).
template <typename T>
__device__ FRW_OUTLINE bool first_transition(const EngineView &E, const DevJob &J, const SView<T> &S, WalkState &w,
                                 T pos[3], const FillList &fl)
{
    typedef Ar<T> A;
    const int N = E.N;
    const uint32_t wl = (uint32_t)w.walk, wh = (uint32_t)(w.walk >> 32);
    const uint4 b0 = philox10(wl, wh, 0u, 0u, J.key0, J.key1);
    const uint4 b1 = philox10(wl, wh, 0u, 1u, J.key0, J.key1);
    const double uf = u53(b0.x, b0.y), ua = u53(b0.z, b0.w), ub = u53(b1.x, b1.y);
    const double tt = __dmul_rn(uf, J.area);
    int f = 0;
    while (f < 5 && !(tt < J.cum[f])) f++;
    const int na = f >> 1, side = f & 1;
    const int o1 = na == 0 ? 1 : 0, o2 = na == 2 ? 1 : 2;
    double r[3];
    r[na] = side ? J.g_hi[na] : J.g_lo[na];
    r[o1] = __dadd_rn(J.g_lo[o1], __dmul_rn(ua, __dsub_rn(J.g_hi[o1], J.g_lo[o1])));
    r[o2] = __dadd_rn(J.g_lo[o2], __dmul_rn(ub, __dsub_rn(J.g_hi[o2], J.g_lo[o2])));
    const double orient = side ? 1.0 : -1.0;
    T rt[3] = {(T)r[0], (T)r[1], (T)r[2]};
    int who;
    T R0 = nearest_electrode(S, rt, who);
    if (E.fp32) R0 = A::sub(R0, S.margin);
    CubeInfo q;
    classify_cube(S, rt, R0, N, q);
    int guard = 0;
    while (q.kind == CUBE_OVERFLOW && guard++ < 40) {
        R0 = A::mul(R0, T(0.5));
        classify_cube(S, rt, R0, N, q);
    }
    if (q.kind == CUBE_OVERFLOW) {          // unreachable in practice: > 14 blocks at 2^-40 R
        atomicOr(&E.status[STAT_ERR], ERR_SHRINK);
        return false;
    }
    int br = 0;
    T Rc = R0;
    CubeInfo qc;
    bool use_qc = false;
    if (q.kind != CUBE_HOM && q.kind != CUBE_STRAT) {
        br = 2;
        for (int m = 1; m <= N / 4; m++) {
            const T Rs = A::div(A::mul(R0, T(N - 2 * m)), T(N));
            classify_cube(S, rt, Rs, N, qc);
            if (qc.kind == CUBE_HOM || qc.kind == CUBE_STRAT) {
                Rc = Rs;
                br = 1;
                use_qc = true;
                break;
            }
        }
    }
    const CubeInfo &qq = use_qc ? qc : q;
    const uint32_t *thr;
    const uint32_t *sgn;
    const uint16_t *guide;
    double keff;
    int fr[3];
    const TableCache &tc = E.tc;
    if (br == 2) {
        const double em = mean_eps(q, N, E.eps);
        thr = tc.thr + (size_t)(tc.cap + 1) * tc.P;
        sgn = tc.sgn + (size_t)(tc.cap + 1) * tc.P32;
        guide = tc.guide + (size_t)(tc.cap + 1) * GUIDE;
        keff = __dmul_rn(em, tc.ktot[tc.cap + 1]);
        frame_sgf(na, fr);
    } else if (qq.kind == CUBE_HOM) {
        thr = tc.thr + (size_t)(tc.cap + 1) * tc.P;
        sgn = tc.sgn + (size_t)(tc.cap + 1) * tc.P32;
        guide = tc.guide + (size_t)(tc.cap + 1) * GUIDE;
        keff = __dmul_rn(E.eps[qq.bg], tc.ktot[tc.cap + 1]);
        frame_sgf(na, fr);
    } else {
        const uint32_t kind = (qq.axis == na) ? TAB_FLUX_PAR : TAB_FLUX_PERP;
        const int e = table_lookup(tc, kind, qq.prof, fl);
        if (e < 0) {
            if (e == -2) atomicOr(&E.status[STAT_ERR], ERR_CACHE_FULL);
            return false;
        }
        thr = tc.thr + (size_t)e * tc.P;
        sgn = tc.sgn + (size_t)e * tc.P32;
        guide = tc.guide + (size_t)e * GUIDE;
        keff = tc.ktot[e];
        if (kind == TAB_FLUX_PAR) frame_sgf(na, fr);
        else frame_perp(na, qq.axis, fr);
    }
    const int m = sample_guided(thr, guide, (int)tc.P, b1.z);
    const double sg = ((__ldg(&sgn[m >> 5]) >> (m & 31)) & 1u) ? -1.0 : 1.0;
    int node[3];
    panel_node(N, fr, m, node);
    const T h = A::div(A::mul(T(2), Rc), T(N));
    w.omega = __dmul_rn(__dmul_rn(__ddiv_rn(__dmul_rn(__dmul_rn(-J.area, EPS0), keff), (double)h), sg), orient);
    w.branch = br;
    node_point(rt, Rc, N, node, pos);
    return true;
}

__device__ __forceinline__ uint32_t nib(uint32_t v, int i) { return (v >> (4 * i)) & 15u; }

__device__ __forceinline__ void store_walk(const EngineView &E, uint32_t s, const WalkState &w)
{
    stcg(&E.s.job[s], w.job);
    stcg(&E.s.hop[s], w.hop);
    stcg(&E.s.walk[s], w.walk);
    stcg(&E.s.steps[s], w.steps);
    stcg(&E.s.cnt_sh[s], w.cnt_sh);
    stcg(&E.s.cnt_mw[s], w.cnt_mw);
    stcg(&E.s.branch[s], w.branch);
    stcg(&E.s.omega[s], w.omega);
}

__device__ __forceinline__ void load_walk(const EngineView &E, uint32_t s, WalkState &w)
{
    w.job = ldcg(&E.s.job[s]);
    w.hop = ldcg(&E.s.hop[s]);
    w.walk = ldcg(&E.s.walk[s]);
    w.steps = ldcg(&E.s.steps[s]);
    w.cnt_sh = ldcg(&E.s.cnt_sh[s]);
    w.cnt_mw = ldcg(&E.s.cnt_mw[s]);
    w.branch = ldcg(&E.s.branch[s]);
    w.omega = ldcg(&E.s.omega[s]);
}

__device__ __forceinline__ bool job_open(const EngineView &E, int j)
{
    return !((volatile int *)E.job_cancel)[j] &&
           ((volatile unsigned long long *)E.job_next)[j] < ((volatile unsigned long long *)E.job_limit)[j];
}

// Walk ids are claimed per CTA, once per epoch, for exactly the number of free
// slots (one compare-and-swap per job on the job's counter, which therefore never
// passes the issue limit the stop rule may move while the kernel runs); free slots
// then take ids from the CTA's claimed ranges through a shared-memory counter.
// Jobs are served oldest first: the scan starts at the lowest undecided job.
constexpr int ISSUE_MAX_JOBS = 64;     // claimed ranges per CTA and epoch
constexpr uint32_t JOB_WINDOW = 256;   // jobs a CTA looks at per epoch
struct IssueRanges {
    uint32_t n;                        // number of ranges
    uint32_t pos;                      // next id to hand out (over the concatenated ranges)
    uint32_t total;
    uint32_t job[ISSUE_MAX_JOBS];
    unsigned long long lo[ISSUE_MAX_JOBS];
    uint32_t cnt[ISSUE_MAX_JOBS];
};

// one warp: claim up to `want` ids over the open jobs among [lo, pub)
__device__ FRW_OUTLINE void claim_ids(const EngineView &E, IssueRanges &ir, uint32_t want, uint32_t lo, uint32_t pub)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        ir.n = 0;
        ir.pos = 0;
        ir.total = 0;
    }
    __syncwarp();
    if (want == 0 || pub <= lo) return;
    const uint32_t span = min(pub - lo, JOB_WINDOW);
    for (uint32_t c = 0; c < span; c += 32) {
        const uint32_t jj = lo + c + (uint32_t)lane;
        const bool open = c + (uint32_t)lane < span && job_open(E, (int)jj);
        uint32_t bal = __ballot_sync(FULL_MASK, open);
        if (lane == 0) {
            while (bal && ir.total < want && ir.n < ISSUE_MAX_JOBS) {
                const uint32_t j = lo + c + (uint32_t)(__ffs(bal) - 1);
                bal &= bal - 1u;
                const unsigned long long lim = ((volatile unsigned long long *)E.job_limit)[j];
                for (int tries = 0; tries < 64; tries++) {
                    const unsigned long long cur = ((volatile unsigned long long *)E.job_next)[j];
                    if (cur >= lim) break;
                    const unsigned long long take = min((unsigned long long)(want - ir.total), lim - cur);
                    if (atomicCAS(&E.job_next[j], cur, cur + take) == cur) {
                        ir.job[ir.n] = j;
                        ir.lo[ir.n] = cur;
                        ir.cnt[ir.n] = (uint32_t)take;
                        ir.n++;
                        ir.total += (uint32_t)take;
                        break;
                    }
                }
            }
        }
        const uint32_t done = __shfl_sync(FULL_MASK, lane == 0 ? (uint32_t)(ir.total >= want || ir.n >= ISSUE_MAX_JOBS) : 0u, 0);
        if (done) break;
    }
    __syncwarp();
}

// one warp, at the start of an epoch: move the job table's low-water mark past the
// leading decided jobs and tell whether any job in the window can take new walks
__device__ FRW_OUTLINE void scan_jobs(const EngineView &E, uint32_t &lo_out, uint32_t &pub_out, uint32_t &open_out)
{
    const int lane = threadIdx.x & 31;
    const uint32_t pub = *(volatile uint32_t *)&E.jctl[JC_PUBLISHED];
    const uint32_t lo0 = *(volatile uint32_t *)&E.jctl[JC_LOW];
    __threadfence();   // jobs below `pub` were written before it (host copies in stream order)
    uint32_t lo = lo0;
    for (int k = 0; k < 8 && lo < pub; k++) {
        const uint32_t j = lo + (uint32_t)lane;
        const bool dec = j < pub && *(volatile uint32_t *)&E.jstate[j].decided != 0u;
        const uint32_t bal = __ballot_sync(FULL_MASK, dec);
        const uint32_t lead = (bal == FULL_MASK) ? 32u : (uint32_t)(__ffs(~bal) - 1);
        lo += lead;
        if (lead < 32u) break;
    }
    if (lane == 0 && lo > lo0) atomicMax(&E.jctl[JC_LOW], lo);
    // a job the host cancelled (job_cancel = 2) is closed here: decided = 3, counted once
    for (uint32_t c = 0; lo + c < pub && c < JOB_WINDOW; c += 32) {
        const uint32_t j = lo + c + (uint32_t)lane;
        if (j < pub && ((volatile int *)E.job_cancel)[j] == 2 && *(volatile uint32_t *)&E.jstate[j].decided == 0u &&
            atomicCAS(&E.jstate[j].decided, 0u, 3u) == 0u)
            atomicAdd(&E.jctl[JC_DECIDED], 1u);
    }
    uint32_t open = 0;
    const uint32_t span = pub > lo ? min(pub - lo, JOB_WINDOW) : 0u;
    for (uint32_t c = 0; c < span && !open; c += 32) {
        const uint32_t jj = lo + c + (uint32_t)lane;
        open = __ballot_sync(FULL_MASK, c + (uint32_t)lane < span && job_open(E, (int)jj)) != 0u;
    }
    lo_out = lo;
    pub_out = pub;
    open_out = open;
}

// a free slot takes the next claimed id (false when the CTA's ranges are used up)
__device__ FRW_OUTLINE bool issue_walk(const EngineView &E, IssueRanges &ir, WalkState &w)
{
    const uint32_t i = atomicAdd(&ir.pos, 1u);
    if (i >= ir.total) return false;
    uint32_t r = 0, off = i;
    while (off >= ir.cnt[r]) {
        off -= ir.cnt[r];
        r++;
    }
    const uint32_t jj = ir.job[r];
    w.job = jj;
    w.walk = E.jobs[jj].walk_begin + ir.lo[r] + off;
    return true;
}


// Geometry-phase work of one slot: a new walk and its first transition if the
// slot is free, then one step of the walk (Algorithm 1 inner loop): absorption
// test, cube sizing, classification, then the analytical route in place or a
// MicroWalk job queued for this CTA through push_mw(o).  Returns the state the
// slot is left in: ST_IDLE (no walk id left), ST_FRESH (the walk ended), ST_FIRST
// or ST_HOP (waiting for a table, or its analytical hops of this round done),
// ST_MW (MicroWalk job queued).
// st_known: the slot's state as the caller read it after a CTA barrier that
// follows every write to the slot, with a cancelled job's walk already turned into
// ST_FRESH; ST_UNKNOWN: read it here (the slot may be handed over concurrently).
constexpr uint32_t ST_UNKNOWN = 7u;
template <typename T, bool MWE, class PushMW>
__device__ uint32_t geo_slot(const EngineView &E, uint32_t s, uint32_t o, const FillList &fl, IssueRanges &ir,
                             const SView<T> *staged, uint32_t st_known, PushMW push_mw)
{
    typedef Ar<T> A;
    const int N = E.N;
    const uint32_t NS = E.NS;
    uint32_t st = st_known;
    if (st_known == ST_UNKNOWN) {
        st = *(volatile uint32_t *)&E.s.state[s];
        __threadfence_block();   // pairs with the MicroWalk warps' fence before they publish ST_MWDONE
    }
    // the position data of the step, loaded together with the walk state (one
    // round trip): the last node's position, or the finished MicroWalk's cube and exit
    double pq[4] = {0.0, 0.0, 0.0, 0.0};
    uint32_t en = 0u;
    if (st == ST_HOP || st == ST_MWDONE) {
        const bool mwd = st == ST_MWDONE;
        const double *src = mwd ? E.s.cube : E.s.pos;
        pq[0] = ldcg(src + s);
        pq[1] = ldcg(src + NS + s);
        pq[2] = ldcg(src + 2 * NS + s);
        if (mwd) {
            pq[3] = ldcg(src + 3 * NS + s);
            en = ldcg(&E.s.exitnode[s]);
        }
    }
    WalkState w;
    load_walk(E, s, w);
    if (st_known == ST_UNKNOWN && st != ST_FRESH && ((volatile int *)E.job_cancel)[w.job]) st = ST_FRESH;   // drop the walk
    if (st == ST_FRESH) {
        if (!issue_walk(E, ir, w)) {
            E.s.state[s] = ST_IDLE;
            E.s.job[s] = w.job;
            return ST_IDLE;
        }
        w.hop = 0; w.steps = 0; w.cnt_sh = 0; w.cnt_mw = 0; w.branch = -1; w.omega = 0.0;
        st = ST_FIRST;
    }
    const DevJob &J = E.jobs[w.job];
    // the CTA's shared-memory copy of the geometry when the walk's structure is the staged one
    const SView<T> &S = (staged != nullptr && J.sid == E.stage_sid) ? *staged : structure_view<T>(E, J.sid);
    T pos[3];
    if (st == ST_FIRST) {
        if (!first_transition<T>(E, J, S, w, pos, fl)) {   // table not ready: retry next epoch
            E.s.state[s] = ST_FIRST;
            store_walk(E, s, w);
            return ST_FIRST;
        }
        w.hop = 1;
    } else if (st == ST_MWDONE) {
        if (MWE && (en & 0x80000000u)) {   // MicroWalk-E: absorbed by a conductor inside its expanded cube
            w.hop++;
            finish_walk(E, J, w, (int)(en & 0xffu));
            E.s.state[s] = ST_FRESH;
            E.s.job[s] = w.job;
            return ST_FRESH;
        }
        const int node[3] = {(int)(en & 255u) - 1, (int)((en >> 8) & 255u) - 1, (int)((en >> 16) & 255u) - 1};
        const T c[3] = {(T)pq[0], (T)pq[1], (T)pq[2]};
        node_point(c, (T)pq[3], N, node, pos);
        w.hop++;
    } else {   // ST_HOP
        pos[0] = (T)pq[0];
        pos[1] = (T)pq[1];
        pos[2] = (T)pq[2];
    }
  T R;
  CubeInfo q;
  uint4 hb;
  for (int hops_here = 0;; hops_here++) {
    int who;
    const T d = nearest_electrode(S, pos, who);
    if (d <= S.tau || (int)w.hop >= E.max_hops) {
        finish_walk(E, J, w, d <= S.tau ? who : -1);
        E.s.state[s] = ST_FRESH;
        E.s.job[s] = w.job;
        return ST_FRESH;
    }
    R = E.fp32 ? A::sub(d, S.margin) : d;
    classify_cube(S, pos, R, N, q);
    int guard = 0;
    while (q.kind == CUBE_OVERFLOW && guard++ < 40) {
        R = A::mul(R, T(0.5));
        classify_cube(S, pos, R, N, q);
    }
    if (q.kind == CUBE_OVERFLOW) {        // unreachable in practice: count the walk as capped
        atomicOr(&E.status[STAT_ERR], ERR_SHRINK);
        finish_walk(E, J, w, -1);
        E.s.state[s] = ST_FRESH;
        E.s.job[s] = w.job;
        return ST_FRESH;
    }
    hb = philox10((uint32_t)w.walk, (uint32_t)(w.walk >> 32), w.hop, 0u, J.key0, J.key1);
    int m = -1, fr[3] = {0, 1, 2};
    bool wait = false;
    if (E.hybrid && q.kind == CUBE_HOM) {
        m = sample_guided(E.tc.thr + (size_t)E.tc.cap * E.tc.P, E.tc.guide + (size_t)E.tc.cap * GUIDE, (int)E.tc.P, hb.x);
        w.cnt_sh += 1u << 16;
    } else if (E.hybrid && q.kind == CUBE_STRAT) {
        const int e = table_lookup(E.tc, TAB_SGF, q.prof, fl);
        if (e < 0) {
            if (e == -2) atomicOr(&E.status[STAT_ERR], ERR_CACHE_FULL);
            wait = true;                   // retry this hop next epoch (same draws)
        } else {
            m = sample_guided(E.tc.thr + (size_t)e * E.tc.P, E.tc.guide + (size_t)e * GUIDE, (int)E.tc.P, hb.x);
            frame_sgf(q.axis, fr);
            w.cnt_sh += 1u;
        }
    }
    if (m >= 0) {
        int node[3];
        panel_node(N, fr, m, node);
        node_point(pos, R, N, node, pos);
        w.hop++;
        if (hops_here + 1 < E.hops_per_epoch) continue;   // next hop of the same walk in this epoch
    }
    if (wait || m >= 0) {
        stcg(&E.s.pos[s], (double)pos[0]);
        stcg(&E.s.pos[NS + s], (double)pos[1]);
        stcg(&E.s.pos[2 * NS + s], (double)pos[2]);
        E.s.state[s] = ST_HOP;
        store_walk(E, s, w);
        return ST_HOP;
    }
    break;
  }
    // MicroWalk-E: expand the cube f-fold (f = mwe .. 2, the first that lists at
    // most KMAX objects) so that it may reach conductors
    if (MWE && S.n_cond <= 254) {
        CubeInfo qe;
        for (int f = E.mwe; f >= 2; f--) {
            const T Re = A::mul(R, T(f));
            if (classify_cube_e<T>(S, pos, Re, N, qe)) {
                q = qe;
                R = Re;
                break;
            }
        }
    }
    // MicroWalk job (Algorithm 3) for this cube, recorded with the slot
    MWJob *jb = E.mwq + s;
    const uint32_t s3 = hb.x >> 29;
    const uint32_t c0 = (uint32_t)(N / 2 - 1);
    const uint32_t start = (c0 + (s3 & 1u)) | ((c0 + ((s3 >> 1) & 1u)) << 8) | ((c0 + ((s3 >> 2) & 1u)) << 16);
    // material nibble map: slot 0 boundary, 1 background, 2 + t listed block t
    uint64_t mm = (uint64_t)BOUNDARY | ((uint64_t)q.bg << 4);
    for (int t = 0; t < q.K; t++) mm |= (uint64_t)rng_mat(q.rng[t]) << (4 * (t + 2));
    uint4 *dst = reinterpret_cast<uint4 *>(jb);
    stcg(&dst[0], make_uint4(s, w.hop, (uint32_t)w.walk, (uint32_t)(w.walk >> 32)));
    stcg(&dst[1], make_uint4(start, (uint32_t)q.K, (uint32_t)mm, (uint32_t)(mm >> 32)));
    stcg(&dst[2], make_uint4(J.key0, J.key1, 0u, 0u));      // pad0 = steps already taken (resume)
    for (int t = 0; t < q.K; t++) stcg(&jb->rng[t], q.rng[t]);
    stcg(&E.s.cube[s], (double)pos[0]);
    stcg(&E.s.cube[NS + s], (double)pos[1]);
    stcg(&E.s.cube[2 * NS + s], (double)pos[2]);
    stcg(&E.s.cube[3 * NS + s], (double)R);
    w.cnt_mw++;
    E.s.state[s] = ST_MW;
    store_walk(E, s, w);
    push_mw(o);
    return ST_MW;
}

// The fixed fields of a MicroWalk job record, read through L2 in three 16-byte loads.
struct MWHead {
    uint32_t slot, hop, walk_lo, walk_hi, start, K, mm_lo, mm_hi, key0, key1, steps;
};
__device__ __forceinline__ MWHead mw_head(const MWJob &b)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(&b);
    const uint4 a = ldcg(p), c = ldcg(p + 1), d = ldcg(p + 2);
    return MWHead{a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w, d.x, d.y, d.z};
}

// ---------------------------------------------------------------------------
// MicroWalk (Algorithm 3).
//
// Lattice masks.  Per warp, shared memory holds one column of 16-bit rows per
// lane, laid out [row][lane] (the 32 lanes of a warp read one row as 64
// contiguous bytes).  Row R = a (N + 4) + c + 2 for axis a and coordinate
// c = -2 .. N + 1.  Bit 0 is set in every row, bit 1 in the rows of the interior
// coordinates 0 .. N - 1, bit 2 + q in the rows whose coordinate lies in listed
// block q's voxel range on that axis (q < KMAX).  The highest set bit of
// mask(0, x) & mask(1, y) & mask(2, z) is the slot of node (x, y, z): 0 for a
// boundary node, 1 for the background, 2 + q for block q (later blocks win).
// Rows -2 and N + 1 exist so that a walker resting on a boundary node (c = -1 or
// N) reads its neighbours' rows in bounds.
//
// Columns.  A slot's material m is a column of the jump-weight table: column
// (m + 1) mod 16, so that column 0 is the boundary (material BOUNDARY, also the
// conductor objects of MicroWalk-E).  A lane keeps its cube's slot -> column
// bytes in four registers A (slots 0-3), B (4-7), C (8-11), D (12-15) and turns a
// mask into a column with bfind and prmt (the permute's sign-replicate mode gives
// 0 for the half of the map a position does not address).
//
// Weight table W'[cv][ck]: the quantised alpha of Eq. 6 of a walker on a node of
// column cv towards a neighbour of column ck (2^24 towards the boundary); row 0,
// a walker on a boundary or conductor node, is all zeros, so that such a walker
// stays where it is.  The lattice step therefore needs no branch: blocks of
// steps run unconditionally and the end of a walk (or of a MicroWalk-E walk on a
// conductor node) is found once per block, from the steps that started on a
// node of non-zero column.

__device__ __forceinline__ int mask_axis_rows(int N) { return N + 4; }
__device__ __forceinline__ int mask_rows(int N) { return 3 * (N + 4); }

__device__ __forceinline__ uint32_t bfind_u32(uint32_t m)
{
    uint32_t p;
    asm("bfind.u32 %0, %1;" : "=r"(p) : "r"(m));
    return p;
}
__device__ __forceinline__ uint32_t prmt_b32(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// A lane's slot -> column map.  Columns decoded by the wide form (slots 0-15) come
// out as column + G, G = byte 0 of C replicated into bytes 1-3; the table address
// of the lane absorbs G (MWTab::bind), so decoding needs no mask.
struct MWMap {
    uint32_t A, B, C, D, G;
};
// from a nibble map of slot -> material (slot 0 BOUNDARY, 1 background, 2 + q block q)
__device__ __forceinline__ MWMap mw_map(uint64_t mm)
{
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const uint32_t m = (uint32_t)(mm >> (4 * (4 * i + b))) & 15u;
            v |= ((m + 1u) & 15u) << (8 * b);
        }
        w[i] = v;
    }
    MWMap M;
    M.A = w[0]; M.B = w[1]; M.C = w[2]; M.D = w[3];
    M.G = (w[2] & 255u) * 0x01010100u;
    return M;
}

template <bool WIDE>
__device__ __forceinline__ uint32_t mw_col(uint32_t m, const MWMap &M)
{
    const uint32_t pos = bfind_u32(m);   // m always has bit 0
    if (!WIDE) return prmt_b32(M.A, M.B, pos);               // slots 0-7: exact column
    return prmt_b32(M.A, M.B, pos) | prmt_b32(M.C, M.D, pos ^ 8u);   // column + G
}

// Weight table as one lane reads it: byte address of W'[0][0] for this lane and
// the byte strides of a row and of a column.  Two layouts: a copy per lane of a
// table of 8 columns ([entry][lane], conflict-free; materials 0-6), or one shared
// table of 16 columns.
struct MWTab {
    uint32_t base, row, col;
    // the base for the wide decode of a lane whose map has offset G
    __device__ __forceinline__ uint32_t wide_base(uint32_t G) const { return base - G * row - G * col; }
    __device__ __forceinline__ MWTab with_base(uint32_t b) const { return MWTab{b, row, col}; }
};
constexpr int WTAB_LANES_WORDS = 64 * 32;   // 8 x 8 entries x 32 lanes
constexpr int WTAB_FULL_WORDS = 256;

__device__ __forceinline__ uint32_t wprime(const uint32_t *__restrict__ Wg, int cv, int ck)
{
    return cv == 0 ? 0u : __ldg(&Wg[((cv - 1) & 15) * 16 + ((ck - 1) & 15)]);
}
// fill the table (all threads of the block); lanes_layout: the per-lane copies
__device__ __forceinline__ void wtab_fill(uint32_t *Wt, const uint32_t *__restrict__ Wg, bool lanes_layout, int tid,
                                          int nthreads)
{
    if (lanes_layout) {
        for (int i = tid; i < WTAB_LANES_WORDS; i += nthreads) {
            const int e = i >> 5;
            Wt[i] = wprime(Wg, e >> 3, e & 7);
        }
    } else {
        for (int i = tid; i < WTAB_FULL_WORDS; i += nthreads) Wt[i] = wprime(Wg, i >> 4, i & 15);
    }
}
__device__ __forceinline__ MWTab wtab_lane(const uint32_t *Wt, bool lanes_layout, int lane)
{
    MWTab t;
    if (lanes_layout) {
        t.base = smem_addr(Wt) + 4u * (uint32_t)lane;
        t.row = 8u * 128u;
        t.col = 128u;
    } else {
        t.base = smem_addr(Wt);
        t.row = 64u;
        t.col = 4u;
    }
    return t;
}

// Every row of the warp's 32 columns set to a boundary row (all nodes boundary
// nodes, so that a lane without a cube rests).
__device__ __forceinline__ void masks_clear(uint16_t *Mw, int N, int lane)
{
    for (int i = lane; i < mask_rows(N) * 32; i += 32) Mw[i] = 1;
}

// Build lane r's mask column (all 32 lanes cooperate).  Lane q < K supplies block
// q's voxel ranges [lo, hi) per axis through rng(lo[3], hi[3]).  Each block's bit
// is toggled at its lo and hi coordinates in the warp's scratch T (32 words), and
// a prefix XOR over the coordinates (one lane per coordinate) gives every row:
// the x and y axes in the low and high halves of one scan, z in a second.
template <class RangeFn>
__device__ __forceinline__ void build_masks(uint16_t *Mw, uint32_t *T, int r, int N, int lane, int K, RangeFn rng)
{
    const int RA = N + 4;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    if (lane < K) rng(lo, hi);
    const uint32_t bit = 4u << (lane & 15);
#pragma unroll
    for (int pass = 0; pass < 2; pass++) {
        T[lane] = 0u;
        __syncwarp();
        if (lane < K) {
            if (pass == 0) {
                atomicXor(&T[lo[0]], bit);
                if (hi[0] < 32) atomicXor(&T[hi[0]], bit);
                atomicXor(&T[lo[1]], bit << 16);
                if (hi[1] < 32) atomicXor(&T[hi[1]], bit << 16);
            } else {
                atomicXor(&T[lo[2]], bit);
                if (hi[2] < 32) atomicXor(&T[hi[2]], bit);
            }
        }
        __syncwarp();
        uint32_t v = T[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t w = __shfl_up_sync(FULL_MASK, v, d);
            if (lane >= d) v ^= w;
        }
        if (lane < N) {
            if (pass == 0) {
                Mw[(lane + 2) * 32 + r] = (uint16_t)((v & 0xffffu) | 3u);
                Mw[(RA + lane + 2) * 32 + r] = (uint16_t)((v >> 16) | 3u);
            } else {
                Mw[(2 * RA + lane + 2) * 32 + r] = (uint16_t)((v & 0xffffu) | 3u);
            }
        }
        __syncwarp();
    }
}

// Row addresses of a lane's column: the byte address of row c = -1 of each axis.
struct MWRows {
    uint32_t x, y, z;
};
__device__ __forceinline__ MWRows mw_rows(const uint16_t *Mw, int N, int lane)
{
    const uint32_t m = smem_addr(Mw + lane);
    const uint32_t RA = (uint32_t)mask_axis_rows(N);
    return MWRows{m + 64u, m + RA * 64u + 64u, m + 2u * RA * 64u + 64u};
}

// One step of the lattice walk from node (x, y, z): weights W'[cv][ck] of Eq. 6
// (quantised) towards the six neighbours (order -x, +x, -y, +y, -z, +z), integer
// prefix sums p0..p5, r = (u p5) >> 32, the first k with r < p_k taken.  With b_k
// = [r >= p_k] the move is dx = 2 b0 - 1 - b1, dy = 2 b2 - b1 - b3, dz = 2 b4 -
// b3 - b5 (b5 = 0 whenever p5 > 0; all six are 1 on a node of column 0, whose
// weights are all 0, so that the walker does not move).  Returns the column of
// the node the step started on (+ G in the wide form): equal to G for a walker
// that rests.
template <bool WIDE>
__device__ __forceinline__ uint32_t mw_step(const MWRows &R, const MWTab &T, const MWMap &M, int &x, int &y, int &z,
                                            uint32_t u)
{
    const uint32_t ax = R.x + (uint32_t)x * 64u, ay = R.y + (uint32_t)y * 64u, az = R.z + (uint32_t)z * 64u;
    const uint32_t xm = lds_u16(ax), x0 = lds_u16(ax + 64u), xp = lds_u16(ax + 128u);
    const uint32_t ym = lds_u16(ay), y0 = lds_u16(ay + 64u), yp = lds_u16(ay + 128u);
    const uint32_t zm = lds_u16(az), z0 = lds_u16(az + 64u), zp = lds_u16(az + 128u);
    const uint32_t yz = y0 & z0, xz = x0 & z0, xy = x0 & y0;
    const uint32_t ev = mw_col<WIDE>(xy & z0, M);
    const uint32_t wr = T.base + ev * T.row;
    const uint32_t w0 = lds_u32(wr + mw_col<WIDE>(xm & yz, M) * T.col);
    const uint32_t w1 = lds_u32(wr + mw_col<WIDE>(xp & yz, M) * T.col);
    const uint32_t w2 = lds_u32(wr + mw_col<WIDE>(ym & xz, M) * T.col);
    const uint32_t w3 = lds_u32(wr + mw_col<WIDE>(yp & xz, M) * T.col);
    const uint32_t w4 = lds_u32(wr + mw_col<WIDE>(zm & xy, M) * T.col);
    const uint32_t w5 = lds_u32(wr + mw_col<WIDE>(zp & xy, M) * T.col);
    const uint32_t p0 = w0, p1 = p0 + w1, p2 = p1 + w2, p3 = p2 + w3, p4 = p3 + w4, p5 = p4 + w5;
    const uint32_t r = __umulhi(u, p5);
    const int b0 = r >= p0, b1 = r >= p1, b2 = r >= p2, b3 = r >= p3, b4 = r >= p4, b5 = r >= p5;
    x += 2 * b0 - 1 - b1;
    y += 2 * b2 - b1 - b3;
    z += 2 * b4 - b3 - b5;
    return ev;
}

// slot of node (x, y, z) (MicroWalk-E: which object a walker rests on)
__device__ __forceinline__ int mw_slot_at(const MWRows &R, int x, int y, int z)
{
    const uint32_t m = lds_u16(R.x + (uint32_t)x * 64u + 64u) & lds_u16(R.y + (uint32_t)y * 64u + 64u) &
                       lds_u16(R.z + (uint32_t)z * 64u + 64u);
    return (int)bfind_u32(m);
}

// Four steps with the words of one Philox block; returns the steps that started
// on a node of non-zero column (the walk's own steps).  T: the lane's table with
// the base for this decode form (MWLane::base_n or base_w).
template <bool WIDE>
__device__ __forceinline__ uint32_t mw_block4(const MWRows &R, const MWTab &T, const MWMap &M, int &x, int &y, int &z,
                                              uint4 w)
{
    const uint32_t rest = WIDE ? M.G : 0u;
    uint32_t moved = 0;
    moved += mw_step<WIDE>(R, T, M, x, y, z, w.x) != rest;
    moved += mw_step<WIDE>(R, T, M, x, y, z, w.y) != rest;
    moved += mw_step<WIDE>(R, T, M, x, y, z, w.z) != rest;
    moved += mw_step<WIDE>(R, T, M, x, y, z, w.w) != rest;
    return moved;
}

// The same four steps in a loop that is not unrolled (one copy of the step: less
// code next to a large kernel's other phases in the instruction cache).
template <bool WIDE>
__device__ __forceinline__ uint32_t mw_block4_compact(const MWRows &R, const MWTab &T, const MWMap &M, int &x, int &y,
                                                      int &z, uint4 w)
{
    const uint32_t rest = WIDE ? M.G : 0u;
    uint32_t moved = 0;
#pragma unroll 1
    for (int k = 0; k < 4; k++) {
        moved += mw_step<WIDE>(R, T, M, x, y, z, w.x) != rest;
        w = make_uint4(w.y, w.z, w.w, w.x);
    }
    return moved;
}

// A lane's walk: identity, cube (block count, column map) and the table bases for
// the narrow and the wide decode.  A warp runs the wide decode while any of its
// walking lanes holds more than 6 blocks; every lane, walking or resting, then
// reads its table through the base of the form in use.
struct MWLane {
    uint32_t walk_lo, walk_hi, hop, key0, key1, tag;
    int K;
    MWMap map;
    uint32_t base_n, base_w;
};
__device__ __forceinline__ void mw_lane_cube(MWLane &L, const MWTab &T0, int K, uint64_t mm)
{
    L.K = K;
    L.map = mw_map(mm);
    L.base_n = T0.base;
    L.base_w = T0.wide_base(L.map.G);
}
__device__ __forceinline__ void mw_lane_reset(MWLane &L, const MWTab &T0)
{
    L.walk_lo = L.walk_hi = L.hop = L.key0 = L.key1 = L.tag = 0;
    L.K = 0;
    L.map = MWMap{0u, 0u, 0u, 0u, 0u};
    L.base_n = L.base_w = T0.base;
}

// Job source: stand-alone cubes given as integer voxel ranges (64 int32 per cube).
struct CubeSource {
    const int32_t *cubes;
    uint64_t n_cubes, spc, total;
    unsigned long long *head;
    uint32_t key0, key1;
    uint64_t mmap_lo;        // local material id -> global id nibbles (ids 0..15)
    uint32_t *d_exit, *d_steps;
    uint32_t *err;
    int N;
    int n_mat;               // material ids of the records index 0 .. n_mat - 1
    int lanes_table;         // 1: per-lane weight-table copies (global materials 0-6)
    uint32_t chunk;          // job ids a warp claims at a time (32 .. MW_CHUNK)
    __device__ uint64_t grab(uint32_t n) const { return atomicAdd(head, (unsigned long long)n); }
    __device__ void overrun() const { atomicOr(err, ERR_MW_STEPS); }
    __device__ bool valid(uint64_t j) const { return j < total; }
    __device__ int gmat(int local) const { return (int)((mmap_lo >> (4 * (local & 15))) & 15ull); }
    __device__ uint64_t cube_of(uint64_t j) const { return j / spc; }
    // (all lanes) check cube `cube`'s record and build lane r's masks from it.  A
    // record is usable when 0 <= K <= 8 (what 64 words hold), every material id is
    // below n_mat and every block range satisfies 0 <= lo < hi <= N; lane q checks
    // block q.  Returns the verdict (the same on every lane); a malformed record
    // builds a cube without blocks.
    __device__ bool build(uint64_t cube, uint16_t *Mw, uint32_t *T, int r, int N_, int lane) const
    {
        const int32_t *c = cubes + cube * 64;
        const int K0 = c[1];
        bool ok = K0 >= 0 && K0 <= 8 && c[0] >= 0 && c[0] < n_mat;
        const int Kc = ok ? K0 : 0;
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        bool mine = true;
        if (lane < Kc) {
            const int m = c[8 + 7 * lane];
            mine = m >= 0 && m < n_mat;
            for (int a = 0; a < 3; a++) {
                lo[a] = c[2 + 7 * lane + 2 * a];
                hi[a] = c[3 + 7 * lane + 2 * a];
                mine = mine && 0 <= lo[a] && lo[a] < hi[a] && hi[a] <= N;
            }
        }
        ok = __all_sync(FULL_MASK, mine) && ok;
        build_masks(Mw, T, r, N_, lane, ok ? Kc : 0, [&](int l[3], int h[3]) {
            for (int a = 0; a < 3; a++) {
                l[a] = lo[a];
                h[a] = hi[a];
            }
        });
        return ok;
    }
    // Start sample j on the lane's cube (fresh: its column map is computed, else
    // kept from the previous sample of the same cube).  False (and the error flag
    // set) for a malformed record: the sample is then written as exit 0, 0 steps
    // and not walked.
    __device__ bool load(uint64_t j, MWLane &L, const MWTab &T0, bool ok, bool fresh, int &x, int &y, int &z) const
    {
        if (!ok) {
            atomicOr(err, ERR_INPUT);
            if (d_exit) d_exit[j] = 0u;
            if (d_steps) d_steps[j] = 0u;
            return false;
        }
        if (fresh) {
            const int32_t *c = cubes + (j / spc) * 64;
            const int K = c[1];
            uint64_t mm = (uint64_t)BOUNDARY | ((uint64_t)gmat(c[0]) << 4);
            for (int t = 0; t < K; t++) mm |= (uint64_t)gmat(c[2 + 7 * t + 6]) << (4 * (t + 2));
            mw_lane_cube(L, T0, K, mm);
        }
        L.walk_lo = (uint32_t)j;
        L.walk_hi = (uint32_t)(j >> 32);
        L.hop = 0;
        L.key0 = key0;
        L.key1 = key1;
        L.tag = 0;
        const uint4 b = philox10(L.walk_lo, L.walk_hi, 0u, 0u, key0, key1);
        const uint32_t s3 = b.x >> 29;
        const int c0 = N / 2 - 1;
        x = c0 + (int)(s3 & 1u);
        y = c0 + (int)((s3 >> 1) & 1u);
        z = c0 + (int)((s3 >> 2) & 1u);
        return true;
    }
    __device__ void finish(const MWLane &L, int x, int y, int z, uint32_t steps) const
    {
        const uint64_t j = (uint64_t)L.walk_lo | ((uint64_t)L.walk_hi << 32);
        if (d_exit) d_exit[j] = (uint32_t)(x + 1) | ((uint32_t)(y + 1) << 8) | ((uint32_t)(z + 1) << 16);
        if (d_steps) d_steps[j] = steps;
    }
};

constexpr uint32_t MW_STEP_CAP = 1u << 26;
// job ids a warp of the stand-alone MicroWalk kernel claims at a time: at most
// this many, fewer (down to 32) when the launch has too few jobs to give every
// warp several chunks
constexpr uint32_t MW_CHUNK = 512;

// Stand-alone MicroWalk over a job source.  Per lane: one walk at a time, in
// blocks of 8 steps (two Philox blocks); a lane whose walk ended rests on a
// boundary node until it is refilled at the next block boundary.  A lane that
// takes its next sample on the cube it already holds keeps its masks.  Warps use
// the narrow column decode while every cube they hold has at most 6 blocks.
template <class Src>
__global__ void __launch_bounds__(512) k_mw(Src src, const uint32_t *__restrict__ Wg, int N)
{
    extern __shared__ uint32_t smem[];
    const bool lanes_table = src.lanes_table != 0;
    uint32_t *Wt = smem;
    const int wt_words = lanes_table ? WTAB_LANES_WORDS : WTAB_FULL_WORDS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *Tw = smem + wt_words + warp * 32;
    uint16_t *Mw = reinterpret_cast<uint16_t *>(smem + wt_words + nwarps * 32) + (size_t)warp * mask_rows(N) * 32;
    wtab_fill(Wt, Wg, lanes_table, threadIdx.x, blockDim.x);
    masks_clear(Mw, N, lane);
    __syncthreads();
    const MWRows R = mw_rows(Mw, N, lane);
    const MWTab T0 = wtab_lane(Wt, lanes_table, lane);
    bool active = false, exhausted = false;
    int x = -1, y = 0, z = 0;
    uint32_t t = 0;
    uint64_t held = ~0ull;   // cube whose masks (and column map) this lane holds
    bool held_ok = false;    // ... and whether its record is well formed
    // the warp's chunk of consecutive job ids [c_next, c_end) (warp-uniform): the
    // lanes' successive jobs stay on one cube, so a lane rarely rebuilds its masks
    uint64_t c_next = 0, c_end = 0;
    MWLane L;
    mw_lane_reset(L, T0);
    for (;;) {
        const bool need = !active && !exhausted;
        const uint32_t bal = __ballot_sync(FULL_MASK, need);
        if (bal) {
            const int leader = __ffs(bal) - 1;
            const uint32_t n = (uint32_t)__popc(bal), rk = (uint32_t)__popc(bal & ((1u << lane) - 1u));
            uint64_t myj;
            if (c_end - c_next >= n) {
                myj = c_next + rk;
                c_next += n;
            } else {
                const uint64_t avail = c_end - c_next;
                unsigned long long nb = 0;
                if (lane == leader) nb = src.grab(src.chunk);   // chunk >= 32 >= n: the ids fit
                nb = __shfl_sync(FULL_MASK, nb, leader);
                myj = rk < avail ? c_next + rk : nb + (rk - avail);
                c_next = nb + (n - avail);
                c_end = nb + src.chunk;
            }
            const bool got = need && src.valid(myj);
            if (need && !got) exhausted = true;
            const uint64_t cube = got ? src.cube_of(myj) : held;
            const bool fresh = got && cube != held;
            uint32_t todo = __ballot_sync(FULL_MASK, fresh);
            while (todo) {
                const int r = __ffs(todo) - 1;
                todo &= todo - 1u;
                const uint64_t cr = __shfl_sync(FULL_MASK, cube, r);
                const bool ok = src.build(cr, Mw, Tw, r, N, lane);
                if (lane == r) held_ok = ok;
            }
            __syncwarp();
            if (got) {
                held = cube;
                t = 0;
                active = src.load(myj, L, T0, held_ok, fresh, x, y, z);
                if (!active) { x = -1; y = 0; z = 0; }
            }
        }
        if (__ballot_sync(FULL_MASK, active) == 0u) break;
        const bool wide = __any_sync(FULL_MASK, active && L.K > 6);
        uint32_t moved;
        const uint4 b0 = philox10(L.walk_lo, L.walk_hi, L.hop, 1u + (t >> 2), L.key0, L.key1);
        const uint4 b1 = philox10(L.walk_lo, L.walk_hi, L.hop, 2u + (t >> 2), L.key0, L.key1);
        if (wide) {
            const MWTab T = T0.with_base(L.base_w);
            moved = mw_block4<true>(R, T, L.map, x, y, z, b0);
            moved += mw_block4<true>(R, T, L.map, x, y, z, b1);
        } else {
            const MWTab T = T0.with_base(L.base_n);
            moved = mw_block4<false>(R, T, L.map, x, y, z, b0);
            moved += mw_block4<false>(R, T, L.map, x, y, z, b1);
        }
        const bool inside = ((unsigned)x < (unsigned)N) & ((unsigned)y < (unsigned)N) & ((unsigned)z < (unsigned)N);
        if (active && (moved < 8u || !inside)) {   // on a boundary node: the walk has ended
            src.finish(L, x, y, z, t + moved);
            active = false;
            x = -1; y = 0; z = 0;
        }
        t += 8;
        if (active && t >= MW_STEP_CAP) {   // safety net: never loop without bound
            src.overrun();
            src.finish(L, x, y, z, t);
            active = false;
            x = -1; y = 0; z = 0;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Analytical table fill (one CTA per table).
//
// A layered lattice (permittivity eps_k along table axis t2) separates: in the
// two lateral axes the FD operator of Eq. 4-5 is (eps_k / 2) T with T the
// cell-centred Dirichlet Laplacian (diagonal 3 at both ends), whose eigenvectors
// are the DST-II vectors u_p(i) = sqrt(2/N) sin(pi p (i + 1/2) / N) (p < N),
// u_N(i) = (-1)^i / sqrt(N), eigenvalues lam_p = 4 sin^2(pi p / (2N)).  In that
// basis the symmetric system S y = b (S = diag(eps) times Eq. 6) becomes one
// tridiagonal system per lateral mode (p, q) along t2, solved by the Thomas
// algorithm; the panel values eps_v y_v (Eq. 8: P = e_c^T A_II^{-1} A_IB) are
// assembled face by face with two small contractions each.  Only the modes that
// the right-hand side excites are kept: odd p and q for the SGF and the
// layer-normal flux kernel, even p with odd q for the flux kernel across layers.
// A group of whole warps that cooperates on a table fill or a batch reduction:
// thread index within the group, group size, and the barrier that synchronises
// it (0: the whole CTA, __syncthreads; else a named barrier of `nt` threads).
struct Grp {
    int tid, nt, bar;
    __device__ __forceinline__ void sync() const
    {
        if (bar == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
    }
};
__device__ __forceinline__ Grp cta_grp() { return Grp{(int)threadIdx.x, (int)blockDim.x, 0}; }

struct FillJob {
    uint32_t kind;
    uint32_t prof[4];
    uint16_t *guide;
    uint32_t *thr;
    uint32_t *sgn;
    double *ktot;
    double *values;        // optional raw panel values (canonical order)
    double *V;             // scratch for the 6N^2 panel values (global memory)
    uint32_t *err;
};

constexpr int FILL_CHUNKS = 256;   // chunks of the table fill's final sums (any block size)

__device__ FRW_OUTLINE void fill_table(const FillJob &F, int N, const double *__restrict__ eps, const FillConsts &C,
                           double *sm, const Grp &G)
{
    const int H = N / 2, M = H * H, P = 6 * N * N;
    const int tid = G.tid, nt = G.nt;
    double *ek = sm;                 // N
    double *yh = ek + MAXN;          // M * N
    double *Z = yh + M * N;          // N * N
    double *red = Z + MAXN * MAXN;   // FILL_CHUNKS + 1
    double *V = F.V;                 // P, global scratch
    const uint32_t kind = F.kind;
    const bool hom = (kind == TAB_SGF_HOM || kind == TAB_FLUX_HOM);
    const bool perp = (kind == TAB_FLUX_PERP);
    const bool flux = (kind == TAB_FLUX_PAR || kind == TAB_FLUX_PERP || kind == TAB_FLUX_HOM);
    for (int k = tid; k < N; k += nt) ek[k] = hom ? 1.0 : eps[nib(F.prof[k >> 3], k & 7)];
    G.sync();
    const int c0 = H - 1, c1 = H;
    // tridiagonal solve per mode
    for (int m = tid; m < M; m += nt) {
        const int ip = m / H, iq = m - ip * H;
        const int p = perp ? 2 * (ip + 1) : 2 * ip + 1;   // 1-based mode numbers
        const int q = 2 * iq + 1;
        const double lam = C.lam[p - 1] + C.lam[q - 1];
        double cp[MAXN], dp[MAXN];
        double prev_off = 0.0;
        for (int k = 0; k < N; k++) {
            const double e = ek[k];
            const double glo = (k == 0) ? e : e * ek[k - 1] / (e + ek[k - 1]);
            const double ghi = (k == N - 1) ? e : e * ek[k + 1] / (e + ek[k + 1]);
            const double diag = 0.5 * e * lam + glo + ghi;
            const double off = (k == N - 1) ? 0.0 : -ghi;
            double rhs = 0.0;
            if (kind == TAB_SGF || kind == TAB_SGF_HOM) {
                if (k == c0 || k == c1) rhs = 0.5 * C.a[p - 1] * C.a[q - 1];
            } else if (perp) {
                if (k == c0 || k == c1) rhs = 0.5 * e * C.d[p - 1] * C.a[q - 1];
            } else {
                const double wgt = 2.0 * ek[c0] * ek[c1] / (ek[c0] + ek[c1]);
                if (k == c1) rhs = wgt * C.a[p - 1] * C.a[q - 1];
                if (k == c0) rhs = -wgt * C.a[p - 1] * C.a[q - 1];
            }
            if (k == 0) {
                cp[0] = off / diag;
                dp[0] = rhs / diag;
            } else {
                const double den = diag - prev_off * cp[k - 1];
                cp[k] = off / den;
                dp[k] = (rhs - prev_off * dp[k - 1]) / den;
            }
            prev_off = off;
        }
        double yk = dp[N - 1];
        yh[m * N + N - 1] = yk;
        for (int k = N - 2; k >= 0; k--) {
            yk = dp[k] - cp[k] * yk;
            yh[m * N + k] = yk;
        }
    }
    G.sync();
    const double *U = C.u;   // U[(p-1)*N + i]
    // faces: f = 2*ta + side; panel (u, w) on the other two table axes in increasing order
    for (int f = 0; f < 6; f++) {
        const int ta = f >> 1, side = f & 1;
        const int fix = side ? N - 1 : 0;
        // stage 1: contract one lateral index
        if (ta == 2) {
            // Z[ip][j] = sum_iq u_q(j) yh[ip,iq][fix]
            for (int o = tid; o < H * N; o += nt) {
                const int ip = o / N, j = o - ip * N;
                double acc = 0.0;
                for (int iq = 0; iq < H; iq++) acc += U[(2 * iq) * N + j] * yh[(ip * H + iq) * N + fix];
                Z[o] = acc;
            }
        } else if (ta == 0) {
            // Z[iq][k] = sum_ip u_p(fix) yh[ip,iq][k]
            for (int o = tid; o < H * N; o += nt) {
                const int iq = o / N, k = o - iq * N;
                double acc = 0.0;
                for (int ip = 0; ip < H; ip++) {
                    const int p = perp ? 2 * (ip + 1) : 2 * ip + 1;
                    acc += U[(p - 1) * N + fix] * yh[(ip * H + iq) * N + k];
                }
                Z[o] = acc;
            }
        } else {
            // Z[ip][k] = sum_iq u_q(fix) yh[ip,iq][k]
            for (int o = tid; o < H * N; o += nt) {
                const int ip = o / N, k = o - ip * N;
                double acc = 0.0;
                for (int iq = 0; iq < H; iq++) acc += U[(2 * iq) * N + fix] * yh[(ip * H + iq) * N + k];
                Z[o] = acc;
            }
        }
        G.sync();
        // stage 2
        for (int o = tid; o < N * N; o += nt) {
            const int u = o / N, w = o - u * N;
            double acc = 0.0, e;
            if (ta == 2) {           // (u, w) = (i, j); layer fix
                for (int ip = 0; ip < H; ip++) {
                    const int p = perp ? 2 * (ip + 1) : 2 * ip + 1;
                    acc += U[(p - 1) * N + u] * Z[ip * N + w];
                }
                e = ek[fix];
            } else if (ta == 0) {    // (u, w) = (j, k)
                for (int iq = 0; iq < H; iq++) acc += U[(2 * iq) * N + u] * Z[iq * N + w];
                e = ek[w];
            } else {                 // (u, w) = (i, k)
                for (int ip = 0; ip < H; ip++) {
                    const int p = perp ? 2 * (ip + 1) : 2 * ip + 1;
                    acc += U[(p - 1) * N + u] * Z[ip * N + w];
                }
                e = ek[w];
            }
            V[f * N * N + o] = e * acc;
        }
        G.sync();
    }
    // totals and thresholds in canonical order: a sequential scan over FILL_CHUNKS
    // fixed chunks, so that the sums round the same way whatever the block size
    // (a table filled by the walk kernel equals the fill kernel's bit for bit)
    const int chunk = (P + FILL_CHUNKS - 1) / FILL_CHUNKS;
    for (int c = tid; c < FILL_CHUNKS; c += nt) {
        const int b0 = min(P, c * chunk), b1 = min(P, b0 + chunk);
        double part = 0.0;
        for (int n = b0; n < b1; n++) part += flux ? fabs(V[n]) : V[n];
        red[c] = part;
    }
    G.sync();
    if (tid == 0) {
        double run = 0.0;
        for (int i = 0; i < FILL_CHUNKS; i++) {
            const double v = red[i];
            red[i] = run;
            run += v;
        }
        red[FILL_CHUNKS] = run;
    }
    G.sync();
    const double total = red[FILL_CHUNKS];
    for (int c = tid; c < FILL_CHUNKS; c += nt) {
        const int b0 = min(P, c * chunk), b1 = min(P, b0 + chunk);
        double cum = red[c];
        for (int n = b0; n < b1; n++) {
            cum += flux ? fabs(V[n]) : V[n];
            double tv = floor((cum / total) * 4294967296.0);
            if (tv > 4294967295.0) tv = 4294967295.0;
            if (tv < 0.0) tv = 0.0;
            F.thr[n] = (uint32_t)tv;
            if (F.values) F.values[n] = V[n];
        }
    }
    const int P32 = (P + 31) / 32;
    for (int wd = tid; wd < P32; wd += nt) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; b++) {
            const int n = wd * 32 + b;
            if (n < P && flux && V[n] < 0.0) bits |= 1u << b;
        }
        F.sgn[wd] = bits;
    }
    if (tid == 0) {
        *F.ktot = total;
        if (!flux && fabs(total - 1.0) > 1e-9) atomicOr(F.err, ERR_FILL);
        if (!(total > 0.0)) atomicOr(F.err, ERR_FILL);
    }
    G.sync();
    // guide table: first panel with threshold > bucket start (binary search)
    for (int k = tid; k < GUIDE; k += nt) {
        const uint32_t start = (uint32_t)k << 21;
        int lo = 0, hi = P - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (F.thr[mid] > start) hi = mid;
            else lo = mid + 1;
        }
        F.guide[k] = (uint16_t)lo;
    }
    G.sync();
}

__global__ void k_fill_one(EngineView E, uint32_t kind, uint4 prof, uint32_t entry, double *values)
{
    extern __shared__ double fsm[];
    FillJob F;
    F.kind = kind;
    F.prof[0] = prof.x; F.prof[1] = prof.y; F.prof[2] = prof.z; F.prof[3] = prof.w;
    F.thr = E.tc.thr + (size_t)entry * E.tc.P;
    F.sgn = E.tc.sgn + (size_t)entry * E.tc.P32;
    F.guide = E.tc.guide + (size_t)entry * GUIDE;
    F.ktot = E.tc.ktot + entry;
    F.values = values;
    F.err = &E.status[STAT_ERR];
    F.V = E.fill_scratch;
    fill_table(F, E.N, E.eps, E.fc, fsm, cta_grp());
}

// ---------------------------------------------------------------------------
// Batch reduction: one CTA per batch folds the batch's walk records into its
// accumulator block (S1, S2 per electrode as exact 128-bit fixed point, counters).
// Integer sums are order-independent, so the result does not depend on which walk
// finished first.  done = number of finished walks of the batch.
__device__ __forceinline__ void smem_add128(unsigned long long *p, unsigned long long lo, unsigned long long hi)
{
    const unsigned long long old = atomicAdd(&p[0], lo);
    atomicAdd(&p[1], hi + ((old + lo < old) ? 1ull : 0ull));
}

__device__ __forceinline__ void to_fixed128(double v, double scale, unsigned long long &lo, unsigned long long &hi)
{
    const double s = rint(v * scale);
    const double a = fabs(s);
    const double ah = floor(a * 5.421010862427522e-20);   // * 2^-64
    const double al = a - ah * 18446744073709551616.0;
    lo = (unsigned long long)al;
    hi = (unsigned long long)ah;
    if (s < 0) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
}

// CTA-cooperative reduction of one complete batch g into its accumulator block;
// sets batch_ready[g] (release) once the block is written.
__device__ FRW_OUTLINE void reduce_batch(const EngineView &E, uint32_t g, unsigned long long *acc_sm, const Grp &G)
{
    const DevJob &J = E.jobs[__ldcg(E.batch_job + g)];
    const int nc1 = J.n_c + 1;
    const uint32_t words = J.acc_stride;
    for (uint32_t i = G.tid; i < words; i += G.nt) acc_sm[i] = 0ull;
    G.sync();
    const uint64_t b = g - J.batch_base;
    const uint64_t w0 = b * J.batch;
    const uint64_t w1 = min(w0 + J.batch, J.walk_count);
    unsigned long long *ex = acc_sm + 4 * nc1;
    unsigned long long loc[ACC_EXTRA];
    for (int x = 0; x < ACC_EXTRA; x++) loc[x] = 0ull;
    for (uint64_t w = w0 + G.tid; w < w1; w += G.nt) {
        const uint64_t r = J.rec_base + w;
        const int k = cuda::atomic_ref<int32_t, cuda::thread_scope_device>(E.rec.k[r]).load(cuda::memory_order_acquire);
        if (k == REC_PENDING) continue;
        loc[0]++;
        loc[1] += E.rec.hops[r];
        loc[2] += E.rec.steps[r];
        const uint32_t sh = E.rec.cnt_sh[r];
        loc[3] += sh & 0xffffu;
        loc[4] += sh >> 16;
        loc[5] += E.rec.cnt_mw[r];
        const int br = E.rec.branch[r];
        if (br >= 0 && br < 3) loc[6 + br]++;
        if (k < 0) {
            loc[9]++;
            continue;
        }
        const double om = E.rec.omega[r];
        unsigned long long lo, hi;
        to_fixed128(om, ACC_S1_SCALE, lo, hi);
        smem_add128(acc_sm + 2 * k, lo, hi);
        to_fixed128(om * om, ACC_S2_SCALE, lo, hi);
        smem_add128(acc_sm + 2 * nc1 + 2 * k, lo, hi);
    }
    for (int x = 0; x < ACC_EXTRA; x++) {
        unsigned long long v = loc[x];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL_MASK, v, o);
        if ((G.tid & 31) == 0 && v) atomicAdd(&ex[x], v);
    }
    G.sync();
    unsigned long long *out = E.acc + J.acc_base + b * words;
    const bool in_range = FRW_CHECKED(E, J.acc_base + (b + 1) * words <= E.acc_cap);
    for (uint32_t i = G.tid; i < words && in_range; i += G.nt) out[i] = acc_sm[i];
    G.sync();
    if (G.tid == 0) {
        __threadfence();
        cuda::atomic_ref<uint32_t, cuda::thread_scope_device>(E.batch_ready[g]).store(1u, cuda::memory_order_release);
    }
    G.sync();
}

// ---------------------------------------------------------------------------
// Stop rule on the device (Sec. IV: standard error below the target on C_ii and on
// the largest |C_ij|, j != i, ground excluded, re-chosen at every check), evaluated
// at every full batch of the completed prefix of walk ids, so the decision does
// not depend on the order in which walks finish.
__device__ __forceinline__ double i128_to_double(unsigned long long lo, unsigned long long hi)
{
    const bool neg = (long long)hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const double v = (double)hi * 18446744073709551616.0 + (double)lo;
    return neg ? -v : v;
}

__device__ __forceinline__ void add128(unsigned long long *d, const unsigned long long *a)
{
    const unsigned long long lo = d[0] + a[0];
    d[1] = d[1] + a[1] + (lo < d[0] ? 1ull : 0ull);
    d[0] = lo;
}

__device__ void rel_errors_dev(const unsigned long long *sum, int nc, int master, double n, double *rs, double *rc)
{
    const int nc1 = nc + 1;
    auto val = [&](int k, double *c, double *se) {
        const double s1 = i128_to_double(sum[2 * k], sum[2 * k + 1]) / ACC_S1_SCALE;
        const double s2 = i128_to_double(sum[2 * nc1 + 2 * k], sum[2 * nc1 + 2 * k + 1]) / ACC_S2_SCALE;
        *c = s1 / n;
        const double v = (s2 - s1 * s1 / n) / (n * (n - 1.0));
        *se = sqrt(v > 0 ? v : 0.0);
    };
    double ci, si;
    val(master, &ci, &si);
    *rs = (ci != 0.0) ? si / fabs(ci) : __longlong_as_double(0x7ff0000000000000ll);
    *rc = 0.0;
    int jb = -1;
    double cb = 0.0;
    for (int j = 0; j < nc; j++) {
        if (j == master) continue;
        double c, sj;
        val(j, &c, &sj);
        if (jb < 0 || fabs(c) > cb) {
            jb = j;
            cb = fabs(c);
        }
    }
    if (jb >= 0) {
        double c, sj;
        val(jb, &c, &sj);
        *rc = (c != 0.0) ? sj / fabs(c) : __longlong_as_double(0x7ff0000000000000ll);
    }
}

// Fold the completed prefix of job j's batches, in walk-id order, into its running
// sums; decide the job when its stop rule holds (sigma jobs, checked at every full
// batch) or its budget is used up; steer a sigma job's issue limit to the
// predicted need (n (r / target)^2 + 5 % + 2 batches) so that the pool does not run
// far past the stopping point.  Caller holds the job's lock.
__device__ void advance_locked(const EngineView &E, uint32_t j, JobState &S)
{
    const DevJob &J = E.jobs[j];
    unsigned long long *sum = E.jsum + __ldcg(E.jsum_off + j);
    if (!FRW_CHECKED(E, __ldcg(E.jsum_off + j) + J.acc_stride <= E.jsum_cap)) return;
    const int nc1 = J.n_c + 1;
    const uint64_t nb = (J.walk_count + J.batch - 1) / J.batch;
    unsigned long long prefix = *(volatile unsigned long long *)&S.prefix;
    bool changed = false, capped = true;
    uint32_t decided = 0;
    for (int it = 0; it < 4096; it++) {
        if (prefix >= nb) {
            capped = false;
            break;
        }
        const uint64_t g = J.batch_base + prefix;
        if (!cuda::atomic_ref<uint32_t, cuda::thread_scope_device>(E.batch_ready[g]).load(cuda::memory_order_acquire)) {
            capped = false;
            break;
        }
        const unsigned long long *blk = E.acc + J.acc_base + prefix * J.acc_stride;
        for (int w = 0; w < 4 * nc1; w += 2) add128(sum + w, blk + w);
        for (int x = 0; x < ACC_EXTRA; x++) sum[4 * nc1 + x] += blk[4 * nc1 + x];
        const uint64_t bsz = min((uint64_t)J.batch, (uint64_t)(J.walk_count - prefix * J.batch));
        prefix++;
        changed = true;
        const double n = (double)min((uint64_t)(prefix * J.batch), (uint64_t)J.walk_count);
        if (J.sigma > 0.0 && bsz == J.batch && n >= 2.0) {
            double rs, rc;
            rel_errors_dev(sum, J.n_c, J.master, n, &rs, &rc);
            if (rs <= J.sigma && rc <= J.sigma) {
                decided = 1;
                S.used = (unsigned long long)n;
                atomicExch(&E.job_cancel[j], 1);
                capped = false;
                break;
            }
        }
    }
    if (!decided && prefix >= nb) {
        decided = 2;
        S.used = J.walk_count;
    }
    S.prefix = prefix;
    if (capped) atomicExch(&S.pending, 1u);   // bounded work per round: the caller takes another
    if (J.sigma > 0.0 && !decided && changed) {
        const double n = (double)min((uint64_t)(prefix * J.batch), (uint64_t)J.walk_count);
        unsigned long long lim = J.walk_count;
        if (n >= (double)J.batch) {
            double rs, rc;
            rel_errors_dev(sum, J.n_c, J.master, n, &rs, &rc);
            const double r = fmax(rs, rc) / J.sigma;
            double need = isfinite(r) ? n * r * r : (double)J.walk_count;
            need = fmin(need * 1.05 + 2.0 * (double)J.batch, (double)J.walk_count);
            lim = ((unsigned long long)need + J.batch - 1) / J.batch * J.batch;
        }
        lim = max(lim, (unsigned long long)((prefix + 1) * J.batch));
        lim = min(lim, (unsigned long long)J.walk_count);
        atomicExch(&E.job_limit[j], lim);
    }
    if (decided) {
        __threadfence();
        if (atomicCAS(&S.decided, 0u, decided) == 0u) atomicAdd(&E.jctl[JC_DECIDED], 1u);
    }
}

// One thread, after reducing a batch of job j: run advance_locked under the job's
// try-lock.  A thread that finds the lock held leaves a pending mark, which the
// holder sees after unlocking and takes the lock again for; every round either
// returns or was asked for by another thread, so the loop ends.
__device__ FRW_OUTLINE void advance_job(const EngineView &E, uint32_t j)
{
    JobState &S = E.jstate[j];
    atomicExch(&S.pending, 1u);
    __threadfence();
    for (int round = 0; round < (1 << 20); round++) {
        if (*(volatile uint32_t *)&S.decided) return;
        if (atomicCAS(&S.lock, 0u, 1u) != 0u) return;
        __threadfence();
        atomicExch(&S.pending, 0u);
        __threadfence();
        if (!*(volatile uint32_t *)&S.decided) advance_locked(E, j, S);
        __threadfence();
        atomicExch(&S.lock, 0u);
        __threadfence();
        if (*(volatile uint32_t *)&S.pending == 0u) return;
    }
}

// Take one completed batch from the reduction queue (compare-and-swap on the
// head; an entry is taken only once its index has been written).
__device__ FRW_OUTLINE uint32_t take_batch(const EngineView &E)
{
    for (int tries = 0; tries < 64; tries++) {
        const uint32_t h = *(volatile uint32_t *)E.rq_head;
        const uint32_t c = min(*(volatile uint32_t *)E.rq_count, E.rq_cap);
        if (h >= c) return 0xffffffffu;
        const uint32_t item = *(volatile uint32_t *)(E.rq + h);
        if (item == 0xffffffffu) return 0xffffffffu;     // not written yet: next epoch
        if (atomicCAS(E.rq_head, h, h + 1u) == h) return item;
    }
    return 0xffffffffu;
}

// ---------------------------------------------------------------------------
// The persistent walk kernel.  Each CTA owns a pool of walk slots and cycles, on
// its own, through four phases per epoch (no CTA ever waits for another):
//   geometry  every slot that is not in MicroWalk makes one step: a free slot takes
//             a walk id and makes the first transition; a walk at a point sizes its
//             cube, classifies it, and either samples the analytical route in place
//             or records a MicroWalk job in the CTA's queue;
//   fill      the CTA fills the analytical tables it claimed (separable FD solve);
//   reduce    completed batches queued by any CTA are folded into accumulators;
//   MicroWalk each warp runs the CTA's queued lattice walks (Algorithm 3), one per
//             lane, refilling lanes at 4-step boundaries; once the queue is empty a
//             warp with few lanes left suspends them (node and step count saved, so
//             the Philox stream continues unchanged) and they resume next epoch.
// The kernel exits when its pool is empty, no walk can be issued and every stop
// rule is decided; an idle wait is bounded by E.idle_timeout_s.
// Block of the walk kernel and CTAs per SM it is compiled for: 2 x 448 threads
// (28 warps per SM at up to 72 registers) measured faster than 3 x 256, 3 x 320,
// 2 x 384, 2 x 512, 4 x 256, 6 x 128 and 1 x 768 on the interconnect workload
#ifndef FRW_WALK_THREADS
#define FRW_WALK_THREADS 448
#endif
#ifndef FRW_POOL_MAX
#define FRW_POOL_MAX 2048   // slot lists of 2048 entries: 12 KB less shared memory than 4096, more L1
#endif
#ifndef FRW_FILL_GLOBAL
#define FRW_FILL_GLOBAL 0
#endif
constexpr int WALK_THREADS = FRW_WALK_THREADS;
// MicroWalk block of the walk kernel: FRW_MW_WIDE_ONLY 1 keeps only the wide
// column decode (one code path), 0 lets a warp whose lanes all hold cubes of at
// most 6 blocks use the narrow decode (two compact loops); FRW_MW_COMPACT 1 runs
// the four steps as a loop.  Measured on the interconnect workload (budget mode,
// 3 x 2^20 walks, N = 24): with two analytical hops per geometry visit the single
// wide loop was fastest (44.7 ms against 45.6 ms with both forms compact, 49.7 ms
// both unrolled, 50.0 ms wide and unrolled); with one hop per visit, which
// relieved the instruction cache, both compact forms are (33.7-33.9 against
// 35.5-35.7 ms)
#ifndef FRW_MW_WIDE_ONLY
#define FRW_MW_WIDE_ONLY 0
#endif
#ifndef FRW_MW_COMPACT
#define FRW_MW_COMPACT 1
#endif
#if FRW_MW_COMPACT
#define FRW_MW_BLOCK mw_block4_compact
#else
#define FRW_MW_BLOCK mw_block4
#endif
// 1: the walk kernel's table fill works in global scratch (per CTA) instead of
// shared memory, so that the shared region holds only the MicroWalk masks
constexpr bool FILL_GLOBAL = FRW_FILL_GLOBAL != 0;
#ifndef FRW_WALK_CTAS
#define FRW_WALK_CTAS 2
#endif
constexpr int WALK_CTAS = FRW_WALK_CTAS;   // CTAs per SM the walk kernel is compiled for
constexpr int WALK_WARPS = WALK_THREADS / 32;
constexpr int MW_WARPS = WALK_WARPS;
constexpr int POOL_MAX = FRW_POOL_MAX;
static_assert(POOL_MAX <= 2048, "slot list entries hold the slot index in 11 bits");
constexpr int FILL_MAX = 128;
constexpr uint32_t SUSPEND_MIN_FINISHED = 32;
// 1: the phased walk kernel keeps a per-lane copy of the weight table (8 KB of
// shared memory) for contexts of at most 7 materials; 0: one shared copy.  Without
// the copies two CTAs fit the 196 KB shared-memory carve-out instead of 228 KB,
// and the larger L1 (60 KB instead of 28 KB) serves the geometry work's stack and
// table reads: measured faster (interconnect, N = 24: 42.9 -> 41.4 ms per
// 3 x 2^20 walks) than conflict-free weight reads.
#ifndef FRW_WALK_WTAB_LANES
#define FRW_WALK_WTAB_LANES 0
#endif // suspension only if this much geometry work is waiting

// Clock read that cannot move above the preceding barrier: it is taken only after
// a shared-memory word loaded after that barrier has been tested.
__device__ __forceinline__ long long clock_after(const uint32_t *anchor)
{
    const uint32_t v = *(const volatile uint32_t *)anchor;
    long long c = 0;
    if (v != 0xfffffffeu) c = clock64();
    return c;
}

#include "fdm_transition.cuh"
constexpr uint32_t FDM_CLAIM_CAP = 8;    // FRW-FDM: walk ids a CTA claims per epoch

struct WalkShared {
    uint32_t W[WTAB_FULL_WORDS];     // jump-weight table W'[centre column][neighbour column] (one copy)
#if FRW_WALK_WTAB_LANES
    uint32_t Wl[WTAB_LANES_WORDS];   // the same table of 8 columns, one copy per lane (materials 0-6)
#endif
    uint32_t scan[32 * (FRW_WALK_THREADS / 32)];   // per-warp scratch of the mask build
    uint32_t g_head, g_back, pad3[2];
    uint32_t q_count, q_head, s_count, g_count;
    uint32_t f_count, active, issuable, stop;
    uint32_t red, finished, n_free, j_lo;
    uint32_t j_pub, pad4[3];
    uint32_t q_next, fdm_sel, progress_seen, pad2;
    unsigned long long idle_t0;      // start of this CTA's idle wait (thread 0)
    IssueRanges ir;
    uint32_t fill[FILL_MAX];
    uint16_t qlist[2][POOL_MAX];
    uint16_t glist[POOL_MAX];
};

// table-fill work space: ek[MAXN], yh[(N/2)^2 N], Z[MAXN^2], red[FILL_CHUNKS + 1]
size_t fill_smem_bytes(int N)
{
    const int H = N / 2;
    return sizeof(double) * (size_t)(MAXN + H * H * N + MAXN * MAXN + FILL_CHUNKS + 1);
}

// stand-alone MicroWalk CTA: weight table (the larger, per-lane layout), one
// 32-word scan scratch per warp, the warps' mask columns
size_t mw_smem_bytes(int N, int warps)
{
    return sizeof(uint32_t) * (WTAB_LANES_WORDS + 32 * (size_t)warps) +
           sizeof(uint16_t) * (size_t)warps * 3 * (N + 4) * 32;
}

// dynamic shared memory of the walk kernel: one region shared in turn by the
// MicroWalk masks, the table fill and the reduction
size_t walk_scratch_bytes(int N, int max_nc)
{
    const size_t masks = sizeof(uint16_t) * (size_t)MW_WARPS * 3 * (N + 4) * 32;
    const size_t fill = FILL_GLOBAL ? 0 : fill_smem_bytes(N);
    const size_t red = sizeof(unsigned long long) * acc_stride_for(max_nc);
    return std::max(masks, std::max(fill, red));
}

// per walk-kernel CTA: doubles of global table-fill scratch (the 6N^2 panel
// values, plus the fill's work arrays when they do not live in shared memory)
size_t walk_fill_scratch_doubles(int N)
{
    // the work arrays too: the warp-specialised kernel fills tables in global memory
    return 6 * (size_t)N * N + (fill_smem_bytes(N) + sizeof(double) - 1) / sizeof(double);
}

// dynamic shared memory of the warp-specialised walk kernel: the reduction's
// accumulator block, then the masks of up to WALK_WARPS - 1 MicroWalk warps
size_t walk_ws_smem_bytes(int N, int max_nc)
{
    const size_t acc = ((size_t)acc_stride_for(max_nc) * 8 + 127) / 128 * 128;
    return acc + sizeof(uint16_t) * (size_t)(WALK_WARPS - 1) * 3 * (N + 4) * 32;
}
int walk_geo_warps_max() { return WALK_WARPS - 1; }

size_t walk_smem_bytes(int N, int max_nc, int transition)
{
    const size_t base = walk_scratch_bytes(N, max_nc);
    return transition == 1 ? std::max(base, fdm_smem_bytes(N)) : base;
}

int walk_pool_slots() { return POOL_MAX; }

// FDM = true: the FRW-FDM comparator, whose non-stratified transitions solve the
// cube's FD system (Algorithm 2) one cube at a time with the whole CTA, in place
// of the MicroWalk phase (one CTA per SM: the solve's vectors fill shared memory).
// Copy the geometry of structure E.stage_sid (the groups of E.stage_flags) into
// `region` and return a view of it whose arrays point there (the groups not
// copied keep their global arrays); nullptr when the groups do not fit the
// E.stage_bytes the host allotted (error bit ERR_CHECK, the walks then read global
// memory).  Every thread of the CTA calls it; the caller synchronises before use.
template <typename T>
__device__ const SView<T> *stage_structure(const EngineView &E, SView<T> &sv, unsigned char *region)
{
    if (!FRW_STAGE_GEOM || E.stage_sid < 0 || E.stage_flags == 0u) return nullptr;
    const int tid = threadIdx.x, nt = blockDim.x;
    const SView<T> &G = structure_view<T>(E, E.stage_sid);
    const int ts = (int)sizeof(T);
    const uint32_t fl = E.stage_flags;
    uint32_t need = 0;
    for (uint32_t g = STAGE_BOXES; g <= STAGE_SLABS; g <<= 1)
        if (fl & g) need += stage_group_bytes(g, G.n_c, G.n_b, G.sl_S, G.sl_words, ts);
    if (need > E.stage_bytes) {
        if (tid == 0) atomicOr(&E.status[STAT_ERR], ERR_CHECK);
        return nullptr;
    }
    const T *clo = G.clo, *chi = G.chi, *blo = G.blo, *bhi = G.bhi;
    const uint8_t *bmat = G.bmat;
    const uint32_t *sL = G.sl_L, *sH = G.sl_H;
    uint32_t off = 0;
    if (fl & STAGE_BOXES) {
        T *d = reinterpret_cast<T *>(region + off);
        const int n = 3 * G.n_c;
        for (int i = tid; i < n; i += nt) {
            d[i] = G.clo[i];
            d[n + i] = G.chi[i];
        }
        clo = d;
        chi = d + n;
        off += stage_group_bytes(STAGE_BOXES, G.n_c, G.n_b, G.sl_S, G.sl_words, ts);
    }
    if ((fl & STAGE_BLOCKS) && G.n_b > 0) {
        T *d = reinterpret_cast<T *>(region + off);
        const int n = 3 * G.n_b;
        for (int i = tid; i < n; i += nt) {
            d[i] = G.blo[i];
            d[n + i] = G.bhi[i];
        }
        uint8_t *m = region + off + stage_round16(6u * (uint32_t)G.n_b * (uint32_t)ts);
        for (int i = tid; i < G.n_b; i += nt) m[i] = G.bmat[i];
        blo = d;
        bhi = d + n;
        bmat = m;
        off += stage_group_bytes(STAGE_BLOCKS, G.n_c, G.n_b, G.sl_S, G.sl_words, ts);
    }
    if (fl & STAGE_SLABS) {
        uint32_t *d = reinterpret_cast<uint32_t *>(region + off);
        const int n = 3 * G.sl_S * G.sl_words;
        for (int i = tid; i < n; i += nt) {
            d[i] = G.sl_L[i];
            d[n + i] = G.sl_H[i];
        }
        sL = d;
        sH = d + n;
    }
    if (tid == 0) {
        sv = G;
        sv.clo = clo; sv.chi = chi; sv.blo = blo; sv.bhi = bhi; sv.bmat = bmat;
        sv.sl_L = sL; sv.sl_H = sH;
        atomicAdd(&E.status[STAT_STAGED], 1u);
    }
    return &sv;
}

template <typename T, bool MWE, bool FDM>
__global__ void __launch_bounds__(WALK_THREADS, FDM ? 1 : WALK_CTAS) k_walk(EngineView E)
{
    extern __shared__ __align__(16) unsigned char dsm_all[];
    __shared__ WalkShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = E.N;
    const uint32_t P = E.pool;
    const uint32_t base = blockIdx.x * P;
    unsigned char *dsm = dsm_all;
    double *fill_v = E.fill_scratch + (size_t)blockIdx.x * E.fill_stride;
    wtab_fill(sh.W, E.W, false, tid, WALK_THREADS);
#if FRW_WALK_WTAB_LANES
    if (E.wtab_lanes) wtab_fill(sh.Wl, E.W, true, tid, WALK_THREADS);
#endif
    // the geometry copy lives above the region the phases share (E.stage_off, set by the host)
    __shared__ SView<T> sview_staged;
    const SView<T> *staged = FDM ? nullptr : stage_structure<T>(E, sview_staged, dsm_all + E.stage_off);
    for (uint32_t o = tid; o < P; o += WALK_THREADS) {
        const uint32_t s = base + o;
        E.s.state[s] = ST_FRESH;
        E.s.job[s] = 0u;
    }
    if (tid == 0) {
        sh.q_count = 0; sh.q_head = 0; sh.s_count = 0; sh.stop = 0; sh.q_next = 0;
        sh.g_count = 0; sh.f_count = 0; sh.active = 0; sh.finished = 0; sh.n_free = 0; sh.red = 0;
        sh.issuable = 0;
        sh.j_lo = 0;
        sh.j_pub = 0;
        sh.idle_t0 = 0;
        sh.progress_seen = 0;
    }
    __syncthreads();
    int cur = 0;
    unsigned long long cyc[5] = {0, 0, 0, 0, 0};
    uint32_t epochs = 0;
    for (;;) {
        const long long c0 = clock64();
        if (warp == 0) {
            uint32_t lo, pub, open;
            scan_jobs(E, lo, pub, open);
            if (lane == 0) {
                sh.g_count = 0; sh.f_count = 0; sh.active = 0; sh.finished = 0; sh.n_free = 0; sh.g_head = 0;
                sh.g_back = 0;
                sh.issuable = open;
                sh.j_lo = lo;
                sh.j_pub = pub;
            }
        }
        __syncthreads();
        uint16_t *q_now = sh.qlist[cur];
        uint16_t *q_next = sh.qlist[cur ^ 1];
        {
            // ---------------- geometry ----------------
            const bool iss = sh.issuable != 0;
            for (uint32_t o = tid; o < P; o += WALK_THREADS) {   // P is a multiple of 32: whole warps
                const uint32_t s = base + o;
                uint32_t st = E.s.state[s];
                if (st == ST_IDLE && iss) {
                    st = ST_FRESH;
                    E.s.state[s] = ST_FRESH;
                }
                const bool act = st != ST_IDLE;
                const bool need = act && st != ST_MW;
                uint32_t wj = 0;
                if (st != ST_FRESH && st != ST_IDLE && st != ST_MW) wj = E.s.job[s];
                const bool cancelled = need && st != ST_FRESH && ((volatile int *)E.job_cancel)[wj];
                const bool free_slot = st == ST_FRESH || cancelled;
                // list entry: slot | effective state << 11 (a cancelled job's walk is dropped)
                const uint32_t entry = o | ((cancelled ? ST_FRESH : st) << 11);
                // slots that start a walk (first transition) are listed from the front,
                // the others from the back: warps then take work of one kind, the
                // costliest first
                const bool first = need && (free_slot || st == ST_FIRST);
                const uint32_t ba = __ballot_sync(FULL_MASK, act);
                const uint32_t b1 = __ballot_sync(FULL_MASK, first), b2 = __ballot_sync(FULL_MASK, need && !first);
                const uint32_t bf = __ballot_sync(FULL_MASK, free_slot);
                uint32_t g1 = 0, g2 = 0;
                if (lane == 0) {
                    if (ba) atomicAdd(&sh.active, (uint32_t)__popc(ba));
                    if (b1) g1 = atomicAdd(&sh.g_count, (uint32_t)__popc(b1));
                    if (b2) g2 = atomicAdd(&sh.g_back, (uint32_t)__popc(b2));
                    if (bf) atomicAdd(&sh.n_free, (uint32_t)__popc(bf));
                }
                g1 = __shfl_sync(FULL_MASK, g1, 0);
                g2 = __shfl_sync(FULL_MASK, g2, 0);
                const uint32_t below = (1u << lane) - 1u;
                if (first) {
                    const uint32_t gi = g1 + __popc(b1 & below);
                    if (FRW_CHECKED(E, gi < P)) sh.glist[gi] = (uint16_t)entry;
                } else if (need) {
                    const uint32_t gi = g2 + __popc(b2 & below);
                    if (FRW_CHECKED(E, gi < P)) sh.glist[P - 1u - gi] = (uint16_t)entry;
                }
            }
            __syncthreads();
            // FRW-FDM: few new walks per CTA and epoch, so that the long FD solves
            // spread over every CTA instead of the first ones to claim
            if (warp == 0) claim_ids(E, sh.ir, FDM ? min(sh.n_free, FDM_CLAIM_CAP) : sh.n_free, sh.j_lo, sh.j_pub);
            __syncthreads();
            const uint32_t n1 = sh.g_count, ng = n1 + sh.g_back;
            const FillList fl{sh.fill, &sh.f_count, (uint32_t)FILL_MAX};
            // dynamic distribution: slot steps differ a lot in cost (first transitions,
            // chains of analytical hops), so threads take the next slot when free
            for (;;) {
                const uint32_t i = atomicAdd(&sh.g_head, 1u);
                if (i >= ng) break;
                const uint32_t ent = i < n1 ? sh.glist[i] : sh.glist[P - 1u - (i - n1)];
                const uint32_t o = ent & 2047u;
                geo_slot<T, MWE>(E, base + o, o, fl, sh.ir, staged, ent >> 11, [&](uint32_t oo) {
                    cg::coalesced_group g = cg::coalesced_threads();
                    uint32_t b0 = 0;
                    if (g.thread_rank() == 0) b0 = atomicAdd(&sh.q_count, (uint32_t)g.size());
                    const uint32_t qi = g.shfl(b0, 0) + g.thread_rank();
                    if (FRW_CHECKED(E, qi < E.pool)) q_now[qi] = (uint16_t)oo;
                });
            }
        }
        __syncthreads();
        const long long cg1 = clock_after(&sh.q_count);
        if constexpr (FDM) {
            // ---------------- FD transitions (Algorithm 2) ----------------
            const uint32_t qn = sh.q_count;
            const FdmSmem S = fdm_smem(dsm, N);
            const FdmScratch X = fdm_scratch(E.fdm_scratch + (size_t)blockIdx.x * fdm_scratch_bytes(N), N);
            const FdmGrid G = fdm_grid(N);
            if (qn) fdm_couplings(S, E.eps);
            for (uint32_t qi = 0; qi < qn; qi++) {
                const uint32_t o = q_now[qi];
                if (!FRW_CHECKED(E, o < P)) continue;
                const MWJob &b = E.mwq[base + o];
                const int K = min((int)b.K, KMAX);
                const uint64_t mm = (uint64_t)b.mm_lo | ((uint64_t)b.mm_hi << 32);
                // voxel materials: background (slot 1), then the listed blocks in order
                fdm_nodes(G, [&](int v, int i, int j, int k) {
                    int slot = 1;
                    for (int t = 0; t < K; t++) {
                        const uint2 r = b.rng[t];
                        if (i >= rng_lo(r, 0) && i < rng_hi(r, 0) && j >= rng_lo(r, 1) && j < rng_hi(r, 1) &&
                            k >= rng_lo(r, 2) && k < rng_hi(r, 2))
                            slot = 2 + t;
                    }
                    S.lat[v] = (uint8_t)((mm >> (4 * slot)) & 15ull);
                });
                __syncthreads();
                // the hop's first word, as MicroWalk's start draw
                const uint32_t u = philox10(b.walk_lo, b.walk_hi, b.hop, 0u, b.key0, b.key1).x;
                const FdmResult r = fdm_solve(N, S, X, u, nullptr, &sh.fdm_sel);
                if (tid == 0) {
                    if (!r.converged) atomicOr(&E.status[STAT_ERR], ERR_FDM);
                    const uint32_t sl = b.slot;
                    E.s.exitnode[sl] = r.exitnode;
                    __threadfence_block();
                    E.s.state[sl] = ST_MWDONE;
                    atomicAdd(&sh.finished, 1u);
                }
                __syncthreads();
            }
        } else {
            // ---------------- MicroWalk ----------------
            // (masks re-cleared: the fill and reduction phases use the same region)
            uint16_t *Mw = reinterpret_cast<uint16_t *>(dsm) + (size_t)warp * mask_rows(N) * 32;
            uint32_t *Tw = sh.scan + warp * 32;
            masks_clear(Mw, N, lane);
            __syncwarp();
            const MWRows R = mw_rows(Mw, N, lane);
#if FRW_WALK_WTAB_LANES
            const bool lanes_table = E.wtab_lanes != 0;
            const MWTab T0 = wtab_lane(lanes_table ? sh.Wl : sh.W, lanes_table, lane);
#else
            const MWTab T0 = wtab_lane(sh.W, false, lane);
#endif
            const uint32_t qn = sh.q_count;
            bool active = false, exhausted = false;
            bool wexh = false;   // warp-uniform: some lane found the queue empty
            int x = -1, y = 0, z = 0;
            uint32_t t = 0, t_in = 0, my_o = 0;
            MWLane L;
            mw_lane_reset(L, T0);
            for (;;) {
                const bool need = !active && !exhausted;
                const uint32_t bal = __ballot_sync(FULL_MASK, need);
                if (bal) {
                    const int leader = __ffs(bal) - 1;
                    uint32_t b0 = 0;
                    if (lane == leader) b0 = atomicAdd(&sh.q_head, (uint32_t)__popc(bal));
                    b0 = __shfl_sync(FULL_MASK, b0, leader);
                    const uint32_t myj = b0 + (uint32_t)__popc(bal & ((1u << lane) - 1u));
                    const bool got = need && myj < qn;
                    if (need && !got) exhausted = true;
                    wexh = __any_sync(FULL_MASK, exhausted);
                    const uint32_t oj = got ? (uint32_t)q_now[myj] : 0u;
                    uint32_t todo = __ballot_sync(FULL_MASK, got);
                    while (todo) {
                        const int r = __ffs(todo) - 1;
                        todo &= todo - 1u;
                        const uint32_t orr = __shfl_sync(FULL_MASK, oj, r);
                        const MWJob &b = E.mwq[base + orr];
                        const int K = min((int)ldcg(&b.K), KMAX);
                        build_masks(Mw, Tw, r, N, lane, K, [&](int lo[3], int hi[3]) {
                            const uint2 rr = ldcg(&b.rng[lane]);
                            lo[0] = (int)(rr.x & 255u); hi[0] = (int)((rr.x >> 8) & 255u);
                            lo[1] = (int)((rr.x >> 16) & 255u); hi[1] = (int)(rr.x >> 24);
                            lo[2] = (int)(rr.y & 255u); hi[2] = (int)((rr.y >> 8) & 255u);
                        });
                    }
                    __syncwarp();
                    if (got) {
                        const MWHead b = mw_head(E.mwq[base + oj]);
                        L.walk_lo = b.walk_lo; L.walk_hi = b.walk_hi; L.hop = b.hop;
                        L.key0 = b.key0; L.key1 = b.key1; L.tag = b.slot;
                        mw_lane_cube(L, T0, min((int)b.K, KMAX), (uint64_t)b.mm_lo | ((uint64_t)b.mm_hi << 32));
                        x = (int)(b.start & 255u); y = (int)((b.start >> 8) & 255u); z = (int)((b.start >> 16) & 255u);
                        t = b.steps;
                        t_in = t;
                        my_o = oj;
                        active = true;
                        if (!FRW_CHECKED(E, (unsigned)x < (unsigned)N && (unsigned)y < (unsigned)N &&
                                                (unsigned)z < (unsigned)N)) {
                            active = false;
                            x = -1; y = 0; z = 0;
                        }
                    }
                }
                const uint32_t ab = __ballot_sync(FULL_MASK, active);
                if (ab == 0u) break;
                // Suspend the few lanes left once the queue is empty (as this warp has
                // seen), if every one of them has made progress this epoch and the CTA
                // has other work waiting (so every job advances every epoch: no livelock).
                bool park = false;
                if (wexh && __popc(ab) <= E.suspend_lanes) {
                    const bool progressed = __all_sync(FULL_MASK, !active || t - t_in >= E.suspend_min_steps);
                    const bool other_work = __shfl_sync(FULL_MASK, (uint32_t)(*(volatile uint32_t *)&sh.finished >=
                                                                               SUSPEND_MIN_FINISHED || sh.issuable), 0) != 0u;
                    park = progressed && other_work;
                }
                if (park) {
                    if (active && FRW_CHECKED(E, (unsigned)x < (unsigned)N && (unsigned)y < (unsigned)N &&
                                                     (unsigned)z < (unsigned)N)) {
                        // a walking lane is always on a node inside the lattice here
                        MWJob &b = E.mwq[base + my_o];
                        stcg(&b.start, (uint32_t)x | ((uint32_t)y << 8) | ((uint32_t)z << 16));
                        stcg(&b.pad0, t);
                        const uint32_t qi = atomicAdd(&sh.q_next, 1u);
                        if (FRW_CHECKED(E, qi < P)) q_next[qi] = (uint16_t)my_o;
                        atomicAdd(&sh.s_count, 1u);
                        active = false;
                    }
                    break;
                }
                // eight steps (two Philox blocks) without a branch; a lane without a
                // walk, or whose walk ended in the first block, rests on a boundary node
                uint32_t moved = 0;
#pragma unroll 1
                for (uint32_t hb = 0; hb < 2u; hb++) {
                    const uint4 blk = philox10(L.walk_lo, L.walk_hi, L.hop, 1u + (t >> 2) + hb, L.key0, L.key1);
#if FRW_MW_WIDE_ONLY
                    moved += FRW_MW_BLOCK<true>(R, T0.with_base(L.base_w), L.map, x, y, z, blk);
#else
                    const bool wide = __any_sync(FULL_MASK, active && L.K > 6);
                    moved += wide ? FRW_MW_BLOCK<true>(R, T0.with_base(L.base_w), L.map, x, y, z, blk)
                                  : FRW_MW_BLOCK<false>(R, T0.with_base(L.base_n), L.map, x, y, z, blk);
#endif
                }
                const bool inside = ((unsigned)x < (unsigned)N) & ((unsigned)y < (unsigned)N) & ((unsigned)z < (unsigned)N);
                if (active && (moved < 8u || !inside)) {
                    // the walk has ended: on a boundary node (the exit node; reached at any of
                    // the four steps), or (MicroWalk-E) it rests on a conductor node inside the
                    // expanded cube (conductor flagged by bit 31)
                    const uint32_t sl2 = L.tag;
                    uint32_t en = (uint32_t)(x + 1) | ((uint32_t)(y + 1) << 8) | ((uint32_t)(z + 1) << 16);
                    if (MWE && inside) {
                        const int slot = mw_slot_at(R, x, y, z);
                        en = FRW_CHECKED(E, slot >= 2 && slot < 2 + KMAX)
                                 ? (0x80000000u | (ldcg(&E.mwq[base + my_o].rng[slot - 2].y) >> 24))
                                 : 0x80000000u;
                    }
                    stcg(&E.s.exitnode[sl2], en);
                    stcg(&E.s.steps[sl2], ldcg(&E.s.steps[sl2]) + t + moved);
                    __threadfence_block();      // exit data before the state (read by geometry warps)
                    E.s.state[sl2] = ST_MWDONE;
                    active = false;
                    x = -1; y = 0; z = 0;
                    atomicAdd(&sh.finished, 1u);
                }
                t += 8;
                if (active && t >= MW_STEP_CAP) {   // safety net: never loop without bound
                    atomicOr(&E.status[STAT_ERR], ERR_MW_STEPS);
                    const uint32_t sl2 = L.tag;
                    E.s.exitnode[sl2] = (uint32_t)(x + 1) | ((uint32_t)(y + 1) << 8) | ((uint32_t)(z + 1) << 16);
                    E.s.steps[sl2] += t;
                    __threadfence_block();
                    E.s.state[sl2] = ST_MWDONE;
                    active = false;
                    x = -1; y = 0; z = 0;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        const long long c1 = clock_after(&sh.q_next);
        if (tid == 0) {
            cyc[0] += (unsigned long long)(cg1 - c0);
            cyc[3] += (unsigned long long)(c1 - cg1);
        }
        // ---------------- fill phase ----------------
        const uint32_t nf = min(sh.f_count, (uint32_t)FILL_MAX);
        for (uint32_t f = 0; f < nf; f++) {
            const uint32_t e = sh.fill[f];
            if (e == 0xffffffffu) continue;
            FillJob F;
            const uint32_t *k = E.tc.keys + 5 * e;
            F.kind = k[0];
            F.prof[0] = k[1]; F.prof[1] = k[2]; F.prof[2] = k[3]; F.prof[3] = k[4];
            F.thr = E.tc.thr + (size_t)e * E.tc.P;
            F.sgn = E.tc.sgn + (size_t)e * E.tc.P32;
            F.guide = E.tc.guide + (size_t)e * GUIDE;
            F.ktot = E.tc.ktot + e;
            F.values = nullptr;
            F.err = &E.status[STAT_ERR];
            F.V = fill_v;
            fill_table(F, N, E.eps, E.fc, FILL_GLOBAL ? fill_v + 6 * N * N : reinterpret_cast<double *>(dsm), cta_grp());
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicExch(&E.tc.state[e], TE_READY);
                atomicAdd(&E.status[STAT_BUILT], 1u);
            }
            __syncthreads();
        }
        __syncthreads();
        const long long c2 = clock_after(&sh.f_count);
        // ---------------- reduction phase ----------------
        for (;;) {
            if (tid == 0) sh.red = take_batch(E);
            __syncthreads();
            const uint32_t g = sh.red;
            __syncthreads();
            if (g == 0xffffffffu) break;
            reduce_batch(E, g, reinterpret_cast<unsigned long long *>(dsm), cta_grp());
            if (tid == 0) advance_job(E, __ldcg(E.batch_job + g));
        }
        const long long c3 = clock_after(&sh.red);
        epochs++;
        if (tid == 0) {
            cyc[1] += (unsigned long long)(c2 - c1);
            cyc[2] += (unsigned long long)(c3 - c2);
            cyc[4] += (unsigned long long)(c3 - c0);
            if (sh.s_count) atomicAdd(&E.status[STAT_SUSPENDED], sh.s_count);
            const bool idle = sh.active == 0u && sh.issuable == 0u && sh.q_next == 0u;
            sh.q_count = sh.q_next;
            sh.q_next = 0;
            sh.q_head = 0;
            sh.s_count = 0;
            uint32_t stop = 0;
            if (*(volatile uint32_t *)&E.ctrl[CTRL_ABORT]) stop = 1;
            if (*(volatile uint32_t *)&E.status[STAT_ERR]) stop = 1;   // any device error ends the run
            const bool undecided =
                *(volatile uint32_t *)&E.jctl[JC_DECIDED] < *(volatile uint32_t *)&E.jctl[JC_PUBLISHED];
            if (idle) {
                if (!undecided && *(volatile uint32_t *)&E.ctrl[CTRL_OPEN] == 0u) {
                    stop = 1;
                } else {
                    // the wait is limited only while no CTA of the run makes progress
                    // (others may still be busy with walks this CTA cannot take over)
                    unsigned long long now;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                    const uint32_t prog = *(volatile uint32_t *)&E.status[STAT_PROGRESS];
                    if (sh.idle_t0 == 0 || prog != sh.progress_seen) {
                        sh.idle_t0 = now;
                        sh.progress_seen = prog;
                    } else if ((double)(now - sh.idle_t0) * 1e-9 > E.idle_timeout_s) {
                        atomicOr(&E.status[STAT_ERR], ERR_IDLE_TIMEOUT);
                        stop = 1;
                    }
                    __nanosleep(20000);
                }
            } else {
                sh.idle_t0 = 0;
                atomicAdd(&E.status[STAT_PROGRESS], 1u);
            }
            sh.stop = stop;
        }
        cur ^= 1;
        __syncthreads();
        if (sh.stop) break;
    }
    if (tid == 0) {
        for (int i = 0; i < 5; i++) atomicAdd(&E.cycles[i], cyc[i]);
        atomicMax(&E.status[STAT_EPOCHS], epochs);
    }
}

// ---------------------------------------------------------------------------
// Warp-specialised walk kernel.  The CTA's warps split into a geometry group
// (warps 0 .. G - 1) and a MicroWalk group (the others), which run at the same
// time and meet only through two bitmaps over the CTA's slots in shared memory:
// gbits (the slot's walk waits for geometry work: a new walk, analytical hops,
// or the follow-up of a finished MicroWalk job) and mbits (the slot holds a
// queued MicroWalk job).  At any time a slot is in at most one of them, or held
// by the one thread working on it, or idle (no walk id).
//  - The geometry group works in rounds, kept together by a named barrier of its
//    own: claim walk ids for idle slots, take every bit of gbits, run geo_slot on
//    each slot (a walk that ends takes the next id in the same slot), fill the
//    analytical tables claimed in the round (work space in global memory), reduce
//    completed batches, and decide whether the run ends.
//  - A MicroWalk warp takes jobs from mbits whenever lanes are free, builds each
//    new lane's masks, walks in blocks of four steps, and hands a finished walk
//    back by setting its bit in gbits.  It never waits for the geometry group.
// Walks are keyed by their ids and accumulated exactly, so the results equal the
// phased kernel's bit for bit; only the schedule differs.

constexpr int WS_WORDS = POOL_MAX / 32;      // bitmap words of a pool of at most POOL_MAX slots
constexpr int WS_BAR = 1;                    // named barrier of the geometry group

struct WalkSharedWS {
    uint32_t W[WTAB_FULL_WORDS];
    uint32_t Wl[WTAB_LANES_WORDS];
    uint32_t scan[32 * WALK_WARPS];
    uint32_t gbits[WS_WORDS], mbits[WS_WORDS], work[WS_WORDS], wpre[WS_WORDS + 1];
    uint16_t idle[POOL_MAX];
    uint32_t n_idle, g_pos, g_total, f_count;
    int32_t m_count;                         // queued MicroWalk jobs (a hint: may lag a push or a claim)
    uint32_t stop, red, issuable, j_lo, j_pub, progress_seen, pad0;
    unsigned long long idle_t0;
    unsigned long long mw_busy;              // cycles MicroWalk warps spent with a lane walking
    IssueRanges ir;
    uint32_t fill[FILL_MAX];
};

__device__ __forceinline__ void ws_set(uint32_t *bm, uint32_t o) { atomicOr(&bm[o >> 5], 1u << (o & 31)); }

// claim one set bit of bm[0 .. nw), scanning from word `start`: the slot, or -1
__device__ __forceinline__ int ws_claim(uint32_t *bm, int nw, int start)
{
    int w = start;
    for (int i = 0; i < nw; i++) {
        uint32_t v = *(volatile uint32_t *)&bm[w];
        while (v) {
            const uint32_t b = v & (0u - v);
            const uint32_t old = atomicAnd(&bm[w], ~b);
            if (old & b) return 32 * w + __ffs((int)b) - 1;
            v = old & ~b;
        }
        if (++w == nw) w = 0;
    }
    return -1;
}

template <typename T, bool MWE>
__global__ void __launch_bounds__(WALK_THREADS, WALK_CTAS) k_walk_ws(EngineView E)
{
    extern __shared__ __align__(16) unsigned char dsm_all[];
    __shared__ WalkSharedWS sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = E.N;
    const uint32_t P = E.pool;
    const int nw = (int)((P + 31) / 32);
    const uint32_t base = blockIdx.x * P;
    const int G = E.geo_warps, NG = 32 * G;
    const bool geo = warp < G;
    double *fill_v = E.fill_scratch + (size_t)blockIdx.x * E.fill_stride;
    unsigned long long *acc_sm = reinterpret_cast<unsigned long long *>(dsm_all);
    const size_t acc_bytes = ((size_t)acc_stride_for(E.max_nc) * 8 + 127) / 128 * 128;
    wtab_fill(sh.W, E.W, false, tid, WALK_THREADS);
    if (E.wtab_lanes) wtab_fill(sh.Wl, E.W, true, tid, WALK_THREADS);
    for (uint32_t o = tid; o < P; o += WALK_THREADS) {
        E.s.state[base + o] = ST_IDLE;
        E.s.job[base + o] = 0u;
        sh.idle[o] = (uint16_t)o;
    }
    for (int w = tid; w < WS_WORDS; w += WALK_THREADS) {
        sh.gbits[w] = 0u;
        sh.mbits[w] = 0u;
    }
    if (tid == 0) {
        sh.n_idle = P; sh.g_pos = 0; sh.g_total = 0; sh.f_count = 0; sh.m_count = 0;
        sh.stop = 0; sh.red = 0; sh.issuable = 0; sh.j_lo = 0; sh.j_pub = 0; sh.progress_seen = 0;
        sh.idle_t0 = 0; sh.mw_busy = 0;
    }
    __syncthreads();
    if (geo) {
        // ======================== geometry group ========================
        const Grp grp{tid, NG, WS_BAR};
        const FillList fl{sh.fill, &sh.f_count, (uint32_t)FILL_MAX};
        unsigned long long cyc[3] = {0, 0, 0};
        const long long t_start = clock64();
        uint32_t rounds = 0;
        auto push_mw = [&](uint32_t o) {
            __threadfence_block();           // job record and slot state before the bit
            ws_set(sh.mbits, o);
            atomicAdd(&sh.m_count, 1);
        };
        for (;;) {
            const long long c0 = clock64();
            // (a) walk ids for the idle slots
            if (warp == 0) {
                uint32_t lo, pub, open;
                scan_jobs(E, lo, pub, open);
                if (lane == 0) {
                    sh.issuable = open;
                    sh.j_lo = lo;
                    sh.j_pub = pub;
                    sh.f_count = 0;
                }
                __syncwarp();
                claim_ids(E, sh.ir, open ? sh.n_idle : 0u, lo, pub);
            }
            grp.sync();
            // (b) idle slots that got an id join the round; (c) take the round's slots
            const uint32_t take = min(sh.n_idle, sh.ir.total);
            for (uint32_t i = tid; i < take; i += NG) {
                const uint32_t o = sh.idle[sh.n_idle - 1u - i];
                E.s.state[base + o] = ST_FRESH;
                ws_set(sh.gbits, o);
            }
            grp.sync();
            for (int w = tid; w < WS_WORDS; w += NG) sh.work[w] = w < nw ? atomicExch(&sh.gbits[w], 0u) : 0u;
            grp.sync();
            if (tid == 0) {
                sh.n_idle -= take;
                uint32_t acc = 0;
                for (int w = 0; w < nw; w++) {
                    sh.wpre[w] = acc;
                    acc += (uint32_t)__popc(sh.work[w]);
                }
                sh.wpre[nw] = acc;
                sh.g_total = acc;
                sh.g_pos = 0;
            }
            grp.sync();
            // (d) geometry work on every taken slot, handed out one at a time
            const uint32_t total = sh.g_total;
            for (;;) {
                const uint32_t k = atomicAdd(&sh.g_pos, 1u);
                if (k >= total) break;
                int lo = 0, hi = nw;                 // word w with wpre[w] <= k < wpre[w + 1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sh.wpre[mid] <= k) lo = mid;
                    else hi = mid;
                }
                uint32_t m = sh.work[lo];
                for (uint32_t q = k - sh.wpre[lo]; q > 0u; q--) m &= m - 1u;   // drop the lower set bits
                if (m == 0u) {                   // cannot happen: the prefix counts say bit k is here
                    atomicOr(&E.status[STAT_ERR], ERR_CHECK);
                    continue;
                }
                const uint32_t o = 32u * (uint32_t)lo + (uint32_t)(__ffs((int)m) - 1);
                if (!FRW_CHECKED(E, o < P)) continue;
                uint32_t st = ST_FRESH;
#pragma unroll 1
                for (int rep = 0; rep < 2; rep++) {   // a walk that ends takes the next id in the same slot
                    st = geo_slot<T, MWE>(E, base + o, o, fl, sh.ir, nullptr, ST_UNKNOWN, push_mw);
                    if (st != ST_FRESH) break;
                }
                if (st == ST_IDLE) {
                    const uint32_t i = atomicAdd(&sh.n_idle, 1u);
                    if (FRW_CHECKED(E, i < P)) sh.idle[i] = (uint16_t)o;
                } else if (st != ST_MW) {
                    ws_set(sh.gbits, o);          // waits for a table, or more hops: next round
                }
            }
            grp.sync();
            const long long c1 = clock_after(&sh.g_pos);
            // (e) tables claimed in this round
            const uint32_t nf = min(sh.f_count, (uint32_t)FILL_MAX);
            for (uint32_t f = 0; f < nf; f++) {
                const uint32_t e = sh.fill[f];
                if (e == 0xffffffffu) continue;
                FillJob F;
                const uint32_t *kk = E.tc.keys + 5 * e;
                F.kind = kk[0];
                F.prof[0] = kk[1]; F.prof[1] = kk[2]; F.prof[2] = kk[3]; F.prof[3] = kk[4];
                F.thr = E.tc.thr + (size_t)e * E.tc.P;
                F.sgn = E.tc.sgn + (size_t)e * E.tc.P32;
                F.guide = E.tc.guide + (size_t)e * GUIDE;
                F.ktot = E.tc.ktot + e;
                F.values = nullptr;
                F.err = &E.status[STAT_ERR];
                F.V = fill_v;
                fill_table(F, N, E.eps, E.fc, fill_v + 6 * N * N, grp);
                grp.sync();
                if (tid == 0) {
                    __threadfence();
                    atomicExch(&E.tc.state[e], TE_READY);
                    atomicAdd(&E.status[STAT_BUILT], 1u);
                }
                grp.sync();
            }
            const long long c2 = clock_after(&sh.f_count);
            // (f) completed batches
            for (;;) {
                if (tid == 0) sh.red = take_batch(E);
                grp.sync();
                const uint32_t g = sh.red;
                grp.sync();
                if (g == 0xffffffffu) break;
                reduce_batch(E, g, acc_sm, grp);
                if (tid == 0) advance_job(E, __ldcg(E.batch_job + g));
            }
            const long long c3 = clock_after(&sh.red);
            rounds++;
            if (tid == 0) {
                cyc[0] += (unsigned long long)(c1 - c0);
                cyc[1] += (unsigned long long)(c2 - c1);
                cyc[2] += (unsigned long long)(c3 - c2);
                // (g) end of the run, or an idle wait limited while no CTA makes progress
                const bool idle = sh.n_idle == P && sh.issuable == 0u;
                uint32_t stop = 0;
                if (*(volatile uint32_t *)&E.ctrl[CTRL_ABORT]) stop = 1;
                if (*(volatile uint32_t *)&E.status[STAT_ERR]) stop = 1;
                const bool undecided =
                    *(volatile uint32_t *)&E.jctl[JC_DECIDED] < *(volatile uint32_t *)&E.jctl[JC_PUBLISHED];
                if (idle) {
                    if (!undecided && *(volatile uint32_t *)&E.ctrl[CTRL_OPEN] == 0u) {
                        stop = 1;
                    } else {
                        unsigned long long now;
                        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                        const uint32_t prog = *(volatile uint32_t *)&E.status[STAT_PROGRESS];
                        if (sh.idle_t0 == 0 || prog != sh.progress_seen) {
                            sh.idle_t0 = now;
                            sh.progress_seen = prog;
                        } else if ((double)(now - sh.idle_t0) * 1e-9 > E.idle_timeout_s) {
                            atomicOr(&E.status[STAT_ERR], ERR_IDLE_TIMEOUT);
                            stop = 1;
                        }
                        __nanosleep(20000);
                    }
                } else {
                    sh.idle_t0 = 0;
                    if ((rounds & 7u) == 0u) atomicAdd(&E.status[STAT_PROGRESS], 1u);
                    if (total == 0u) __nanosleep(2000);   // walks held by MicroWalk: let it run
                }
                if (stop) *(volatile uint32_t *)&sh.stop = 1u;
            }
            grp.sync();
            if (*(volatile uint32_t *)&sh.stop) break;
        }
        if (tid == 0) {
            const long long t_all = clock64() - t_start;
            atomicAdd(&E.cycles[0], cyc[0]);
            atomicAdd(&E.cycles[1], cyc[1]);
            atomicAdd(&E.cycles[2], cyc[2]);
            atomicAdd(&E.cycles[4], (unsigned long long)t_all);
            atomicMax(&E.status[STAT_EPOCHS], rounds);
        }
    } else {
        // ======================== MicroWalk group ========================
        const int mwarp = warp - G;
        uint16_t *Mw = reinterpret_cast<uint16_t *>(dsm_all + acc_bytes) + (size_t)mwarp * mask_rows(N) * 32;
        uint32_t *Tw = sh.scan + warp * 32;
        masks_clear(Mw, N, lane);
        __syncwarp();
        const MWRows R = mw_rows(Mw, N, lane);
        const bool lanes_table = E.wtab_lanes != 0;
        const MWTab T0 = wtab_lane(lanes_table ? sh.Wl : sh.W, lanes_table, lane);
        bool active = false;
        int x = -1, y = 0, z = 0;
        uint32_t t = 0, my_o = 0;
        MWLane L;
        mw_lane_reset(L, T0);
        int rot = (mwarp * 7 + lane * 3) % nw;
        unsigned long long busy = 0;
        for (;;) {
            const bool need = !active;
            // warp-uniform: stop, and whether to look for jobs
            const uint32_t flags = __shfl_sync(FULL_MASK, (*(volatile uint32_t *)&sh.stop ? 1u : 0u) |
                                                              (*(volatile int32_t *)&sh.m_count > 0 ? 2u : 0u), 0);
            if ((flags & 1u) && !__any_sync(FULL_MASK, active && *(volatile uint32_t *)&E.status[STAT_ERR] == 0u))
                break;                           // the run is over (or failed: walks in flight are dropped)
            if (__any_sync(FULL_MASK, need) && (flags & 2u)) {
                int o = -1;
                if (need) {
                    o = ws_claim(sh.mbits, nw, rot);
                    if (o >= 0) atomicSub(&sh.m_count, 1);
                    if (++rot == nw) rot = 0;
                }
                const bool got = o >= 0;
                uint32_t todo = __ballot_sync(FULL_MASK, got);
                if (todo) __threadfence_block();     // pairs with the pusher's fence
                while (todo) {
                    const int r = __ffs(todo) - 1;
                    todo &= todo - 1u;
                    const uint32_t orr = (uint32_t)__shfl_sync(FULL_MASK, o, r);
                    const MWJob &b = E.mwq[base + orr];
                    const int K = min((int)ldcg(&b.K), KMAX);
                    build_masks(Mw, Tw, r, N, lane, K, [&](int lo[3], int hi[3]) {
                        const uint2 rr = ldcg(&b.rng[lane]);
                        lo[0] = (int)(rr.x & 255u); hi[0] = (int)((rr.x >> 8) & 255u);
                        lo[1] = (int)((rr.x >> 16) & 255u); hi[1] = (int)(rr.x >> 24);
                        lo[2] = (int)(rr.y & 255u); hi[2] = (int)((rr.y >> 8) & 255u);
                    });
                }
                __syncwarp();
                if (got) {
                    const MWHead b = mw_head(E.mwq[base + (uint32_t)o]);
                    L.walk_lo = b.walk_lo; L.walk_hi = b.walk_hi; L.hop = b.hop;
                    L.key0 = b.key0; L.key1 = b.key1; L.tag = b.slot;
                    mw_lane_cube(L, T0, min((int)b.K, KMAX), (uint64_t)b.mm_lo | ((uint64_t)b.mm_hi << 32));
                    x = (int)(b.start & 255u); y = (int)((b.start >> 8) & 255u); z = (int)((b.start >> 16) & 255u);
                    t = b.steps;
                    my_o = (uint32_t)o;
                    active = true;
                    if (!FRW_CHECKED(E, (unsigned)x < (unsigned)N && (unsigned)y < (unsigned)N &&
                                            (unsigned)z < (unsigned)N)) {
                        active = false;
                        x = -1; y = 0; z = 0;
                    }
                }
            }
            if (__ballot_sync(FULL_MASK, active) == 0u) {
                __nanosleep(1000);
                continue;
            }
            const long long cb = clock64();
            const uint4 blk = philox10(L.walk_lo, L.walk_hi, L.hop, 1u + (t >> 2), L.key0, L.key1);
#if FRW_MW_WIDE_ONLY
            const uint32_t moved = FRW_MW_BLOCK<true>(R, T0.with_base(L.base_w), L.map, x, y, z, blk);
#else
            const bool wide = __any_sync(FULL_MASK, active && L.K > 6);
            const uint32_t moved = wide ? FRW_MW_BLOCK<true>(R, T0.with_base(L.base_w), L.map, x, y, z, blk)
                                        : FRW_MW_BLOCK<false>(R, T0.with_base(L.base_n), L.map, x, y, z, blk);
#endif
            const bool inside = ((unsigned)x < (unsigned)N) & ((unsigned)y < (unsigned)N) & ((unsigned)z < (unsigned)N);
            if (active && (moved < 4u || !inside)) {
                // the walk has ended (see the phased kernel): exit node or conductor
                const uint32_t sl2 = L.tag;
                uint32_t en = (uint32_t)(x + 1) | ((uint32_t)(y + 1) << 8) | ((uint32_t)(z + 1) << 16);
                if (MWE && inside) {
                    const int slot = mw_slot_at(R, x, y, z);
                    en = FRW_CHECKED(E, slot >= 2 && slot < 2 + KMAX)
                             ? (0x80000000u | (ldcg(&E.mwq[base + my_o].rng[slot - 2].y) >> 24))
                             : 0x80000000u;
                }
                stcg(&E.s.exitnode[sl2], en);
                stcg(&E.s.steps[sl2], ldcg(&E.s.steps[sl2]) + t + moved);
                __threadfence_block();          // exit data before the state and the bit
                E.s.state[sl2] = ST_MWDONE;
                ws_set(sh.gbits, my_o);
                active = false;
                x = -1; y = 0; z = 0;
            }
            t += 4;
            if (active && t >= MW_STEP_CAP) {   // safety net: never loop without bound
                atomicOr(&E.status[STAT_ERR], ERR_MW_STEPS);
                const uint32_t sl2 = L.tag;
                E.s.exitnode[sl2] = (uint32_t)(x + 1) | ((uint32_t)(y + 1) << 8) | ((uint32_t)(z + 1) << 16);
                E.s.steps[sl2] += t;
                __threadfence_block();
                E.s.state[sl2] = ST_MWDONE;
                ws_set(sh.gbits, my_o);
                active = false;
                x = -1; y = 0; z = 0;
            }
            busy += (unsigned long long)(clock64() - cb);
            __syncwarp();
        }
        if (lane == 0) atomicAdd(&sh.mw_busy, busy);
    }
    __syncthreads();
    if (tid == 0) atomicAdd(&E.cycles[3], sh.mw_busy / (unsigned long long)max(1, WALK_WARPS - G));
}

// Shared-memory carve-out for the resident CTAs of the walk kernel (WALK_CTAS;
// one for the FDM comparator): no more than they need, so that the rest of the
// SM's on-chip memory serves as L1 (the geometry phase's structure data and stack
// live there).
template <typename T, bool MWE> static cudaError_t set_walk_ws_attributes(int smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_walk_ws<T, MWE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k_walk_ws<T, MWE>)) != cudaSuccess) return e;
    const size_t need = (size_t)WALK_CTAS * ((size_t)smem + fa.sharedSizeBytes + 1024);
    const int pct = (int)std::min<size_t>(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024));
    return cudaFuncSetAttribute(k_walk_ws<T, MWE>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

template <typename T, bool MWE, bool FDM> static cudaError_t set_walk_attributes(int smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_walk<T, MWE, FDM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k_walk<T, MWE, FDM>)) != cudaSuccess) return e;
    const size_t need = (size_t)(FDM ? 1 : WALK_CTAS) * ((size_t)smem + fa.sharedSizeBytes + 1024);
    const int pct = (int)std::min<size_t>(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024));
    return cudaFuncSetAttribute(k_walk<T, MWE, FDM>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

// dynamic shared memory of one launch of the phased walk kernel: the phases'
// region, then the geometry copy when the view has one
static size_t walk_view_smem(const EngineView &E)
{
    const size_t base = walk_smem_bytes(E.N, E.max_nc, E.transition);
    if (E.stage_sid < 0 || E.stage_flags == 0u || E.transition == 1) return base;
    return std::max(base, (size_t)E.stage_off + E.stage_bytes);
}

static cudaError_t walk_attributes(int N, int max_nc, int fp32, int mwe, int transition, size_t smem_bytes)
{
    const int smem = (int)smem_bytes;
    if (transition == 1)
        return fp32 ? set_walk_attributes<float, false, true>(smem) : set_walk_attributes<double, false, true>(smem);
    if (mwe > 1)
        return fp32 ? set_walk_attributes<float, true, false>(smem) : set_walk_attributes<double, true, false>(smem);
    return fp32 ? set_walk_attributes<float, false, false>(smem) : set_walk_attributes<double, false, false>(smem);
}

cudaError_t prepare_walk(const EngineView &E)
{
    if (E.geo_warps > 0 && E.transition != 1) {
        const int smem = (int)walk_ws_smem_bytes(E.N, E.max_nc);
        if (E.mwe > 1) return E.fp32 ? set_walk_ws_attributes<float, true>(smem) : set_walk_ws_attributes<double, true>(smem);
        return E.fp32 ? set_walk_ws_attributes<float, false>(smem) : set_walk_ws_attributes<double, false>(smem);
    }
    return walk_attributes(E.N, E.max_nc, E.fp32, E.mwe, E.transition, walk_view_smem(E));
}

cudaError_t launch_walk(const EngineView &E, const LaunchShape &L, cudaStream_t st)
{
    (void)L;
    const unsigned grid = E.NS / E.pool;
    if (E.geo_warps > 0 && E.transition != 1) {
        if (E.geo_warps >= WALK_WARPS || E.pool > (uint32_t)POOL_MAX) return cudaErrorInvalidValue;
        const size_t smem = walk_ws_smem_bytes(E.N, E.max_nc);
        if (E.mwe > 1) {
            if (E.fp32) k_walk_ws<float, true><<<grid, WALK_THREADS, smem, st>>>(E);
            else k_walk_ws<double, true><<<grid, WALK_THREADS, smem, st>>>(E);
        } else {
            if (E.fp32) k_walk_ws<float, false><<<grid, WALK_THREADS, smem, st>>>(E);
            else k_walk_ws<double, false><<<grid, WALK_THREADS, smem, st>>>(E);
        }
        return cudaGetLastError();
    }
    const size_t smem = walk_view_smem(E);
    if (E.transition == 1) {
        if (E.fp32) k_walk<float, false, true><<<grid, WALK_THREADS, smem, st>>>(E);
        else k_walk<double, false, true><<<grid, WALK_THREADS, smem, st>>>(E);
    } else if (E.mwe > 1) {
        if (E.fp32) k_walk<float, true, false><<<grid, WALK_THREADS, smem, st>>>(E);
        else k_walk<double, true, false><<<grid, WALK_THREADS, smem, st>>>(E);
    } else {
        if (E.fp32) k_walk<float, false, false><<<grid, WALK_THREADS, smem, st>>>(E);
        else k_walk<double, false, false><<<grid, WALK_THREADS, smem, st>>>(E);
    }
    return cudaGetLastError();
}

// FD transitions of stand-alone cubes (records as for the MicroWalk kernel: 64
// int32, [0] background, [1] K <= 8, then (i0, i1, j0, j1, k0, k1, mat) per block;
// local material ids mapped to the context's ids through the nibble map mmap)
__global__ void __launch_bounds__(FDM_THREADS, 1)
    k_fdm_cubes(int N, const int32_t *__restrict__ cubes, uint32_t n_cubes, uint64_t mmap,
                const double *__restrict__ eps, const uint32_t *__restrict__ u, double *P, uint32_t *exit_out,
                uint32_t *iters, unsigned char *scratch, uint32_t *err)
{
    extern __shared__ __align__(16) unsigned char dsm_fdm[];
    __shared__ uint32_t sel;
    const FdmSmem S = fdm_smem(dsm_fdm, N);
    const FdmScratch X = fdm_scratch(scratch + (size_t)blockIdx.x * fdm_scratch_bytes(N), N);
    const FdmGrid G = fdm_grid(N);
    fdm_couplings(S, eps);
    for (uint32_t c = blockIdx.x; c < n_cubes; c += gridDim.x) {
        const int32_t *rec = cubes + (size_t)c * 64;
        const int K = min(max(rec[1], 0), 8);
        const int bgm = (int)((mmap >> (4 * (rec[0] & 15))) & 15ull);
        fdm_nodes(G, [&](int v, int i, int j, int k) {
            int m = bgm;
            for (int t = 0; t < K; t++) {
                const int32_t *bk = rec + 2 + 7 * t;
                if (i >= bk[0] && i < bk[1] && j >= bk[2] && j < bk[3] && k >= bk[4] && k < bk[5])
                    m = (int)((mmap >> (4 * (bk[6] & 15))) & 15ull);
            }
            S.lat[v] = (uint8_t)m;
        });
        __syncthreads();
        const FdmResult r =
            fdm_solve(N, S, X, u ? u[c] : 0xffffffffu, P ? P + (size_t)c * 6 * N * N : nullptr, &sel);
        if (threadIdx.x == 0) {
            if (exit_out) exit_out[c] = r.exitnode;
            if (iters) iters[c] = r.inner | (r.outer << 24);
            if (!r.converged) atomicOr(err, ERR_FDM);
        }
        __syncthreads();
    }
}

size_t fdm_cube_scratch_bytes(int N) { return fdm_scratch_bytes(N); }

cudaError_t launch_fdm_cubes(int N, const int32_t *d_cubes, uint32_t n_cubes, const uint8_t *map, const double *eps,
                             const uint32_t *d_u, double *d_P, uint32_t *d_exit, uint32_t *d_iters,
                             unsigned char *scratch, int grid, uint32_t *d_err, cudaStream_t st)
{
    const int smem = (int)fdm_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(k_fdm_cubes, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    uint64_t mm = 0;
    for (int i = 0; i < 16; i++) mm |= (uint64_t)(map[i] & 15u) << (4 * i);
    k_fdm_cubes<<<grid, FDM_THREADS, smem, st>>>(N, d_cubes, n_cubes, mm, eps, d_u, d_P, d_exit, d_iters, scratch,
                                                  d_err);
    return cudaGetLastError();
}

cudaError_t set_kernel_attributes(int N, int mw_warps, int max_nc)
{
    (void)max_nc;
    cudaError_t e = cudaFuncSetAttribute(k_fill_one, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fill_smem_bytes(N));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mw<CubeSource>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mw_smem_bytes(N, mw_warps));
}

cudaError_t launch_fill_one(const EngineView &E, uint32_t kind, const uint32_t prof[4], uint32_t entry,
                            double *values_out, cudaStream_t st)
{
    k_fill_one<<<1, 256, fill_smem_bytes(E.N), st>>>(E, kind, make_uint4(prof[0], prof[1], prof[2], prof[3]),
                                                      entry, values_out);
    return cudaGetLastError();
}

cudaError_t launch_mw_cubes(int N, const int32_t *d_cubes, uint64_t n_cubes, uint64_t spc, uint32_t key0,
                            uint32_t key1, int n_mat, int n_global_mat, const uint8_t *map, const uint32_t *W, uint32_t *d_exit,
                            uint32_t *d_steps, unsigned long long *d_head, uint32_t *d_err,
                            const LaunchShape &L, cudaStream_t st)
{
    CubeSource src;
    src.err = d_err;
    src.cubes = d_cubes;
    src.n_cubes = n_cubes;
    src.spc = spc;
    src.total = n_cubes * spc;
    src.head = d_head;
    src.key0 = key0;
    src.key1 = key1;
    uint64_t mm = 0;
    for (int i = 0; i < 16; i++) mm |= (uint64_t)(map[i] & 15u) << (4 * i);
    src.mmap_lo = mm;
    src.d_exit = d_exit;
    src.d_steps = d_steps;
    src.N = N;
    src.n_mat = n_mat;
    src.lanes_table = n_global_mat <= 7 ? 1 : 0;   // columns 0-7 only: the per-lane table copies
    const uint64_t warps = (uint64_t)L.sms * L.mw_ctas_per_sm * L.mw_warps;
    src.chunk = (uint32_t)std::min<uint64_t>(MW_CHUNK, std::max<uint64_t>(32, src.total / (4 * std::max<uint64_t>(warps, 1))));
    const int threads = 32 * L.mw_warps;
    k_mw<CubeSource><<<L.sms * L.mw_ctas_per_sm, threads, mw_smem_bytes(N, L.mw_warps), st>>>(src, W, N);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Candidate lists of the uniform grid of the max-cube query (Sec. II-A), built
// on the device when a structure is loaded.  Cell c lists, in ascending order,
// every conductor box whose L-infinity distance to the cell (grown by 2 % of a
// cell on each side) is at most U + tol, U the smallest upper bound of the
// nearest-electrode distance over the grown cell (walls and boxes), so that the
// box nearest to any point of the cell, and every box tied with it, is listed.
// Pass 0 writes each cell's count into off[cell]; an exclusive scan turns the
// counts into offsets; pass 1 writes the lists.  The arithmetic is written out
// operation by operation (no contraction) in double precision.
__device__ __forceinline__ double dmin_rn(double a, double b) { return b < a ? b : a; }
__device__ __forceinline__ double dmax_rn(double a, double b) { return a < b ? b : a; }

__global__ void k_grid_lists(GridBuild G, uint32_t *off, uint16_t *ids, int pass)
{
    const uint32_t plane = (uint32_t)G.gdim[1] * (uint32_t)G.gdim[2];
    const uint32_t cells = (uint32_t)G.gdim[0] * plane;
    const uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= cells) return;
    const int ii[3] = {(int)(cell / plane), (int)((cell / (uint32_t)G.gdim[2]) % (uint32_t)G.gdim[1]),
                       (int)(cell % (uint32_t)G.gdim[2])};
    double lo[3], hi[3];
    double U = __longlong_as_double(0x7ff0000000000000ll);   // +inf
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double w = G.w[a], m = __dmul_rn(0.02, w);
        lo[a] = __dsub_rn(__dadd_rn(G.dlo[a], __dmul_rn((double)ii[a], w)), m);
        hi[a] = __dadd_rn(__dadd_rn(G.dlo[a], __dmul_rn((double)(ii[a] + 1), w)), m);
        U = dmin_rn(U, dmin_rn(__dsub_rn(hi[a], G.dlo[a]), __dsub_rn(G.dhi[a], lo[a])));
    }
    const int n = G.n_box;
    for (int k = 0; k < n; k++) {
        double dmax = 0.0;
#pragma unroll
        for (int a = 0; a < 3; a++)
            dmax = dmax_rn(dmax, dmax_rn(__dsub_rn(G.clo[a * n + k], lo[a]), __dsub_rn(hi[a], G.chi[a * n + k])));
        U = dmin_rn(U, dmax);
    }
    const double lim = __dadd_rn(U, G.tol);
    const uint32_t base = pass ? off[cell] : 0u;
    uint32_t c = 0;
    for (int k = 0; k < n; k++) {
        double dm = 0.0;
#pragma unroll
        for (int a = 0; a < 3; a++)
            dm = dmax_rn(dm, dmax_rn(__dsub_rn(G.clo[a * n + k], hi[a]), __dsub_rn(lo[a], G.chi[a * n + k])));
        if (dm <= lim) {
            if (pass) ids[base + c] = (uint16_t)k;
            c++;
        }
    }
    if (!pass) off[cell] = c;
}

// One CTA: a[0 .. n) (counts) -> exclusive prefix sums, a[n] = the total.
__global__ void k_scan_exclusive(uint32_t *a, uint32_t n)
{
    __shared__ uint32_t part[1024];
    const uint32_t t = threadIdx.x, nt = blockDim.x;
    const uint32_t chunk = (n + nt - 1) / nt;
    const uint32_t b = min(t * chunk, n), e = min(b + chunk, n);
    uint32_t s = 0;
    for (uint32_t i = b; i < e; i++) s += a[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        uint32_t acc = 0;
        for (uint32_t i = 0; i < nt; i++) {
            const uint32_t v = part[i];
            part[i] = acc;
            acc += v;
        }
        a[n] = acc;
    }
    __syncthreads();
    uint32_t acc = part[t];
    for (uint32_t i = b; i < e; i++) {
        const uint32_t v = a[i];
        a[i] = acc;
        acc += v;
    }
}

cudaError_t launch_grid_lists(const GridBuild &G, uint32_t *off, uint16_t *ids, int pass, cudaStream_t st)
{
    const uint64_t cells = (uint64_t)G.gdim[0] * G.gdim[1] * G.gdim[2];
    if (cells == 0 || cells >= (1ull << 31)) return cudaErrorInvalidValue;
    k_grid_lists<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(G, off, ids, pass);
    if (pass == 0) k_scan_exclusive<<<1, 1024, 0, st>>>(off, (uint32_t)cells);
    return cudaGetLastError();
}

}  // namespace frw

// ---------------------------------------------------------------------------
// Allocation-free MicroWalk entry point (see frw_microwalk_cubes_noalloc in frw.h).
// Its scratch lives in this fixed device array; host code only ever uses the
// address returned by cudaGetSymbolAddress for the current device.
#include <mutex>

#include "frw.h"

namespace frw {
namespace {

constexpr int NOALLOC_WORDS = 512;                   // 2 KB
constexpr int NOALLOC_W_OFFSET = 64;                 // weight table at word 64 (256 words)
static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_WORDS];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
uint32_t *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on `dev` (looked up once per device).
cudaError_t noalloc_scratch(int dev, uint32_t **out)
{
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace frw

extern "C" int frw_microwalk_cubes_noalloc(int32_t N, int32_t n_cubes, const int32_t *d_cubes, const double *eps_r,
                                           int32_t n_mat, uint64_t seed, uint64_t samples_per_cube,
                                           uint64_t request_id, uint32_t *d_exit, uint32_t *d_steps,
                                           void *cuda_stream)
{
    using namespace frw;
    if (N < 2 || N > FRW_MAX_N || (N & 1) || n_cubes < 0 || !eps_r || n_mat < 1) return FRW_EINVAL;
    if (n_mat > FRW_MAX_MATERIALS) return FRW_ECAPACITY;
    for (int i = 0; i < n_mat; i++)
        if (!(eps_r[i] > 0.0) || !std::isfinite(eps_r[i])) return FRW_EINVAL;
    if (n_cubes == 0 || samples_per_cube == 0) return FRW_OK;
    if (!d_cubes) return FRW_EINVAL;
    if (samples_per_cube > UINT64_MAX / (uint64_t)n_cubes) return FRW_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FRW_EDEVICE;
    uint32_t *scr = nullptr;
    if (noalloc_scratch(dev, &scr) != cudaSuccess) return FRW_EDEVICE;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // jump weights of Eq. 6, quantised as in the context path
    uint32_t W[256];
    for (int i = 0; i < 256; i++) W[i] = 0;
    for (int v = 0; v < n_mat; v++) {
        for (int i = 0; i < n_mat; i++) {
            const double al = eps_r[i] / (eps_r[i] + eps_r[v]);
            W[v * 16 + i] = (uint32_t)std::floor(al * 16777216.0 + 0.5);
        }
        W[v * 16 + BOUNDARY] = 16777216u;
    }
    uint8_t map[16];
    for (int i = 0; i < 16; i++) map[i] = (uint8_t)i;
    LaunchShape L;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return FRW_EDEVICE;
    L.sms = sms;
    L.mw_warps = 16;
    L.mw_ctas_per_sm = 2;
    L.geom_threads = 128;
    L.fill_ctas = sms;
    if (cudaFuncSetAttribute(k_mw<CubeSource>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mw_smem_bytes(N, L.mw_warps)) != cudaSuccess)
        return FRW_EDEVICE;
    // counter and error word start at zero; the weight table is rewritten every call
    if (cudaMemsetAsync(scr, 0, 4 * sizeof(uint32_t), st) != cudaSuccess) return FRW_EDEVICE;
    if (cudaMemcpyAsync(scr + NOALLOC_W_OFFSET, W, sizeof(W), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FRW_EDEVICE;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32) ^ (uint32_t)request_id;
    if (launch_mw_cubes(N, d_cubes, (uint64_t)n_cubes, samples_per_cube, key0, key1, n_mat, n_mat, map, scr + NOALLOC_W_OFFSET,
                        d_exit, d_steps, reinterpret_cast<unsigned long long *>(scr), scr + 2, L,
                        st) != cudaSuccess)
        return FRW_EDEVICE;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, scr + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FRW_EDEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FRW_EDEVICE;
    if (err & ERR_INPUT) return FRW_EINVAL;
    return err ? FRW_EDEVICE : FRW_OK;
}

namespace frw {
// CTAs of the walk kernel resident per SM at this lattice edge (2 by design at
// N = 24: at most 72 registers per thread and about 97 KB of shared memory each;
// one for the FDM comparator)
template <typename T, bool MWE, bool FDM> static int walk_occupancy(int smem)
{
    int n = 0;
    set_walk_attributes<T, MWE, FDM>(smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_walk<T, MWE, FDM>, WALK_THREADS, smem);
    return n;
}

uint32_t walk_stage_cap(const EngineView &E, int ctas_per_sm)
{
    if (!FRW_STAGE_GEOM || E.transition == 1 || E.geo_warps > 0 || ctas_per_sm < 1) return 0;
    cudaFuncAttributes fa;
    cudaError_t e;
    if (E.mwe > 1) e = E.fp32 ? cudaFuncGetAttributes(&fa, k_walk<float, true, false>) : cudaFuncGetAttributes(&fa, k_walk<double, true, false>);
    else e = E.fp32 ? cudaFuncGetAttributes(&fa, k_walk<float, false, false>) : cudaFuncGetAttributes(&fa, k_walk<double, false, false>);
    int dev = 0, per_sm = 0, per_block = 0, reserved = 0;
    if (e != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const long long base = (long long)stage_round16((uint32_t)walk_smem_bytes(E.N, E.max_nc, 0));
    // stay within the shared-memory carve-out the kernel needs without the copy
    // (the SM's supported capacities), so that the copy never takes L1 away
    const long long need0 = (long long)ctas_per_sm * ((long long)fa.sharedSizeBytes + base + reserved);
    static const int tiers_kb[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
    long long tier = per_sm;
    for (int kb : tiers_kb)
        if ((long long)kb * 1024 >= need0) {
            tier = std::min<long long>((long long)kb * 1024, per_sm);
            break;
        }
    const long long fit = std::min<long long>(tier / ctas_per_sm - reserved, per_block) -
                          (long long)fa.sharedSizeBytes - base;
    const long long cap = std::min<long long>(fit, 32 * 1024) / 128 * 128;
    if (cap <= 0) return 0u;
    // confirm with the occupancy calculator at the enlarged size
    const int smem = (int)(base + cap);
    int n = 0;
    if (E.mwe > 1) n = E.fp32 ? walk_occupancy<float, true, false>(smem) : walk_occupancy<double, true, false>(smem);
    else n = E.fp32 ? walk_occupancy<float, false, false>(smem) : walk_occupancy<double, false, false>(smem);
    cudaGetLastError();
    return n >= ctas_per_sm ? (uint32_t)cap : 0u;
}

int walk_ctas_per_sm(int N, int fp32, int mwe, int transition)
{
    const int smem = (int)walk_smem_bytes(N, 200, transition);
    int n;
    if (transition == 1)
        n = fp32 ? walk_occupancy<float, false, true>(smem) : walk_occupancy<double, false, true>(smem);
    else if (mwe > 1)
        n = fp32 ? walk_occupancy<float, true, false>(smem) : walk_occupancy<double, true, false>(smem);
    else
        n = fp32 ? walk_occupancy<float, false, false>(smem) : walk_occupancy<double, false, false>(smem);
    return n > 0 ? n : 1;
}
}  // namespace frw
