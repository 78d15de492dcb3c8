// fdm_transition.cuh -- FD-based transition (Algorithm 2, the FRW-FDM comparator)
// computed by one CTA per transition cube.  Included by frw_kernels.cu.
//
// The discrete SGF of Eq. 8 is P = e_c^T A_II^{-1} A_IB.  Multiplying row v of
// the FD equations (Eq. 6) by eps_v makes the system symmetric positive definite:
//   (S y)_v = sum over the six neighbours of  s_vw (y_v - y_w)   (interior w)
//                                          +  eps_v y_v          (boundary panel)
// with s_vw = eps_v eps_w / (eps_v + eps_w), and A_II^{-1} A_IB = S^{-1} S_IB, so
// P_b = eps_v y_v at the interior node v next to panel b, where S y = e_c (e_c
// averages the 8 central nodes, as MicroWalk's start).
//
// Solve: mixed-precision iterative refinement.  The outer loop keeps y in FP64
// (global scratch) and forms the residual r = e_c - S y in FP64; the inner loop
// solves S d = r approximately by Jacobi-preconditioned conjugate gradients in
// FP32 (dot products: FP32 per thread, the 256 partial sums added in FP64; the
// FP64 pipe of this GPU is too narrow for per-node FP64 work); y += d.  The inner vectors p, z = D^-1 r and d live
// in shared memory (r is carried as z and the diagonal D, recomputed with each
// stencil from the same neighbour lookups), so an inner iteration touches no
// global memory.  The outer loop stops when ||e_c - S y||_2 <=
// FDM_TOL ||e_c||_2.  The panel values eps_v y_v are then summed in natural face
// order (face 2a + side, then the other two axes in increasing order) and one
// panel is sampled with a 32-bit word u: the first panel whose threshold
// min(floor(2^32 cum / total), 2^32 - 1) exceeds u, the last panel otherwise.
#pragma once

constexpr int FDM_THREADS = 256;          // block of the stand-alone kernel (the solve works for any
                                          // multiple of 32 up to 1024: the walk kernel's block)
constexpr int FDM_MAX_OUTER = 12;
constexpr int FDM_MAX_INNER = 3000;
constexpr double FDM_TOL = 1e-12;         // outer stop, FP64 residual relative to ||e_c||_2
constexpr double FDM_INNER_TOL2 = 1e-10;  // inner stop, squared FP32 residual reduction

// dynamic shared memory: [sig64 256][sig32 256][red 64 doubles][lat N^3 (16-aligned)][p N^3][z N^3][d N^3]
__host__ __device__ inline size_t fdm_lat_bytes(int N) { return ((size_t)N * N * N + 15) & ~(size_t)15; }
__host__ __device__ inline size_t fdm_smem_bytes(int N)
{
    return 256 * sizeof(double) + 256 * sizeof(float) + 64 * sizeof(double) + fdm_lat_bytes(N) +
           3 * sizeof(float) * (size_t)N * N * N;
}
// global scratch per CTA: y (FP64)
__host__ __device__ inline size_t fdm_scratch_bytes(int N)
{
    return ((size_t)N * N * N * sizeof(double) + 255) & ~(size_t)255;
}

struct FdmSmem {
    double *sig64;     // [m][w], column BOUNDARY = eps_m
    float *sig32;
    double *red;       // reduction scratch
    uint8_t *lat;      // material id per voxel, natural order v = (i N + j) N + k
    float *p, *z, *d;
};

__device__ __forceinline__ FdmSmem fdm_smem(unsigned char *base, int N)
{
    FdmSmem S;
    S.sig64 = reinterpret_cast<double *>(base);
    S.sig32 = reinterpret_cast<float *>(base + 256 * sizeof(double));
    S.red = reinterpret_cast<double *>(base + 256 * sizeof(double) + 256 * sizeof(float));
    S.lat = base + 256 * sizeof(double) + 256 * sizeof(float) + 64 * sizeof(double);
    S.p = reinterpret_cast<float *>(S.lat + fdm_lat_bytes(N));
    S.z = S.p + (size_t)N * N * N;
    S.d = S.z + (size_t)N * N * N;
    return S;
}

struct FdmScratch {
    double *y;
};

__device__ __forceinline__ FdmScratch fdm_scratch(unsigned char *base, int)
{
    FdmScratch X;
    X.y = reinterpret_cast<double *>(base);
    return X;
}

// couplings of every material pair from the permittivity table (16 entries; ids
// with eps <= 0 are unused and get 0)
__device__ __forceinline__ void fdm_couplings(const FdmSmem &S, const double *__restrict__ eps)
{
    for (int e = threadIdx.x; e < 256; e += blockDim.x) {
        const int m = e >> 4, w = e & 15;
        const double em = eps[m], ew = eps[w];
        double s = 0.0;
        if (w == BOUNDARY) s = em > 0.0 ? em : 0.0;
        else if (em > 0.0 && ew > 0.0) s = __ddiv_rn(__dmul_rn(em, ew), __dadd_rn(em, ew));
        S.sig64[e] = s;
        S.sig32[e] = (float)s;
    }
}

// Nodes of this thread: v = tid + nt t (nt = the block size) with coordinates
// (i, j, k) kept by carries
struct FdmGrid {
    int N, NN, n3, nt;
    int di, dj, dk;    // nt written in base N
};

__device__ __forceinline__ FdmGrid fdm_grid(int N)
{
    FdmGrid G;
    G.N = N;
    G.NN = N * N;
    G.n3 = N * N * N;
    G.nt = (int)blockDim.x;
    G.dk = G.nt % N;
    G.dj = (G.nt / N) % N;
    G.di = G.nt / G.NN;
    return G;
}

template <class F> __device__ __forceinline__ void fdm_nodes(const FdmGrid &G, F f)
{
    int v = threadIdx.x;
    int i = v / G.NN, j = (v / G.N) % G.N, k = v % G.N;
    for (; v < G.n3; v += G.nt) {
        f(v, i, j, k);
        k += G.dk;
        if (k >= G.N) { k -= G.N; j++; }
        j += G.dj;
        if (j >= G.N) { j -= G.N; i++; }
        i += G.di;
    }
}

// (S y)_v, neighbours in the order -x, +x, -y, +y, -z, +z
template <typename R>
__device__ __forceinline__ R fdm_apply(const FdmGrid &G, const uint8_t *lat, const R *sig, const R *y, int v, int i,
                                       int j, int k)
{
    const int m = lat[v];
    const R *row = sig + m * 16;
    const R yv = y[v], eb = row[BOUNDARY];
    R acc = R(0);
    acc += (i > 0) ? row[lat[v - G.NN]] * (yv - y[v - G.NN]) : eb * yv;
    acc += (i < G.N - 1) ? row[lat[v + G.NN]] * (yv - y[v + G.NN]) : eb * yv;
    acc += (j > 0) ? row[lat[v - G.N]] * (yv - y[v - G.N]) : eb * yv;
    acc += (j < G.N - 1) ? row[lat[v + G.N]] * (yv - y[v + G.N]) : eb * yv;
    acc += (k > 0) ? row[lat[v - 1]] * (yv - y[v - 1]) : eb * yv;
    acc += (k < G.N - 1) ? row[lat[v + 1]] * (yv - y[v + 1]) : eb * yv;
    return acc;
}

// diagonal of S at v (sum of the six couplings)
template <typename R>
__device__ __forceinline__ R fdm_diag(const FdmGrid &G, const uint8_t *lat, const R *sig, int v, int i, int j, int k)
{
    const int m = lat[v];
    const R *row = sig + m * 16;
    const R eb = row[BOUNDARY];
    R acc = R(0);
    acc += (i > 0) ? row[lat[v - G.NN]] : eb;
    acc += (i < G.N - 1) ? row[lat[v + G.NN]] : eb;
    acc += (j > 0) ? row[lat[v - G.N]] : eb;
    acc += (j < G.N - 1) ? row[lat[v + G.N]] : eb;
    acc += (k > 0) ? row[lat[v - 1]] : eb;
    acc += (k < G.N - 1) ? row[lat[v + 1]] : eb;
    return acc;
}

// (S y)_v and the diagonal at v from one set of neighbour lookups (FP32)
__device__ __forceinline__ float fdm_apply_diag(const FdmGrid &G, const uint8_t *lat, const float *sig, const float *y,
                                                int v, int i, int j, int k, float &dg)
{
    const int m = lat[v];
    const float *row = sig + m * 16;
    const float yv = y[v], eb = row[BOUNDARY];
    const float s0 = (i > 0) ? row[lat[v - G.NN]] : eb;
    const float s1 = (i < G.N - 1) ? row[lat[v + G.NN]] : eb;
    const float s2 = (j > 0) ? row[lat[v - G.N]] : eb;
    const float s3 = (j < G.N - 1) ? row[lat[v + G.N]] : eb;
    const float s4 = (k > 0) ? row[lat[v - 1]] : eb;
    const float s5 = (k < G.N - 1) ? row[lat[v + 1]] : eb;
    float acc = 0.0f;
    acc += s0 * ((i > 0) ? yv - y[v - G.NN] : yv);
    acc += s1 * ((i < G.N - 1) ? yv - y[v + G.NN] : yv);
    acc += s2 * ((j > 0) ? yv - y[v - G.N] : yv);
    acc += s3 * ((j < G.N - 1) ? yv - y[v + G.N] : yv);
    acc += s4 * ((k > 0) ? yv - y[v - 1] : yv);
    acc += s5 * ((k < G.N - 1) ? yv - y[v + 1] : yv);
    dg = ((((s0 + s1) + s2) + s3) + s4) + s5;
    return acc;
}

// CTA-wide sums in a fixed order (warp butterflies, then the warp totals in
// order): every thread gets the same value
__device__ __forceinline__ double fdm_warp_sum(double a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(FULL_MASK, a, o);
    return a;
}

__device__ __forceinline__ double2 fdm_block_sum2(double a, double b, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = fdm_warp_sum(a);
    b = fdm_warp_sum(b);
    __syncthreads();   // earlier readers of red are done
    if (lane == 0) {
        red[warp] = a;
        red[32 + warp] = b;
    }
    __syncthreads();
    double sa = 0.0, sb = 0.0;
    const int nw = (int)(blockDim.x >> 5);
    for (int w = 0; w < nw; w++) {
        sa += red[w];
        sb += red[32 + w];
    }
    return make_double2(sa, sb);
}

__device__ __forceinline__ bool fdm_is_centre(int N, int i, int j, int k)
{
    const int c = N / 2 - 1;
    return (unsigned)(i - c) < 2u && (unsigned)(j - c) < 2u && (unsigned)(k - c) < 2u;
}

// interior node next to panel m (natural face order) and the panel's boundary node
__device__ __forceinline__ int fdm_panel(int N, int m, int node[3])
{
    const int f = m / (N * N), rem = m - f * N * N;
    const int u = rem / N, w = rem - u * N;
    const int a = f >> 1, side = f & 1;
    const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
    int c[3];
    c[a] = side ? N - 1 : 0;
    c[o1] = u;
    c[o2] = w;
    node[a] = side ? N : -1;
    node[o1] = u;
    node[o2] = w;
    return (c[0] * N + c[1]) * N + c[2];
}

struct FdmResult {
    uint32_t exitnode;   // packed (x+1) | (y+1) << 8 | (z+1) << 16
    uint32_t inner, outer;
    bool converged;
};

// Solve and sample for the lattice already in S.lat (all threads of the CTA
// call this; the couplings must be in S.sig*).  P_out (may be null) receives the
// 6 N^2 panel values.  sel is a shared word used for the sampled panel.
__device__ FRW_OUTLINE FdmResult fdm_solve(int N, const FdmSmem &S, const FdmScratch &X, uint32_t u, double *P_out,
                                           uint32_t *sel)
{
    const FdmGrid G = fdm_grid(N);
    const int tid = threadIdx.x;
    fdm_nodes(G, [&](int v, int, int, int) { X.y[v] = 0.0; });
    __syncthreads();
    const double bnorm2 = 8.0 * 0.125 * 0.125;
    FdmResult res;
    res.inner = 0;
    res.outer = 0;
    res.converged = false;
    for (; res.outer < (uint32_t)FDM_MAX_OUTER; res.outer++) {
        // FP64 residual of the current y; the inner solve starts from z = D^-1 r, p = z, d = 0
        double rr = 0.0, rz = 0.0;
        fdm_nodes(G, [&](int v, int i, int j, int k) {
            const double b = fdm_is_centre(N, i, j, k) ? 0.125 : 0.0;
            const double rv = b - fdm_apply<double>(G, S.lat, S.sig64, X.y, v, i, j, k);
            const float z = (float)rv / fdm_diag<float>(G, S.lat, S.sig32, v, i, j, k);
            S.z[v] = z;
            S.p[v] = z;
            S.d[v] = 0.0f;
            rr += rv * rv;
            rz += rv * (double)z;
        });
        const double2 s0 = fdm_block_sum2(rr, rz, S.red);
        rr = s0.x;
        rz = s0.y;
        if (rr <= FDM_TOL * FDM_TOL * bnorm2) {
            res.converged = true;
            break;
        }
        // FP32 Jacobi-preconditioned CG on S d = r
        for (int it = 0; it < FDM_MAX_INNER && rz > 0.0; it++) {
            float pq_t = 0.0f;
            fdm_nodes(G, [&](int v, int i, int j, int k) {
                pq_t += S.p[v] * fdm_apply<float>(G, S.lat, S.sig32, S.p, v, i, j, k);
            });
            const double pq = fdm_block_sum2((double)pq_t, 0.0, S.red).x;
            res.inner++;
            if (!(pq > 0.0)) break;
            const float alpha = (float)(rz / pq);
            float rn_t = 0.0f, rz_t = 0.0f;
            fdm_nodes(G, [&](int v, int i, int j, int k) {
                float dg;
                const float q = fdm_apply_diag(G, S.lat, S.sig32, S.p, v, i, j, k, dg);
                const float rv = dg * S.z[v] - alpha * q;
                const float z = rv / dg;
                S.d[v] += alpha * S.p[v];
                S.z[v] = z;
                rn_t += rv * rv;
                rz_t += rv * z;
            });
            const double2 s2 = fdm_block_sum2((double)rn_t, (double)rz_t, S.red);
            if (s2.x <= FDM_INNER_TOL2 * rr) break;
            const float beta = (float)(s2.y / rz);
            rz = s2.y;
            fdm_nodes(G, [&](int v, int, int, int) { S.p[v] = S.z[v] + beta * S.p[v]; });
            __syncthreads();
        }
        fdm_nodes(G, [&](int v, int, int, int) { X.y[v] += (double)S.d[v]; });
        __syncthreads();
    }
    // panel values eps_v y_v, prefix sums over contiguous chunks of panels
    const int P = 6 * N * N;
    const int nt = (int)blockDim.x;
    const int chunk = (P + nt - 1) / nt;
    const int m0 = min(tid * chunk, P), m1 = min(m0 + chunk, P);
    double loc = 0.0;
    for (int m = m0; m < m1; m++) {
        int node[3];
        const int v = fdm_panel(N, m, node);
        const double val = S.sig64[S.lat[v] * 16 + BOUNDARY] * X.y[v];
        if (P_out) P_out[m] = val;
        loc += val;
    }
    // exclusive scan of the chunk sums (inclusive warp scan, then warp offsets)
    const int lane = tid & 31, warp = tid >> 5;
    double inc = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();
    if (lane == 31) S.red[warp] = inc;
    if (tid == 0) *sel = (uint32_t)(P - 1);
    __syncthreads();
    double off = 0.0, total = 0.0;
    for (int w = 0; w < nt / 32; w++) {
        if (w < warp) off += S.red[w];
        total += S.red[w];
    }
    double cum = off + (inc - loc);
    for (int m = m0; m < m1 && m < P - 1; m++) {
        int node[3];
        const int v = fdm_panel(N, m, node);
        cum += S.sig64[S.lat[v] * 16 + BOUNDARY] * X.y[v];
        double t = floor(__dmul_rn(__ddiv_rn(cum, total), 4294967296.0));
        if (t > 4294967295.0) t = 4294967295.0;
        if (t < 0.0) t = 0.0;
        if (u < (uint32_t)t) {
            atomicMin(sel, (uint32_t)m);
            break;
        }
    }
    __syncthreads();
    int node[3];
    fdm_panel(N, (int)*sel, node);
    res.exitnode = (uint32_t)(node[0] + 1) | ((uint32_t)(node[1] + 1) << 8) | ((uint32_t)(node[2] + 1) << 16);
    __syncthreads();   // *sel may be reused
    return res;
}
