// sph_pairs.cu -- the cell-linked-list density and force loops (paper Section 2.1 steps 1-2).
//
// One CTA per cell (the paper's per-cell compute kernel, Section 2.1 / 2.3): the cell's particles are the local
// set, the particles of its 3^3 vertex-connected neighbour cells (periodic wrap) the active set.  Loop order is
// local-active (Section 5.4): every local particle gathers its sum, so there are no atomics on results.  Pair
// symmetry is not exploited (Section 5.3): every ordered pair is evaluated once from each side.
//
// Per CTA:
//   1. a 27-entry neighbour table (first slot, count, running prefix, periodic shift) in shared memory;
//   2. the active set is staged through shared memory in tiles of TJ particles (only the SoA members the
//      loop body reads);
//   3. each warp takes one local particle i at a time: its 32 lanes sweep the staged tile with a cheap FP32
//      distance test, the survivors are compacted into a per-warp queue (ballot + popc), and whenever 32 are
//      queued the lanes evaluate the full pair term in the path's precision, one pair per lane, with the exact
//      support test applied as a mask (the neutral-element formulation of Section 5.6: out-of-support pairs
//      contribute zero, no per-pair branch decides whether a term is summed);
//   4. the warp's per-lane partial sums are combined by a shuffle tree and added to the particle's
//      shared-memory accumulator; after the last tile each accumulator is finalised and written to the SoA.
// The compaction keeps the expensive pair evaluation at ~90 % lane occupancy although only ~14 % of the
// 3^3-stencil candidates lie inside the support (cell edge 2h).
//
// FP64 path: positions are the FP64 members; x_i - x_j gets the periodic shift (+-box) of j's cell exactly as a
// minimum-image wrap would.  The FP32 filter uses cell-relative float copies of the positions (k_pos32) with a
// conservative radius, so it never drops a pair the FP64 test keeps.
// FP32 path: positions are cell-relative floats (the FP32 view), so x_i - x_j = r_i - (r_j + d * edge) with d the
// neighbour cell offset; the filter is the exact test; all sums are Kahan-compensated.
#include <math.h>

#include "sph_internal.cuh"

namespace sphk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPairThreads = 128;
constexpr int kPairWarps = kPairThreads / 32;
constexpr int kMaxLocal = 128;

struct NbrTable {
    int start[27];
    int pref[28];
    double shift[27][3];  // added to x_i - x_j for a j of neighbour q (0 or +-box)
    float offf[27][3];    // origin of neighbour cell q relative to the local cell origin: (float)(d * edge)
    int wrap;             // any shift != 0
};

__device__ __forceinline__ void build_nbr_table(NbrTable &nb, int c, const Grid &g, const int *cell_start)
{
    const int tid = threadIdx.x;
    const int kc[3] = {c % g.n[0], (c / g.n[0]) % g.n[1], c / (g.n[0] * g.n[1])};
    if (tid == 0) nb.wrap = 0;
    __syncthreads();
    if (tid < 27) {
        const int d[3] = {tid % 3 - 1, (tid / 3) % 3 - 1, tid / 9 - 1};
        int kk[3];
        bool valid = true;
        bool wr = false;
        for (int a = 0; a < 3; ++a) {
            int k = kc[a] + d[a];
            double s = 0.0;
            if (k < 0) {
                if (g.periodic) {
                    k += g.n[a];
                    s = g.box[a];
                } else {
                    valid = false;
                }
            } else if (k >= g.n[a]) {
                if (g.periodic) {
                    k -= g.n[a];
                    s = -g.box[a];
                } else {
                    valid = false;
                }
            }
            kk[a] = k;
            nb.shift[tid][a] = s;
            nb.offf[tid][a] = __double2float_rn((double)d[a] * g.edge[a]);
            wr = wr || (s != 0.0);
        }
        int cnt = 0, st = 0;
        if (valid) {
            const int c2 = kk[0] + g.n[0] * (kk[1] + g.n[1] * kk[2]);
            st = cell_start[c2];
            cnt = cell_start[c2 + 1] - st;
        }
        nb.start[tid] = st;
        nb.pref[tid + 1] = cnt;  // counts, turned into a prefix below
        if (wr && cnt > 0) atomicOr(&nb.wrap, 1);
    }
    __syncthreads();
    if (tid == 0) {
        nb.pref[0] = 0;
        for (int q = 0; q < 27; ++q) nb.pref[q + 1] += nb.pref[q];
    }
    __syncthreads();
}

// Neighbour index q with pref[q] <= jj < pref[q+1] (empty neighbours have pref[q] == pref[q+1]).
__device__ __forceinline__ int find_nbr(const NbrTable &nb, int jj)
{
    int lo = 0, hi = 27;  // invariant: pref[lo] <= jj < pref[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (nb.pref[mid] <= jj) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Kahan accumulator (FP32 path): value = s - c.
struct Kahan {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float y)
    {
        const float yy = __fsub_rn(y, c);
        const float t = __fadd_rn(s, yy);
        c = __fsub_rn(__fsub_rn(t, s), yy);
        s = t;
    }
    // Combine with another compensated sum (TwoSum of the heads, compensations added).
    __device__ __forceinline__ void merge(float s2, float c2)
    {
        const float t = __fadd_rn(s, s2);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
        c = __fsub_rn(__fadd_rn(c, c2), err);
        s = t;
    }
    __device__ __forceinline__ void warp_reduce()
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_xor_sync(kFull, s, o);
            const float c2 = __shfl_xor_sync(kFull, c, o);
            merge(s2, c2);
        }
    }
};

// ------------------------------------------------------------------------------------------------------------
// Loop bodies
// ------------------------------------------------------------------------------------------------------------
struct PairCommon {
    const int *cell_start;
    Grid g;
    unsigned *status;
    Counters *counters;
    int tj;  // staged particles per tile
};

// ---- density, FP64 ----
struct DensF64 {
    struct Args {
        PairCommon cm;
        const double *x, *y, *z, *m, *h, *u;
        const float *xf, *yf, *zf;  // cell-relative float positions (filter only)
        double *rho, *P, *cs;
        double gamma;
    };
    struct Tile {
        double *x, *y, *z, *m;
        float *fx, *fy, *fz;
        unsigned char *q;
    };
    struct Lhs {
        double x, y, z, h, hinv;
        float fx, fy, fz, b2;
    };
    struct Part {
        double rho;
        __device__ __forceinline__ void zero() { rho = 0.0; }
        __device__ __forceinline__ void reduce() { rho = warp_sum(rho); }
    };
    using Acc = double;
    static constexpr int kStageBytes = 4 * 8 + 3 * 4 + 1;

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        t.x = reinterpret_cast<double *>(s);
        t.y = t.x + tj;
        t.z = t.y + tj;
        t.m = t.z + tj;
        t.fx = reinterpret_cast<float *>(t.m + tj);
        t.fy = t.fx + tj;
        t.fz = t.fy + tj;
        t.q = reinterpret_cast<unsigned char *>(t.fz + tj);
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        T.x[t] = A.x[slot];
        T.y[t] = A.y[slot];
        T.z[t] = A.z[slot];
        T.m[t] = A.m[slot];
        T.fx[t] = A.xf[slot] + nb.offf[q][0];
        T.fy[t] = A.yf[slot] + nb.offf[q][1];
        T.fz[t] = A.zf[slot] + nb.offf[q][2];
        T.q[t] = (unsigned char)q;
    }
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float margin)
    {
        Lhs L;
        L.x = A.x[i];
        L.y = A.y[i];
        L.z = A.z[i];
        L.h = A.h[i];
        L.hinv = 1.0 / L.h;
        L.fx = A.xf[i];
        L.fy = A.yf[i];
        L.fz = A.zf[i];
        const float rf = __fmaf_ru(2.0f * (1.0f + 4e-6f), __double2float_ru(L.h), margin);
        L.b2 = __fmul_ru(rf, rf);
        return L;
    }
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float dx = L.fx - T.fx[k], dy = L.fy - T.fy[k], dz = L.fz - T.fz[k];
        return dx * dx + dy * dy + dz * dz < L.b2;
    }
    static __device__ __forceinline__ bool eval(const Args &, const Lhs &L, const Tile &T, const NbrTable &nb,
                                                bool wrap, int, int k, Part &P)
    {
        double dx = L.x - T.x[k], dy = L.y - T.y[k], dz = L.z - T.z[k];
        if (wrap) {
            const int q = T.q[k];
            dx += nb.shift[q][0];
            dy += nb.shift[q][1];
            dz += nb.shift[q][2];
        }
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double q = sqrt(r2) * L.hinv;
        const double w1 = fma(q * q, fma(0.75, q, -1.5), 1.0);
        const double t = 2.0 - q;
        const double w2 = 0.25 * (t * t * t);
        const double w = (q < 1.0) ? w1 : ((q < 2.0) ? w2 : 0.0);
        P.rho = fma(T.m[k], w, P.rho);
        return q < 2.0;
    }
    static __device__ __forceinline__ void accumulate(Acc &a, const Part &P) { a += P.rho; }
    static __device__ __forceinline__ void finish(const Args &A, int i, const Acc &a)
    {
        const double h = A.h[i];
        const double hinv = 1.0 / h;
        const double rho = a * (kInvPi * hinv * hinv * hinv);
        const double P = (A.gamma - 1.0) * rho * A.u[i];
        const double cs = sqrt(A.gamma * P / rho);
        A.rho[i] = rho;
        A.P[i] = P;
        A.cs[i] = cs;
        unsigned bits = 0;
        if (!(rho > 0.0) || !isfinite(rho) || !isfinite(P) || !isfinite(cs)) bits |= SPH_DEV_NONFINITE;
        if (!(2.0 * h <= A.cm.g.min_edge)) bits |= SPH_DEV_H_TOO_BIG;
        if (bits) atomicOr(A.cm.status, bits);
    }
    static __device__ __forceinline__ void count(const Args &A, unsigned long long cand,
                                                 unsigned long long pairs)
    {
        atomicAdd(&A.cm.counters->dens_cand, cand);
        atomicAdd(&A.cm.counters->dens_pairs, pairs);
    }
};

// ---- density, FP32 (cell-relative float positions, Kahan sums) ----
struct DensF32 {
    struct Args {
        PairCommon cm;
        const float *x, *y, *z, *m, *h, *u;
        float *rho, *P, *cs;
        float gamma;
    };
    struct Tile {
        float *x, *y, *z, *m;
    };
    struct Lhs {
        float x, y, z, h, hinv, b2;
    };
    struct Part {
        Kahan rho;
        __device__ __forceinline__ void zero() { rho.zero(); }
        __device__ __forceinline__ void reduce() { rho.warp_reduce(); }
    };
    using Acc = float2;  // (s, c)
    static constexpr int kStageBytes = 4 * 4;

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        t.x = reinterpret_cast<float *>(s);
        t.y = t.x + tj;
        t.z = t.y + tj;
        t.m = t.z + tj;
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        T.x[t] = A.x[slot] + nb.offf[q][0];
        T.y[t] = A.y[slot] + nb.offf[q][1];
        T.z[t] = A.z[slot] + nb.offf[q][2];
        T.m[t] = A.m[slot];
    }
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float)
    {
        Lhs L;
        L.x = A.x[i];
        L.y = A.y[i];
        L.z = A.z[i];
        L.h = A.h[i];
        L.hinv = __frcp_rn(L.h);
        L.b2 = 4.0f * L.h * L.h;
        return L;
    }
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float dx = L.x - T.x[k], dy = L.y - T.y[k], dz = L.z - T.z[k];
        return dx * dx + dy * dy + dz * dz < L.b2;
    }
    static __device__ __forceinline__ bool eval(const Args &, const Lhs &L, const Tile &T, const NbrTable &,
                                                bool, int, int k, Part &P)
    {
        const float dx = L.x - T.x[k], dy = L.y - T.y[k], dz = L.z - T.z[k];
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float q = sqrtf(r2) * L.hinv;
        const float w1 = fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f);
        const float t = 2.0f - q;
        const float w2 = 0.25f * (t * t * t);
        const float w = (q < 1.0f) ? w1 : ((q < 2.0f) ? w2 : 0.0f);
        P.rho.add(T.m[k] * w);
        return q < 2.0f;
    }
    static __device__ __forceinline__ void accumulate(Acc &a, const Part &P)
    {
        Kahan k;
        k.s = a.x;
        k.c = a.y;
        k.merge(P.rho.s, P.rho.c);
        a.x = k.s;
        a.y = k.c;
    }
    static __device__ __forceinline__ void finish(const Args &A, int i, const Acc &a)
    {
        const float h = A.h[i];
        const float hinv = __frcp_rn(h);
        const float rho = __fsub_rn(a.x, a.y) * ((float)kInvPi * hinv * hinv * hinv);
        const float P = (A.gamma - 1.0f) * rho * A.u[i];
        const float cs = sqrtf(A.gamma * P / rho);
        A.rho[i] = rho;
        A.P[i] = P;
        A.cs[i] = cs;
        unsigned bits = 0;
        if (!(rho > 0.0f) || !isfinite(rho) || !isfinite(P) || !isfinite(cs)) bits |= SPH_DEV_NONFINITE;
        // h is the float cast of the record's h (at most half an ulp above it): allow that rounding
        if (!(2.0 * (double)h <= A.cm.g.min_edge * (1.0 + 2.4e-7))) bits |= SPH_DEV_H_TOO_BIG;
        if (bits) atomicOr(A.cm.status, bits);
    }
    static __device__ __forceinline__ void count(const Args &A, unsigned long long cand,
                                                 unsigned long long pairs)
    {
        atomicAdd(&A.cm.counters->dens_cand, cand);
        atomicAdd(&A.cm.counters->dens_pairs, pairs);
    }
};

// ---- force, FP64 ----
struct ForceF64 {
    struct Args {
        PairCommon cm;
        const double *x, *y, *z, *vx, *vy, *vz, *m, *h, *rho, *cs;
        const double *hinv, *k5, *A;      // derived per particle (k_force_prep)
        const float *xf, *yf, *zf, *hf;  // filter copies
        double *ax, *ay, *az, *dudt;
        double alpha, beta, eps;
    };
    struct Tile {
        double *x, *y, *z, *vx, *vy, *vz, *m, *h, *hinv, *k5, *A, *c, *rho;
        float *fx, *fy, *fz, *fh;
        int *slot;
        unsigned char *q;
    };
    struct Lhs {
        double x, y, z, vx, vy, vz, h, hinv, k5, A, c, rho;
        float fx, fy, fz, fh, margin;
    };
    struct Part {
        double ax, ay, az, du;
        __device__ __forceinline__ void zero() { ax = ay = az = du = 0.0; }
        __device__ __forceinline__ void reduce()
        {
            ax = warp_sum(ax);
            ay = warp_sum(ay);
            az = warp_sum(az);
            du = warp_sum(du);
        }
    };
    struct Acc {
        double ax, ay, az, du;
    };
    static constexpr int kStageBytes = 13 * 8 + 4 * 4 + 4 + 1;

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        double *d = reinterpret_cast<double *>(s);
        t.x = d;
        t.y = d + tj;
        t.z = d + 2 * tj;
        t.vx = d + 3 * tj;
        t.vy = d + 4 * tj;
        t.vz = d + 5 * tj;
        t.m = d + 6 * tj;
        t.h = d + 7 * tj;
        t.hinv = d + 8 * tj;
        t.k5 = d + 9 * tj;
        t.A = d + 10 * tj;
        t.c = d + 11 * tj;
        t.rho = d + 12 * tj;
        float *f = reinterpret_cast<float *>(d + 13 * tj);
        t.fx = f;
        t.fy = f + tj;
        t.fz = f + 2 * tj;
        t.fh = f + 3 * tj;
        t.slot = reinterpret_cast<int *>(f + 4 * tj);
        t.q = reinterpret_cast<unsigned char *>(t.slot + tj);
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        T.x[t] = A.x[slot];
        T.y[t] = A.y[slot];
        T.z[t] = A.z[slot];
        T.vx[t] = A.vx[slot];
        T.vy[t] = A.vy[slot];
        T.vz[t] = A.vz[slot];
        T.m[t] = A.m[slot];
        T.h[t] = A.h[slot];
        T.hinv[t] = A.hinv[slot];
        T.k5[t] = A.k5[slot];
        T.A[t] = A.A[slot];
        T.c[t] = A.cs[slot];
        T.rho[t] = A.rho[slot];
        T.fx[t] = A.xf[slot] + nb.offf[q][0];
        T.fy[t] = A.yf[slot] + nb.offf[q][1];
        T.fz[t] = A.zf[slot] + nb.offf[q][2];
        T.fh[t] = A.hf[slot];
        T.slot[t] = slot;
        T.q[t] = (unsigned char)q;
    }
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float margin)
    {
        Lhs L;
        L.x = A.x[i];
        L.y = A.y[i];
        L.z = A.z[i];
        L.vx = A.vx[i];
        L.vy = A.vy[i];
        L.vz = A.vz[i];
        L.h = A.h[i];
        L.hinv = A.hinv[i];
        L.k5 = A.k5[i];
        L.A = A.A[i];
        L.c = A.cs[i];
        L.rho = A.rho[i];
        L.fx = A.xf[i];
        L.fy = A.yf[i];
        L.fz = A.zf[i];
        L.fh = A.hf[i];
        L.margin = margin;
        return L;
    }
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float dx = L.fx - T.fx[k], dy = L.fy - T.fy[k], dz = L.fz - T.fz[k];
        const float rf = __fmaf_ru(2.0f * (1.0f + 4e-6f), fmaxf(L.fh, T.fh[k]), L.margin);
        return dx * dx + dy * dy + dz * dz < __fmul_ru(rf, rf);
    }
    static __device__ __forceinline__ bool eval(const Args &A, const Lhs &L, const Tile &T, const NbrTable &nb,
                                                bool wrap, int i, int k, Part &P)
    {
        double dx = L.x - T.x[k], dy = L.y - T.y[k], dz = L.z - T.z[k];
        if (wrap) {
            const int q = T.q[k];
            dx += nb.shift[q][0];
            dy += nb.shift[q][1];
            dz += nb.shift[q][2];
        }
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double hj = T.h[k];
        const double hm = fmax(L.h, hj);
        const bool in = (r2 < 4.0 * hm * hm) && (T.slot[k] != i) && (r2 > 0.0);
        const double rinv = rsqrt(in ? r2 : 1.0);
        const double r = r2 * rinv;
        const double qi = r * L.hinv, qj = r * T.hinv[k];
        const double ti = 2.0 - qi, tj = 2.0 - qj;
        // g(q) = f'(q)/q; on the outer piece 1/q = h/r
        const double gi = (qi < 1.0) ? fma(2.25, qi, -3.0) : ((qi < 2.0) ? (-0.75 * ti * ti) * (L.h * rinv) : 0.0);
        const double gj = (qj < 1.0) ? fma(2.25, qj, -3.0) : ((qj < 2.0) ? (-0.75 * tj * tj) * (hj * rinv) : 0.0);
        const double Fi = L.k5 * gi, Fj = T.k5[k] * gj;  // grad_i W(r_ij, h) = F r_ij
        const double dvx = L.vx - T.vx[k], dvy = L.vy - T.vy[k], dvz = L.vz - T.vz[k];
        const double vdotr = dvx * dx + dvy * dy + dvz * dz;
        double visc = 0.0;
        if (in && vdotr < 0.0) {
            const double hb = 0.5 * (L.h + hj);
            const double D1 = fma(A.eps * hb, hb, r2);   // r^2 + eps hbar^2
            const double D2 = 0.5 * (L.rho + T.rho[k]);  // rhobar
            const double rr = 1.0 / (D1 * D2);
            const double mu = hb * vdotr * (D2 * rr);
            const double cb = 0.5 * (L.c + T.c[k]);
            visc = mu * fma(A.beta, mu, -A.alpha * cb) * (D1 * rr);
        }
        const double Fb = 0.5 * (Fi + Fj);
        const double mj = T.m[k];
        const double aF = L.A * Fi;
        double coef = mj * (aF + T.A[k] * Fj + visc * Fb);
        double dcoef = mj * (aF + 0.5 * visc * Fb) * vdotr;
        if (!in) {
            coef = 0.0;
            dcoef = 0.0;
        }
        P.ax = fma(-coef, dx, P.ax);
        P.ay = fma(-coef, dy, P.ay);
        P.az = fma(-coef, dz, P.az);
        P.du += dcoef;
        return in;
    }
    static __device__ __forceinline__ void accumulate(Acc &a, const Part &P)
    {
        a.ax += P.ax;
        a.ay += P.ay;
        a.az += P.az;
        a.du += P.du;
    }
    static __device__ __forceinline__ void finish(const Args &A, int i, const Acc &a)
    {
        A.ax[i] = a.ax;
        A.ay[i] = a.ay;
        A.az[i] = a.az;
        A.dudt[i] = a.du;
        if (!isfinite(a.ax) || !isfinite(a.ay) || !isfinite(a.az) || !isfinite(a.du))
            atomicOr(A.cm.status, SPH_DEV_NONFINITE);
    }
    static __device__ __forceinline__ void count(const Args &A, unsigned long long cand,
                                                 unsigned long long pairs)
    {
        atomicAdd(&A.cm.counters->force_cand, cand);
        atomicAdd(&A.cm.counters->force_pairs, pairs);
    }
};

// ---- force, FP32 ----
struct ForceF32 {
    struct Args {
        PairCommon cm;
        const float *x, *y, *z, *vx, *vy, *vz, *m, *h, *rho, *cs;
        const float *hinv, *k5, *A;
        float *ax, *ay, *az, *dudt;
        float alpha, beta, eps;
    };
    struct Tile {
        float *x, *y, *z, *vx, *vy, *vz, *m, *h, *hinv, *k5, *A, *c, *rho;
        int *slot;
    };
    struct Lhs {
        float x, y, z, vx, vy, vz, h, hinv, k5, A, c, rho;
    };
    struct Part {
        Kahan ax, ay, az, du;
        __device__ __forceinline__ void zero()
        {
            ax.zero();
            ay.zero();
            az.zero();
            du.zero();
        }
        __device__ __forceinline__ void reduce()
        {
            ax.warp_reduce();
            ay.warp_reduce();
            az.warp_reduce();
            du.warp_reduce();
        }
    };
    struct Acc {
        float2 ax, ay, az, du;
    };
    static constexpr int kStageBytes = 13 * 4 + 4;

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        float *f = reinterpret_cast<float *>(s);
        t.x = f;
        t.y = f + tj;
        t.z = f + 2 * tj;
        t.vx = f + 3 * tj;
        t.vy = f + 4 * tj;
        t.vz = f + 5 * tj;
        t.m = f + 6 * tj;
        t.h = f + 7 * tj;
        t.hinv = f + 8 * tj;
        t.k5 = f + 9 * tj;
        t.A = f + 10 * tj;
        t.c = f + 11 * tj;
        t.rho = f + 12 * tj;
        t.slot = reinterpret_cast<int *>(f + 13 * tj);
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        T.x[t] = A.x[slot] + nb.offf[q][0];
        T.y[t] = A.y[slot] + nb.offf[q][1];
        T.z[t] = A.z[slot] + nb.offf[q][2];
        T.vx[t] = A.vx[slot];
        T.vy[t] = A.vy[slot];
        T.vz[t] = A.vz[slot];
        T.m[t] = A.m[slot];
        T.h[t] = A.h[slot];
        T.hinv[t] = A.hinv[slot];
        T.k5[t] = A.k5[slot];
        T.A[t] = A.A[slot];
        T.c[t] = A.cs[slot];
        T.rho[t] = A.rho[slot];
        T.slot[t] = slot;
    }
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float)
    {
        Lhs L;
        L.x = A.x[i];
        L.y = A.y[i];
        L.z = A.z[i];
        L.vx = A.vx[i];
        L.vy = A.vy[i];
        L.vz = A.vz[i];
        L.h = A.h[i];
        L.hinv = A.hinv[i];
        L.k5 = A.k5[i];
        L.A = A.A[i];
        L.c = A.cs[i];
        L.rho = A.rho[i];
        return L;
    }
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float dx = L.x - T.x[k], dy = L.y - T.y[k], dz = L.z - T.z[k];
        const float hm = fmaxf(L.h, T.h[k]);
        return dx * dx + dy * dy + dz * dz < 4.0f * hm * hm;
    }
    static __device__ __forceinline__ bool eval(const Args &A, const Lhs &L, const Tile &T, const NbrTable &,
                                                bool, int i, int k, Part &P)
    {
        const float dx = L.x - T.x[k], dy = L.y - T.y[k], dz = L.z - T.z[k];
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float hj = T.h[k];
        const float hm = fmaxf(L.h, hj);
        const bool in = (r2 < 4.0f * hm * hm) && (T.slot[k] != i) && (r2 > 0.0f);
        const float rinv = rsqrtf(in ? r2 : 1.0f);
        const float r = r2 * rinv;
        const float qi = r * L.hinv, qj = r * T.hinv[k];
        const float ti = 2.0f - qi, tj = 2.0f - qj;
        const float gi = (qi < 1.0f) ? fmaf(2.25f, qi, -3.0f) : ((qi < 2.0f) ? (-0.75f * ti * ti) * (L.h * rinv) : 0.0f);
        const float gj = (qj < 1.0f) ? fmaf(2.25f, qj, -3.0f) : ((qj < 2.0f) ? (-0.75f * tj * tj) * (hj * rinv) : 0.0f);
        const float Fi = L.k5 * gi, Fj = T.k5[k] * gj;
        const float dvx = L.vx - T.vx[k], dvy = L.vy - T.vy[k], dvz = L.vz - T.vz[k];
        const float vdotr = dvx * dx + dvy * dy + dvz * dz;
        float visc = 0.0f;
        if (in && vdotr < 0.0f) {
            const float hb = 0.5f * (L.h + hj);
            const float D1 = fmaf(A.eps * hb, hb, r2);
            const float D2 = 0.5f * (L.rho + T.rho[k]);
            const float rr = __frcp_rn(D1 * D2);
            const float mu = hb * vdotr * (D2 * rr);
            const float cb = 0.5f * (L.c + T.c[k]);
            visc = mu * fmaf(A.beta, mu, -A.alpha * cb) * (D1 * rr);
        }
        const float Fb = 0.5f * (Fi + Fj);
        const float mj = T.m[k];
        const float aF = L.A * Fi;
        float coef = mj * (aF + T.A[k] * Fj + visc * Fb);
        float dcoef = mj * (aF + 0.5f * visc * Fb) * vdotr;
        if (!in) {
            coef = 0.0f;
            dcoef = 0.0f;
        }
        P.ax.add(-coef * dx);
        P.ay.add(-coef * dy);
        P.az.add(-coef * dz);
        P.du.add(dcoef);
        return in;
    }
    static __device__ __forceinline__ void merge2(float2 &a, const Kahan &p)
    {
        Kahan k;
        k.s = a.x;
        k.c = a.y;
        k.merge(p.s, p.c);
        a.x = k.s;
        a.y = k.c;
    }
    static __device__ __forceinline__ void accumulate(Acc &a, const Part &P)
    {
        merge2(a.ax, P.ax);
        merge2(a.ay, P.ay);
        merge2(a.az, P.az);
        merge2(a.du, P.du);
    }
    static __device__ __forceinline__ void finish(const Args &A, int i, const Acc &a)
    {
        const float ax = __fsub_rn(a.ax.x, a.ax.y), ay = __fsub_rn(a.ay.x, a.ay.y);
        const float az = __fsub_rn(a.az.x, a.az.y), du = __fsub_rn(a.du.x, a.du.y);
        A.ax[i] = ax;
        A.ay[i] = ay;
        A.az[i] = az;
        A.dudt[i] = du;
        if (!isfinite(ax) || !isfinite(ay) || !isfinite(az) || !isfinite(du)) atomicOr(A.cm.status, SPH_DEV_NONFINITE);
    }
    static __device__ __forceinline__ void count(const Args &A, unsigned long long cand,
                                                 unsigned long long pairs)
    {
        atomicAdd(&A.cm.counters->force_cand, cand);
        atomicAdd(&A.cm.counters->force_pairs, pairs);
    }
};

template <class K>
__device__ __forceinline__ void zero_acc(typename K::Acc &a);
template <>
__device__ __forceinline__ void zero_acc<DensF64>(double &a) { a = 0.0; }
template <>
__device__ __forceinline__ void zero_acc<DensF32>(float2 &a) { a = make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ void zero_acc<ForceF64>(ForceF64::Acc &a) { a.ax = a.ay = a.az = a.du = 0.0; }
template <>
__device__ __forceinline__ void zero_acc<ForceF32>(ForceF32::Acc &a)
{
    a.ax = a.ay = a.az = a.du = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------------------------------------------------------
// The per-cell driver shared by all loop bodies.
// ------------------------------------------------------------------------------------------------------------
template <class K>
__global__ void __launch_bounds__(kPairThreads) k_cell_pairs(const typename K::Args A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ NbrTable nb;
    __shared__ typename K::Acc acc[kMaxLocal];
    __shared__ int queue[kPairWarps][64];
    __shared__ unsigned long long sh_pairs;

    const int c = blockIdx.x;
    const int ls = A.cm.cell_start[c], le = A.cm.cell_start[c + 1];
    if (ls >= le) return;  // CTA-uniform
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int tj = A.cm.tj;
    const typename K::Tile T = K::carve(smem, tj);
    if (tid == 0) sh_pairs = 0ull;
    build_nbr_table(nb, c, A.cm.g, A.cm.cell_start);
    const int NJ = nb.pref[27];
    const bool wrap = nb.wrap != 0;
    // conservative slack of the FP32 filter: float rounding of cell-relative coordinates (|coord| <= 2 edges)
    const float margin = (float)(4e-6 * fmax(A.cm.g.edge[0], fmax(A.cm.g.edge[1], A.cm.g.edge[2])));
    unsigned long long my_pairs = 0;

    for (int ib = ls; ib < le; ib += kMaxLocal) {
        const int nloc = min(kMaxLocal, le - ib);
        for (int t = tid; t < nloc; t += kPairThreads) zero_acc<K>(acc[t]);
        for (int tb = 0; tb < NJ; tb += tj) {
            const int tn = min(tj, NJ - tb);
            __syncthreads();  // accumulators zeroed, previous tile consumed
            for (int t = tid; t < tn; t += kPairThreads) {
                const int jj = tb + t;
                const int q = find_nbr(nb, jj);
                const int slot = nb.start[q] + (jj - nb.pref[q]);
                K::stage(A, T, nb, t, slot, q);
            }
            __syncthreads();
            for (int li = warp; li < nloc; li += kPairWarps) {
                const int i = ib + li;
                const typename K::Lhs L = K::load(A, i, margin);
                typename K::Part P;
                P.zero();
                int nq = 0;
                for (int jb = 0; jb < tn; jb += 32) {
                    const int k = jb + lane;
                    const bool p = (k < tn) && K::filter(L, T, k);
                    const unsigned bal = __ballot_sync(kFull, p);
                    if (p) queue[warp][nq + __popc(bal & lt_mask)] = k;
                    nq += __popc(bal);
                    __syncwarp();
                    if (nq >= 32) {
                        const bool in = K::eval(A, L, T, nb, wrap, i, queue[warp][lane], P);
                        const unsigned bin = __ballot_sync(kFull, in);  // every lane votes
                        if (lane == 0) my_pairs += __popc(bin);
                        __syncwarp();
                        if (lane < nq - 32) queue[warp][lane] = queue[warp][lane + 32];
                        nq -= 32;
                        __syncwarp();
                    }
                }
                if (nq > 0) {
                    bool in = false;
                    if (lane < nq) in = K::eval(A, L, T, nb, wrap, i, queue[warp][lane], P);
                    const unsigned b = __ballot_sync(kFull, in);
                    if (lane == 0) my_pairs += __popc(b);
                }
                __syncwarp();
                P.reduce();
                if (lane == 0) K::accumulate(acc[li], P);
            }
        }
        __syncthreads();
        for (int t = tid; t < nloc; t += kPairThreads) K::finish(A, ib + t, acc[t]);
    }
    if (lane == 0 && my_pairs) atomicAdd(&sh_pairs, my_pairs);
    __syncthreads();
    if (tid == 0) K::count(A, (unsigned long long)(le - ls) * (unsigned long long)NJ, sh_pairs);
}

// FP32 cell-relative copies of FP64 positions (filter input of the FP64 path), plus (float) h.
__global__ void k_pos32(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                        const double *__restrict__ h, const int *__restrict__ cell_of_slot, int n, Grid g,
                        float *__restrict__ xf, float *__restrict__ yf, float *__restrict__ zf,
                        float *__restrict__ hf)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int c = cell_of_slot[s];
    const int kx = c % g.n[0], ky = (c / g.n[0]) % g.n[1], kz = c / (g.n[0] * g.n[1]);
    xf[s] = __double2float_rn(x[s] - (double)kx * g.edge[0]);
    yf[s] = __double2float_rn(y[s] - (double)ky * g.edge[1]);
    zf[s] = __double2float_rn(z[s] - (double)kz * g.edge[2]);
    if (hf) hf[s] = __double2float_ru(h[s]);
}

// Per-particle quantities of the force loop: 1/h, 1/(pi h^5), P/rho^2.
template <typename T>
__global__ void k_force_prep(const T *__restrict__ h, const T *__restrict__ P, const T *__restrict__ rho, int n,
                             T *__restrict__ hinv, T *__restrict__ k5, T *__restrict__ A)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const T hi = T(1) / h[s];
    const T h2 = hi * hi;
    hinv[s] = hi;
    k5[s] = T(kInvPi) * h2 * h2 * hi;
    const T r = rho[s];
    A[s] = P[s] / (r * r);
}

template <class K>
cudaError_t run_cells(const typename K::Args &A, int ncells, cudaStream_t st)
{
    const size_t smem = (size_t)A.cm.tj * K::kStageBytes + 16;
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_cell_pairs<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    k_cell_pairs<K><<<ncells, kPairThreads, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_density_prep(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_of_slot, int n,
                                const Grid &g, cudaStream_t st, int *nl)
{
    if (n <= 0 || f32) return cudaSuccess;  // FP32 views are already cell-relative floats
    k_pos32<<<(n + 255) / 256, 256, 0, st>>>((const double *)soa.p[SPH_X][0], (const double *)soa.p[SPH_X][1],
                                             (const double *)soa.p[SPH_X][2], nullptr, cell_of_slot, n, g, scr.xf,
                                             scr.yf, scr.zf, nullptr);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_force_prep(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_of_slot, int n,
                              const Grid &g, cudaStream_t st, int *nl)
{
    if (n <= 0) return cudaSuccess;
    const int nb = (n + 255) / 256;
    if (!f32) {
        k_pos32<<<nb, 256, 0, st>>>((const double *)soa.p[SPH_X][0], (const double *)soa.p[SPH_X][1],
                                    (const double *)soa.p[SPH_X][2], (const double *)soa.p[SPH_H][0], cell_of_slot,
                                    n, g, scr.xf, scr.yf, scr.zf, scr.hf);
        k_force_prep<double><<<nb, 256, 0, st>>>((const double *)soa.p[SPH_H][0], (const double *)soa.p[SPH_P][0],
                                                 (const double *)soa.p[SPH_RHO][0], n, (double *)scr.hinv,
                                                 (double *)scr.k5, (double *)scr.A);
        *nl += 2;
    } else {
        k_force_prep<float><<<nb, 256, 0, st>>>((const float *)soa.p[SPH_H][0], (const float *)soa.p[SPH_P][0],
                                                (const float *)soa.p[SPH_RHO][0], n, (float *)scr.hinv,
                                                (float *)scr.k5, (float *)scr.A);
        *nl += 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_density_pairs(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_start,
                                 int ncells, int n, const Grid &g, double gamma, int tj, unsigned *status,
                                 Counters *counters, cudaStream_t st, int *nl)
{
    if (n <= 0) return cudaSuccess;
    ++*nl;
    PairCommon cm{cell_start, g, status, counters, 0};
    if (!f32) {
        DensF64::Args A;
        cm.tj = tj > 0 ? tj : 512;
        A.cm = cm;
        A.x = (const double *)soa.p[SPH_X][0];
        A.y = (const double *)soa.p[SPH_X][1];
        A.z = (const double *)soa.p[SPH_X][2];
        A.m = (const double *)soa.p[SPH_MASS][0];
        A.h = (const double *)soa.p[SPH_H][0];
        A.u = (const double *)soa.p[SPH_U][0];
        A.xf = scr.xf;
        A.yf = scr.yf;
        A.zf = scr.zf;
        A.rho = (double *)soa.p[SPH_RHO][0];
        A.P = (double *)soa.p[SPH_P][0];
        A.cs = (double *)soa.p[SPH_CS][0];
        A.gamma = gamma;
        return run_cells<DensF64>(A, ncells, st);
    }
    DensF32::Args A;
    cm.tj = tj > 0 ? tj : 1024;
    A.cm = cm;
    A.x = (const float *)soa.p[SPH_X][0];
    A.y = (const float *)soa.p[SPH_X][1];
    A.z = (const float *)soa.p[SPH_X][2];
    A.m = (const float *)soa.p[SPH_MASS][0];
    A.h = (const float *)soa.p[SPH_H][0];
    A.u = (const float *)soa.p[SPH_U][0];
    A.rho = (float *)soa.p[SPH_RHO][0];
    A.P = (float *)soa.p[SPH_P][0];
    A.cs = (float *)soa.p[SPH_CS][0];
    A.gamma = (float)gamma;
    return run_cells<DensF32>(A, ncells, st);
}

cudaError_t launch_force_pairs(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_start,
                               int ncells, int n, const Grid &g, const sph_params &prm, int tj, unsigned *status,
                               Counters *counters, cudaStream_t st, int *nl)
{
    if (n <= 0) return cudaSuccess;
    ++*nl;
    PairCommon cm{cell_start, g, status, counters, 0};
    if (!f32) {
        ForceF64::Args A;
        cm.tj = tj > 0 ? tj : 512;
        A.cm = cm;
        A.x = (const double *)soa.p[SPH_X][0];
        A.y = (const double *)soa.p[SPH_X][1];
        A.z = (const double *)soa.p[SPH_X][2];
        A.vx = (const double *)soa.p[SPH_V][0];
        A.vy = (const double *)soa.p[SPH_V][1];
        A.vz = (const double *)soa.p[SPH_V][2];
        A.m = (const double *)soa.p[SPH_MASS][0];
        A.h = (const double *)soa.p[SPH_H][0];
        A.rho = (const double *)soa.p[SPH_RHO][0];
        A.cs = (const double *)soa.p[SPH_CS][0];
        A.hinv = (const double *)scr.hinv;
        A.k5 = (const double *)scr.k5;
        A.A = (const double *)scr.A;
        A.xf = scr.xf;
        A.yf = scr.yf;
        A.zf = scr.zf;
        A.hf = scr.hf;
        A.ax = (double *)soa.p[SPH_A][0];
        A.ay = (double *)soa.p[SPH_A][1];
        A.az = (double *)soa.p[SPH_A][2];
        A.dudt = (double *)soa.p[SPH_DUDT][0];
        A.alpha = prm.alpha;
        A.beta = prm.beta;
        A.eps = prm.eps;
        return run_cells<ForceF64>(A, ncells, st);
    }
    ForceF32::Args A;
    cm.tj = tj > 0 ? tj : 512;
    A.cm = cm;
    A.x = (const float *)soa.p[SPH_X][0];
    A.y = (const float *)soa.p[SPH_X][1];
    A.z = (const float *)soa.p[SPH_X][2];
    A.vx = (const float *)soa.p[SPH_V][0];
    A.vy = (const float *)soa.p[SPH_V][1];
    A.vz = (const float *)soa.p[SPH_V][2];
    A.m = (const float *)soa.p[SPH_MASS][0];
    A.h = (const float *)soa.p[SPH_H][0];
    A.rho = (const float *)soa.p[SPH_RHO][0];
    A.cs = (const float *)soa.p[SPH_CS][0];
    A.hinv = (const float *)scr.hinv;
    A.k5 = (const float *)scr.k5;
    A.A = (const float *)scr.A;
    A.ax = (float *)soa.p[SPH_A][0];
    A.ay = (float *)soa.p[SPH_A][1];
    A.az = (float *)soa.p[SPH_A][2];
    A.dudt = (float *)soa.p[SPH_DUDT][0];
    A.alpha = (float)prm.alpha;
    A.beta = (float)prm.beta;
    A.eps = (float)prm.eps;
    return run_cells<ForceF32>(A, ncells, st);
}

}  // namespace sphk
