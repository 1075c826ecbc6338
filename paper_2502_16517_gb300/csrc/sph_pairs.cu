// sph_pairs.cu -- the cell-linked-list density and force loops (paper Section 2.1 steps 1-2).
//
// One CTA per cell (the paper's per-cell compute kernel, Section 2.1 / 2.3): the cell's particles are the local
// set, the particles of its 3^3 vertex-connected neighbour cells (periodic wrap) the active set.  Loop order is
// local-active (Section 5.4): every local particle gathers its sum, so there are no atomics on results.  Pair
// symmetry is not exploited (Section 5.3): every ordered pair is evaluated once from each side.
//
// Per CTA (FP64 loop bodies):
//   1. a 27-entry neighbour table (first slot, count, running prefix, periodic shift) in shared memory;
//   2. the active set is staged through shared memory in tiles of TJ particles holding only the SoA members the
//      loop body reads, plus one float4 per particle for the distance filter; each tile is padded to a multiple
//      of 64 with sentinel particles that no filter accepts;
//   3. each warp takes two local particles at a time (their FP64 members in two per-warp shared slots): its 32
//      lanes sweep the tile 32 candidates per step with the FP32 distance filter for both, the survivors of both
//      are compacted (ballot + popc) into one per-warp ring of 128 slots, tagged with their particle, and
//      whenever 32 are queued the lanes evaluate the full pair term in the path's precision, one pair per lane.
//      Inside the term the support is applied as a mask (the neutral-element formulation of Section 5.6:
//      out-of-support coefficients are zero, no branch decides whether a term is summed);
//   4. the per-lane partial sums are combined by reduce-scatters over the warp and added to the particles'
//      shared-memory accumulators; after the last tile each accumulator is finalised and written to the SoA
//      arrays.
// The compaction keeps the expensive evaluation at ~95 % lane occupancy although only ~15 % of the
// 3^3-stencil candidates lie inside the support (cell edge 2h).
//
// FP64 path: positions are the FP64 members; a neighbour across the periodic boundary is staged at its image
// x_j -+ box, so x_i - x_j needs no wrap test in the pair term (the image differs from the minimum-image difference
// by the rounding of one addition at the box scale).  The FP32 filter uses cell-relative float copies of the
// positions with a conservative radius, so it never drops a pair the FP64 test keeps.  The FP64 pipe (1/64 of the FP32 rate on this part) is
// the bound, so every per-pair FP64 instruction is counted: piece selection and masks run on the integer pipe,
// reciprocals are FP32-seeded Newton iterations, per-particle factors are precomputed.
// FP32 path: positions are cell-relative floats (the FP32 view), so x_i - x_j = r_i - (r_j + d * edge) with d the
// neighbour cell offset; the filter is the exact test; all sums are Kahan-compensated.  The FP32 loop bodies run
// under the lane driver (process_cell_lanes below): each thread owns one (local particle, candidate stream) pair
// and keeps its sums in registers over all tiles.  Their arithmetic is written for the FMA pipe: clamps are
// saturating adds, the spline pieces are combined arithmetically rather than selected, the viscosity switch is
// min(v.r, 0) = (v.r - |v.r|) / 2, so the half-rate ALU pipe carries almost no per-pair work.
#include <math.h>

#include <algorithm>
#include <climits>

#include "sph_internal.cuh"

namespace sphk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr long long kSignBit = (long long)0x8000000000000000ULL;  // sign bit of an FP64 bit pattern
constexpr int kMaxLocal = 128;  // local particles per round of the FP64 driver (shared accumulators)
// Threads per pair CTA ("warps per cell"): 128 or 256, chosen per loop by the view (autotuner).
constexpr int kRing = 128;   // per-warp queue slots (at most 31 + 2 x 32 pending)
constexpr int kStep = 64;    // tile granularity: a staged tile is padded to a multiple of kStep
constexpr float kFar = 1e30f;  // sentinel coordinate: its squared distance overflows to +inf

struct NbrTable {
    int start[27];
    int pref[32];  // prefix counts pref[0..27]; pref[28..31] = INT_MAX (sentinels of find_nbr's search)
    double shift[27][3];  // added to x_i - x_j for a j of neighbour q (0 or +-box)
    float offf[27][3];    // origin of neighbour cell q relative to the local cell origin: (float)(d * edge)
    int wrap;             // any shift != 0
    float margin;         // slack of the FP64 paths' FP32 filter
};

// n, ncells, status: the checked build's range checks of the neighbour cells and their slot ranges (a neighbour
// that fails one counts as empty).
__device__ __forceinline__ void build_nbr_table(NbrTable &nb, int c, const CellSpace &cs, const int *cell_start,
                                                int n, int ncells, unsigned *status)
{
    // one warp: lane q < 27 fills neighbour q, then the counts are prefix-summed with shuffles
    const int tid = threadIdx.x;
    if (tid < 32) {
        const bool periodic = cs.npatch == 0 && cs.g.periodic;
        CellLoc L;
        locate_cell(cs, c, L);
        int cnt = 0;
        bool wr = false;
        if (tid < 27) {
            const int d[3] = {tid % 3 - 1, (tid / 3) % 3 - 1, tid / 9 - 1};
            int kk[3];
            bool valid = true;
            for (int a = 0; a < 3; ++a) {
                int k = L.k[a] + d[a];
                double sh = 0.0;
                if (k < 0) {
                    if (periodic) {
                        k += L.n[a];
                        sh = cs.g.box[a];
                    } else {
                        valid = false;
                    }
                } else if (k >= L.n[a]) {
                    if (periodic) {
                        k -= L.n[a];
                        sh = -cs.g.box[a];
                    } else {
                        valid = false;
                    }
                }
                kk[a] = k;
                nb.shift[tid][a] = sh;
                // (float)(d edge) for d in {-1, 0, 1} is d (float)edge exactly
                const float ef = cs.npatch == 0 ? cs.g.edgef[a] : __double2float_rn(cell_edge(cs, L, a));
                nb.offf[tid][a] = (float)d[a] * ef;
                wr = wr || (sh != 0.0);
            }
            int st = 0;
            if (valid) {
                const int c2 = L.base + kk[0] + L.n[0] * (kk[1] + L.n[1] * kk[2]);
                if (SPH_CHECK(c2 >= 0 && c2 < ncells, status)) {
                    st = cell_start[c2];
                    cnt = cell_start[c2 + 1] - st;
                    if (!SPH_CHECK(st >= 0 && cnt >= 0 && st <= n - cnt, status)) st = cnt = 0;
                }
            }
            nb.start[tid] = st;
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int up = __shfl_up_sync(kFull, incl, o);
            if (tid >= o) incl += up;
        }
        if (tid < 27) nb.pref[tid + 1] = incl;
        else if (tid < 31) nb.pref[tid + 1] = INT_MAX;
        const bool any_wrap = __any_sync(kFull, wr && cnt > 0);
        if (tid == 0) {
            nb.pref[0] = 0;
            nb.wrap = any_wrap ? 1 : 0;
            // conservative slack of the FP32 filter: float rounding of cell-relative coordinates (|coord| <= 2 edges)
            const float emax = cs.npatch == 0
                                   ? fmaxf(cs.g.edgef[0], fmaxf(cs.g.edgef[1], cs.g.edgef[2]))
                                   : __double2float_rn(fmax(cell_edge(cs, L, 0),
                                                            fmax(cell_edge(cs, L, 1), cell_edge(cs, L, 2))));
            nb.margin = 4e-6f * emax;
        }
    }
    __syncthreads();
}

// Neighbour index q with pref[q] <= jj < pref[q+1] for 0 <= jj < pref[27] (empty neighbours have pref[q] ==
// pref[q+1]): the largest q with pref[q] <= jj, found by five fixed, branch-free halving steps over pref[0..31].
__device__ __forceinline__ int find_nbr(const NbrTable &nb, int jj)
{
    int q = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (nb.pref[q + step] <= jj) q += step;
    return q;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Single-instruction FP32 forms (PTX): approximate reciprocal square root and reciprocal, and saturating
// (clamped to [0, 1]) multiply-add / add / multiply.  Subnormal inputs and results flush to zero; the FP32
// pair terms stay far above the subnormal range, so this changes no result and saves the subnormal fix-up
// sequences of the default forms.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float fma_sat(float a, float b, float c)
{
    float y;
    asm("fma.rn.ftz.sat.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
    return y;
}
__device__ __forceinline__ float mul_sat(float a, float b)
{
    float y;
    asm("mul.rn.ftz.sat.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
    return y;
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
};

// Two Kahan accumulators side by side (value = s - c per component), updated with paired FP32 instructions: the
// same IEEE operations, in the same order, as two Kahan::add.
struct Kahan2 {
    float2 s, c;
    __device__ __forceinline__ void zero()
    {
        s = make_float2(0.f, 0.f);
        c = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void add(float2 y)
    {
        const float2 neg = make_float2(-1.0f, -1.0f);
        const float2 yy = __ffma2_rn(c, neg, y);  // y - c
        const float2 t = __fadd2_rn(s, yy);
        c = __ffma2_rn(yy, neg, __ffma2_rn(s, neg, t));  // (t - s) - yy
        s = t;
    }
};

// ------------------------------------------------------------------------------------------------------------
// Pair-term arithmetic of the FP64 loop bodies.
//
// The cubic spline is piecewise cubic in q = r/h.  Instead of evaluating both pieces and selecting, the
// coefficients of the one piece that applies are selected and a single polynomial is evaluated:
//   f(q)     = d0 + d1 q + d2 q^2 + d3 q^3     inner (q < 1): (1, 0, -3/2, 3/4), outer (1 <= q < 2): (2, -3, 3/2, -1/4)
//   f'(q)/q  = c0/q + c1 + c2 q                inner: (0, -3, 9/4),             outer: (-3, 3, -3/4)
// with every coefficient 0 for q >= 2 (outside the support): the masking of Section 5.6.  The coefficients are
// scaled by powers of 1/h per particle (so the polynomials run in r) and the piece is chosen by integer compares
// of bit patterns: for doubles >= 0 the bit patterns order like the values.  (The FP32 bodies use another form
// of the same spline, suited to the FP32 pipes; see DensF32.)
// ------------------------------------------------------------------------------------------------------------
// FP32 approximation of a positive double by bit manipulation on the integer pipe (exponent re-bias, mantissa
// truncated to 23 bits; the input is first clamped into the float normal range), and the exact reverse.
__device__ __forceinline__ float dbl_to_flt_bits(double x)
{
    unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    hi = min(max(hi, 0x38100000u), 0x47EFFFFFu);
    return __uint_as_float(((hi - 0x38000000u) << 3) | (lo >> 29));
}
__device__ __forceinline__ double flt_to_dbl_bits(float y)
{
    const unsigned f = __float_as_uint(y);
    return __hiloint2double((int)((f >> 3) + 0x38000000u), (int)(f << 29));
}

// 1/sqrt(x), x >= 0: FP32 seed y0 (no conversion instructions, relative error e0 below ~2^-22), then one
// third-order step in FP64: with e = 1 - x y0^2, x^(-1/2) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + 5e^3/16 ...),
// truncated after e^2, which leaves ~(5/16) e0^3 < 2^-66, below FP64 rounding -- five FP64 operations instead of
// the seven of two Newton steps.  For x = 0 (or x below the float range) the result is large but finite, so
// r = x / sqrt(x) comes out 0 (or tiny).
__device__ __forceinline__ double rsqrt_seeded(double x)
{
    const double y = flt_to_dbl_bits(rsqrt_ftz(dbl_to_flt_bits(x)));
    const double e = fma(-(x * y), y, 1.0);
    return fma(y * e, fma(0.375, e, 0.5), y);
}

// sqrt(x), x >= 0, from the same FP32 seed y0 of 1/sqrt(x): g = x y0 and e = 1 - g y0 give
// sqrt(x) = g (1 - e)^(-1/2) = g (1 + e/2 + 3e^2/8 + ...), truncated after e^2 (remainder ~(5/16) e0^3, below FP64
// rounding): five FP64 operations, one fewer than x * rsqrt_seeded(x).  x = 0 gives 0 (g = 0).
__device__ __forceinline__ double sqrt_seeded(double x)
{
    const double y = flt_to_dbl_bits(rsqrt_ftz(dbl_to_flt_bits(x)));
    const double g = x * y;
    const double e = fma(-g, y, 1.0);
    return fma(g * e, fma(0.375, e, 0.5), g);
}

// 1/x, x > 0 within the float range: FP32 seed y0, then 1/x = y0 / (1 - e) = y0 (1 + e + e^2 ...) with
// e = 1 - x y0, truncated after e^2 (remainder ~e0^3, below FP64 rounding): three FMAs.
__device__ __forceinline__ double rcp_seeded(double x)
{
    const double y = flt_to_dbl_bits(rcp_ftz(dbl_to_flt_bits(x)));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// Shared-memory loads the compiler may not hoist or merge (asm volatile): for values read again on purpose in
// every round of a loop, so that they do not occupy registers across it.
__device__ __forceinline__ double lds(const double *p)
{
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}
__device__ __forceinline__ float ldsf(const float *p)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}

// ------------------------------------------------------------------------------------------------------------
// Loop bodies.  Each provides: Args, Tile (carve / stage / sentinel), Lhs (load), filter, eval, Part (per-lane
// partial sums, reduce), Acc (shared accumulator), accumulate, finish, count.
// ------------------------------------------------------------------------------------------------------------
struct PairCommon {
    const int *cell_start;
    CellSpace cs;
    unsigned *status;
    Counters *counters;
    int tj;            // staged particles per tile (a multiple of kStep)
    const int *skip;   // device flag: nonzero = return at once (a converged smoothing-length iteration)
    int n, ncells;     // particles and cells (patch views: the cell capacity), for the checked build's checks
};

// ---- density, FP64 ----
// Per pair: r from one seeded square root, the piece of the spline chosen by integer compares of the bit
// patterns of r against h_i and 2 h_i, and f evaluated as a cubic in r whose coefficients d_k h_i^-k come from
// the per-particle set-up kernel.
struct DensF64 {
    // The FP64 members of the local particle a pair term reads (per-particle arrays in Args, the warp's shared
    // slot in Lhs), in this order.
    enum { X, Y, Z, H, E2, E3, O1, O2, O3, NF };
    struct Args {
        PairCommon cm;
        const double *f[NF];                   // x, y, z, h and (k_density_prep_f64) e2 .. o3
        const double *m, *u;
        const double *rk, *cs0;                // per particle (k_density_prep_f64): 1/(pi h^3), c_s
        const float *xf, *yf, *zf;             // cell-relative float positions (filter only)
        double *rho, *P, *cs;
        double gamma;
    };
    struct Tile {
        double *x, *y, *z, *m;
        float4 *f4;  // filter: cell-relative position seen from the local cell, unused
    };
    // The local particle: FP64 members in the warp's shared slot s (re-read every evaluation round), the
    // filter's FP32 copies in registers.
    struct Lhs {
        const double *s;
        float fx, fy, fz, b2;
    };
    struct Part {
        double rho;
        __device__ __forceinline__ void zero() { rho = 0.0; }
    };
    using Acc = double;
    static constexpr int kStageBytes = 4 * 8 + 16;
    static constexpr int kSlotDoubles = 17;  // slot of a local particle's members (odd: see PairShared)
    // rho_i includes m_i W(0, h_i) = m_i / (pi h^3): the filter drops the self candidate and finish adds m_i f(0) =
    // m_i to the sum of the others (kSelfInFinish: the self pair is still counted)
    static constexpr bool kSkipSelf = true;
    static constexpr bool kSelfInFinish = true;
    static constexpr bool kSplit = false;     // one queue (see tile_pairs_split)
    // CTAs per SM the register allocation must allow: shared memory allows seven of 128 threads at a 512 tile
    static constexpr int min_ctas(int nt) { return nt == 128 ? 7 : 3; }
    // The warp's lane partials of four local particles (u = 0..3) are reduced together: a reduce-scatter (xor 16
    // keeps two of the four sums per half-warp, xor 8 one per quarter, then xor 4, 2, 1) takes 6 additions per
    // lane instead of 4 x 5.  Each particle's sum still runs over the same tree as a butterfly sum (xor 16, 8, 4,
    // 2, 1), so the result does not depend on the grouping.
    static constexpr int kGroup = 4;
    struct Group {
        double p0, p1, p2, p3;
        int l0, l1, l2, l3;
        __device__ __forceinline__ void zero() { p0 = p1 = p2 = p3 = 0.0; }
        __device__ __forceinline__ void put(int u, const Part &P, int li)
        {
            if (u == 0) { p0 = P.rho; l0 = li; }
            else if (u == 1) { p1 = P.rho; l1 = li; }
            else if (u == 2) { p2 = P.rho; l2 = li; }
            else { p3 = P.rho; l3 = li; }
        }
        // Adds sum u to acc[l_u] for u < nu (lane 8u holds sum u); called by the whole warp.
        __device__ __forceinline__ void accumulate(Acc *acc, int nu, int lane)
        {
            const bool up16 = (lane & 16) != 0;
            double s0 = up16 ? p2 : p0, s1 = up16 ? p3 : p1;
            const double o0 = up16 ? p0 : p2, o1 = up16 ? p1 : p3;
            s0 += __shfl_xor_sync(kFull, o0, 16);
            s1 += __shfl_xor_sync(kFull, o1, 16);
            const bool up8 = (lane & 8) != 0;
            double t = up8 ? s1 : s0;
            const double o = up8 ? s0 : s1;
            t += __shfl_xor_sync(kFull, o, 8);
            t += __shfl_xor_sync(kFull, t, 4);
            t += __shfl_xor_sync(kFull, t, 2);
            t += __shfl_xor_sync(kFull, t, 1);
            const int u = lane >> 3;
            if ((lane & 7) == 0 && u < nu) acc[u == 0 ? l0 : u == 1 ? l1 : u == 2 ? l2 : l3] += t;
        }
    };

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        t.x = reinterpret_cast<double *>(s);
        t.y = t.x + tj;
        t.z = t.y + tj;
        t.m = t.z + tj;
        t.f4 = reinterpret_cast<float4 *>(t.m + tj);
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        // a neighbour across the periodic boundary is staged at its image position: shift is what the minimum image
        // adds to x_i - x_j, so the image is x_j - shift (only cells next to the boundary have shifts)
        double xs = A.f[X][slot], ys = A.f[Y][slot], zs = A.f[Z][slot];
        if (nb.wrap) {
            xs -= nb.shift[q][0];
            ys -= nb.shift[q][1];
            zs -= nb.shift[q][2];
        }
        T.x[t] = xs;
        T.y[t] = ys;
        T.z[t] = zs;
        T.m[t] = A.m[slot];
        T.f4[t] = make_float4(A.xf[slot] + nb.offf[q][0], A.yf[slot] + nb.offf[q][1], A.zf[slot] + nb.offf[q][2],
                              0.0f);
    }
    static __device__ __forceinline__ void sentinel(const Tile &T, int t) { T.f4[t] = make_float4(kFar, kFar, kFar, 0.f); }
    // Called by the whole warp; ws is a slot of kSlotDoubles doubles of shared memory.
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float margin, double *ws)
    {
        const int lane = threadIdx.x & 31;
        if (lane < NF) ws[lane] = A.f[lane][i];
        __syncwarp();
        Lhs L;
        L.s = ws;
        L.fx = A.xf[i];
        L.fy = A.yf[i];
        L.fz = A.zf[i];
        const float rf = __fmaf_ru(2.0f * (1.0f + 4e-6f), __double2float_ru(A.f[H][i]), margin);
        L.b2 = __fmul_ru(rf, rf);
        return L;
    }
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float4 p = T.f4[k];
        const float dx = L.fx - p.x, dy = L.fy - p.y, dz = L.fz - p.z;
        return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < L.b2;
    }
    static __device__ __forceinline__ bool eval(const Args &, const Lhs &L, const Tile &T, const NbrTable &nb,
                                                bool wrap, int, int k, Part &P)
    {
        const double *s = L.s;
        const double dx = lds(s + X) - T.x[k], dy = lds(s + Y) - T.y[k], dz = lds(s + Z) - T.z[k];
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double r = sqrt_seeded(r2);
        const long long rb = __double_as_longlong(r);
        // bit patterns of h and 2 h: for r >= 0, r < h exactly when bits(r) < bits(h)
        const long long hb1 = __double_as_longlong(lds(s + H)), hb2 = hb1 + (1LL << 52);
        const bool inner = rb < hb1, supp = rb < hb2;
        const double c0 = inner ? 1.0 : (supp ? 2.0 : 0.0);
        const double c1 = inner ? 0.0 : (supp ? lds(s + O1) : 0.0);
        const double c2 = inner ? lds(s + E2) : (supp ? lds(s + O2) : 0.0);
        const double c3 = inner ? lds(s + E3) : (supp ? lds(s + O3) : 0.0);
        const double w = fma(fma(fma(c3, r, c2), r, c1), r, c0);
        P.rho = fma(T.m[k], w, P.rho);
        return supp;
    }
    static __device__ __forceinline__ void finish(const Args &A, int i, const Acc &a)
    {
        const double h = A.f[H][i];
        const double rho = (a + A.m[i]) * A.rk[i];  // + the self term m_i f(0), f(0) = 1
        const double P = (A.gamma - 1.0) * rho * A.u[i];
        const double cs = A.cs0[i];
        A.rho[i] = rho;
        A.P[i] = P;
        A.cs[i] = cs;
        unsigned bits = 0;
        if (!(rho > 0.0) || !isfinite(rho) || !isfinite(P) || !isfinite(cs)) bits |= SPH_DEV_NONFINITE;
        if (!(2.0 * h <= A.cm.cs.g.min_edge)) bits |= SPH_DEV_H_TOO_BIG;
        if (bits) atomicOr(A.cm.status, bits);
    }
    static __device__ __forceinline__ void count(const Args &A, unsigned long long cand,
                                                 unsigned long long pairs)
    {
        atomicAdd(&A.cm.counters->dens_cand, cand);
        atomicAdd(&A.cm.counters->dens_pairs, pairs);
    }
};

// ---- density, FP32 (cell-relative float positions, Kahan sums; lane driver, every candidate evaluated) ----
// f(q) = 2 s^3 - t^3 with s = sat(1 - q/2), t = sat(1 - q): the outer piece 1/4 (2-q)^3 = 2 s^3, and for q < 1 the
// inner piece 1 - 3/2 q^2 + 3/4 q^3 = 1/4 (2-q)^3 - (1-q)^3; beyond q = 2 both clamps are 0 (the support mask).
// The self term (r = 0) is included, as in the definition of rho_i.  s > 0 exactly when q < 2 and then
// s >= 2^-24, so sat(2^24 s) counts the pairs in the support.
struct DensF32 {
    static constexpr bool kMasked = true;
    // CTAs per SM the register allocation must allow: 40 registers keep twelve 128-thread CTAs (the 1024 tile's
    // shared memory allows twelve as well)
    static constexpr int min_ctas(int nt) { return nt == 128 ? 12 : 6; }
    static constexpr int min_ctas_persist(int nt) { return min_ctas(nt); }
    struct Args {
        PairCommon cm;
        const float *x, *y, *z, *m, *h, *u;
        float *rho, *P, *cs;
        float gamma;
    };
    // Candidates stored pair-interleaved (candidates 2p and 2p+1 side by side), so that each 16-byte load gives
    // two aligned float2 operands and the sweep runs two candidates per paired FP32 instruction.
    struct Tile {
        float4 *pa;  // pair p: x_2p, x_2p+1, y_2p, y_2p+1 (positions seen from the local cell)
        float4 *pb;  // pair p: z_2p, z_2p+1, m_2p, m_2p+1
    };
    struct Lhs {
        float x, y, z, hinv;
    };
    struct Part {
        Kahan rho;
        float npair;
        __device__ __forceinline__ void zero()
        {
            rho.zero();
            npair = 0.f;
        }
    };
    using Acc = float2;  // (s, c)
    static constexpr int kStageBytes = 16;

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        t.pa = reinterpret_cast<float4 *>(s);
        t.pb = t.pa + tj / 2;
        return t;
    }
    static __device__ __forceinline__ void put(const Tile &T, int t, float x, float y, float z, float m)
    {
        float *a = reinterpret_cast<float *>(T.pa + (t >> 1)) + (t & 1);
        float *b = reinterpret_cast<float *>(T.pb + (t >> 1)) + (t & 1);
        a[0] = x;
        a[2] = y;
        b[0] = z;
        b[2] = m;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        put(T, t, A.x[slot] + nb.offf[q][0], A.y[slot] + nb.offf[q][1], A.z[slot] + nb.offf[q][2], A.m[slot]);
    }
    // The partner of an odd last candidate: massless and far away (finite, so no inf * 0): it adds 0 and is
    // never counted.
    static __device__ __forceinline__ void pad(const Tile &T, int t) { put(T, t, 1e18f, 1e18f, 1e18f, 0.f); }
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float, double *)
    {
        Lhs L;
        L.x = A.x[i];
        L.y = A.y[i];
        L.z = A.z[i];
        L.hinv = __frcp_rn(A.h[i]);
        return L;
    }
    // m_j f(q_ij) of candidate pair p (two candidates at once); adds the pair's in-support count to cnt.
    static __device__ __forceinline__ float2 term2(const Lhs &L, const Tile &T, int p, float2 &cnt)
    {
        const float4 a = T.pa[p], b = T.pb[p];
        const float2 neg = make_float2(-1.0f, -1.0f);
        const float2 dx = __ffma2_rn(make_float2(a.x, a.y), neg, make_float2(L.x, L.x));
        const float2 dy = __ffma2_rn(make_float2(a.z, a.w), neg, make_float2(L.y, L.y));
        const float2 dz = __ffma2_rn(make_float2(b.x, b.y), neg, make_float2(L.z, L.z));
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        const float2 r2e = __fadd2_rn(r2, make_float2(1e-30f, 1e-30f));
        const float2 rs = make_float2(rsqrt_ftz(r2e.x), rsqrt_ftz(r2e.y));
        const float2 q = __fmul2_rn(__fmul2_rn(r2, rs), make_float2(L.hinv, L.hinv));
        const float2 sq = make_float2(fma_sat(-0.5f, q.x, 1.0f), fma_sat(-0.5f, q.y, 1.0f));
        const float2 t = make_float2(fma_sat(-1.0f, q.x, 1.0f), fma_sat(-1.0f, q.y, 1.0f));
        const float2 s3 = __fmul2_rn(__fmul2_rn(sq, sq), sq);
        const float2 t3 = __fmul2_rn(__fmul2_rn(t, t), t);
        const float2 w = __ffma2_rn(s3, make_float2(2.0f, 2.0f), make_float2(-t3.x, -t3.y));
        cnt = __fadd2_rn(cnt, make_float2(mul_sat(sq.x, 16777216.0f), mul_sat(sq.y, 16777216.0f)));
        return __fmul2_rn(make_float2(b.z, b.w), w);
    }
    // Candidate pairs p, p + ns, ... covering candidates < tn (an odd tail was padded): two pairs (four terms)
    // summed plainly, then added to the compensated sum.
    static __device__ __forceinline__ void sweep(const Lhs &L, const Tile &T, int p, int ns, int tn, Part &P)
    {
        const int np = (tn + 1) >> 1;
        float2 cnt = make_float2(0.f, 0.f);
        for (; p + ns < np; p += 2 * ns) {
            const float2 u = term2(L, T, p, cnt), v = term2(L, T, p + ns, cnt);
            P.rho.add((u.x + u.y) + (v.x + v.y));
        }
        if (p < np) {
            const float2 u = term2(L, T, p, cnt);
            P.rho.add(u.x + u.y);
        }
        P.npair += cnt.x + cnt.y;
    }
    static __device__ __forceinline__ void merge_part(Acc &a, const Part &P)
    {
        Kahan k;
        k.s = a.x;
        k.c = a.y;
        k.merge(P.rho.s, P.rho.c);
        a.x = k.s;
        a.y = k.c;
    }
    static __device__ __forceinline__ unsigned pairs_of(const Part &P) { return (unsigned)P.npair; }
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
        if (!(2.0 * (double)h <= A.cm.cs.g.min_edge * (1.0 + 2.4e-7))) bits |= SPH_DEV_H_TOO_BIG;
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
// Per particle (k_force_prep_f64): q2 = (h/2)^2 and the gradient coefficients S0 = -3/(pi h^4), K1 = 3/(pi h^5),
// K2i = 2.25/(pi h^6), K2o = -0.75/(pi h^6), so that grad_i W(r_ij, h) = F r_ij with
//   F = (K2i r^2) / r - K1            (r < h)
//   F = (S0 + K2o r^2) / r + K1       (h <= r < 2h),   0 beyond,
// i.e. F = fma(fma(a, r^2, b), 1/r, c) with (a, b, c) of the piece, which the pair picks for each side by integer
// compares of bits(r^2) - 2^53 (= bits(r^2/4)) and bits(r^2) - 2^54 (= bits(r^2/16)) against bits(q2): r itself is
// never formed.  A = P / rho^2.
// The viscosity (Monaghan): mu = hbar w / D1 with w = v_ij . r_ij, D1 = r^2 + eps hbar^2, hbar = (h_i + h_j)/2,
// D2 = rho_i + rho_j, and Pi / 2 = mu (beta mu - alpha cbar) / D2.  With soft (eps > 0) and s = sqrt(eps), each
// particle carries hs = s h/2 and acs = alpha c / (2 s): then hbs = hs_i + hs_j = s hbar, D1 = hbs^2 + r^2, and
// with R = 1 / (D1 D2), g = hbs w R (= s mu / D2) and mu' = g D2 (= s mu),
//   Pi / 2 = g (beta/eps mu' - (acs_i + acs_j)),
// the same value with no multiplication by eps per pair.  Without softening (eps = 0): s = 1 and D1 = r^2.
template <bool kSoft>
struct ForceF64 {
    // The 15 FP64 members a pair term reads from either particle, in this order (per-particle arrays in Args,
    // one row per candidate in the tile); q2 is staged beside the rows.
    enum { X, Y, Z, VX, VY, VZ, M, HS, S0, K1, K2I, K2O, AP, ACS, RHO, NF };
    static constexpr int Q2 = NF;  // its place in the local particle's slot
    struct Args {
        PairCommon cm;
        const double *f[NF];                // x, y, z, v, m, rho and (k_force_prep_f64) hs .. acs
        const double *q2;                   // (h/2)^2 (k_force_prep_f64)
        const float *xf, *yf, *zf, *hf;     // filter copies
        double *ax, *ay, *az, *dudt;
        double beta_s;                      // beta / eps (soft), else beta
    };
    // Candidate k's members at d[k * NF + f]: one row address serves all fifteen loads (NF is odd, so 64-bit
    // loads of 32 different rows hit distinct bank pairs); its q2 at q[k] (likewise).
    struct Tile {
        double *d;
        double *q;
        float4 *f4;  // filter: cell-relative position seen from the local cell, its filter radius
    };
    // The local particle: its FP64 members sit in the warp's shared slot (s[f], read again in every evaluation
    // round, which keeps them out of the registers), and so does its FP32 velocity (read by the receding
    // estimate); only the filter's FP32 copies stay in registers.
    struct Lhs {
        const double *s;
        float fx, fy, fz, rf;
    };
    struct Part {
        double ax, ay, az, du;
        __device__ __forceinline__ void zero() { ax = ay = az = du = 0.0; }
    };
    struct Acc {
        double ax, ay, az, du;
    };
    static constexpr int kStageBytes = NF * 8 + 8 + 16;
    // slot of a local particle: its members, q2, then its FP32 velocity (two doubles' room); odd: see PairShared
    static constexpr int kSlotDoubles = 19;
    static constexpr int kVelF = 16;  // the FP32 velocity's place in the slot (in doubles)
    // The self pair contributes nothing (j != i in the sums), so the queue driver drops it at the filter.
    static constexpr bool kSkipSelf = true;
    static constexpr bool kSelfInFinish = false;
    // Receding pairs (v_ij . r_ij >= 0) have no viscosity: the queued hits are sorted by an FP32 estimate of
    // v_ij . r_ij, and rounds of estimated receding pairs skip the viscosity terms (tile_pairs_split).
    static constexpr bool kSplit = true;
    // CTAs per SM the register allocation must allow: shared memory allows three at a 448 tile (85 registers
    // at 256 threads)
    static constexpr int min_ctas(int) { return 3; }
    // The two local particles of a warp's queue are reduced together: one reduce-scatter of their eight sums
    // (xor 16 keeps one particle per half-warp, xor 8 two of its sums, xor 4 one, then xor 2, 1) takes 9
    // additions per lane instead of 2 x 6.  Every sum still runs over the butterfly tree (xor 16, 8, 4, 2, 1).
    static constexpr int kGroup = 2;
    struct Group {
        Part P0, P1;
        int l0, l1;
        __device__ __forceinline__ void zero() {}
        __device__ __forceinline__ void put(int u, const Part &P, int li)
        {
            if (u == 0) { P0 = P; l0 = li; }
            else { P1 = P; l1 = li; }
        }
        // Adds the sums of particle u < nu to acc[l_u]; called by the whole warp.  Afterwards lanes 4g .. 4g + 3
        // hold sum g = 4 u + c (c: 0 ax, 1 ay, 2 az, 3 du).
        __device__ __forceinline__ void accumulate(Acc *acc, int nu, int lane)
        {
            const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0, up4 = (lane & 4) != 0;
            const Part &K = up16 ? P1 : P0, &O = up16 ? P0 : P1;
            double a0 = K.ax + __shfl_xor_sync(kFull, O.ax, 16);
            double a1 = K.ay + __shfl_xor_sync(kFull, O.ay, 16);
            double a2 = K.az + __shfl_xor_sync(kFull, O.az, 16);
            double a3 = K.du + __shfl_xor_sync(kFull, O.du, 16);
            double b0 = up8 ? a2 : a0, b1 = up8 ? a3 : a1;
            b0 += __shfl_xor_sync(kFull, up8 ? a0 : a2, 8);
            b1 += __shfl_xor_sync(kFull, up8 ? a1 : a3, 8);
            double t = up4 ? b1 : b0;
            t += __shfl_xor_sync(kFull, up4 ? b0 : b1, 4);
            t += __shfl_xor_sync(kFull, t, 2);
            t += __shfl_xor_sync(kFull, t, 1);
            const int u = lane >> 4, c = (lane >> 2) & 3;
            if ((lane & 3) == 0 && u < nu) {
                Acc &a = acc[u == 0 ? l0 : l1];
                if (c == 0) a.ax += t;
                else if (c == 1) a.ay += t;
                else if (c == 2) a.az += t;
                else a.du += t;
            }
        }
    };

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        t.d = reinterpret_cast<double *>(s);
        t.q = t.d + NF * tj;
        t.f4 = reinterpret_cast<float4 *>(t.q + tj);
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        // a neighbour across the periodic boundary is staged at its image position: shift is what the minimum image
        // adds to x_i - x_j, so the image is x_j - shift (only cells next to the boundary have shifts)
        double *row = T.d + t * NF;
        double xs = A.f[X][slot], ys = A.f[Y][slot], zs = A.f[Z][slot];
        if (nb.wrap) {
            xs -= nb.shift[q][0];
            ys -= nb.shift[q][1];
            zs -= nb.shift[q][2];
        }
        row[X] = xs;
        row[Y] = ys;
        row[Z] = zs;
#pragma unroll
        for (int f = VX; f < NF; ++f) row[f] = A.f[f][slot];
        T.q[t] = A.q2[slot];
        T.f4[t] = make_float4(A.xf[slot] + nb.offf[q][0], A.yf[slot] + nb.offf[q][1], A.zf[slot] + nb.offf[q][2],
                              radius(A.hf[slot], nb.margin));
    }
    static __device__ __forceinline__ void sentinel(const Tile &T, int t) { T.f4[t] = make_float4(kFar, kFar, kFar, 0.f); }
    // Called by the whole warp; ws is the warp's slot (kSlotDoubles doubles of shared memory).
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float margin, double *ws)
    {
        const int lane = threadIdx.x & 31;
        if (lane < NF) ws[lane] = A.f[lane][i];
        else if (lane == Q2) ws[Q2] = A.q2[i];
        else if (lane < Q2 + 4)
            reinterpret_cast<float *>(ws + kVelF)[lane - Q2 - 1] = __double2float_rn(A.f[VX + lane - Q2 - 1][i]);
        __syncwarp();
        Lhs L;
        L.s = ws;
        L.fx = A.xf[i];
        L.fy = A.yf[i];
        L.fz = A.zf[i];
        L.rf = radius(A.hf[i], margin);
        return L;
    }
    // The filter radius of a particle: 2 h (1 + 4e-6) + margin, rounded up, from the float h rounded up (the slack
    // covers the rounding of the cell-relative FP32 positions).  Rounding up is monotone, so the larger of two
    // particles' radii is the radius of the larger h.
    static __device__ __forceinline__ float radius(float hf, float margin)
    {
        return __fmaf_ru(2.0f * (1.0f + 4e-6f), hf, margin);
    }
    // r < 2 max(h_i, h_j) with a conservative FP32 radius, so that it never drops a pair the FP64 test keeps.
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float4 p = T.f4[k];
        const float dx = L.fx - p.x, dy = L.fy - p.y, dz = L.fz - p.z;
        const float rf = fmaxf(L.rf, p.w);
        return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < __fmul_ru(rf, rf);
    }
    // Candidate k's velocity, approximately: the FP32 pattern of each member's sign, exponent and top 20 mantissa
    // bits (the high word of the double, re-biased; exact truncation in the FP32 normal range, meaningless
    // outside it).  It serves only the queue choice below, which costs time when wrong, never accuracy.
    static __device__ __forceinline__ float3 vel_estimate(const Tile &T, int k)
    {
        const int *w = reinterpret_cast<const int *>(T.d + k * NF);
        const auto f = [](int h) {
            const unsigned m = ((unsigned)h & 0x7fffffffu) - 0x38000000u;  // exponent bias 1023 -> 127
            return __uint_as_float((m << 3) | ((unsigned)h & 0x80000000u));
        };
        return make_float3(f(w[2 * VX + 1]), f(w[2 * VY + 1]), f(w[2 * VZ + 1]));
    }
    // Whether the FP32 estimate of v_ij . r_ij is positive (the pair of the local particle L and candidate k
    // probably recedes): cell-relative FP32 positions, the local particle's FP32 velocity from its slot.
    static __device__ __forceinline__ bool receding(const Lhs &L, const Tile &T, int k)
    {
        const float4 p = T.f4[k];
        const float3 vj = vel_estimate(T, k);
        const float *v = reinterpret_cast<const float *>(L.s + kVelF);
        const float dx = L.fx - p.x, dy = L.fy - p.y, dz = L.fz - p.z;
        return fmaf(ldsf(v) - vj.x, dx, fmaf(ldsf(v + 1) - vj.y, dy, (ldsf(v + 2) - vj.z) * dz)) > 0.0f;
    }
    // visc (warp-uniform): the whole term.  !visc (a round of pairs estimated receding): the viscosity terms only
    // where the FP64 v_ij . r_ij is negative after all (bits of -0 included), exactly as the whole term takes them;
    // elsewhere they are zero and skipped (the acceleration and du/dt then differ from the whole term's at most in
    // the sign of an exact zero).
    static __device__ __forceinline__ bool eval(const Args &A, const Lhs &L, const Tile &T, const NbrTable &nb,
                                                bool wrap, int i, int k, Part &P, bool visc)
    {
        const double *R_ = T.d + k * NF;
        const double *L_ = L.s;
        const double dx = lds(L_ + X) - R_[X], dy = lds(L_ + Y) - R_[Y], dz = lds(L_ + Z) - R_[Z];
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double rinv = rsqrt_seeded(r2);
        const long long rb = __double_as_longlong(r2);
        const long long r4 = rb - (2LL << 52), r16 = rb - (4LL << 52);  // bits of r^2/4 and r^2/16
        const long long qbi = __double_as_longlong(lds(L_ + Q2)), qbj = __double_as_longlong(T.q[k]);
        const bool ii = r4 < qbi, io = r16 < qbi;  // r < h_i, r < 2 h_i
        const bool ji = r4 < qbj, jo = r16 < qbj;  // r < h_j, r < 2 h_j
        // c = -K1 (inner), K1 (outer), 0 (beyond): the sign bit is flipped on the integer pipe
        const long long k1i = __double_as_longlong(lds(L_ + K1)), k1j = __double_as_longlong(R_[K1]);
        const double Ci = __longlong_as_double(io ? (ii ? k1i ^ kSignBit : k1i) : 0LL);
        const double Cj = __longlong_as_double(jo ? (ji ? k1j ^ kSignBit : k1j) : 0LL);
        const double Fi = fma(fma(ii ? lds(L_ + K2I) : (io ? lds(L_ + K2O) : 0.0), r2, ii ? 0.0 : (io ? lds(L_ + S0) : 0.0)),
                              rinv, Ci);
        const double Fj = fma(fma(ji ? R_[K2I] : (jo ? R_[K2O] : 0.0), r2, ji ? 0.0 : (jo ? R_[S0] : 0.0)), rinv, Cj);
        const double dvx = lds(L_ + VX) - R_[VX], dvy = lds(L_ + VY) - R_[VY], dvz = lds(L_ + VZ) - R_[VZ];
        const double vdotr = fma(dvx, dx, fma(dvy, dy, dvz * dz));
        const double aF = lds(L_ + AP) * Fi;
        double cpart = aF, dpart = aF;  // aF + V and aF + V/2
        if (visc || __double2hiint(vdotr) < 0) {
            const double hbs = lds(L_ + HS) + R_[HS];
            const double D1 = kSoft ? fma(hbs, hbs, r2) : r2;
            const double D2 = lds(L_ + RHO) + R_[RHO];
            const double R = rcp_seeded(D1 * D2);
            const double g = (hbs * vdotr) * R;
            const double mu = g * D2;
            const double t = fma(A.beta_s, mu, -(lds(L_ + ACS) + R_[ACS]));
            double Ph = g * t;
            if (__double2hiint(vdotr) >= 0) Ph = 0.0;  // receding (or v.r = +0): no viscosity
            const double V = Ph * (Fi + Fj);             // Pi * gradbar / r_ij
            cpart = aF + V;
            dpart = fma(0.5, V, aF);
        }
        const double mj = R_[M];
        const double coef = mj * fma(R_[AP], Fj, cpart);
        P.ax = fma(-coef, dx, P.ax);
        P.ay = fma(-coef, dy, P.ay);
        P.az = fma(-coef, dz, P.az);
        P.du = fma(mj * vdotr, dpart, P.du);
        return io || jo;
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

// ------------------------------------------------------------------------------------------------------------
// Kernel families and the fuller views (FP64, single-grid views).  The two bodies below serve every
// (kernel, scheme) pair except (cubic, minimal), which DensF64 / ForceF64 cover with the cubic's piece
// coefficients in r.  Here the kernel is evaluated from q = r/h; as sums of truncated powers (t)_+ = max(t, 0):
//   cubic M4 (support 2h, sigma 1/pi):         f = 1/4 (2 - q)_+^3 - (1 - q)_+^3
//   quartic M5 (support 5h/2, sigma 1/(20 pi), the paper's kernel, Section 2.1):
//                                              f = (5/2 - q)_+^4 - 5 (3/2 - q)_+^4 + 10 (1/2 - q)_+^4
// W = sigma f / h^3, dW/dr = sigma f' / h^4 and dW/dh = -sigma (3 f + q f') / h^4: beyond the support every
// coefficient is zero, which is the masking of Section 5.6.
// ------------------------------------------------------------------------------------------------------------
// f on each piece as a polynomial in q, f = sum_k a_k q^k, the piece chosen by integer compares of the bit
// pattern of q (for doubles >= 0 the bit patterns order like the values) and every coefficient 0 beyond the
// support: four FMAs for f, three for f', where the truncated powers cost about twice as many FP64 operations.
// The expansions (of the truncated-power forms above, term by term):
//   M4:  q < 1:  1 - 3/2 q^2 + 3/4 q^3            q < 2:  2 - 3q + 3/2 q^2 - 1/4 q^3
//   M5:  q < 1/2: 115/8 - 15 q^2 + 6 q^4          q < 3/2: 55/4 + 5q - 30 q^2 + 20 q^3 - 4 q^4
//        q < 5/2: 625/16 - 125/2 q + 75/2 q^2 - 10 q^3 + q^4
struct KerM4 {
    static constexpr double kappa = 2.0;
    static constexpr float kappaf = 2.0f;
    static constexpr double sigma = kInvPi;
    static __device__ __forceinline__ void f_fp(double q, double &f, double &fp)
    {
        const long long qb = __double_as_longlong(q);
        const bool in = qb < 0x3FF0000000000000LL, out = qb < 0x4000000000000000LL;  // q < 1, q < 2
        const double a3 = in ? 0.75 : (out ? -0.25 : 0.0), a2 = in ? -1.5 : (out ? 1.5 : 0.0);
        const double a1 = in ? 0.0 : (out ? -3.0 : 0.0), a0 = in ? 1.0 : (out ? 2.0 : 0.0);
        f = fma(fma(fma(a3, q, a2), q, a1), q, a0);
        const double b2 = in ? 2.25 : (out ? -0.75 : 0.0), b1 = in ? -3.0 : (out ? 3.0 : 0.0);
        fp = fma(fma(b2, q, b1), q, a1);
    }
    static __device__ __forceinline__ double fp_only(double q)
    {
        const long long qb = __double_as_longlong(q);
        const bool in = qb < 0x3FF0000000000000LL, out = qb < 0x4000000000000000LL;
        const double b2 = in ? 2.25 : (out ? -0.75 : 0.0), b1 = in ? -3.0 : (out ? 3.0 : 0.0);
        const double b0 = in ? 0.0 : (out ? -3.0 : 0.0);
        return fma(fma(b2, q, b1), q, b0);
    }
};
struct KerM5 {
    static constexpr double kappa = 2.5;
    static constexpr float kappaf = 2.5f;
    static constexpr double sigma = kInvPi / 20.0;
    static __device__ __forceinline__ void f_fp(double q, double &f, double &fp)
    {
        const long long qb = __double_as_longlong(q);
        // q < 1/2, q < 3/2, q < 5/2
        const bool p0 = qb < 0x3FE0000000000000LL, p1 = qb < 0x3FF8000000000000LL, p2 = qb < 0x4004000000000000LL;
        const double a4 = p0 ? 6.0 : (p1 ? -4.0 : (p2 ? 1.0 : 0.0));
        const double a3 = p0 ? 0.0 : (p1 ? 20.0 : (p2 ? -10.0 : 0.0));
        const double a2 = p0 ? -15.0 : (p1 ? -30.0 : (p2 ? 37.5 : 0.0));
        const double a1 = p0 ? 0.0 : (p1 ? 5.0 : (p2 ? -62.5 : 0.0));
        const double a0 = p0 ? 14.375 : (p1 ? 13.75 : (p2 ? 39.0625 : 0.0));
        f = fma(fma(fma(fma(a4, q, a3), q, a2), q, a1), q, a0);
        const double b3 = p0 ? 24.0 : (p1 ? -16.0 : (p2 ? 4.0 : 0.0));    // 4 a4
        const double b2 = p0 ? 0.0 : (p1 ? 60.0 : (p2 ? -30.0 : 0.0));    // 3 a3
        const double b1 = p0 ? -30.0 : (p1 ? -60.0 : (p2 ? 75.0 : 0.0));  // 2 a2
        fp = fma(fma(fma(b3, q, b2), q, b1), q, a1);
    }
    static __device__ __forceinline__ double fp_only(double q)
    {
        const long long qb = __double_as_longlong(q);
        const bool p0 = qb < 0x3FE0000000000000LL, p1 = qb < 0x3FF8000000000000LL, p2 = qb < 0x4004000000000000LL;
        const double b3 = p0 ? 24.0 : (p1 ? -16.0 : (p2 ? 4.0 : 0.0));
        const double b2 = p0 ? 0.0 : (p1 ? 60.0 : (p2 ? -30.0 : 0.0));
        const double b1 = p0 ? -30.0 : (p1 ? -60.0 : (p2 ? 75.0 : 0.0));
        const double b0 = p0 ? 0.0 : (p1 ? 5.0 : (p2 ? -62.5 : 0.0));
        return fma(fma(fma(b3, q, b2), q, b1), q, b0);
    }
};

// Reduce-scatter of NV (a power of two <= 32) per-lane values over the warp: afterwards lane l holds the warp
// sum of value l >> (5 - log2 NV).  Every value is summed over the butterfly tree xor 16, 8, 4, 2, 1.
template <int NV>
__device__ __forceinline__ double reduce_scatter(const double (&v)[NV], int lane)
{
    double cur[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) cur[k] = v[k];
    int n = NV;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (n > 1) {
            const bool up = (lane & o) != 0;
            n >>= 1;
#pragma unroll
            for (int k = 0; k < NV / 2; ++k) {
                if (k < n) {
                    const double keep = up ? cur[k + n] : cur[k];
                    const double send = up ? cur[k] : cur[k + n];
                    cur[k] = keep + __shfl_xor_sync(kFull, send, o);
                }
            }
        } else {
            cur[0] += __shfl_xor_sync(kFull, cur[0], o);
        }
    }
    return cur[0];
}

// Density of the kernel family Ker; with Ext also the fuller density view: drho/dh (for Omega), the neighbour
// count, and the velocity divergence and curl estimates
//   (div v)_i = -1/rho_i sum_j m_j v_ij . grad_i W(r_ij, h_i),  (curl v)_i = 1/rho_i sum_j m_j v_ij x grad_i W.
template <class Ker, bool Ext>
struct DensF64G {
    enum { X, Y, Z, VX, VY, VZ, HINV, S0, S1, NF };  // slot members (VX..VZ read only with Ext)
    struct Args {
        PairCommon cm;
        const double *f[NF];  // x, y, z, v, and (prep) 1/h, sigma/h^3, sigma/h^4
        const double *m, *h, *u, *cs0;
        const float *xf, *yf, *zf;
        double *rho, *P, *cs;
        double *nnb, *divv, *cx, *cy, *cz, *omega;  // Ext only
        double gamma;
    };
    static constexpr int kRow = Ext ? 7 : 5;  // odd row length: x, y, z, m (, vx, vy, vz) and padding
    struct Tile {
        double *d;
        float4 *f4;
    };
    struct Lhs {
        const double *s;
        float fx, fy, fz, b2;
    };
    struct Part {
        double rho, drho, dv, cx, cy, cz;
        int cnt;
        __device__ __forceinline__ void zero()
        {
            rho = drho = dv = cx = cy = cz = 0.0;
            cnt = 0;
        }
    };
    struct Acc {
        double rho, drho, dv, cx, cy, cz;
        int cnt;
    };
    static constexpr int kStageBytes = kRow * 8 + 16;
    static constexpr int kSlotDoubles = 17;
    static constexpr bool kSkipSelf = false;  // the sums include the self term
    static constexpr bool kSelfInFinish = false;
    static constexpr bool kSplit = false;
    static constexpr int min_ctas(int nt) { return nt == 128 ? 6 : 3; }
    // the two particles of a warp's queue: Ext reduces 12 sums with one 16-value reduce-scatter, the plain
    // density its 2 sums; the neighbour counts are integer warp sums
    static constexpr int kGroup = 2;
    struct Group {
        Part P0, P1;
        int l0, l1;
        __device__ __forceinline__ void zero() {}
        __device__ __forceinline__ void put(int u, const Part &P, int li)
        {
            if (u == 0) { P0 = P; l0 = li; }
            else { P1 = P; l1 = li; }
        }
        __device__ __forceinline__ void accumulate(Acc *acc, int nu, int lane)
        {
            if constexpr (Ext) {
                const double v[16] = {P0.rho, P0.drho, P0.dv, P0.cx, P0.cy, P0.cz,
                                      P1.rho, P1.drho, P1.dv, P1.cx, P1.cy, P1.cz, 0.0, 0.0, 0.0, 0.0};
                const double t = reduce_scatter<16>(v, lane);
                const int c0 = __reduce_add_sync(kFull, P0.cnt), c1 = __reduce_add_sync(kFull, P1.cnt);
                const int g = lane >> 1;  // value index
                if ((lane & 1) == 0 && g < 12) {
                    const int u = g / 6, c = g - 6 * u;
                    if (u < nu) {
                        Acc &a = acc[u == 0 ? l0 : l1];
                        if (c == 0) a.rho += t;
                        else if (c == 1) a.drho += t;
                        else if (c == 2) a.dv += t;
                        else if (c == 3) a.cx += t;
                        else if (c == 4) a.cy += t;
                        else a.cz += t;
                    }
                }
                if (lane == 0) acc[l0].cnt += c0;
                if (lane == 0 && nu > 1) acc[l1].cnt += c1;
            } else {
                const double v[2] = {P0.rho, P1.rho};
                const double t = reduce_scatter<2>(v, lane);
                const int u = lane >> 4;
                if ((lane & 15) == 0 && u < nu) acc[u == 0 ? l0 : l1].rho += t;
                const int c0 = __reduce_add_sync(kFull, P0.cnt), c1 = __reduce_add_sync(kFull, P1.cnt);
                if (lane == 0) acc[l0].cnt += c0;
                if (lane == 0 && nu > 1) acc[l1].cnt += c1;
            }
        }
    };

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        t.d = reinterpret_cast<double *>(s);
        t.f4 = reinterpret_cast<float4 *>(t.d + kRow * tj);
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        double xs = A.f[X][slot], ys = A.f[Y][slot], zs = A.f[Z][slot];
        if (nb.wrap) {  // the image of a neighbour across the periodic boundary
            xs -= nb.shift[q][0];
            ys -= nb.shift[q][1];
            zs -= nb.shift[q][2];
        }
        double *row = T.d + t * kRow;
        row[0] = xs;
        row[1] = ys;
        row[2] = zs;
        row[3] = A.m[slot];
        if constexpr (Ext) {
            row[4] = A.f[VX][slot];
            row[5] = A.f[VY][slot];
            row[6] = A.f[VZ][slot];
        }
        T.f4[t] = make_float4(A.xf[slot] + nb.offf[q][0], A.yf[slot] + nb.offf[q][1], A.zf[slot] + nb.offf[q][2],
                              0.0f);
    }
    static __device__ __forceinline__ void sentinel(const Tile &T, int t) { T.f4[t] = make_float4(kFar, kFar, kFar, 0.f); }
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float margin, double *ws)
    {
        const int lane = threadIdx.x & 31;
        if (lane < NF && (Ext || lane < VX || lane > VZ)) ws[lane] = A.f[lane][i];
        __syncwarp();
        Lhs L;
        L.s = ws;
        L.fx = A.xf[i];
        L.fy = A.yf[i];
        L.fz = A.zf[i];
        const float rf = __fmaf_ru(Ker::kappaf * (1.0f + 4e-6f), __double2float_ru(A.h[i]), margin);
        L.b2 = __fmul_ru(rf, rf);
        return L;
    }
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float4 p = T.f4[k];
        const float dx = L.fx - p.x, dy = L.fy - p.y, dz = L.fz - p.z;
        return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < L.b2;
    }
    static __device__ __forceinline__ bool eval(const Args &, const Lhs &L, const Tile &T, const NbrTable &,
                                                bool, int, int k, Part &P)
    {
        const double *R_ = T.d + k * kRow;
        const double *s = L.s;
        const double dx = lds(s + X) - R_[0], dy = lds(s + Y) - R_[1], dz = lds(s + Z) - R_[2];
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double rinv = rsqrt_seeded(r2);
        const double r = r2 * rinv;
        const double q = r * lds(s + HINV);
        double f, fp;
        Ker::f_fp(q, f, fp);
        const double mj = R_[3];
        P.rho = fma(mj, lds(s + S0) * f, P.rho);
        const bool supp = q < Ker::kappa;
        P.cnt += supp ? 1 : 0;
        if constexpr (Ext) {
            const double s1 = lds(s + S1);
            P.drho = fma(mj, -s1 * fma(q, fp, 3.0 * f), P.drho);
            const double mG = mj * ((s1 * fp) * rinv);  // m_j dW/dr / r
            const double vx = lds(s + VX) - R_[4], vy = lds(s + VY) - R_[5], vz = lds(s + VZ) - R_[6];
            P.dv = fma(mG, fma(vx, dx, fma(vy, dy, vz * dz)), P.dv);
            P.cx = fma(mG, fma(vy, dz, -(vz * dy)), P.cx);
            P.cy = fma(mG, fma(vz, dx, -(vx * dz)), P.cy);
            P.cz = fma(mG, fma(vx, dy, -(vy * dx)), P.cz);
        }
        return supp;
    }
    static __device__ __forceinline__ void finish(const Args &A, int i, const Acc &a)
    {
        const double h = A.h[i];
        const double rho = a.rho;
        const double P = (A.gamma - 1.0) * rho * A.u[i];
        const double cs = A.cs0[i];
        A.rho[i] = rho;
        A.P[i] = P;
        A.cs[i] = cs;
        unsigned bits = 0;
        if constexpr (Ext) {
            const double ri = 1.0 / rho;
            A.nnb[i] = (double)(a.cnt - 1);  // the local particle itself is in its own tile once
            A.divv[i] = -a.dv * ri;
            A.cx[i] = a.cx * ri;
            A.cy[i] = a.cy * ri;
            A.cz[i] = a.cz * ri;
            const double om = 1.0 + h / (3.0 * rho) * a.drho;
            A.omega[i] = om;
            if (!isfinite(om) || !isfinite(a.dv) || !isfinite(a.cx) || !isfinite(a.cy) || !isfinite(a.cz))
                bits |= SPH_DEV_NONFINITE;
        }
        if (!(rho > 0.0) || !isfinite(rho) || !isfinite(P) || !isfinite(cs)) bits |= SPH_DEV_NONFINITE;
        if (!(Ker::kappa * h <= A.cm.cs.g.min_edge)) bits |= SPH_DEV_H_TOO_BIG;
        if (bits) atomicOr(A.cm.status, bits);
    }
    static __device__ __forceinline__ void count(const Args &A, unsigned long long cand,
                                                 unsigned long long pairs)
    {
        atomicAdd(&A.cm.counters->dens_cand, cand);
        atomicAdd(&A.cm.counters->dens_pairs, pairs);
    }
};

// Force of the kernel family Ker; with Ext the fuller force view: P/rho^2 becomes P/(Omega rho^2) (grad-h
// terms), the viscosity is scaled by the pair mean of the Balsara switch B, and the signal velocity
// max_j (c_i + c_j - 3 min(v_ij . r_ij / r, 0)) is written too.  The per-particle A = P/(Omega rho^2) and B come
// from the prep kernel (Omega = B = 1 without Ext).
template <class Ker, bool Ext>
struct ForceF64G {
    enum { X, Y, Z, VX, VY, VZ, M, HH, HINV, S1, AP, ACH, RHO, CS, BAL, NF };
    struct Args {
        PairCommon cm;
        const double *f[NF];
        const float *xf, *yf, *zf, *hf;
        double *ax, *ay, *az, *dudt, *vsig;
        double beta, eps;
    };
    struct Tile {
        double *d;
        float4 *f4;
    };
    struct Lhs {
        const double *s;
        float fx, fy, fz, fh, margin;
    };
    struct Part {
        double ax, ay, az, du, vs;
        __device__ __forceinline__ void zero() { ax = ay = az = du = vs = 0.0; }
    };
    struct Acc {
        double ax, ay, az, du, vs;
    };
    static constexpr int kStageBytes = NF * 8 + 16;
    static constexpr int kSlotDoubles = 17;
    static constexpr bool kSkipSelf = true;  // as ForceF64
    static constexpr bool kSelfInFinish = false;
    static constexpr bool kSplit = false;
    // three 256-thread CTAs per SM, as ForceF64 (the 448 tile's shared memory allows three)
    static constexpr int min_ctas(int) { return 3; }
    static constexpr int kGroup = 2;
    struct Group {
        Part P0, P1;
        int l0, l1;
        __device__ __forceinline__ void zero() {}
        __device__ __forceinline__ void put(int u, const Part &P, int li)
        {
            if (u == 0) { P0 = P; l0 = li; }
            else { P1 = P; l1 = li; }
        }
        __device__ __forceinline__ void accumulate(Acc *acc, int nu, int lane)
        {
            const double v[8] = {P0.ax, P0.ay, P0.az, P0.du, P1.ax, P1.ay, P1.az, P1.du};
            const double t = reduce_scatter<8>(v, lane);
            const int g = lane >> 2, u = g >> 2, c = g & 3;
            if ((lane & 3) == 0 && u < nu) {
                Acc &a = acc[u == 0 ? l0 : l1];
                if (c == 0) a.ax += t;
                else if (c == 1) a.ay += t;
                else if (c == 2) a.az += t;
                else a.du += t;
            }
            if constexpr (Ext) {  // maxima are exact in any order
                double m0 = P0.vs, m1 = P1.vs;
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    m0 = fmax(m0, __shfl_xor_sync(kFull, m0, o));
                    m1 = fmax(m1, __shfl_xor_sync(kFull, m1, o));
                }
                if (lane == 0) acc[l0].vs = fmax(acc[l0].vs, m0);
                if (lane == 0 && nu > 1) acc[l1].vs = fmax(acc[l1].vs, m1);
            }
        }
    };

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        t.d = reinterpret_cast<double *>(s);
        t.f4 = reinterpret_cast<float4 *>(t.d + NF * tj);
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        double *row = T.d + t * NF;
        double xs = A.f[X][slot], ys = A.f[Y][slot], zs = A.f[Z][slot];
        if (nb.wrap) {
            xs -= nb.shift[q][0];
            ys -= nb.shift[q][1];
            zs -= nb.shift[q][2];
        }
        row[X] = xs;
        row[Y] = ys;
        row[Z] = zs;
#pragma unroll
        for (int f = VX; f < NF; ++f) row[f] = A.f[f][slot];
        T.f4[t] = make_float4(A.xf[slot] + nb.offf[q][0], A.yf[slot] + nb.offf[q][1], A.zf[slot] + nb.offf[q][2],
                              A.hf[slot]);
    }
    static __device__ __forceinline__ void sentinel(const Tile &T, int t) { T.f4[t] = make_float4(kFar, kFar, kFar, 0.f); }
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float margin, double *ws)
    {
        const int lane = threadIdx.x & 31;
        if (lane < NF) ws[lane] = A.f[lane][i];
        __syncwarp();
        Lhs L;
        L.s = ws;
        L.fx = A.xf[i];
        L.fy = A.yf[i];
        L.fz = A.zf[i];
        L.fh = A.hf[i];
        L.margin = margin;
        return L;
    }
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float4 p = T.f4[k];
        const float dx = L.fx - p.x, dy = L.fy - p.y, dz = L.fz - p.z;
        const float rf = __fmaf_ru(Ker::kappaf * (1.0f + 4e-6f), fmaxf(L.fh, p.w), L.margin);
        return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < __fmul_ru(rf, rf);
    }
    static __device__ __forceinline__ bool eval(const Args &A, const Lhs &L, const Tile &T, const NbrTable &,
                                                bool, int i, int k, Part &P)
    {
        const double *R_ = T.d + k * NF;
        const double *L_ = L.s;
        const double dx = lds(L_ + X) - R_[X], dy = lds(L_ + Y) - R_[Y], dz = lds(L_ + Z) - R_[Z];
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double rinv = rsqrt_seeded(r2);
        const double r = r2 * rinv;
        const double qi = r * lds(L_ + HINV), qj = r * R_[HINV];
        const double Fi = (lds(L_ + S1) * Ker::fp_only(qi)) * rinv;  // dW/dr(r, h_i) / r
        const double Fj = (R_[S1] * Ker::fp_only(qj)) * rinv;
        const double dvx = lds(L_ + VX) - R_[VX], dvy = lds(L_ + VY) - R_[VY], dvz = lds(L_ + VZ) - R_[VZ];
        const double vdotr = fma(dvx, dx, fma(dvy, dy, dvz * dz));
        // Monaghan viscosity, the unscaled form of ForceF64's: Ph = Pi / 2 = g (beta mu - alpha cbar), g = w R,
        // mu = g D2, with D1 = r^2 + eps hbar^2 formed per pair
        const double hb = lds(L_ + HH) + R_[HH];
        const double D1 = fma(A.eps * hb, hb, r2);
        const double D2 = lds(L_ + RHO) + R_[RHO];
        const double R = rcp_seeded(D1 * D2);
        const double g = (hb * vdotr) * R;
        const double mu = g * D2;
        const double t = fma(A.beta, mu, -(lds(L_ + ACH) + R_[ACH]));
        double Ph = g * t;
        if constexpr (Ext) Ph = Ph * (0.5 * (lds(L_ + BAL) + R_[BAL]));
        if (__double2hiint(vdotr) >= 0) Ph = 0.0;  // receding (or v.r = +0): no viscosity
        const double V = Ph * (Fi + Fj);
        const double aF = lds(L_ + AP) * Fi;
        const double mj = R_[M];
        const double coef = mj * fma(R_[AP], Fj, aF + V);
        const bool in = qi < Ker::kappa || qj < Ker::kappa;
        P.ax = fma(-coef, dx, P.ax);
        P.ay = fma(-coef, dy, P.ay);
        P.az = fma(-coef, dz, P.az);
        P.du = fma(mj * vdotr, fma(0.5, V, aF), P.du);
        if constexpr (Ext) {
            const double w = vdotr * rinv;
            const double vs = (lds(L_ + CS) + R_[CS]) - 3.0 * fmin(w, 0.0);
            if (in) P.vs = fmax(P.vs, vs);
        }
        return in;
    }
    static __device__ __forceinline__ void finish(const Args &A, int i, const Acc &a)
    {
        A.ax[i] = a.ax;
        A.ay[i] = a.ay;
        A.az[i] = a.az;
        A.dudt[i] = a.du;
        if constexpr (Ext) A.vsig[i] = a.vs;
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

// ---- force, FP32 (lane driver: candidates filtered into a per-lane hit mask, only hits evaluated) ----
// grad_i W(r_ij, h) = F r_ij with F = 3 (t^2 - s^2) / (pi h^4 r), s = sat(1 - q/2), t = sat(1 - q) (the derivative
// of f = 2 s^3 - t^3); 3/(pi h^4) comes per particle from k_force_prep_f32.  The viscosity uses
// min(v_ij . r_ij, 0), which makes Pi_ij vanish for receding pairs without a branch.  A pair at r = 0 (the self
// pair, or two coincident particles) contributes exactly 0: q = 0 gives F = 0, r_ij = 0, and D1 >= 1e-30 keeps
// the viscosity finite (0) there when eps = 0.  The pairs counted are the filter's hits,
// r^2 < 4 max(h_i, h_j)^2, minus the self pair of every local particle.
struct ForceF32 {
    static constexpr bool kMasked = false;
    // One CTA per cell: no register bound (0); the compiler's own choice (70 registers, seven 128-thread CTAs per
    // SM) measured faster than a bound of seven CTAs (72 registers), and a bound of eight spills.  The
    // persistent form (patch views) measured faster with the bound of seven.
    static constexpr int min_ctas(int) { return 0; }
    static constexpr int min_ctas_persist(int nt) { return nt == 128 ? 7 : 3; }
    struct Args {
        PairCommon cm;
        const float *x, *y, *z, *vx, *vy, *vz, *m, *h, *rho, *cs;
        const float *hinv, *k4, *A;
        float *ax, *ay, *az, *dudt;
        float alpha, beta, eps;
    };
    // Staged members in four float4 groups (one 16-byte shared load each): the filter reads only p4.
    struct Tile {
        float4 *p4;  // position seen from the local cell, 4 h^2
        float4 *v4;  // velocity, mass
        float4 *g4;  // h, 1/h, 3/(pi h^4), P/rho^2
        float2 *c2;  // c_s, rho
    };
    struct Lhs {
        float x, y, z, vx, vy, vz, h, hinv, k4, A, c, rho, b2;
    };
    // The four compensated sums as two pairs, (a_x, a_y) and (a_z, du/dt), for paired FP32 updates.
    struct Part {
        Kahan2 axy, azd;
        __device__ __forceinline__ void zero()
        {
            axy.zero();
            azd.zero();
        }
    };
    struct Acc {
        float2 ax, ay, az, du;
    };
    static constexpr int kStageBytes = 3 * 16 + 8;

    static __device__ Tile carve(unsigned char *s, int tj)
    {
        Tile t;
        t.p4 = reinterpret_cast<float4 *>(s);
        t.v4 = t.p4 + tj;
        t.g4 = t.v4 + tj;
        t.c2 = reinterpret_cast<float2 *>(t.g4 + tj);
        return t;
    }
    static __device__ __forceinline__ void stage(const Args &A, const Tile &T, const NbrTable &nb, int t,
                                                 int slot, int q)
    {
        const float h = A.h[slot];
        T.p4[t] = make_float4(A.x[slot] + nb.offf[q][0], A.y[slot] + nb.offf[q][1], A.z[slot] + nb.offf[q][2],
                              4.0f * h * h);
        T.v4[t] = make_float4(A.vx[slot], A.vy[slot], A.vz[slot], A.m[slot]);
        T.g4[t] = make_float4(h, A.hinv[slot], A.k4[slot], A.A[slot]);
        T.c2[t] = make_float2(A.cs[slot], A.rho[slot]);
    }
    static __device__ __forceinline__ Lhs load(const Args &A, int i, float, double *)
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
        L.k4 = A.k4[i];
        L.A = A.A[i];
        L.c = A.cs[i];
        L.rho = A.rho[i];
        L.b2 = 4.0f * L.h * L.h;
        return L;
    }
    // r < 2 max(h_i, h_j), as r^2 < max(4 h_i^2, 4 h_j^2) (the same float products the staging formed).
    static __device__ __forceinline__ bool filter(const Lhs &L, const Tile &T, int k)
    {
        const float4 p = T.p4[k];
        const float dx = L.x - p.x, dy = L.y - p.y, dz = L.z - p.z;
        return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < fmaxf(L.b2, p.w);
    }
    // Where two quantities go through the same operation (the x and y components, the i and j sides of the
    // kernel gradient, ...) they share one paired FP32 instruction; every operation and its order is that of the
    // scalar form, so the results are the same.
    static __device__ __forceinline__ void eval(const Args &A, const Lhs &L, const Tile &T, int k, Part &P)
    {
        const float4 p = T.p4[k];
        const float4 vm = T.v4[k];
        const float4 g = T.g4[k];
        const float2 cr = T.c2[k];
        const float2 neg = make_float2(-1.0f, -1.0f);
        const float2 dxy = __ffma2_rn(make_float2(p.x, p.y), neg, make_float2(L.x, L.y));
        const float dz = L.z - p.z;
        const float r2 = fmaf(dxy.x, dxy.x, fmaf(dxy.y, dxy.y, dz * dz));
        const float r2e = r2 + 1e-30f;  // > 0 at r = 0; equal to r2 for r2 >= 2^-75
        const float rinv = rsqrt_ftz(r2e);
        const float r = r2 * rinv;
        const float2 q = __fmul2_rn(make_float2(r, r), make_float2(L.hinv, g.y));  // q_i, q_j
        const float2 sq = make_float2(fma_sat(-0.5f, q.x, 1.0f), fma_sat(-0.5f, q.y, 1.0f));
        const float2 tq = make_float2(fma_sat(-1.0f, q.x, 1.0f), fma_sat(-1.0f, q.y, 1.0f));
        // (F_i, F_j) = (k4 / r) ((t - s) (t + s)) for each side
        const float2 F = __fmul2_rn(__fmul2_rn(make_float2(L.k4, g.z), make_float2(rinv, rinv)),
                                    __fmul2_rn(__ffma2_rn(sq, neg, tq), __fadd2_rn(tq, sq)));
        const float2 dvxy = __ffma2_rn(make_float2(vm.x, vm.y), neg, make_float2(L.vx, L.vy));
        const float dvz = L.vz - vm.z;
        const float vdotr = fmaf(dvxy.x, dxy.x, fmaf(dvxy.y, dxy.y, dvz * dz));
        const float vneg = 0.5f * (vdotr - fabsf(vdotr));  // min(v_ij . r_ij, 0)
        const float2 hc = __fmul2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(make_float2(L.h, L.c), make_float2(g.x, cr.x)));
        const float hb = hc.x, cb = hc.y;  // hbar, cbar
        const float D1 = fmaf(A.eps * hb, hb, r2e);  // finite R at r = 0 even for eps = 0
        const float D2 = L.rho + cr.y;
        const float R = rcp_ftz(D1 * D2);
        const float2 m1 = __fmul2_rn(make_float2(hb, D2), make_float2(vneg, R));
        const float mu = m1.x * m1.y;  // (hbar v-) (D2 R)
        const float2 m2 = __fmul2_rn(make_float2(mu, D1), make_float2(fmaf(A.beta, mu, -A.alpha * cb), R));
        const float Ph = m2.x * m2.y;
        const float Fs = F.x + F.y;
        const float aF = L.A * F.x;
        const float mj = vm.w;
        const float ncoef = -mj * fmaf(Ph, Fs, fmaf(g.w, F.y, aF));  // -coef
        const float2 m3 = __fmul2_rn(make_float2(mj, 0.5f), make_float2(vdotr, Ph));
        const float dcoef = m3.x * fmaf(m3.y, Fs, aF);
        P.axy.add(__fmul2_rn(make_float2(ncoef, ncoef), dxy));
        P.azd.add(make_float2(ncoef * dz, dcoef));
    }
    static __device__ __forceinline__ void merge2(float2 &a, float ps, float pc)
    {
        Kahan k;
        k.s = a.x;
        k.c = a.y;
        k.merge(ps, pc);
        a.x = k.s;
        a.y = k.c;
    }
    static __device__ __forceinline__ void merge_part(Acc &a, const Part &P)
    {
        merge2(a.ax, P.axy.s.x, P.axy.c.x);
        merge2(a.ay, P.axy.s.y, P.axy.c.y);
        merge2(a.az, P.azd.s.x, P.azd.c.x);
        merge2(a.du, P.azd.s.y, P.azd.c.y);
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

// Every accumulator starts at zero (value initialisation zeroes each member).
template <class K>
__device__ __forceinline__ void zero_acc(typename K::Acc &a)
{
    a = typename K::Acc{};
}

// ------------------------------------------------------------------------------------------------------------
// The per-cell driver of the FP64 loop bodies.
// ------------------------------------------------------------------------------------------------------------
template <class K, int NT>
struct PairShared {
    NbrTable nb;
    typename K::Acc acc[kMaxLocal];
    union {
        int ring[NT / 32][kRing];                 // tile_pairs: one queue per warp
        unsigned short ring2[NT / 32][2][kRing];  // tile_pairs_split: Q, then A and B (half a ring each)
    };
    // per warp: its two local particles (K::load); an odd slot length puts member f of the two slots in
    // different banks, so a round that mixes the two particles reads both without a bank conflict
    double lslot[NT / 32][2][K::kSlotDoubles];
    unsigned long long pairs;
};

// One staged tile against the local particles, two at a time per warp (particles 2m and 2m + 1 for m = warp,
// warp + W, ...: the pairing does not depend on the warp count).  Both particles' filter hits go to the warp's one
// queue, tagged with the particle, and every evaluation round takes 32 queue entries whichever particle they
// belong to: only the last round of the pair of particles runs part-full, where one particle per warp would leave
// a part-full round per particle.  Each lane evaluates with the members of its entry's particle (shared slot 0 or
// 1) into that particle's partial sums; the partials are reduced over the warp kGroup particles at a time.
// With K::kSkipSelf the filter drops each particle's own entry: the local cell is neighbour 13 of the table (the
// periodic domains have at least 3 cells per axis, so it appears once), which puts slot i at tile position
// pref[13] + (i - start[13]) - tb.
template <class K, int NT>
__device__ __forceinline__ void tile_pairs(const typename K::Args &A, const typename K::Tile &T,
                                           PairShared<K, NT> &S, int ib, int nloc, int tb, int tnp, float margin,
                                           bool wrap, unsigned long long &my_pairs)
{
    constexpr int W = NT / 32;
    constexpr int kTag = 1 << 14;  // entry = candidate | kTag for the second particle (candidates < 4096)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    int *q = S.ring[warp];
    const NbrTable &nb = S.nb;
    typename K::Group G;  // groups of kGroup > 2 particles span several pairs
    G.zero();
    int nu = 0;  // particles held by G (warp-uniform)
    for (int li0 = 2 * warp; li0 < nloc; li0 += 2 * W) {
        const bool two = li0 + 1 < nloc;  // warp-uniform
        const int i0 = ib + li0, i1 = two ? i0 + 1 : i0;
        const typename K::Lhs L0 = K::load(A, i0, margin, S.lslot[warp][0]);
        const typename K::Lhs L1 = K::load(A, i1, margin, S.lslot[warp][1]);
        typename K::Part P0, P1;
        P0.zero();
        P1.zero();
        int head = 0, tail = 0;  // warp-uniform ring cursors; tail - head <= 31 + 64
        auto round = [&](bool act) {
            bool in = false;
            if (act) {
                const int e = q[(head + lane) & (kRing - 1)];
                const bool tag = (e & kTag) != 0;
                typename K::Part Pt = tag ? P1 : P0;
                in = K::eval(A, tag ? L1 : L0, T, nb, wrap, tag ? i1 : i0, e & (kTag - 1), Pt);
                if (tag) P1 = Pt; else P0 = Pt;
            }
            const unsigned b = __ballot_sync(kFull, in);  // every lane votes
            if (lane == 0) my_pairs += __popc(b);
        };
        const int self0 = nb.pref[13] + (i0 - nb.start[13]) - tb;  // tile position of i0 (i1 follows it)
        for (int jb = 0; jb < tnp; jb += 32) {
            const int k = jb + lane;
            const bool p0 = K::filter(L0, T, k) && (!K::kSkipSelf || k != self0);
            const bool p1 = two && K::filter(L1, T, k) && (!K::kSkipSelf || k != self0 + 1);
            const unsigned b0 = __ballot_sync(kFull, p0);
            const unsigned b1 = __ballot_sync(kFull, p1);
            const int c0 = __popc(b0);
            if (p0) q[(tail + __popc(b0 & lt_mask)) & (kRing - 1)] = k;
            if (p1) q[(tail + c0 + __popc(b1 & lt_mask)) & (kRing - 1)] = k | kTag;
            tail += c0 + __popc(b1);
            while (tail - head >= 32) {
                __syncwarp();
                round(true);
                head += 32;
            }
        }
        const int rem = tail - head;
        if (rem > 0) {
            __syncwarp();
            round(lane < rem);
        }
        __syncwarp();  // the ring and the slots are reused by the next two particles
        if constexpr (K::kGroup == 2) {  // one reduction per pair of particles
            typename K::Group G2;
            G2.put(0, P0, li0);
            G2.put(1, P1, li0 + 1);  // (all zero when the warp has a single particle)
            G2.accumulate(S.acc, two ? 2 : 1, lane);
        } else {
            G.put(nu++, P0, li0);
            if (two) G.put(nu++, P1, li0 + 1);
            if (nu == K::kGroup || li0 + 2 * W >= nloc) {
                G.accumulate(S.acc, nu, lane);
                G.zero();
                nu = 0;
            }
        }
    }
}

// tile_pairs for loop bodies whose term has a part that vanishes for receding pairs (K::kSplit: the force's
// viscosity).  The filter queues its hits in the warp's ring Q as tile_pairs does; 32 of them at a time are then
// sorted by an FP32 estimate of v_ij . r_ij into two lists, A (approaching, or the estimate not positive) and B
// (receding).  Rounds of 32 A entries take the whole term, rounds of 32 B entries the term without the viscosity
// (which still takes it where the FP64 v_ij . r_ij is negative, so a wrong estimate costs time only).  What is left
// after the tile (fewer than 32 in each list) goes into one round of the whole term, A entries first, then B
// entries (or, without A entries, of the term without the viscosity); B entries beyond 32 take a last round
// without the viscosity.  The entries, their order and the rounds follow from the tile and the pair of particles
// alone, as in tile_pairs.  The term has one call site: the loop below visits every round in one place.
template <class K, int NT>
__device__ __forceinline__ void tile_pairs_split(const typename K::Args &A, const typename K::Tile &T,
                                                 PairShared<K, NT> &S, int ib, int nloc, int tb, int tnp,
                                                 float margin, bool wrap, unsigned long long &my_pairs)
{
    static_assert(K::kSkipSelf && K::kGroup == 2,
                  "split queues: self pairs dropped, sums reduced two particles at a time");
    constexpr int W = NT / 32;
    constexpr int kTag = 1 << 14;  // entry = candidate | kTag for the second particle (candidates < 4096)
    constexpr int kQ = kRing - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned short *q = S.ring2[warp][0], *qa = S.ring2[warp][1], *qb = S.ring2[warp][1] + kRing / 2;
    const NbrTable &nb = S.nb;
    unsigned npair = 0;  // lane 0: in-support pairs of this tile (added to my_pairs at the end)
    for (int li0 = 2 * warp; li0 < nloc; li0 += 2 * W) {
        const bool two = li0 + 1 < nloc;  // warp-uniform
        const int i0 = ib + li0, i1 = two ? i0 + 1 : i0;
        const typename K::Lhs L0 = K::load(A, i0, margin, S.lslot[warp][0]);
        const typename K::Lhs L1 = K::load(A, i1, margin, S.lslot[warp][1]);
        typename K::Part P0, P1;
        P0.zero();
        P1.zero();
        // warp-uniform: the cursors of ring Q (at most 31 + 64 entries) and the lengths of A and B (at most 31 + 32
        // each; their entries start at 0)
        int head = 0, tail = 0, na = 0, nbq = 0;
        const int self0 = nb.pref[13] + (i0 - nb.start[13]) - tb;  // tile position of i0 (i1 follows it)
        for (int jb = 0;; jb += 32) {
            const bool more = jb < tnp;  // warp-uniform
            if (more) {
                const int k = jb + lane;
                const bool p0 = K::filter(L0, T, k) && k != self0;
                const bool p1 = two && K::filter(L1, T, k) && k != self0 + 1;
                const unsigned b0 = __ballot_sync(kFull, p0);
                const unsigned b1 = __ballot_sync(kFull, p1);
                const int c0 = __popc(b0);
                if (p0) q[(tail + __popc(b0 & lt_mask)) & kQ] = (unsigned short)k;
                if (p1) q[(tail + c0 + __popc(b1 & lt_mask)) & kQ] = (unsigned short)(k | kTag);
                tail += c0 + __popc(b1);
            }
            // Rounds of 32 A or 32 B entries while there are, else 32 entries of Q (after the tile: the rest) sorted
            // into A and B, else (after the tile) the rest of A and B.  A and B thus hold fewer than 32 entries
            // before each sort and at most 31 + 32 after it.
            for (;;) {
                const int nq = tail - head;
                int n1, ca;  // entries of the round, of them from A (first)
                if (na >= 32) {
                    n1 = 32;
                    ca = 32;
                } else if (nbq >= 32) {
                    n1 = 32;
                    ca = 0;
                } else if (nq >= 32 || (!more && nq > 0)) {
                    __syncwarp();
                    const int n = min(32, nq);
                    const bool act = lane < n;
                    const int e = act ? q[(head + lane) & kQ] : 0;
                    const bool tag = (e & kTag) != 0;
                    const bool rec = act && K::receding(tag ? L1 : L0, T, e & (kTag - 1));
                    const unsigned ma = __ballot_sync(kFull, act && !rec), mb = __ballot_sync(kFull, rec);
                    if (act) {
                        if (rec) qb[nbq + __popc(mb & lt_mask)] = (unsigned short)e;
                        else qa[na + __popc(ma & lt_mask)] = (unsigned short)e;
                    }
                    head += n;
                    na += __popc(ma);
                    nbq += __popc(mb);
                    continue;
                } else if (!more && na + nbq > 0) {
                    n1 = min(32, na + nbq);
                    ca = na;
                } else {
                    break;
                }
                __syncwarp();
                const int e = lane < ca ? qa[lane] : (lane < n1 ? qb[lane - ca] : 0);
                bool in = false;
                if (lane < n1) {
                    const bool tag = (e & kTag) != 0;
                    typename K::Part Pt = tag ? P1 : P0;
                    in = K::eval(A, tag ? L1 : L0, T, nb, wrap, tag ? i1 : i0, e & (kTag - 1), Pt, ca > 0);
                    if (tag) P1 = Pt; else P0 = Pt;
                }
                const unsigned b = __ballot_sync(kFull, in);  // every lane votes (and the reads above are done)
                if (lane == 0) npair += __popc(b);
                // the list the round drew from keeps its rest (fewer than 32 entries) at the front
                unsigned short *r = ca == 32 ? qa : qb;
                const int used = ca == 32 ? 32 : n1 - ca, len = ca == 32 ? na : nbq;
                const int rem = len - used;
                const int ek = lane < rem ? r[used + lane] : 0;
                __syncwarp();
                if (lane < rem) r[lane] = (unsigned short)ek;
                if (ca == 32) {
                    na = rem;
                } else {
                    nbq = rem;
                    na -= ca;
                }
            }
            if (!more) break;
        }
        __syncwarp();  // the rings and the slots are reused by the next two particles
        typename K::Group G2;  // one reduction per pair of particles
        G2.put(0, P0, li0);
        G2.put(1, P1, li0 + 1);  // (all zero when the warp has a single particle)
        G2.accumulate(S.acc, two ? 2 : 1, lane);
    }
    my_pairs += npair;
}

// One cell: local set = the cell's particles, active set = its 3^3 neighbour cells, all of the CTA's threads.
template <class K, int NT>
__device__ __forceinline__ void process_cell(const typename K::Args &A, int c, const typename K::Tile &T,
                                             PairShared<K, NT> &S)
{
    if (A.cm.skip && *A.cm.skip) return;  // CTA-uniform
    const int ls = A.cm.cell_start[c], le = A.cm.cell_start[c + 1];
    if (ls >= le) return;  // CTA-uniform
    if (!SPH_CHECK(ls >= 0 && le <= A.cm.n, A.cm.status)) return;  // CTA-uniform
    const int tid = threadIdx.x, lane = tid & 31;
    const int tj = A.cm.tj;
    NbrTable &nb = S.nb;
    if (tid == 0) S.pairs = 0ull;
    build_nbr_table(nb, c, A.cm.cs, A.cm.cell_start, A.cm.n, A.cm.ncells, A.cm.status);
    const int NJ = nb.pref[27];
    const bool wrap = nb.wrap != 0;
    const float margin = nb.margin;
    unsigned long long my_pairs = 0;

    for (int ib = ls; ib < le; ib += kMaxLocal) {
        const int nloc = min(kMaxLocal, le - ib);
        for (int t = tid; t < nloc; t += NT) zero_acc<K>(S.acc[t]);
        for (int tb = 0; tb < NJ; tb += tj) {
            const int tn = min(tj, NJ - tb);
            const int tnp = (tn + kStep - 1) / kStep * kStep;  // padded to a multiple of kStep (<= tj)
            __syncthreads();  // accumulators zeroed, previous tile consumed
            for (int t = tid; t < tnp; t += NT) {
                if (t < tn) {
                    const int jj = tb + t;
                    const int nq = find_nbr(nb, jj);
                    K::stage(A, T, nb, t, nb.start[nq] + (jj - nb.pref[nq]), nq);
                } else {
                    K::sentinel(T, t);
                }
            }
            __syncthreads();
            if constexpr (K::kSplit) {
                tile_pairs_split<K, NT>(A, T, S, ib, nloc, tb, tnp, margin, wrap, my_pairs);
            } else {
                tile_pairs<K, NT>(A, T, S, ib, nloc, tb, tnp, margin, wrap, my_pairs);
            }
        }
        __syncthreads();
        for (int t = tid; t < nloc; t += NT) K::finish(A, ib + t, S.acc[t]);
    }
    if (lane == 0 && my_pairs) atomicAdd(&S.pairs, my_pairs);
    __syncthreads();
    if (tid == 0) {
        // a self term added in finish is still a pair of the sum
        const unsigned long long self = K::kSelfInFinish ? (unsigned long long)(le - ls) : 0ull;
        K::count(A, (unsigned long long)(le - ls) * (unsigned long long)NJ, S.pairs + self);
    }
}

// Lane driver of the FP32 loop bodies: each of the CTA's threads owns one (local particle, candidate stream)
// pair.  With nloc local particles, ns = min(32, 128 / nloc) threads share a particle; thread t takes particle
// t / ns and the candidates s, s + ns, s + 2 ns, ... of every tile (s = t mod ns).  The thread's partial sums
// live in registers across all tiles; at the end the ns partials of a particle are merged in stream order
// (deterministic) through shared memory and finalised.  Two sweeps:
//   K::kMasked:  every candidate is evaluated, the support acting only as a mask (Section 5.6) -- the density,
//                whose term is barely dearer than the distance test;
//   otherwise:   the lane tests 32 of its candidates into a bit mask, then evaluates its hits -- the force,
//                whose term costs several times the test and covers ~15 % of the candidates.
template <class K>
struct LaneShared {
    NbrTable nb;
    unsigned long long pairs;
};

template <class K>
__device__ __forceinline__ unsigned hit_sweep(const typename K::Args &A, const typename K::Lhs &L,
                                              const typename K::Tile &T, int s, int ns, int tn,
                                              typename K::Part &P)
{
    unsigned nhit = 0;
    int k0 = s;
    for (; k0 + 31 * ns < tn; k0 += 32 * ns) {  // whole windows: no bounds test per candidate
        unsigned hits = 0;
#pragma unroll
        for (int b = 0; b < 32; ++b)
            if (K::filter(L, T, k0 + b * ns)) hits |= 1u << b;
        nhit += __popc(hits);
        while (hits) {
            const int b = __ffs(hits) - 1;
            hits &= hits - 1u;
            K::eval(A, L, T, k0 + b * ns, P);
        }
    }
    if (k0 < tn) {  // the last, partial window
        unsigned hits = 0;
#pragma unroll
        for (int b = 0; b < 32; ++b) {
            const int k = k0 + b * ns;
            if (k < tn && K::filter(L, T, k)) hits |= 1u << b;
        }
        nhit += __popc(hits);
        while (hits) {
            const int b = __ffs(hits) - 1;
            hits &= hits - 1u;
            K::eval(A, L, T, k0 + b * ns, P);
        }
    }
    return nhit;
}

template <class K, int NT>
__device__ __forceinline__ void process_cell_lanes(const typename K::Args &A, int c, const typename K::Tile &T,
                                                   LaneShared<K> &S, unsigned char *smem)
{
    if (A.cm.skip && *A.cm.skip) return;  // CTA-uniform
    const int ls = A.cm.cell_start[c], le = A.cm.cell_start[c + 1];
    if (ls >= le) return;  // CTA-uniform
    if (!SPH_CHECK(ls >= 0 && le <= A.cm.n, A.cm.status)) return;  // CTA-uniform
    const int tid = threadIdx.x, lane = tid & 31;
    const int tj = A.cm.tj;
    NbrTable &nb = S.nb;
    if (tid == 0) S.pairs = 0ull;
    build_nbr_table(nb, c, A.cm.cs, A.cm.cell_start, A.cm.n, A.cm.ncells, A.cm.status);
    const int NJ = nb.pref[27];
    unsigned my_pairs = 0;
    typename K::Part *part = reinterpret_cast<typename K::Part *>(smem);  // reuses the tile after the last one

    for (int ib = ls; ib < le; ib += NT) {
        const int nloc = min(NT, le - ib);
        const int ns = min(32, NT / nloc);  // lanes per local particle
        const int li = tid / ns, s = tid - li * ns;
        const bool active = li < nloc;
        const int i = ib + (active ? li : 0);
        const typename K::Lhs L = K::load(A, i, 0.f, nullptr);
        typename K::Part P;
        P.zero();
        for (int tb = 0; tb < NJ; tb += tj) {
            const int tn = min(tj, NJ - tb);
            __syncthreads();  // previous tile consumed
            for (int t = tid; t < tn; t += NT) {
                const int jj = tb + t;
                const int nq = find_nbr(nb, jj);
                K::stage(A, T, nb, t, nb.start[nq] + (jj - nb.pref[nq]), nq);
            }
            if constexpr (K::kMasked) {
                if (tid == 0 && (tn & 1)) K::pad(T, tn);  // tn < tj here: tiles are multiples of 64
            }
            __syncthreads();
            if (active) {
                if constexpr (K::kMasked) {
                    K::sweep(L, T, s, ns, tn, P);
                } else {
                    my_pairs += hit_sweep<K>(A, L, T, s, ns, tn, P);
                }
            }
        }
        if constexpr (K::kMasked) {
            if (active) my_pairs += K::pairs_of(P);
        }
        __syncthreads();  // last tile consumed: its space holds the partials now
        part[tid] = P;
        __syncthreads();
        if (tid < nloc) {
            typename K::Acc acc;
            zero_acc<K>(acc);
            for (int q = 0; q < ns; ++q) K::merge_part(acc, part[tid * ns + q]);
            K::finish(A, ib + tid, acc);
        }
    }
    const unsigned long long wp = warp_sum((unsigned long long)my_pairs);
    if (lane == 0 && wp) atomicAdd(&S.pairs, wp);
    __syncthreads();
    if (tid == 0) {
        // the hit count of the filtered sweep includes every local particle's self pair
        const unsigned long long self = K::kMasked ? 0ull : (unsigned long long)(le - ls);
        K::count(A, (unsigned long long)(le - ls) * (unsigned long long)NJ, S.pairs - self);
    }
}

template <class K, int NT>
__global__ void __launch_bounds__(NT, K::min_ctas(NT)) k_cell_lanes(const typename K::Args A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LaneShared<K> S;
    const typename K::Tile T = K::carve(smem, A.cm.tj);
    process_cell_lanes<K, NT>(A, blockIdx.x, T, S, smem);
}

template <class K, int NT>
__global__ void __launch_bounds__(NT, K::min_ctas_persist(NT)) k_cell_lanes_persist(const typename K::Args A,
                                                                     const int *__restrict__ order,
                                                                     const int *__restrict__ count, int *next)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LaneShared<K> S;
    __shared__ int w;
    const typename K::Tile T = K::carve(smem, A.cm.tj);
    const int total = *count;
    for (;;) {
        if (threadIdx.x == 0) w = atomicAdd(next, 1);
        __syncthreads();
        const int wi = w;
        __syncthreads();
        if (wi >= total) break;
        const int c = order[wi];
        if (SPH_CHECK(c >= 0 && c < A.cm.ncells, A.cm.status)) process_cell_lanes<K, NT>(A, c, T, S, smem);
    }
}

// One CTA per cell (single-grid views).
template <class K, int NT>
__global__ void __launch_bounds__(NT, K::min_ctas(NT)) k_cell_pairs(const typename K::Args A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PairShared<K, NT> S;
    const typename K::Tile T = K::carve(smem, A.cm.tj);
    process_cell<K, NT>(A, blockIdx.x, T, S);
}

// Persistent CTAs pulling cells from a work list (patch views: cells in descending cost order, so the largest
// cells start first and the small ones fill the tail).
template <class K, int NT>
__global__ void __launch_bounds__(NT, K::min_ctas(NT)) k_cell_pairs_persist(const typename K::Args A,
                                                                     const int *__restrict__ order,
                                                                     const int *__restrict__ count, int *next)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PairShared<K, NT> S;
    __shared__ int w;
    const typename K::Tile T = K::carve(smem, A.cm.tj);
    const int total = *count;
    for (;;) {
        if (threadIdx.x == 0) w = atomicAdd(next, 1);
        __syncthreads();
        const int wi = w;
        __syncthreads();  // every thread has read w before thread 0 fetches the next item
        if (wi >= total) break;
        const int c = order[wi];
        if (SPH_CHECK(c >= 0 && c < A.cm.ncells, A.cm.status)) process_cell<K, NT>(A, c, T, S);
    }
}

// Cost of every non-empty cell (local particles x active particles), bucketed by floor(log2(cost)); one CTA per
// patch (patch views only), the bucket histogram gathered in shared memory first.
__global__ void __launch_bounds__(256) k_cell_cost(const CellSpace cs, const int *__restrict__ cell_start,
                                                   int *__restrict__ cell_bucket, int *__restrict__ bucket_count)
{
    __shared__ int hist[64];
    const int p = blockIdx.x;
    if (threadIdx.x < 64) hist[threadIdx.x] = 0;
    __syncthreads();
    const int base = cs.patch_cell_base[p], nc = cs.patch_cell_base[p + 1] - base;
    const int nx = cs.patch_n[3 * p], ny = cs.patch_n[3 * p + 1], nz = cs.patch_n[3 * p + 2];
    for (int l = threadIdx.x; l < nc; l += blockDim.x) {
        const int c = base + l;
        const int nloc = cell_start[c + 1] - cell_start[c];
        int b = -1;
        if (nloc > 0) {
            const int k0 = l % nx, k1 = (l / nx) % ny, k2 = l / (nx * ny);
            long long nj = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int kx = k0 + dx, ky = k1 + dy, kz = k2 + dz;
                        if (kx < 0 || ky < 0 || kz < 0 || kx >= nx || ky >= ny || kz >= nz) continue;
                        const int c2 = base + kx + nx * (ky + ny * kz);
                        nj += cell_start[c2 + 1] - cell_start[c2];
                    }
            const unsigned long long cost = (unsigned long long)nloc * (unsigned long long)nj;
            b = 63 - __clzll((long long)cost);
            atomicAdd(&hist[b], 1);
        }
        cell_bucket[c] = b;
    }
    __syncthreads();
    if (threadIdx.x < 64 && hist[threadIdx.x]) atomicAdd(&bucket_count[threadIdx.x], hist[threadIdx.x]);
}

// Offsets of the 64 cost buckets, largest first; the work count.
__global__ void k_work_offsets(int *__restrict__ bucket_count, int *__restrict__ work_count)
{
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 63; b >= 0; --b) {
            const int cnt = bucket_count[b];
            bucket_count[b] = run;  // becomes the bucket's cursor
            run += cnt;
        }
        *work_count = run;
    }
}

// Work list: every non-empty cell takes a place in its bucket's range (order inside a bucket is immaterial: every
// cell's result is independent of when it runs).  One CTA per patch: it counts its cells per bucket in shared
// memory, reserves one range per bucket with a single global atomic each, then places its cells through
// shared-memory cursors.
__global__ void __launch_bounds__(256) k_work_place(const CellSpace cs, const int *__restrict__ cell_bucket,
                                                    int *__restrict__ cursor, int *__restrict__ order)
{
    __shared__ int cnt[64], at[64];
    const int p = blockIdx.x;
    if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = cs.patch_cell_base[p], nc = cs.patch_cell_base[p + 1] - base;
    for (int l = threadIdx.x; l < nc; l += blockDim.x) {
        const int b = cell_bucket[base + l];
        if (b >= 0) atomicAdd(&cnt[b], 1);
    }
    __syncthreads();
    if (threadIdx.x < 64) at[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&cursor[threadIdx.x], cnt[threadIdx.x]) : 0;
    __syncthreads();
    for (int l = threadIdx.x; l < nc; l += blockDim.x) {
        const int b = cell_bucket[base + l];
        if (b >= 0) order[atomicAdd(&at[b], 1)] = base + l;
    }
}

// The magnitudes the FP64 pair loops need.  They refine FP32-seeded reciprocals and square roots of r^2 (r below
// kappa h in the support) and of (r^2 + eps hbar^2)(rho_i + rho_j), which must lie in the float normal range
// (2^-126 .. 2^128).  That holds, with room for kappa^2, the pair means and pairs down to h/100 apart (closer
// pairs give a tiny r^2, whose seeded forms stay finite and whose terms vanish), when 2^-50 <= h < 2^50 and
// 2^-105 <= h^2 rho < 2^105.  The set-up kernels flag a particle outside these bounds (SPH_DEV_MAGNITUDE: its
// results may be wrong; rescale the units).  rho alone is never seeded there.  Exponents are compared on the
// integer pipe.
__device__ __forceinline__ bool h_in_band(double h)
{
    const unsigned hi = (unsigned)__double2hiint(h);  // negative values and NaN fall outside
    return hi >= 0x3CD00000u && hi < 0x43100000u;     // 2^-50 <= h < 2^50
}
__device__ __forceinline__ void check_h_band(double h, unsigned *status)
{
    if (!h_in_band(h)) atomicOr(status, SPH_DEV_MAGNITUDE);
}
__device__ __forceinline__ void check_h_rho_band(double h, double rho, unsigned *status)
{
    const unsigned hr = (unsigned)__double2hiint(rho);
    const int eh = (int)((unsigned)__double2hiint(h) >> 20) - 1023, er = (int)(hr >> 20) - 1023;  // exponents
    const bool rho_ok = hr >= 0x00100000u && hr < 0x7FF00000u;  // positive, normal, finite
    const int e = 2 * eh + er;                                   // h^2 rho in [2^e, 2^(e+3))
    if (!h_in_band(h) || !rho_ok || e < -105 || e > 101) atomicOr(status, SPH_DEV_MAGNITUDE);
}

// FP32 cell-relative copies of FP64 positions, (float)(x - k edge) with the product and the difference each rounded
// once (as the FP32 view's positions and BlockCells form them): the filter inputs of the FP64 loops.
__device__ __forceinline__ void cell_relative_f32(const CellSpace &cs, int c, double x, double y, double z,
                                                  float &xf, float &yf, float &zf)
{
    CellLoc L;
    locate_cell(cs, c, L);
    xf = __double2float_rn(__dsub_rn(x, __dmul_rn((double)L.k[0], cell_edge(cs, L, 0))));
    yf = __double2float_rn(__dsub_rn(y, __dmul_rn((double)L.k[1], cell_edge(cs, L, 1))));
    zf = __double2float_rn(__dsub_rn(z, __dmul_rn((double)L.k[2], cell_edge(cs, L, 2))));
}

__global__ void k_pos32(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                        const double *__restrict__ h, const int *__restrict__ cell_of_slot, int n, CellSpace cs,
                        float *__restrict__ xf, float *__restrict__ yf, float *__restrict__ zf,
                        float *__restrict__ hf, unsigned *status)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    cell_relative_f32(cs, cell_of_slot[s], x[s], y[s], z[s], xf[s], yf[s], zf[s]);
    hf[s] = __double2float_ru(h[s]);
    check_h_band(h[s], status);
}

// ---- per-particle set-up of the FP64 loops ----
// These kernels are bound by the FP64 pipe (1/64 of the FP32 rate on this part), so they avoid its long
// sequences: 1/x and sqrt(x) come from the seeded forms above (an FP32 seed, one FP64 correction, within an ulp
// or two of the IEEE results) where x lies well inside the float range, and from the IEEE operations elsewhere (a
// branch that physical inputs never take); and each cell's origin is formed once per block (BlockCells).
__device__ __forceinline__ bool seedable(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
    return hi >= 0x38200000u && hi < 0x47C00000u;  // 2^-125 <= |x| < 2^125: seed and result are float normals
}
__device__ __forceinline__ double rcp_prep(double x) { return seedable(x) ? rcp_seeded(x) : 1.0 / x; }
__device__ __forceinline__ double sqrt_prep(double x) { return seedable(x) ? sqrt_seeded(x) : sqrt(x); }

// The cell origins of a block's slots.  Slots are in cell order, so the block's slots lie in the cells c0 .. c0 +
// ncl - 1; with at most kPrepThreads of them each origin k edge is formed once per cell in shared memory, and a
// slot outside that range (none, for slots in cell order) forms its own.  The FP32 copy of a position is then
// (float)(x - origin), as the FP32 view's positions are.  The range lives in each thread's registers (BlockCells),
// the origins in shared memory.
constexpr int kPrepThreads = 256;
struct BlockCells {
    int c0, ncl;
    // called by the whole block (one __syncthreads); o: the block's shared origins
    __device__ __forceinline__ void build(double (*o)[3], const CellSpace &cs, const int *cell_of_slot, int n)
    {
        const int base = blockIdx.x * kPrepThreads;
        const int cnt = min(kPrepThreads, n - base);
        c0 = cell_of_slot[base];
        ncl = cell_of_slot[base + cnt - 1] - c0 + 1;
        if (ncl >= 1 && ncl <= kPrepThreads) {
            for (int j = threadIdx.x; j < ncl; j += kPrepThreads) {
                CellLoc L;
                locate_cell(cs, c0 + j, L);
#pragma unroll
                for (int a = 0; a < 3; ++a) o[j][a] = __dmul_rn((double)L.k[a], cell_edge(cs, L, a));
            }
        }
        __syncthreads();
    }
    __device__ __forceinline__ void rel_f32(const double (*o)[3], const CellSpace &cs, int c, double x, double y,
                                            double z, float &xf, float &yf, float &zf) const
    {
        double ox, oy, oz;
        const int j = c - c0;
        if (ncl >= 1 && ncl <= kPrepThreads && (unsigned)j < (unsigned)ncl) {
            ox = o[j][0];
            oy = o[j][1];
            oz = o[j][2];
        } else {
            CellLoc L;
            locate_cell(cs, c, L);
            ox = __dmul_rn((double)L.k[0], cell_edge(cs, L, 0));
            oy = __dmul_rn((double)L.k[1], cell_edge(cs, L, 1));
            oz = __dmul_rn((double)L.k[2], cell_edge(cs, L, 2));
        }
        xf = __double2float_rn(__dsub_rn(x, ox));
        yf = __double2float_rn(__dsub_rn(y, oy));
        zf = __double2float_rn(__dsub_rn(z, oz));
    }
};

// Per-particle set-up of the FP64 density loop: cell-relative float positions (filter) and f(r/h) of the cubic
// spline as a cubic in r: inner piece 1 - 3/2 (r/h)^2 + 3/4 (r/h)^3, outer 2 - 3 (r/h) + 3/2 (r/h)^2 - 1/4 (r/h)^3.
// g1 = gamma (gamma - 1).
__global__ void __launch_bounds__(kPrepThreads) k_density_prep_f64(
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ h, const int *__restrict__ cell_of_slot, int n, CellSpace cs, float *__restrict__ xf,
    float *__restrict__ yf, float *__restrict__ zf, double *__restrict__ e2, double *__restrict__ e3,
    double *__restrict__ o1, double *__restrict__ o2, double *__restrict__ o3, const double *__restrict__ u,
    double g1, double *__restrict__ rk, double *__restrict__ cs0, unsigned *status)
{
    __shared__ double org[kPrepThreads][3];
    BlockCells B;
    B.build(org, cs, cell_of_slot, n);
    const int s = blockIdx.x * kPrepThreads + threadIdx.x;
    if (s >= n) return;
    B.rel_f32(org, cs, cell_of_slot[s], x[s], y[s], z[s], xf[s], yf[s], zf[s]);
    check_h_band(h[s], status);
    const double hi = rcp_prep(h[s]), h2 = hi * hi, h3 = h2 * hi;
    e2[s] = -1.5 * h2;
    e3[s] = 0.75 * h3;
    o1[s] = -3.0 * hi;
    o2[s] = 1.5 * h2;
    o3[s] = -0.25 * h3;
    // the density's normalisation 1/(pi h^3), and the sound speed of the ideal-gas EOS: with P = (gamma - 1) rho u,
    // c_s = sqrt(gamma P / rho) = sqrt(gamma (gamma - 1) u), which needs no density (so the pair kernel's per-particle
    // epilogue, run by few lanes of a warp, has no division or square root left)
    rk[s] = kInvPi * h3;
    cs0[s] = sqrt_prep(g1 * u[s]);
}

// Per-particle quantities of the FP32 force loop: 1/h, 3/(pi h^4), P/rho^2.
__global__ void k_force_prep_f32(const float *__restrict__ h, const float *__restrict__ P,
                                 const float *__restrict__ rho, int n, float *__restrict__ hinv,
                                 float *__restrict__ k4, float *__restrict__ A)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float hi = 1.0f / h[s];
    const float h2 = hi * hi;
    hinv[s] = hi;
    k4[s] = (float)(3.0 * kInvPi) * h2 * h2;
    const float r = rho[s];
    A[s] = P[s] / (r * r);
}

// Per-particle quantities of the FP64 force loop (see ForceF64); sc = sqrt(eps) with softening, else 1, and
// acs_k = alpha / (2 sc).  Also the filter's FP32 copies (k_pos32's work, in the same pass over the particles).
__global__ void __launch_bounds__(kPrepThreads) k_force_prep_f64(
    const double *__restrict__ h, const double *__restrict__ P, const double *__restrict__ rho,
    const double *__restrict__ cs, double acs_k, double sc, int n, double *__restrict__ hs, double *__restrict__ q2,
    double *__restrict__ S0, double *__restrict__ K1, double *__restrict__ K2i, double *__restrict__ K2o,
    double *__restrict__ A, double *__restrict__ acs, const double *__restrict__ x, const double *__restrict__ y,
    const double *__restrict__ z, const int *__restrict__ cell_of_slot, CellSpace g, float *__restrict__ xf,
    float *__restrict__ yf, float *__restrict__ zf, float *__restrict__ hf, unsigned *status)
{
    __shared__ double org[kPrepThreads][3];
    BlockCells B;
    B.build(org, g, cell_of_slot, n);
    const int s = blockIdx.x * kPrepThreads + threadIdx.x;
    if (s >= n) return;
    B.rel_f32(org, g, cell_of_slot[s], x[s], y[s], z[s], xf[s], yf[s], zf[s]);
    const double hv = h[s];
    hf[s] = __double2float_ru(hv);
    check_h_rho_band(hv, rho[s], status);
    const double hi = rcp_prep(hv), h2 = hi * hi;
    const double s4 = kInvPi * h2 * h2;  // 1/(pi h^4)
    const double hh = 0.5 * hv;
    hs[s] = sc * hh;
    q2[s] = hh * hh;
    S0[s] = -3.0 * s4;
    K1[s] = 3.0 * s4 * hi;
    K2i[s] = 2.25 * s4 * h2;
    K2o[s] = -0.75 * s4 * h2;
    const double ri = rcp_prep(rho[s]);  // P / rho^2 as P (1/rho)^2: 1/rho^2 may leave the float range, 1/rho not
    A[s] = P[s] * (ri * ri);
    acs[s] = acs_k * cs[s];
}

// Per-particle set-up of the kernel-family density (DensF64G): cell-relative float positions (filter), 1/h,
// sigma/h^3, sigma/h^4 and the sound speed sqrt(gamma (gamma - 1) u) of the ideal-gas EOS.
template <class Ker>
__global__ void k_density_prep_g(const double *__restrict__ x, const double *__restrict__ y,
                                 const double *__restrict__ z, const double *__restrict__ h,
                                 const double *__restrict__ u, const int *__restrict__ cell_of_slot, int n,
                                 CellSpace cs, double gamma, float *__restrict__ xf, float *__restrict__ yf,
                                 float *__restrict__ zf, double *__restrict__ hinv, double *__restrict__ s0,
                                 double *__restrict__ s1, double *__restrict__ cs0, unsigned *status)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    cell_relative_f32(cs, cell_of_slot[s], x[s], y[s], z[s], xf[s], yf[s], zf[s]);
    check_h_band(h[s], status);
    const double hi = 1.0 / h[s], h3 = hi * hi * hi;
    hinv[s] = hi;
    s0[s] = Ker::sigma * h3;
    s1[s] = Ker::sigma * (h3 * hi);
    cs0[s] = sqrt(gamma * (gamma - 1.0) * u[s]);
}

// Per-particle set-up of the kernel-family force (ForceF64G): h/2, 1/h, sigma/h^4, A = P / (Omega rho^2),
// alpha c / 2 and the Balsara switch B = |div v| / (|div v| + |curl v| + 1e-4 c / h); Omega = B = 1 without Ext.
template <class Ker, bool Ext>
__global__ void k_force_prep_g(const double *__restrict__ h, const double *__restrict__ P,
                               const double *__restrict__ rho, const double *__restrict__ cs,
                               const double *__restrict__ omega, const double *__restrict__ divv,
                               const double *__restrict__ cx, const double *__restrict__ cy,
                               const double *__restrict__ cz, double alpha, int n, double *__restrict__ hh,
                               double *__restrict__ hinv, double *__restrict__ s1, double *__restrict__ A,
                               double *__restrict__ ach, double *__restrict__ bal, unsigned *status)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    check_h_rho_band(h[s], rho[s], status);
    const double hv = h[s];
    const double hi = 1.0 / hv, h2 = hi * hi;
    hh[s] = 0.5 * hv;
    hinv[s] = hi;
    s1[s] = Ker::sigma * (h2 * h2);
    const double r = rho[s];
    if constexpr (Ext) {
        A[s] = P[s] / (omega[s] * r * r);
        const double d = fabs(divv[s]);
        const double c = sqrt(cx[s] * cx[s] + cy[s] * cy[s] + cz[s] * cz[s]);
        bal[s] = d / (d + c + 1e-4 * cs[s] * hi);
    } else {
        A[s] = P[s] / (r * r);
        bal[s] = 1.0;
    }
    ach[s] = 0.5 * alpha * cs[s];
}

template <class K>
struct UsesLanes {
    static constexpr bool value = false;
};
template <>
struct UsesLanes<DensF32> {
    static constexpr bool value = true;
};
template <>
struct UsesLanes<ForceF32> {
    static constexpr bool value = true;
};

template <class K, bool Lanes, int NT>
struct CellKernels {
    static auto grid() { return k_cell_pairs<K, NT>; }
    static auto persist() { return k_cell_pairs_persist<K, NT>; }
};
template <class K, int NT>
struct CellKernels<K, true, NT> {
    static auto grid() { return k_cell_lanes<K, NT>; }
    static auto persist() { return k_cell_lanes_persist<K, NT>; }
};

// Shared memory of a pair CTA: the tile, or (lane driver) the lane partials merged after the last tile if larger.
template <class K, int NT>
size_t pair_smem(int tj)
{
    size_t b = (size_t)tj * K::kStageBytes;
    if (UsesLanes<K>::value) b = std::max(b, (size_t)NT * sizeof(typename K::Part));
    return b + 16;
}

template <class K, int NT>
cudaError_t run_cells_nt(const typename K::Args &A, int ncells, const PairLaunch &pl, cudaStream_t st)
{
    void (*const kgrid)(const typename K::Args) = CellKernels<K, UsesLanes<K>::value, NT>::grid();
    void (*const kpers)(const typename K::Args, const int *, const int *, int *) =
        CellKernels<K, UsesLanes<K>::value, NT>::persist();
    const size_t smem = pair_smem<K, NT>(A.cm.tj);
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kgrid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kpers, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    if (pl.work_order) {
        // persistent CTAs: as many as fit on the device at once (occupancy of this kernel at this tile size)
        static size_t sized_for = 0;
        static int ctas = 0;
        if (sized_for != smem || ctas <= 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kpers, NT, smem);
            ctas = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
            sized_for = smem;
        }
        cudaError_t e = cudaMemsetAsync(pl.work_next, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        kpers<<<pl.persistent_ctas > 0 ? pl.persistent_ctas : ctas, NT, smem, st>>>(A, pl.work_order, pl.work_count,
                                                                                  pl.work_next);
    } else {
        kgrid<<<ncells, NT, smem, st>>>(A);
    }
    return cudaGetLastError();
}

template <class K>
cudaError_t run_cells(const typename K::Args &A, int ncells, const PairLaunch &pl, cudaStream_t st)
{
    return pl.threads == 256 ? run_cells_nt<K, 256>(A, ncells, pl, st) : run_cells_nt<K, 128>(A, ncells, pl, st);
}

int tile_or_default(int tj, int dflt)
{
    const int t = tj > 0 ? tj : dflt;
    return (t + kStep - 1) / kStep * kStep;
}

}  // namespace

cudaError_t launch_density_prep(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_of_slot, int n,
                                const CellSpace &g, const sph_params &prm, unsigned *status, cudaStream_t st,
                                int *nl)
{
    if (n <= 0 || f32) return cudaSuccess;  // FP32 views are already cell-relative floats
    const double gamma = prm.gamma;
    const int nb = (n + 255) / 256;
    const double *x = (const double *)soa.p[SPH_X][0], *y = (const double *)soa.p[SPH_X][1],
                 *z = (const double *)soa.p[SPH_X][2], *h = (const double *)soa.p[SPH_H][0],
                 *u = (const double *)soa.p[SPH_U][0];
    double *const *d = reinterpret_cast<double *const *>(scr.d);
    if (prm.kernel == SPH_KERNEL_M4 && prm.scheme == SPH_SCHEME_MINIMAL) {
        k_density_prep_f64<<<(n + kPrepThreads - 1) / kPrepThreads, kPrepThreads, 0, st>>>(
            x, y, z, h, cell_of_slot, n, g, scr.xf, scr.yf, scr.zf, d[0], d[1], d[2], d[3], d[4], u,
            gamma * (gamma - 1.0), d[5], d[6], status);
    } else if (prm.kernel == SPH_KERNEL_M5) {
        k_density_prep_g<KerM5><<<nb, 256, 0, st>>>(x, y, z, h, u, cell_of_slot, n, g, gamma, scr.xf, scr.yf,
                                                    scr.zf, d[0], d[1], d[2], d[6], status);
    } else {
        k_density_prep_g<KerM4><<<nb, 256, 0, st>>>(x, y, z, h, u, cell_of_slot, n, g, gamma, scr.xf, scr.yf,
                                                    scr.zf, d[0], d[1], d[2], d[6], status);
    }
    ++*nl;
    return cudaGetLastError();
}

namespace {

template <class Ker, bool Ext>
void force_prep_g(const SoaPtrs &soa, const Scratch &scr, int n, double alpha, unsigned *status, cudaStream_t st)
{
    double *const *d = reinterpret_cast<double *const *>(scr.d);
    const double *omega = Ext ? (const double *)soa.p[SPH_OMEGA][0] : nullptr;
    const double *divv = Ext ? (const double *)soa.p[SPH_DIVV][0] : nullptr;
    const double *cx = Ext ? (const double *)soa.p[SPH_CURLV][0] : nullptr;
    const double *cy = Ext ? (const double *)soa.p[SPH_CURLV][1] : nullptr;
    const double *cz = Ext ? (const double *)soa.p[SPH_CURLV][2] : nullptr;
    k_force_prep_g<Ker, Ext><<<(n + 255) / 256, 256, 0, st>>>(
        (const double *)soa.p[SPH_H][0], (const double *)soa.p[SPH_P][0], (const double *)soa.p[SPH_RHO][0],
        (const double *)soa.p[SPH_CS][0], omega, divv, cx, cy, cz, alpha, n, d[0], d[1], d[2], d[3], d[4], d[5],
        status);
}

}  // namespace

cudaError_t launch_force_prep(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_of_slot, int n,
                              const CellSpace &g, const sph_params &prm, unsigned *status, cudaStream_t st,
                              int *nl)
{
    if (n <= 0) return cudaSuccess;
    const int nb = (n + 255) / 256;
    const double alpha = prm.alpha;
    if (!f32) {
        const bool ext = prm.scheme == SPH_SCHEME_EXTENDED;
        if (prm.kernel == SPH_KERNEL_M4 && !ext) {
            const double sc = prm.eps > 0.0 ? sqrt(prm.eps) : 1.0;
            k_force_prep_f64<<<(n + kPrepThreads - 1) / kPrepThreads, kPrepThreads, 0, st>>>(
                                                 (const double *)soa.p[SPH_H][0], (const double *)soa.p[SPH_P][0],
                                                 (const double *)soa.p[SPH_RHO][0],
                                                 (const double *)soa.p[SPH_CS][0], 0.5 * alpha / sc, sc, n,
                                                 (double *)scr.d[0],
                                                 (double *)scr.d[7], (double *)scr.d[1], (double *)scr.d[2],
                                                 (double *)scr.d[3], (double *)scr.d[4], (double *)scr.d[5],
                                                 (double *)scr.d[6], (const double *)soa.p[SPH_X][0],
                                                 (const double *)soa.p[SPH_X][1], (const double *)soa.p[SPH_X][2],
                                                 cell_of_slot, g, scr.xf, scr.yf, scr.zf, scr.hf, status);
            *nl += 1;
        } else {
            k_pos32<<<nb, 256, 0, st>>>((const double *)soa.p[SPH_X][0], (const double *)soa.p[SPH_X][1],
                                        (const double *)soa.p[SPH_X][2], (const double *)soa.p[SPH_H][0],
                                        cell_of_slot, n, g, scr.xf, scr.yf, scr.zf, scr.hf, status);
            if (prm.kernel == SPH_KERNEL_M5) {
                if (ext) force_prep_g<KerM5, true>(soa, scr, n, alpha, status, st);
                else force_prep_g<KerM5, false>(soa, scr, n, alpha, status, st);
            } else {
                force_prep_g<KerM4, true>(soa, scr, n, alpha, status, st);
            }
            *nl += 2;
        }
    } else {
        k_force_prep_f32<<<nb, 256, 0, st>>>((const float *)soa.p[SPH_H][0], (const float *)soa.p[SPH_P][0],
                                             (const float *)soa.p[SPH_RHO][0], n, (float *)scr.d[0],
                                             (float *)scr.d[1], (float *)scr.d[2]);
        *nl += 1;
    }
    return cudaGetLastError();
}

namespace {

template <class Ker, bool Ext>
cudaError_t density_pairs_g(const SoaPtrs &soa, const Scratch &scr, PairCommon cm, int tj, double gamma,
                            int ncells, const PairLaunch &pl, cudaStream_t st)
{
    using D = DensF64G<Ker, Ext>;
    typename D::Args A;
    cm.tj = tile_or_default(tj, 448);
    A.cm = cm;
    A.f[D::X] = (const double *)soa.p[SPH_X][0];
    A.f[D::Y] = (const double *)soa.p[SPH_X][1];
    A.f[D::Z] = (const double *)soa.p[SPH_X][2];
    A.f[D::VX] = Ext ? (const double *)soa.p[SPH_V][0] : nullptr;
    A.f[D::VY] = Ext ? (const double *)soa.p[SPH_V][1] : nullptr;
    A.f[D::VZ] = Ext ? (const double *)soa.p[SPH_V][2] : nullptr;
    A.f[D::HINV] = (const double *)scr.d[0];
    A.f[D::S0] = (const double *)scr.d[1];
    A.f[D::S1] = (const double *)scr.d[2];
    A.m = (const double *)soa.p[SPH_MASS][0];
    A.h = (const double *)soa.p[SPH_H][0];
    A.u = (const double *)soa.p[SPH_U][0];
    A.cs0 = (const double *)scr.d[6];
    A.xf = scr.xf;
    A.yf = scr.yf;
    A.zf = scr.zf;
    A.rho = (double *)soa.p[SPH_RHO][0];
    A.P = (double *)soa.p[SPH_P][0];
    A.cs = (double *)soa.p[SPH_CS][0];
    A.nnb = Ext ? (double *)soa.p[SPH_NNB][0] : nullptr;
    A.divv = Ext ? (double *)soa.p[SPH_DIVV][0] : nullptr;
    A.cx = Ext ? (double *)soa.p[SPH_CURLV][0] : nullptr;
    A.cy = Ext ? (double *)soa.p[SPH_CURLV][1] : nullptr;
    A.cz = Ext ? (double *)soa.p[SPH_CURLV][2] : nullptr;
    A.omega = Ext ? (double *)soa.p[SPH_OMEGA][0] : nullptr;
    A.gamma = gamma;
    return run_cells<D>(A, ncells, pl, st);
}

template <class Ker, bool Ext>
cudaError_t force_pairs_g(const SoaPtrs &soa, const Scratch &scr, PairCommon cm, int tj, const sph_params &prm,
                          int ncells, const PairLaunch &pl, cudaStream_t st)
{
    using F = ForceF64G<Ker, Ext>;
    typename F::Args A;
    cm.tj = tile_or_default(tj, 448);
    A.cm = cm;
    A.f[F::X] = (const double *)soa.p[SPH_X][0];
    A.f[F::Y] = (const double *)soa.p[SPH_X][1];
    A.f[F::Z] = (const double *)soa.p[SPH_X][2];
    A.f[F::VX] = (const double *)soa.p[SPH_V][0];
    A.f[F::VY] = (const double *)soa.p[SPH_V][1];
    A.f[F::VZ] = (const double *)soa.p[SPH_V][2];
    A.f[F::M] = (const double *)soa.p[SPH_MASS][0];
    A.f[F::HH] = (const double *)scr.d[0];
    A.f[F::HINV] = (const double *)scr.d[1];
    A.f[F::S1] = (const double *)scr.d[2];
    A.f[F::AP] = (const double *)scr.d[3];
    A.f[F::ACH] = (const double *)scr.d[4];
    A.f[F::BAL] = (const double *)scr.d[5];
    A.f[F::RHO] = (const double *)soa.p[SPH_RHO][0];
    A.f[F::CS] = (const double *)soa.p[SPH_CS][0];
    A.xf = scr.xf;
    A.yf = scr.yf;
    A.zf = scr.zf;
    A.hf = scr.hf;
    A.ax = (double *)soa.p[SPH_A][0];
    A.ay = (double *)soa.p[SPH_A][1];
    A.az = (double *)soa.p[SPH_A][2];
    A.dudt = (double *)soa.p[SPH_DUDT][0];
    A.vsig = Ext ? (double *)soa.p[SPH_VSIG][0] : nullptr;
    A.beta = prm.beta;
    A.eps = prm.eps;
    return run_cells<F>(A, ncells, pl, st);
}

}  // namespace

cudaError_t launch_density_pairs(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_start,
                                 int ncells, int n, const CellSpace &g, const sph_params &prm, const PairLaunch &pl,
                                 unsigned *status, Counters *counters, cudaStream_t st, int *nl)
{
    if (n <= 0) return cudaSuccess;
    ++*nl;
    PairCommon cm{cell_start, g, status, counters, 0, pl.skip, n, ncells};
    const int tj = pl.tj;
    const double gamma = prm.gamma;
    if (!f32 && prm.kernel == SPH_KERNEL_M5) {
        return prm.scheme == SPH_SCHEME_EXTENDED ? density_pairs_g<KerM5, true>(soa, scr, cm, tj, gamma, ncells, pl, st)
                                                 : density_pairs_g<KerM5, false>(soa, scr, cm, tj, gamma, ncells, pl, st);
    }
    if (!f32 && prm.scheme == SPH_SCHEME_EXTENDED) return density_pairs_g<KerM4, true>(soa, scr, cm, tj, gamma, ncells, pl, st);
    if (!f32) {
        DensF64::Args A;
        cm.tj = tile_or_default(tj, 512);
        A.cm = cm;
        using D = DensF64;
        A.f[D::X] = (const double *)soa.p[SPH_X][0];
        A.f[D::Y] = (const double *)soa.p[SPH_X][1];
        A.f[D::Z] = (const double *)soa.p[SPH_X][2];
        A.f[D::H] = (const double *)soa.p[SPH_H][0];
        A.f[D::E2] = (const double *)scr.d[0];
        A.f[D::E3] = (const double *)scr.d[1];
        A.f[D::O1] = (const double *)scr.d[2];
        A.f[D::O2] = (const double *)scr.d[3];
        A.f[D::O3] = (const double *)scr.d[4];
        A.m = (const double *)soa.p[SPH_MASS][0];
        A.u = (const double *)soa.p[SPH_U][0];
        A.rk = (const double *)scr.d[5];
        A.cs0 = (const double *)scr.d[6];
        A.xf = scr.xf;
        A.yf = scr.yf;
        A.zf = scr.zf;
        A.rho = (double *)soa.p[SPH_RHO][0];
        A.P = (double *)soa.p[SPH_P][0];
        A.cs = (double *)soa.p[SPH_CS][0];
        A.gamma = gamma;
        return run_cells<DensF64>(A, ncells, pl, st);
    }
    DensF32::Args A;
    cm.tj = tile_or_default(tj, 1024);
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
    return run_cells<DensF32>(A, ncells, pl, st);
}

namespace {

template <bool kSoft>
cudaError_t force_pairs_f64(const SoaPtrs &soa, const Scratch &scr, PairCommon cm, int tj, const sph_params &prm,
                            int ncells, const PairLaunch &pl, cudaStream_t st)
{
    using F = ForceF64<kSoft>;
    typename F::Args A;
    cm.tj = tile_or_default(tj, 448);  // 144 B per staged particle: three 256-thread CTAs per SM
    A.cm = cm;
    A.f[F::X] = (const double *)soa.p[SPH_X][0];
    A.f[F::Y] = (const double *)soa.p[SPH_X][1];
    A.f[F::Z] = (const double *)soa.p[SPH_X][2];
    A.f[F::VX] = (const double *)soa.p[SPH_V][0];
    A.f[F::VY] = (const double *)soa.p[SPH_V][1];
    A.f[F::VZ] = (const double *)soa.p[SPH_V][2];
    A.f[F::M] = (const double *)soa.p[SPH_MASS][0];
    A.f[F::RHO] = (const double *)soa.p[SPH_RHO][0];
    A.f[F::HS] = (const double *)scr.d[0];
    A.f[F::S0] = (const double *)scr.d[1];
    A.f[F::K1] = (const double *)scr.d[2];
    A.f[F::K2I] = (const double *)scr.d[3];
    A.f[F::K2O] = (const double *)scr.d[4];
    A.f[F::AP] = (const double *)scr.d[5];
    A.f[F::ACS] = (const double *)scr.d[6];
    A.q2 = (const double *)scr.d[7];
    A.xf = scr.xf;
    A.yf = scr.yf;
    A.zf = scr.zf;
    A.hf = scr.hf;
    A.ax = (double *)soa.p[SPH_A][0];
    A.ay = (double *)soa.p[SPH_A][1];
    A.az = (double *)soa.p[SPH_A][2];
    A.dudt = (double *)soa.p[SPH_DUDT][0];
    A.beta_s = kSoft ? prm.beta / prm.eps : prm.beta;
    return run_cells<F>(A, ncells, pl, st);
}

}  // namespace

cudaError_t launch_force_pairs(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_start,
                               int ncells, int n, const CellSpace &g, const sph_params &prm, const PairLaunch &pl,
                               unsigned *status, Counters *counters, cudaStream_t st, int *nl)
{
    if (n <= 0) return cudaSuccess;
    ++*nl;
    PairCommon cm{cell_start, g, status, counters, 0, pl.skip, n, ncells};
    const int tj = pl.tj;
    if (!f32 && prm.kernel == SPH_KERNEL_M5) {
        return prm.scheme == SPH_SCHEME_EXTENDED ? force_pairs_g<KerM5, true>(soa, scr, cm, tj, prm, ncells, pl, st)
                                                 : force_pairs_g<KerM5, false>(soa, scr, cm, tj, prm, ncells, pl, st);
    }
    if (!f32 && prm.scheme == SPH_SCHEME_EXTENDED) return force_pairs_g<KerM4, true>(soa, scr, cm, tj, prm, ncells, pl, st);
    if (!f32) return prm.eps > 0.0 ? force_pairs_f64<true>(soa, scr, cm, tj, prm, ncells, pl, st)
                                   : force_pairs_f64<false>(soa, scr, cm, tj, prm, ncells, pl, st);
    ForceF32::Args A;
    cm.tj = tile_or_default(tj, 512);
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
    A.hinv = (const float *)scr.d[0];
    A.k4 = (const float *)scr.d[1];
    A.A = (const float *)scr.d[2];
    A.ax = (float *)soa.p[SPH_A][0];
    A.ay = (float *)soa.p[SPH_A][1];
    A.az = (float *)soa.p[SPH_A][2];
    A.dudt = (float *)soa.p[SPH_DUDT][0];
    A.alpha = (float)prm.alpha;
    A.beta = (float)prm.beta;
    A.eps = (float)prm.eps;
    return run_cells<ForceF32>(A, ncells, pl, st);
}

cudaError_t launch_work_list(const CellSpace &cs, const int *cell_start, int ncells_cap, int *cell_bucket,
                             int *bucket_count, int *work_order, int *work_count, cudaStream_t st, int *nl)
{
    (void)ncells_cap;
    if (cs.npatch <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(bucket_count, 0, 64 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_cell_cost<<<cs.npatch, 256, 0, st>>>(cs, cell_start, cell_bucket, bucket_count);
    k_work_offsets<<<1, 32, 0, st>>>(bucket_count, work_count);
    k_work_place<<<cs.npatch, 256, 0, st>>>(cs, cell_bucket, bucket_count, work_order);
    *nl += 3;
    return cudaGetLastError();
}

}  // namespace sphk
