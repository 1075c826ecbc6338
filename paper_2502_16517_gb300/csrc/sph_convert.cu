// sph_convert.cu -- cell bucketing and the field-selective AoS<->SoA view conversions.
//
// Bucketing (paper Section 2.1: particles sorted into cells at least as wide as the interaction radius; Section
// 2.2 / 5.2: the particles of a cell form one contiguous chunk indexed by a CSR-like list):
//   k_bin_count   one thread per record: cell coordinate floor(x * n/box) per axis, clamped, linear cell id,
//                 histogram by atomicAdd;
//   k_scan_cells  one CTA: exclusive scan of the histogram into cell_start (CSR) and the fill cursors (small
//                 grids); large grids use k_scan_block_sums + k_scan_cells over the block sums + k_scan_apply;
//   k_bin_place   one thread per record: claims a slot of its cell (atomic cursor);
//   k_cell_sort   one warp per cell: ranks the claimed record indices so that each cell holds ascending record
//                 indices (the slot order is then independent of atomic timing, i.e. deterministic).
//
// Patch views (independent open boxes): k_patch_grid gives every patch its own grid with cell edge >= 2 h_max of
// the patch (capped), k_bin_count_patches (one CTA per patch) maps records to global cell ids, and the same scan
// / place / sort follow, with the cell count read on the device.
//
// Views (Section 4, Eq. 3-5; prologue/epilogue of Section 3.1):
//   k_gather      CTA per tile of 256 slots.  Phase 1 reads, per record, only the 16-byte chunks that hold a
//                 member of the mask (128-bit loads; consecutive threads take consecutive chunks of one record)
//                 into shared memory; phase 2 transposes them out of shared memory into one SoA array per
//                 member component, consecutive threads writing consecutive slots (coalesced).  After a drift,
//                 v and u can arrive predicted (v + a dt/2, u + du/dt dt/2 from the same record, in FP64): the
//                 view then carries the values the leapfrog's force needs, and the records keep theirs.
//   k_scatter     the reverse: phase 1 reads the SoA arrays coalesced into shared memory, phase 2 writes each
//                 member's 8 bytes back into its record; no other byte of a record is written (the leapfrog's
//                 second kick, when fused in, also rewrites v and u of the record).
// The leapfrog's first kick and drift run inside k_bin_count / k_bin_count_patches of the pass that follows them,
// which read the records anyway.
#include "sph_internal.cuh"

namespace sphk {

namespace {

constexpr int kTile = 256;
constexpr int kUnroll = 8;  // independent global loads a conversion thread issues before it stores any of them
constexpr int kHmaxSlots = 8;  // patches of a record-pass tile whose h maximum is gathered in shared memory
constexpr unsigned kFull = 0xffffffffu;

// q / d for 0 <= q < 256 d and 1 <= d <= 40 by multiplication with inv = ceil(2^20 / d) and a shift (exact in that
// range, checked exhaustively; the product stays below 2^29): the conversion kernels' index arithmetic without
// integer division.
__host__ __device__ __forceinline__ unsigned div_inv(unsigned d) { return ((1u << 20) + d - 1) / d; }
__device__ __forceinline__ int div_small(int q, unsigned inv) { return (int)(((unsigned)q * inv) >> 20); }

// cell_coord on the integer pipe: the same value and the same range flag as cell_coord below, with one FP64
// multiply; the compares and the floor work on the bit patterns (for doubles >= 0 they order like the values; a
// set sign bit is a negative value, -0.0 or a negative NaN; an all-ones exponent is an infinity or a NaN).
__device__ __forceinline__ int cell_coord_bits(double x, double inv, int n, double box, bool &bad)
{
    const long long kNeg0 = (long long)0x8000000000000000ULL;
    const long long xb = __double_as_longlong(x);
    const long long bb = __double_as_longlong(box);  // box > 0, finite
    // x >= 0 && x <= box, false for NaN: -0.0 counts as 0; a positive NaN or +inf has bits above any finite box
    if (!((xb >= 0 && xb <= bb) || xb == kNeg0)) bad = true;
    const long long yb = __double_as_longlong(__dmul_rn(x, inv));
    if (yb < 0) return 0;                                   // negative, -0.0 or negative NaN: floor < 0 or NaN
    const int ex = (int)(yb >> 52);                          // biased exponent (sign clear)
    if (ex == 2047) return (yb & 0xFFFFFFFFFFFFFLL) ? 0 : n - 1;  // NaN: 0; +inf: clamped
    const int e = ex - 1023;
    if (e < 0) return 0;                                     // 0 <= y < 1
    if (e >= 31) return n - 1;                               // y >= 2^31 > n - 1
    const long long m = (yb & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int f = (int)(m >> (52 - e));                      // floor(y)
    return f > n - 1 ? n - 1 : f;
}

__device__ __forceinline__ int cell_coord(double x, double inv, int n, double box, bool &bad)
{
    if (!(x >= 0.0 && x <= box)) bad = true;
    const double f = floor(__dmul_rn(x, inv));
    int k;
    if (!(f >= 0.0)) {
        k = 0;  // also NaN
    } else if (f > (double)(n - 1)) {
        k = n - 1;
    } else {
        k = (int)f;
    }
    return k;
}

// v + a d, each operation rounded on its own (no contraction), as the leapfrog is written.
__device__ __forceinline__ double kick1(double v, double a, double d) { return __dadd_rn(v, __dmul_rn(a, d)); }

// The leapfrog's first kick and its drift on one record (in place): v += a dtk, u += du/dt dtk, then x += v dt,
// wrapped into [0, box) on a periodic grid, or mirrored at the walls of an open box (that velocity component turns;
// a position still outside after one mirror, |v dt| > box, is put on the wall).  Returns the new position in x.
__device__ __forceinline__ void kick_drift(double x[3], double v[3], double &u, const double a[3], double du,
                                           double dtk, double dt, const Grid &g)
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        v[d] = kick1(v[d], a[d], dtk);
        double xn = __dadd_rn(x[d], __dmul_rn(v[d], dt));
        if (g.periodic) {
            if (xn >= g.box[d]) xn = __dsub_rn(xn, g.box[d]);
            else if (xn < 0.0) xn = __dadd_rn(xn, g.box[d]);
        } else {
            if (xn < 0.0) {
                xn = -xn;
                v[d] = -v[d];
            } else if (xn > g.box[d]) {
                xn = __dsub_rn(__dadd_rn(g.box[d], g.box[d]), xn);
                v[d] = -v[d];
            }
            if (xn < 0.0) xn = 0.0;
            else if (xn > g.box[d]) xn = g.box[d];
        }
        x[d] = xn;
    }
    u = kick1(u, du, dtk);
}

// kick_drift with the reuse of the product a dtk for the predicted velocity (v_pred = v_half + a dtk, the oracle's
// second application of the same kick: the same product, so the same bits), and the position compares on the
// integer pipe (bit patterns as in cell_coord_bits).  vp, up receive the predicted v, u.
__device__ __forceinline__ void kick_drift_predict(double x[3], double v[3], double &u, const double a[3], double du,
                                                   double dtk, double dt, const Grid &g, double vp[3], double &up)
{
    const long long kNeg0 = (long long)0x8000000000000000ULL;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double ad = __dmul_rn(a[d], dtk);
        v[d] = __dadd_rn(v[d], ad);
        double xn = __dadd_rn(x[d], __dmul_rn(v[d], dt));
        const long long xb = __double_as_longlong(xn), bb = __double_as_longlong(g.box[d]);
        const bool nan = ((xb >> 52) & 0x7FF) == 0x7FF && (xb & 0xFFFFFFFFFFFFFLL) != 0;
        const bool neg = xb < 0 && xb != kNeg0 && !nan;      // xn < 0
        const bool ge = xb >= 0 && xb >= bb && !nan;         // xn >= box (positive, not NaN)
        const bool gt = ge && xb != bb;                      // xn > box
        if (g.periodic) {
            if (ge) xn = __dsub_rn(xn, g.box[d]);
            else if (neg) xn = __dadd_rn(xn, g.box[d]);
        } else {
            if (neg) {
                xn = -xn;
                v[d] = -v[d];
            } else if (gt) {
                xn = __dsub_rn(__dadd_rn(g.box[d], g.box[d]), xn);
                v[d] = -v[d];
            }
            // still outside after one mirror: onto the wall
            const long long yb = __double_as_longlong(xn);
            const bool ynan = ((yb >> 52) & 0x7FF) == 0x7FF && (yb & 0xFFFFFFFFFFFFFLL) != 0;
            if (yb < 0 && yb != kNeg0 && !ynan) xn = 0.0;
            else if (yb >= 0 && yb > bb && !ynan) xn = g.box[d];
        }
        x[d] = xn;
        vp[d] = __dadd_rn(v[d], ad);
    }
    const double ud = __dmul_rn(du, dtk);
    u = __dadd_rn(u, ud);
    up = __dadd_rn(u, ud);
}

__device__ __forceinline__ void kick_drift_record(uint8_t *rec, int off_x, const KickDrift &kd, const Grid &g,
                                                  double x[3])
{
    double *xp = reinterpret_cast<double *>(rec + off_x);
    double *vp = reinterpret_cast<double *>(rec + kd.off_v);
    double *up = reinterpret_cast<double *>(rec + kd.off_u);
    const double *ap = reinterpret_cast<const double *>(rec + kd.off_a);
    const double a[3] = {ap[0], ap[1], ap[2]};
    double v[3] = {vp[0], vp[1], vp[2]};
    double u = *up;
    x[0] = xp[0];
    x[1] = xp[1];
    x[2] = xp[2];
    kick_drift(x, v, u, a, *reinterpret_cast<const double *>(rec + kd.off_du), kd.dtk, kd.dt, g);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xp[d] = x[d];
        vp[d] = v[d];
    }
    *up = u;
}

// KD: the records are kicked and drifted first (the leapfrog fused into the bin); their new positions are binned.
template <bool KD>
__global__ void k_bin_count(const uint8_t *__restrict__ aos, int64_t stride, int off_x, int n, Grid g,
                            int *__restrict__ cell_of, int *__restrict__ count, unsigned *status, KickDrift kd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3];
    if (KD) {
        kick_drift_record(kd.aos + (int64_t)i * stride, off_x, kd, g, x);
    } else {
        const double *xp = reinterpret_cast<const double *>(aos + (int64_t)i * stride + off_x);
        x[0] = __ldg(xp + 0);
        x[1] = __ldg(xp + 1);
        x[2] = __ldg(xp + 2);
    }
    bool bad = false;
    const int kx = cell_coord(x[0], g.inv[0], g.n[0], g.box[0], bad);
    const int ky = cell_coord(x[1], g.inv[1], g.n[1], g.box[1], bad);
    const int kz = cell_coord(x[2], g.inv[2], g.n[2], g.box[2], bad);
    const int c = kx + g.n[0] * (ky + g.n[1] * kz);
    cell_of[i] = c;
    atomicAdd(&count[c], 1);
    if (bad) atomicOr(status, SPH_DEV_POS_RANGE);
}

// Single-CTA exclusive scan over the cell histogram, 4 cells per thread per round.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_scan_cells(const int *__restrict__ count, int ncells_host,
                                                             const int *__restrict__ ncells_dev,
                                                             int *__restrict__ cell_start, int *__restrict__ fill)
{
    __shared__ int warp_tot[32];
    __shared__ int carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncells = ncells_dev ? *ncells_dev : ncells_host;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < ncells; base += kScanThreads * 4) {
        const int idx = base + tid * 4;
        int v[4];
        int t = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (idx + k < ncells) ? count[idx + k] : 0;
            t += v[k];
        }
        // inclusive warp scan of t
        int incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = warp_tot[lane];
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += y;
            }
            warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
        }
        __syncthreads();
        const int carry = carry_s;
        int run = carry + warp_tot[warp] + incl - t;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (idx + k < ncells) {
                cell_start[idx + k] = run;
                fill[idx + k] = run;
            }
            run += v[k];
        }
        __syncthreads();
        if (tid == kScanThreads - 1) carry_s = run;  // last thread's running total = carry + round total
        __syncthreads();
    }
    if (tid == 0) cell_start[ncells] = carry_s;
}

// Multi-CTA exclusive scan for large grids, in three deterministic launches: every CTA sums its kScanChunk cells
// (k_scan_block_sums), one CTA scans those sums (k_scan_cells on the block sums), every CTA rescans its chunk from
// its block offset (k_scan_apply).  The cell count may live on the device (patch views); CTAs past it idle.
constexpr int kScanChunk = kScanThreads * 4;

__global__ void __launch_bounds__(kScanThreads) k_scan_block_sums(const int *__restrict__ count, int ncells_host,
                                                                  const int *__restrict__ ncells_dev,
                                                                  int *__restrict__ block_sum)
{
    __shared__ int warp_tot[32];
    const int ncells = ncells_dev ? *ncells_dev : ncells_host;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int idx = blockIdx.x * kScanChunk + tid * 4;
    int t = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) t += (idx + k < ncells) ? count[idx + k] : 0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    if (lane == 0) warp_tot[warp] = t;
    __syncthreads();
    if (warp == 0) {
        int w = warp_tot[lane];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
        if (lane == 0) block_sum[blockIdx.x] = w;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int *__restrict__ count, int ncells_host,
                                                             const int *__restrict__ ncells_dev,
                                                             const int *__restrict__ block_off,
                                                             int *__restrict__ cell_start, int *__restrict__ fill)
{
    __shared__ int warp_tot[32];
    const int ncells = ncells_dev ? *ncells_dev : ncells_host;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.x == 0 && tid == 0) cell_start[ncells] = block_off[gridDim.x];  // the total
    const int base = blockIdx.x * kScanChunk;
    if (base >= ncells) return;  // CTA-uniform
    const int idx = base + tid * 4;
    int v[4];
    int t = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (idx + k < ncells) ? count[idx + k] : 0;
        t += v[k];
    }
    int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = warp_tot[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;
    }
    __syncthreads();
    int run = block_off[blockIdx.x] + warp_tot[warp] + incl - t;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (idx + k < ncells) {
            cell_start[idx + k] = run;
            fill[idx + k] = run;
        }
        run += v[k];
    }
}

__global__ void k_bin_place(const int *__restrict__ cell_of, int n, int *__restrict__ fill,
                            int *__restrict__ perm_tmp, unsigned *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = atomicAdd(&fill[cell_of[i]], 1);
    if (SPH_CHECK(s >= 0 && s < n, status)) perm_tmp[s] = i;
}

// One warp per cell: rank every record index of the cell among the cell's indices (all distinct), write it to
// its sorted slot.  O(L^2 / 32) per cell of L particles, with the compared values broadcast by shuffles.
__global__ void k_cell_sort(const int *__restrict__ cell_start, int ncells_host, const int *__restrict__ ncells_dev,
                            const int *__restrict__ perm_tmp, int *__restrict__ perm, int *__restrict__ cell_of_slot)
{
    const int ncells = ncells_dev ? *ncells_dev : ncells_host;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncells; c += nwarps) {
    const int b = cell_start[c], L = cell_start[c + 1] - b;
    for (int k0 = 0; k0 < L; k0 += 32) {
        const int k = k0 + lane;
        const int v = (k < L) ? perm_tmp[b + k] : 0x7fffffff;
        int rank = 0;
        for (int t0 = 0; t0 < L; t0 += 32) {
            const int w = (t0 + lane < L) ? perm_tmp[b + t0 + lane] : 0x7fffffff;
#pragma unroll 8
            for (int t = 0; t < 32; ++t) rank += (__shfl_sync(kFull, w, t) < v) ? 1 : 0;
        }
        if (k < L) {
            perm[b + rank] = v;
            cell_of_slot[b + rank] = c;
        }
    }
    }
}

// Grid of patch p from its largest h: per axis n = floor(box / (2 h_max)) cells (at least 1, at most ncap,
// lowered while box / n < 2 h_max after rounding), the cell edge box / n and the inverse n / box, each rounded once
// in FP64, and the patch's cell count.
__device__ __forceinline__ void patch_grid_one(int p, double hm, const Grid &g, int ncap, int *patch_n,
                                               double *patch_edge, double *patch_inv, int *patch_cells)
{
    int cells = 1;
    for (int a = 0; a < 3; ++a) {
        int nn = ncap;
        if (hm > 0.0) {
            const double f = floor(g.box[a] / (2.0 * hm));
            nn = f >= (double)ncap ? ncap : (f >= 1.0 ? (int)f : 1);
            while (nn > 1 && __ddiv_rn(g.box[a], (double)nn) < 2.0 * hm) --nn;
        }
        patch_n[3 * p + a] = nn;
        patch_edge[3 * p + a] = __ddiv_rn(g.box[a], (double)nn);
        patch_inv[3 * p + a] = __ddiv_rn((double)nn, g.box[a]);
        cells *= nn;
    }
    patch_cells[p] = cells;
}

// Patch grids: per patch (one CTA) the largest h of its records, then per axis n = floor(box / (2 h_max)) cells
// (at least 1, at most ncap, lowered while box / n < 2 h_max after rounding), the cell edge box / n and the inverse
// n / box, each rounded once in FP64, and the patch's cell count.
__global__ void __launch_bounds__(256) k_patch_grid(const uint8_t *__restrict__ aos, int64_t stride, int off_h,
                                                    const int64_t *__restrict__ patch_start, Grid g, int ncap,
                                                    int *__restrict__ patch_n, double *__restrict__ patch_edge,
                                                    double *__restrict__ patch_inv, int *__restrict__ patch_cells)
{
    __shared__ double red[8];
    const int p = blockIdx.x;
    const int64_t s = patch_start[p], e = patch_start[p + 1];
    double hm = 0.0;
    for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x)
        hm = fmax(hm, *reinterpret_cast<const double *>(aos + i * stride + off_h));
    for (int o = 16; o > 0; o >>= 1) hm = fmax(hm, __shfl_xor_sync(kFull, hm, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = hm;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) hm = fmax(hm, red[w]);
        patch_grid_one(p, hm, g, ncap, patch_n, patch_edge, patch_inv, patch_cells);
    }
}

// The same grids from the per-patch h_max the record pass gathered (bit patterns of positive doubles, which
// order like the values), one thread per patch.
__global__ void k_patch_grid_hmax(const unsigned long long *__restrict__ hmax_bits, int npatch, Grid g, int ncap,
                                  int *__restrict__ patch_n, double *__restrict__ patch_edge,
                                  double *__restrict__ patch_inv, int *__restrict__ patch_cells)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npatch) return;
    patch_grid_one(p, __longlong_as_double((long long)hmax_bits[p]), g, ncap, patch_n, patch_edge, patch_inv,
                   patch_cells);
}

// Global cell of every record of a patch view, one CTA per patch: floor(x * (n / box)) per axis in the patch's
// grid, clamped (positions outside [0, box] set SPH_DEV_POS_RANGE).  KD: each record is kicked and drifted (walls
// of the patch box) first.
template <bool KD>
__global__ void __launch_bounds__(256) k_bin_count_patches(const uint8_t *__restrict__ aos, int64_t stride, int off_x,
                                                           const int64_t *__restrict__ patch_start, Grid g,
                                                           const int *__restrict__ patch_n,
                                                           const double *__restrict__ patch_inv,
                                                           const int *__restrict__ patch_cell_base,
                                                           int *__restrict__ cell_of, int *__restrict__ count,
                                                           unsigned *status, KickDrift kd)
{
    const int p = blockIdx.x;
    const int64_t s = patch_start[p], e = patch_start[p + 1];
    const int nx = patch_n[3 * p], ny = patch_n[3 * p + 1], nz = patch_n[3 * p + 2];
    const double ix = patch_inv[3 * p], iy = patch_inv[3 * p + 1], iz = patch_inv[3 * p + 2];
    const int cb = patch_cell_base[p];
    bool bad = false;
    for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
        double x[3];
        if (KD) {
            kick_drift_record(kd.aos + i * stride, off_x, kd, g, x);
        } else {
            const double *xp = reinterpret_cast<const double *>(aos + i * stride + off_x);
            x[0] = __ldg(xp + 0);
            x[1] = __ldg(xp + 1);
            x[2] = __ldg(xp + 2);
        }
        const int kx = cell_coord(x[0], ix, nx, g.box[0], bad);
        const int ky = cell_coord(x[1], iy, ny, g.box[1], bad);
        const int kz = cell_coord(x[2], iz, nz, g.box[2], bad);
        const int c = cb + kx + nx * (ky + ny * kz);
        cell_of[i] = c;
        atomicAdd(&count[c], 1);
    }
    if (bad) atomicOr(status, SPH_DEV_POS_RANGE);
}

// Origin of the slot's cell along an axis: k * edge, the product rounded once in FP64.
__device__ __forceinline__ double cell_origin(const CellSpace &cs, int c, int axis)
{
    CellLoc L;
    locate_cell(cs, c, L);
    const int k = axis == 0 ? L.k[0] : (axis == 1 ? L.k[1] : L.k[2]);
    return __dmul_rn((double)k, cell_edge(cs, L, axis));
}

// Gather: VEC16 selects 16-byte chunks (record stride and buffer 16-byte aligned) or 8-byte items.
template <bool VEC16, bool F32>
__global__ void __launch_bounds__(kTile) k_gather(const uint8_t *__restrict__ aos, int64_t stride,
                                                  const int *__restrict__ perm,
                                                  const int *__restrict__ cell_of_slot, int n,
                                                  const ConvPlan plan, const CellSpace cs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int srec[kTile];
    __shared__ double sorg[F32 ? 3 * kTile : 1];  // FP32 views: origin of each slot's cell
    __shared__ int prange[2];
    const int base = blockIdx.x * kTile;
    const int cnt = min(kTile, n - base);
    const int tid = threadIdx.x;
    for (int s = tid; s < cnt; s += kTile) {
        const int r = perm[base + s];
        srec[s] = SPH_CHECK(r >= 0 && r < n, plan.status) ? r : 0;  // checked build: a bad entry reads record 0
    }
    bool haspos = false;
    if (F32) {
        for (int k = 0; k < plan.nitems; ++k) haspos = haspos || plan.item_pos[k] >= 0;
        if (haspos && cs.npatch > 0 && tid < 2) {
            // the tile's slots are cell-ordered, so its cells lie in the patches between these two
            CellLoc L;
            locate_cell(cs, cell_of_slot[base + (tid == 0 ? 0 : cnt - 1)], L);
            prange[tid] = L.patch;
        }
    }
    __syncthreads();
    if (F32 && haspos) {
        const int lo = cs.npatch > 0 ? prange[0] : 0, hi = cs.npatch > 0 ? prange[1] + 1 : 0;
        for (int s = tid; s < cnt; s += kTile) {
            CellLoc L;
            locate_cell_in(cs, cell_of_slot[base + s], lo, hi, L);
#pragma unroll
            for (int a = 0; a < 3; ++a) sorg[3 * s + a] = __dmul_rn((double)L.k[a], cell_edge(cs, L, a));
        }
    }
    const int nch = plan.nchunks;
    const int nload = cnt * nch;
    const int cw = VEC16 ? 2 : 1;  // doubles per chunk
    // a slot's chunks occupy rs doubles of shared memory, rs odd: the same member of 32 consecutive slots then
    // falls on distinct bank pairs when phase 2 reads across slots
    const int rs = (cw * nch) | 1;
    double *dbuf = reinterpret_cast<double *>(smem);
    // several independent loads in flight per thread before the first store (see k_record_pass)
    const unsigned inv_nch = div_inv(nch);
    if (VEC16) {
        for (int i0 = tid; i0 < nload; i0 += kUnroll * kTile) {
            double2 w[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int idx = i0 + u * kTile;
                if (idx < nload) {
                    const int s = div_small(idx, inv_nch);
                    w[u] = __ldg(reinterpret_cast<const double2 *>(aos + (int64_t)srec[s] * stride +
                                                                   plan.chunk_off[idx - s * nch]));
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int idx = i0 + u * kTile;
                if (idx < nload) {
                    const int s = div_small(idx, inv_nch);
                    const int c = idx - s * nch;
                    dbuf[s * rs + 2 * c] = w[u].x;
                    dbuf[s * rs + 2 * c + 1] = w[u].y;
                }
            }
        }
    } else {
        for (int i0 = tid; i0 < nload; i0 += kUnroll * kTile) {
            double w[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int idx = i0 + u * kTile;
                if (idx < nload) {
                    const int s = div_small(idx, inv_nch);
                    w[u] = __ldg(reinterpret_cast<const double *>(aos + (int64_t)srec[s] * stride +
                                                                  plan.chunk_off[idx - s * nch]));
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int idx = i0 + u * kTile;
                if (idx < nload) {
                    const int s = div_small(idx, inv_nch);
                    dbuf[s * rs + idx - s * nch] = w[u];
                }
            }
        }
    }
    __syncthreads();
    for (int kk = 0; kk < plan.nitems * (tid < cnt ? 1 : 0); ++kk) {  // one slot per thread, item by item
        const int k = kk, s = tid;
        double v = dbuf[s * rs + plan.item_chunk[k] * cw + plan.item_sub[k]];
        const int pc = plan.item_pred_chunk[k];
        if (pc >= 0) v = __dadd_rn(v, __dmul_rn(dbuf[s * rs + pc * cw + plan.item_pred_sub[k]], plan.pred_dt));
        if (!F32) {
            static_cast<double *>(plan.soa[k])[base + s] = v;
        } else {
            const int axis = plan.item_pos[k];
            float o;
            if (axis >= 0) {
                o = __double2float_rn(__dsub_rn(v, sorg[3 * s + axis]));
            } else {
                o = __double2float_rn(v);
            }
            static_cast<float *>(plan.soa[k])[base + s] = o;
        }
    }
}

template <bool F32>
__global__ void __launch_bounds__(kTile) k_scatter(uint8_t *__restrict__ aos, int64_t stride,
                                                   const int *__restrict__ perm,
                                                   const int *__restrict__ cell_of_slot, int n,
                                                   const ConvPlan plan, const CellSpace cs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int srec[kTile];
    double *sval = reinterpret_cast<double *>(smem);
    const int base = blockIdx.x * kTile;
    const int cnt = min(kTile, n - base);
    const int tid = threadIdx.x;
    const int ni = plan.nitems;
    const int sst = ni | 1;  // odd stride of a slot's values in shared memory (no bank conflicts across slots)
    const bool kick = plan.kick_dt != 0.0;
    double *skick = sval + (size_t)kTile * sst;  // with the kick: the records' v (3) and u, 4 per slot
    if (tid < cnt) {
        // phase 1, one slot per thread: its record, its SoA values and (kick) the record's v and u, all loads
        // independent, so they are in flight together
        const int s = tid;
        int rec = perm[base + s];
        if (!SPH_CHECK(rec >= 0 && rec < n, plan.status)) rec = -1;  // checked build: nothing of it is read or written
        srec[s] = rec;
        double w[kMaxItems];
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) {
            if (k < ni)
                w[k] = F32 ? (double)static_cast<const float *>(plan.soa[k])[base + s]
                           : static_cast<const double *>(plan.soa[k])[base + s];
        }
        double kv[4];
        if (kick && rec >= 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                kv[c] = *reinterpret_cast<const double *>(aos + (int64_t)rec * stride + plan.kick_off[c]);
        }
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) {
            if (k >= ni) break;
            double v = w[k];
            if (F32) {
                const int axis = plan.item_pos[k];
                if (axis >= 0) v = __dadd_rn(cell_origin(cs, cell_of_slot[base + s], axis), v);
            }
            sval[s * sst + k] = v;
        }
        if (kick) {
#pragma unroll
            for (int c = 0; c < 4; ++c) skick[4 * s + c] = kv[c];
        }
    }
    __syncthreads();
    // phase 2: consecutive threads write consecutive members of a record (a warp's stores cover few records)
    const int nin = cnt * ni;
    const unsigned inv_ni = div_inv(ni);
    for (int idx = tid; idx < nin; idx += kTile) {
        const int s = div_small(idx, inv_ni);
        const int k = idx - s * ni;
#ifdef SPH_CHECKED
        if (srec[s] < 0) continue;
#endif
        double *p = reinterpret_cast<double *>(aos + (int64_t)srec[s] * stride + plan.item_off[k]);
        *p = sval[s * sst + k];
    }
    if (kick) {
        // the leapfrog's second kick fused into the epilogue: v += a dt/2, u += du/dt dt/2 with the values just
        // written (the same doubles the record now holds)
        for (int idx = tid; idx < 4 * cnt; idx += kTile) {
            const int s = idx >> 2, c = idx & 3;
#ifdef SPH_CHECKED
            if (srec[s] < 0) continue;
#endif
            double *p = reinterpret_cast<double *>(aos + (int64_t)srec[s] * stride + plan.kick_off[c]);
            *p = kick1(skick[idx], sval[s * sst + plan.kick_item[c]], plan.kick_dt);
        }
    }
}

// Record pass (RecordPlan): CTA per tile of kTile consecutive records.  Phase 1 loads the plan's 16-byte chunks of
// the tile's records into shared memory, consecutive threads on consecutive chunks (coalesced).  Phase 2, one
// thread per record: with KD the kick and drift on the shared copies (written back to the record: x, v, u), then
// the cell of the position in the grid or in its patch's grid, the histogram and the range check.  Phase 3 writes
// the staged items in record order (coalesced), v and u predicted where the plan asks.
template <bool KD, bool PATCH, bool F32>
__global__ void __launch_bounds__(kTile, 6) k_record_pass(uint8_t *__restrict__ aos, int64_t stride, int n,
                                                       const RecordPlan rp, Grid g,
                                                       const int64_t *__restrict__ patch_start, int npatch,
                                                       const int *__restrict__ patch_n,
                                                       const double *__restrict__ patch_inv,
                                                       const int *__restrict__ patch_cell_base,
                                                       int *__restrict__ cell_of, int *__restrict__ count,
                                                       unsigned *status, unsigned long long *__restrict__ hmax_bits)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int prange[2];
    __shared__ unsigned long long hmx[kHmaxSlots];  // patch views: the tile's largest h per patch (bit patterns)
    const int base = blockIdx.x * kTile;
    const int cnt = min(kTile, n - base);
    const int tid = threadIdx.x;
    const int nch = rp.conv.nchunks;
    // a record's chunks occupy rs = 2 nch + 1 doubles of shared memory: the odd stride puts the same member of 32
    // consecutive records on distinct bank pairs (phases 2 and 3 read across records)
    const int rs = 2 * nch + 1;
    double *dbuf = reinterpret_cast<double *>(smem);
    const uint8_t *tile = aos + (int64_t)base * stride;
    // kUnroll independent 16-byte loads per thread are issued before the first of them is stored, so that each
    // thread keeps several loads in flight (one at a time bounds the pass by memory latency, not bandwidth)
    const unsigned inv_nch = div_inv(nch);
    constexpr int kU = 4;  // loads in flight per thread (six CTAs per SM keep 48 warps issuing them)
    for (int i0 = tid; i0 < cnt * nch; i0 += kU * kTile) {
        double2 w[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int idx = i0 + u * kTile;
            if (idx < cnt * nch) {
                const int s = div_small(idx, inv_nch);
                w[u] = *reinterpret_cast<const double2 *>(tile + (int64_t)s * stride + rp.conv.chunk_off[idx - s * nch]);
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int idx = i0 + u * kTile;
            if (idx < cnt * nch) {
                const int s = div_small(idx, inv_nch);
                const int c = idx - s * nch;
                dbuf[s * rs + 2 * c] = w[u].x;
                dbuf[s * rs + 2 * c + 1] = w[u].y;
            }
        }
    }
    if (PATCH && tid < kHmaxSlots) hmx[tid] = 0ull;
    if (PATCH && tid < 2) {
        // patch of the tile's first / last record: the largest p with patch_start[p] <= i
        const int64_t i = base + (tid == 0 ? 0 : cnt - 1);
        int lo = 0, hi = npatch;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (patch_start[mid] <= i) lo = mid; else hi = mid;
        }
        prange[tid] = lo;
    }
    __syncthreads();
    if (tid < cnt) {
        double *r = dbuf + (size_t)tid * rs;
        double x[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) x[d] = r[rp.x_ch[d] * 2 + rp.x_sub[d]];
        if (KD) {
            double v[3], a[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                v[d] = r[rp.kd_ch[3 + d] * 2 + rp.kd_sub[3 + d]];
                a[d] = r[rp.kd_ch[6 + d] * 2 + rp.kd_sub[6 + d]];
            }
            double u = r[rp.kd_ch[9] * 2 + rp.kd_sub[9]];
            const double du = r[rp.kd_ch[10] * 2 + rp.kd_sub[10]];
            double vp[3], up;
            kick_drift_predict(x, v, u, a, du, rp.dtk, rp.dt, g, vp, up);
            // the records get the half-step v, u; the staged view gets the predicted ones (kd_pred) or those
            const double nv[7] = {x[0], x[1], x[2], v[0], v[1], v[2], u};
            const double sv[7] = {x[0], x[1], x[2], rp.kd_pred ? vp[0] : v[0], rp.kd_pred ? vp[1] : v[1],
                                  rp.kd_pred ? vp[2] : v[2], rp.kd_pred ? up : u};
            uint8_t *rec = aos + (int64_t)(base + tid) * stride;
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                r[rp.kd_ch[k < 6 ? k : 9] * 2 + rp.kd_sub[k < 6 ? k : 9]] = sv[k];
                *reinterpret_cast<double *>(rec + rp.kd_off[k]) = nv[k];
            }
        }
        if (PATCH) {
            // patch views bin later, per patch (k_patch_bin), once the patch grids are known; here the largest h
            // of each patch is gathered for them (h > 0, infinities included, NaN left out, as fmax would)
            int lo = prange[0], hi = prange[1] + 1;
            const int64_t i = base + tid;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (patch_start[mid] <= i) lo = mid; else hi = mid;
            }
            const long long hb = __double_as_longlong(r[rp.h_ch * 2 + rp.h_sub]);
            if (hb > 0 && hb <= 0x7FF0000000000000LL) {
                const int slot = lo - prange[0];
                if (slot < kHmaxSlots) atomicMax(&hmx[slot], (unsigned long long)hb);
                else atomicMax(&hmax_bits[lo], (unsigned long long)hb);
            }
        } else {
            bool bad = false;
            const int kx = cell_coord_bits(x[0], g.inv[0], g.n[0], g.box[0], bad);
            const int ky = cell_coord_bits(x[1], g.inv[1], g.n[1], g.box[1], bad);
            const int kz = cell_coord_bits(x[2], g.inv[2], g.n[2], g.box[2], bad);
            const int c = kx + g.n[0] * (ky + g.n[1] * kz);
            cell_of[base + tid] = c;
            atomicAdd(&count[c], 1);
            if (bad) atomicOr(status, SPH_DEV_POS_RANGE);
        }
    }
    __syncthreads();
    if (PATCH && tid < kHmaxSlots && tid <= prange[1] - prange[0] && hmx[tid] != 0ull)
        atomicMax(&hmax_bits[prange[0] + tid], hmx[tid]);
    const ConvPlan &plan = rp.conv;
    if (tid < cnt) {  // one record per thread (kTile records per tile): its packed row
        const double *r = dbuf + (size_t)tid * rs;
        uint8_t *row = rp.rows + (int64_t)(base + tid) * rp.row_bytes;
        for (int k = 0; k < plan.nitems; ++k) {
            double v = r[plan.item_chunk[k] * 2 + plan.item_sub[k]];
            const int pc = plan.item_pred_chunk[k];
            if (pc >= 0) v = __dadd_rn(v, __dmul_rn(r[pc * 2 + plan.item_pred_sub[k]], plan.pred_dt));
            if (!F32 || plan.item_pos[k] >= 0) {
                *reinterpret_cast<double *>(row + rp.row_off[k]) = v;
            } else {
                *reinterpret_cast<float *>(row + rp.row_off[k]) = __double2float_rn(v);
            }
        }
    }
}

// Permutation of staged items into slot order (PermutePlan), CTA per tile of kTile slots; FP32 positions become
// (float)(x - origin of the slot's cell), with the origin as the gather computes it.  Slots are in cell order, so
// a tile's slots lie in the cells cell_of_slot[base] .. cell_of_slot[base + cnt - 1]: when there are at most
// kTile of them, each origin is formed once per cell in shared memory, else once per slot (the same products
// either way).  The other FP32 members move as the float bits the record pass stored.  Conversions to and from
// FP64 run on the FP64 pipe, 1/64 of the FP32 rate on this part: per slot, only the positions' subtraction and
// rounding remain.
template <bool F32>
__global__ void __launch_bounds__(kTile) k_permute(const int *__restrict__ perm, const int *__restrict__ cell_of_slot,
                                                   int n, const PermutePlan pp, const CellSpace cs)
{
    __shared__ int srec[kTile];
    __shared__ double sorg[F32 ? 3 * kTile : 1];
    __shared__ int prange[2];
    const int base = blockIdx.x * kTile;
    const int cnt = min(kTile, n - base);
    const int tid = threadIdx.x;
    for (int s = tid; s < cnt; s += kTile) {
        const int r = perm[base + s];
        srec[s] = SPH_CHECK(r >= 0 && r < n, pp.status) ? r : 0;  // checked build: a bad entry reads row 0
    }
    bool haspos = false;
    int c0 = 0, ncl = 0;  // the tile's cells c0 .. c0 + ncl - 1 (FP32 positions)
    if (F32) {
        for (int k = 0; k < pp.nitems; ++k) haspos = haspos || pp.item_pos[k] >= 0;
        if (haspos) {
            c0 = cell_of_slot[base];
            ncl = cell_of_slot[base + cnt - 1] - c0 + 1;
            if (cs.npatch > 0 && tid < 2) {
                CellLoc L;
                locate_cell(cs, tid == 0 ? c0 : c0 + ncl - 1, L);
                prange[tid] = L.patch;
            }
        }
    }
    __syncthreads();
    const bool per_cell = ncl >= 1 && ncl <= kTile;  // CTA-uniform
    int lo = 0, hi = 0;                               // the patches of the tile's cells
    if (F32 && haspos) {
        lo = cs.npatch > 0 ? prange[0] : 0;
        hi = cs.npatch > 0 ? prange[1] + 1 : 0;
        for (int j = tid; j < (per_cell ? ncl : cnt); j += kTile) {
            CellLoc L;
            locate_cell_in(cs, per_cell ? c0 + j : cell_of_slot[base + j], lo, hi, L);
#pragma unroll
            for (int a = 0; a < 3; ++a) sorg[3 * j + a] = __dmul_rn((double)L.k[a], cell_edge(cs, L, a));
        }
        __syncthreads();
    }
    if (tid < cnt) {  // one slot per thread: its record's packed row, all loads in flight before the stores
        const int s = tid;
        const uint8_t *row = pp.rows + (int64_t)srec[s] * pp.row_bytes;
        unsigned long long w[kMaxItems];  // an item's bits: a double, or an FP32 member's float (not a position)
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) {
            if (k < pp.nitems)
                w[k] = (!F32 || pp.item_pos[k] >= 0)
                           ? *reinterpret_cast<const unsigned long long *>(row + pp.row_off[k])
                           : (unsigned long long)*reinterpret_cast<const unsigned *>(row + pp.row_off[k]);
        }
        double org[3] = {0.0, 0.0, 0.0};
        if (F32 && haspos) {
            // the slot's cell in the tile's range (always, for slots in cell order); else its origin afresh
            const int j = per_cell ? cell_of_slot[base + s] - c0 : s;
            if (!per_cell || (unsigned)j < (unsigned)ncl) {
#pragma unroll
                for (int a = 0; a < 3; ++a) org[a] = sorg[3 * j + a];
            } else {
                CellLoc L;
                locate_cell(cs, cell_of_slot[base + s], L);
#pragma unroll
                for (int a = 0; a < 3; ++a) org[a] = __dmul_rn((double)L.k[a], cell_edge(cs, L, a));
            }
        }
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) {
            if (k >= pp.nitems) break;
            if (!F32) {
                static_cast<unsigned long long *>(pp.dst[k])[base + s] = w[k];
            } else {
                const int axis = pp.item_pos[k];
                if (axis >= 0) {  // (float)(x - origin)
                    double o = org[0];
                    if (axis == 1) o = org[1];
                    if (axis == 2) o = org[2];
                    static_cast<float *>(pp.dst[k])[base + s] =
                        __double2float_rn(__dsub_rn(__longlong_as_double((long long)w[k]), o));
                } else {
                    static_cast<unsigned *>(pp.dst[k])[base + s] = (unsigned)w[k];
                }
            }
        }
    }
}

constexpr int kPatchThreads = 512;
constexpr int kPatchCap = 8192;  // records of a patch whose cells k_patch_bin keeps in shared memory

// Bin of one patch, CTA per patch (patch views, after the record pass and the patch grids): the cell of every
// record from its staged (drifted) position, the patch's cell counts, cell_start of its cells (global slot
// offsets: the patch's slots are its record range), and the stable slot order -- ascending record index inside a
// cell.  Each warp owns a contiguous range of the patch's records: it counts per cell (lanes with the same cell
// found by __match_any_sync), the counts are turned into per-warp bases (cell-major, warp order), and each warp
// places its records in order, ranked among equal cells by lane.  Cells of a key (up to kPatchCap records) are
// kept in shared memory between the passes.
constexpr int kBinWarps = kPatchThreads / 32;
constexpr int kBinCellCap = 512;  // cells of a patch grid: ncap^3 <= 512 (ncap <= 8)

__device__ __forceinline__ int patch_cell_of(const uint8_t *rows, int row_bytes, int x_off, int i, const Grid &g,
                                             int nx, int ny, int nz, const double *inv, bool &bad)
{
    const double *x = reinterpret_cast<const double *>(rows + (int64_t)i * row_bytes + x_off);
    const int kx = cell_coord_bits(x[0], inv[0], nx, g.box[0], bad);
    const int ky = cell_coord_bits(x[1], inv[1], ny, g.box[1], bad);
    const int kz = cell_coord_bits(x[2], inv[2], nz, g.box[2], bad);
    return kx + nx * (ky + ny * kz);
}

__global__ void __launch_bounds__(kPatchThreads) k_patch_bin(const uint8_t *__restrict__ rows, int row_bytes,
                                                             int x_off,
                                                             const int64_t *__restrict__ patch_start, Grid g,
                                                             const int *__restrict__ patch_n,
                                                             const double *__restrict__ patch_inv,
                                                             const int *__restrict__ patch_cell_base,
                                                             const int *__restrict__ ncells_dev, int n,
                                                             int *__restrict__ cell_start, int *__restrict__ perm,
                                                             int *__restrict__ cell_of_slot, unsigned *status)
{
    extern __shared__ __align__(16) int bsm[];
    int *cnt = bsm;                              // [kBinWarps][kBinCellCap]
    int *off = cnt + kBinWarps * kBinCellCap;    // [kBinCellCap]
    unsigned short *key = reinterpret_cast<unsigned short *>(off + kBinCellCap);  // [kPatchCap]
    const int p = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (p == 0 && tid == 0) cell_start[*ncells_dev] = n;
    const int ps = (int)patch_start[p], np = (int)(patch_start[p + 1] - ps);
    const int nx = patch_n[3 * p], ny = patch_n[3 * p + 1], nz = patch_n[3 * p + 2];
    const int ncp = nx * ny * nz, cb = patch_cell_base[p];
    const double inv[3] = {patch_inv[3 * p], patch_inv[3 * p + 1], patch_inv[3 * p + 2]};
    if (np <= 0) {  // CTA-uniform: an empty patch's cells all start at its offset
        for (int c = tid; c < ncp; c += kPatchThreads) cell_start[cb + c] = ps;
        return;
    }
    for (int i = tid; i < kBinWarps * kBinCellCap; i += kPatchThreads) cnt[i] = 0;
    __syncthreads();
    const bool keyed = np <= kPatchCap;
    const int R = (np + kBinWarps - 1) / kBinWarps;
    const int r0 = min(np, w * R), r1 = min(np, r0 + R);
    int *mine = cnt + w * kBinCellCap;
    bool bad = false;
    for (int b = r0; b < r1; b += 32) {
        const int i = b + lane;
        int c = -1;
        if (i < r1) {
            c = patch_cell_of(rows, row_bytes, x_off, ps + i, g, nx, ny, nz, inv, bad);
            if (keyed) key[i] = (unsigned short)c;
        }
        const unsigned grp = __match_any_sync(kFull, c);
        if (c >= 0 && lane == __ffs(grp) - 1) mine[c] += __popc(grp);
        __syncwarp();
    }
    __syncthreads();
    // per cell: warp bases in warp order, then the exclusive scan over cells
    for (int c = tid; c < ncp; c += kPatchThreads) {
        int run = 0;
        for (int ww = 0; ww < kBinWarps; ++ww) {
            const int t = cnt[ww * kBinCellCap + c];
            cnt[ww * kBinCellCap + c] = run;
            run += t;
        }
        off[c] = run;
    }
    __syncthreads();
    if (w == 0) {  // one warp scans the (at most 512) cell totals: 16 consecutive cells per lane
        constexpr int per = kBinCellCap / 32;
        int v[per], sum = 0;
#pragma unroll
        for (int k = 0; k < per; ++k) {
            const int c = lane * per + k;
            v[k] = c < ncp ? off[c] : 0;
            sum += v[k];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        int run = incl - sum;
#pragma unroll
        for (int k = 0; k < per; ++k) {
            const int c = lane * per + k;
            if (c < ncp) off[c] = run;
            run += v[k];
        }
    }
    __syncthreads();
    for (int c = tid; c < ncp; c += kPatchThreads) {
        const int o = off[c];
        cell_start[cb + c] = ps + o;
        for (int ww = 0; ww < kBinWarps; ++ww) cnt[ww * kBinCellCap + c] += o;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int b = r0; b < r1; b += 32) {
        const int i = b + lane;
        int c = -1;
        if (i < r1) c = keyed ? (int)key[i] : patch_cell_of(rows, row_bytes, x_off, ps + i, g, nx, ny, nz, inv, bad);
        const unsigned grp = __match_any_sync(kFull, c);
        if (c >= 0) {
            const int slot = ps + mine[c] + __popc(grp & lt);
            perm[slot] = ps + i;
            cell_of_slot[slot] = cb + c;
        }
        __syncwarp();
        if (c >= 0 && lane == __ffs(grp) - 1) mine[c] += __popc(grp);
        __syncwarp();
    }
    if (bad) atomicOr(status, SPH_DEV_POS_RANGE);
}

}  // namespace

int scan_tmp_ints(int ncells_cap) { return 3 * ((ncells_cap + kScanChunk - 1) / kScanChunk) + 4; }

namespace {

// Exclusive scan of count[0 .. ncells) into cell_start (ncells + 1 entries) and fill; ncells is ncells_dev's
// value when given, else ncells_host, and at most ncells_cap.  Small capacities (or no scratch): one CTA.
void launch_scan(const int *count, int ncells_host, const int *ncells_dev, int ncells_cap, int *cell_start, int *fill,
                 int *scan_tmp, cudaStream_t st, int *nl)
{
    if (!scan_tmp || ncells_cap <= 4 * kScanChunk) {
        k_scan_cells<<<1, kScanThreads, 0, st>>>(count, ncells_host, ncells_dev, cell_start, fill);
        ++*nl;
        return;
    }
    const int nb = (ncells_cap + kScanChunk - 1) / kScanChunk;
    int *block_sum = scan_tmp, *block_off = scan_tmp + nb, *block_fill = scan_tmp + 2 * nb + 1;
    k_scan_block_sums<<<nb, kScanThreads, 0, st>>>(count, ncells_host, ncells_dev, block_sum);
    k_scan_cells<<<1, kScanThreads, 0, st>>>(block_sum, nb, nullptr, block_off, block_fill);
    k_scan_apply<<<nb, kScanThreads, 0, st>>>(count, ncells_host, ncells_dev, block_off, cell_start, fill);
    *nl += 3;
}

}  // namespace

cudaError_t launch_bin(const uint8_t *aos, int64_t stride, int off_x, int n, const Grid &g, int ncells,
                       int *cell_of, int *count, int *cell_start, int *fill, int *perm_tmp, int *perm,
                       int *cell_of_slot, int *scan_tmp, unsigned *status, cudaStream_t st, int *nl,
                       const KickDrift *kd)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncells, st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        if (kd) {
            k_bin_count<true><<<(n + 255) / 256, 256, 0, st>>>(aos, stride, off_x, n, g, cell_of, count, status, *kd);
        } else {
            k_bin_count<false><<<(n + 255) / 256, 256, 0, st>>>(aos, stride, off_x, n, g, cell_of, count, status,
                                                                KickDrift{});
        }
        ++*nl;
    }
    launch_scan(count, ncells, nullptr, ncells, cell_start, fill, scan_tmp, st, nl);
    if (n > 0) {
        *nl += 2;
        k_bin_place<<<(n + 255) / 256, 256, 0, st>>>(cell_of, n, fill, perm_tmp, status);
        const long long threads = (long long)ncells * 32;
        const long long blocks = (threads + 255) / 256;
        k_cell_sort<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(cell_start, ncells, nullptr,
                                                                                perm_tmp, perm, cell_of_slot);
    }
    return cudaGetLastError();
}

cudaError_t launch_bin_patches(const uint8_t *aos, int64_t stride, int off_x, int off_h, int n,
                               const int64_t *patch_start, int npatch, const Grid &box, int ncap, int ncells_cap,
                               int *patch_n, double *patch_edge, int *patch_cells, int *patch_cell_base,
                               int *ncells_dev, int *cell_of, int *count, int *cell_start, int *fill,
                               int *perm_tmp, int *perm, int *cell_of_slot, int *scan_tmp, unsigned *status,
                               cudaStream_t st, int *nl, const KickDrift *kd)
{
    // patch_edge holds 3 * npatch edges followed by 3 * npatch inverses
    double *patch_inv = patch_edge + 3 * (size_t)npatch;
    k_patch_grid<<<npatch, 256, 0, st>>>(aos, stride, off_h, patch_start, box, ncap, patch_n, patch_edge, patch_inv,
                                         patch_cells);
    k_scan_cells<<<1, kScanThreads, 0, st>>>(patch_cells, npatch, nullptr, patch_cell_base, fill);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncells_cap, st);
    if (e != cudaSuccess) return e;
    *nl += 2;
    if (n > 0) {
        if (kd) {
            k_bin_count_patches<true><<<npatch, 256, 0, st>>>(aos, stride, off_x, patch_start, box, patch_n,
                                                              patch_inv, patch_cell_base, cell_of, count, status, *kd);
        } else {
            k_bin_count_patches<false><<<npatch, 256, 0, st>>>(aos, stride, off_x, patch_start, box, patch_n,
                                                               patch_inv, patch_cell_base, cell_of, count, status,
                                                               KickDrift{});
        }
        ++*nl;
    }
    launch_scan(count, ncells_cap, ncells_dev, ncells_cap, cell_start, fill, scan_tmp, st, nl);
    if (n > 0) {
        k_bin_place<<<(n + 255) / 256, 256, 0, st>>>(cell_of, n, fill, perm_tmp, status);
        k_cell_sort<<<2048, 256, 0, st>>>(cell_start, ncells_cap, ncells_dev, perm_tmp, perm, cell_of_slot);
        *nl += 2;
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const uint8_t *aos, int64_t stride, bool vec16, const int *perm,
                          const int *cell_of_slot, int n, const ConvPlan &plan, const CellSpace &g, bool f32,
                          cudaStream_t st, int *nl)
{
    if (n <= 0 || plan.nitems == 0) return cudaSuccess;
    ++*nl;
    const int blocks = (n + kTile - 1) / kTile;
    const size_t smem = (size_t)kTile * (((vec16 ? 2 : 1) * plan.nchunks) | 1) * 8;
    if (vec16) {
        if (f32) {
            cudaFuncSetAttribute(k_gather<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_gather<true, true><<<blocks, kTile, smem, st>>>(aos, stride, perm, cell_of_slot, n, plan, g);
        } else {
            cudaFuncSetAttribute(k_gather<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_gather<true, false><<<blocks, kTile, smem, st>>>(aos, stride, perm, cell_of_slot, n, plan, g);
        }
    } else {
        if (f32) {
            cudaFuncSetAttribute(k_gather<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_gather<false, true><<<blocks, kTile, smem, st>>>(aos, stride, perm, cell_of_slot, n, plan, g);
        } else {
            cudaFuncSetAttribute(k_gather<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_gather<false, false><<<blocks, kTile, smem, st>>>(aos, stride, perm, cell_of_slot, n, plan, g);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter(uint8_t *aos, int64_t stride, const int *perm, const int *cell_of_slot, int n,
                           const ConvPlan &plan, const CellSpace &g, bool f32, cudaStream_t st, int *nl)
{
    if (n <= 0 || plan.nitems == 0) return cudaSuccess;
    ++*nl;
    const int blocks = (n + kTile - 1) / kTile;
    const size_t smem = (size_t)kTile * ((plan.nitems | 1) + (plan.kick_dt != 0.0 ? 4 : 0)) * 8;
    if (f32) {
        cudaFuncSetAttribute(k_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_scatter<true><<<blocks, kTile, smem, st>>>(aos, stride, perm, cell_of_slot, n, plan, g);
    } else {
        cudaFuncSetAttribute(k_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_scatter<false><<<blocks, kTile, smem, st>>>(aos, stride, perm, cell_of_slot, n, plan, g);
    }
    return cudaGetLastError();
}

namespace {

template <bool KD, bool PATCH, bool F32>
void record_pass(uint8_t *aos, int64_t stride, int n, const RecordPlan &rp, const Grid &g, const int64_t *patch_start,
                 int npatch, const int *patch_n, const double *patch_inv, const int *patch_cell_base, int *cell_of,
                 int *count, unsigned *status, unsigned long long *hmax, cudaStream_t st)
{
    const size_t smem = (size_t)kTile * (2 * rp.conv.nchunks + 1) * 8;
    cudaFuncSetAttribute(k_record_pass<KD, PATCH, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_record_pass<KD, PATCH, F32><<<(n + kTile - 1) / kTile, kTile, smem, st>>>(
        aos, stride, n, rp, g, patch_start, npatch, patch_n, patch_inv, patch_cell_base, cell_of, count, status, hmax);
}

template <bool KD, bool PATCH>
void record_pass_p(bool f32, uint8_t *aos, int64_t stride, int n, const RecordPlan &rp, const Grid &g,
                   const int64_t *patch_start, int npatch, int *cell_of, int *count, unsigned *status,
                   unsigned long long *hmax, cudaStream_t st)
{
    if (f32) {
        record_pass<KD, PATCH, true>(aos, stride, n, rp, g, patch_start, npatch, nullptr, nullptr, nullptr, cell_of,
                                     count, status, hmax, st);
    } else {
        record_pass<KD, PATCH, false>(aos, stride, n, rp, g, patch_start, npatch, nullptr, nullptr, nullptr, cell_of,
                                      count, status, hmax, st);
    }
}

}  // namespace

cudaError_t launch_bin_staged(uint8_t *aos, int64_t stride, int n, const RecordPlan &rp, bool f32, const Grid &g,
                              int ncells, const int64_t *patch_start, int npatch, int ncap, int *patch_n,
                              double *patch_edge, int *patch_cells, int *patch_cell_base, int *ncells_dev,
                              unsigned long long *hmax, int x_off, int *cell_of, int *count,
                              int *cell_start, int *fill, int *perm_tmp, int *perm, int *cell_of_slot, int *scan_tmp,
                              unsigned *status, cudaStream_t st, int *nl)
{
    if (npatch > 0) {
        // patch views: record pass (leapfrog, staging, h maxima), patch grids, then one bin per patch
        double *patch_inv = patch_edge + 3 * (size_t)npatch;
        cudaError_t e = cudaMemsetAsync(hmax, 0, sizeof(unsigned long long) * (size_t)npatch, st);
        if (e != cudaSuccess) return e;
        if (n > 0) {
            ++*nl;
            if (rp.kd) {
                record_pass_p<true, true>(f32, aos, stride, n, rp, g, patch_start, npatch, nullptr, nullptr, status,
                                          hmax, st);
            } else {
                record_pass_p<false, true>(f32, aos, stride, n, rp, g, patch_start, npatch, nullptr, nullptr, status,
                                           hmax, st);
            }
        }
        k_patch_grid_hmax<<<(npatch + 255) / 256, 256, 0, st>>>(hmax, npatch, g, ncap, patch_n, patch_edge,
                                                                 patch_inv, patch_cells);
        k_scan_cells<<<1, kScanThreads, 0, st>>>(patch_cells, npatch, nullptr, patch_cell_base, fill);
        const size_t smem = (size_t)(kBinWarps * kBinCellCap + kBinCellCap) * 4 + (size_t)kPatchCap * 2;
        cudaFuncSetAttribute(k_patch_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_patch_bin<<<npatch, kPatchThreads, smem, st>>>(rp.rows, rp.row_bytes, x_off, patch_start, g, patch_n, patch_inv,
                                                          patch_cell_base, ncells_dev, n, cell_start, perm,
                                                          cell_of_slot, status);
        *nl += 3;
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncells, st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        ++*nl;
        if (rp.kd) {
            record_pass_p<true, false>(f32, aos, stride, n, rp, g, nullptr, 0, cell_of, count, status, nullptr, st);
        } else {
            record_pass_p<false, false>(f32, aos, stride, n, rp, g, nullptr, 0, cell_of, count, status, nullptr, st);
        }
    }
    launch_scan(count, ncells, nullptr, ncells, cell_start, fill, scan_tmp, st, nl);
    if (n > 0) {
        *nl += 2;
        k_bin_place<<<(n + 255) / 256, 256, 0, st>>>(cell_of, n, fill, perm_tmp, status);
        const long long threads = (long long)ncells * 32;
        const long long blocks = (threads + 255) / 256;
        k_cell_sort<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(cell_start, ncells, nullptr,
                                                                                perm_tmp, perm, cell_of_slot);
    }
    return cudaGetLastError();
}

cudaError_t launch_permute(const int *perm, const int *cell_of_slot, int n, const PermutePlan &pp,
                           const CellSpace &cs, bool f32, cudaStream_t st, int *nl)
{
    if (n <= 0 || pp.nitems == 0) return cudaSuccess;
    ++*nl;
    const int blocks = (n + kTile - 1) / kTile;
    if (f32) {
        k_permute<true><<<blocks, kTile, 0, st>>>(perm, cell_of_slot, n, pp, cs);
    } else {
        k_permute<false><<<blocks, kTile, 0, st>>>(perm, cell_of_slot, n, pp, cs);
    }
    return cudaGetLastError();
}

}  // namespace sphk
