// sph_internal.cuh -- definitions shared by the translation units of libsph (device side and host runtime).
//
// Nothing here is visible through the C ABI; include/sph.h is the public surface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sph.h"

namespace sphk {

// Index checks of the checked build (compiled with -DSPH_CHECKED): where an index is read from device data (a
// cell's slot range, a neighbour cell, a work-list entry, a placement slot, a permutation entry), SPH_CHECK(ok,
// status) is ok, and a false ok also sets SPH_DEV_BOUNDS in the status word; the caller then skips the access it
// guards.  In the default build the check is the constant true and compiles away.
#ifdef SPH_CHECKED
#define SPH_CHECK(ok, status) ((ok) ? true : (atomicOr((status), SPH_DEV_BOUNDS), false))
#else
#define SPH_CHECK(ok, status) true
#endif

// 1/pi: normalisation of the 3D cubic spline W(r,h) = f(r/h) / (pi h^3) (Monaghan & Lattanzio 1985).
constexpr double kInvPi = 0.318309886183790671537767526745028724;

constexpr int kMaxItems = 17;   // double components of all ten members (x, v, a are three each)
constexpr int kMaxChunks = 40;  // 16-byte chunks loaded per record by the gather (stride <= 640 B), or items

// Cell grid of a domain (host fills it once per view).
struct Grid {
    int n[3];          // cells per axis
    int periodic;      // wrap every axis
    double box[3];     // domain edge
    double edge[3];    // cell edge = box / n, rounded once in FP64
    double inv[3];     // n / box, rounded once in FP64: cell coordinate = floor(x * inv)
    float edgef[3];    // (float) edge
    double min_edge;   // smallest cell edge: every 2h must fit
};

// Cell space of a view: either one grid over the domain (npatch == 0), or npatch independent patches, each an
// open box of size g.box with its own grid of patch_n[3p..3p+2] cells (chosen per step from the patch's largest h).
// Global cell ids of patch p are patch_cell_base[p] .. patch_cell_base[p+1]-1; inside a grid the id is
// kx + nx (ky + ny kz).
struct CellSpace {
    Grid g;
    int npatch;
    const int *patch_cell_base;  // [npatch + 1]
    const int *patch_n;          // [3 npatch]
    const double *patch_edge;    // [3 npatch]: g.box[a] / patch_n[3p+a], rounded once in FP64
    const int *ncells_dev;       // total cells (device word; patches only)
};

struct CellLoc {
    int k[3];  // cell coordinates inside its grid
    int n[3];  // grid size
    int base;  // first global cell of the grid
    int patch;
};

// Coordinates of global cell c.  Patches: binary search of c in patch_cell_base over the patches [lo, hi), which
// must contain c's patch (locate_cell searches all of them).
__device__ __forceinline__ void locate_cell_in(const CellSpace &cs, int c, int lo, int hi, CellLoc &L)
{
    int local = c;
    if (cs.npatch == 0) {
        L.n[0] = cs.g.n[0];
        L.n[1] = cs.g.n[1];
        L.n[2] = cs.g.n[2];
        L.base = 0;
        L.patch = 0;
    } else {
        while (hi - lo > 1) {  // patch_cell_base[lo] <= c < patch_cell_base[hi]
            const int mid = (lo + hi) >> 1;
            if (cs.patch_cell_base[mid] <= c) lo = mid; else hi = mid;
        }
        L.patch = lo;
        L.base = cs.patch_cell_base[lo];
        L.n[0] = cs.patch_n[3 * lo];
        L.n[1] = cs.patch_n[3 * lo + 1];
        L.n[2] = cs.patch_n[3 * lo + 2];
        local = c - L.base;
    }
    L.k[0] = local % L.n[0];
    L.k[1] = (local / L.n[0]) % L.n[1];
    L.k[2] = local / (L.n[0] * L.n[1]);
}

__device__ __forceinline__ void locate_cell(const CellSpace &cs, int c, CellLoc &L)
{
    locate_cell_in(cs, c, 0, cs.npatch, L);
}

// Cell edge along an axis: box / n rounded once in FP64 (precomputed for the uniform grid and per patch).
__device__ __forceinline__ double cell_edge(const CellSpace &cs, const CellLoc &L, int axis)
{
    if (cs.npatch == 0) return axis == 0 ? cs.g.edge[0] : (axis == 1 ? cs.g.edge[1] : cs.g.edge[2]);
    return cs.patch_edge[3 * L.patch + axis];
}

// Field-selective conversion plan (host builds it from a member mask and the record layout).
// Items are the double components moved; for the 16-byte path the record bytes holding them are loaded as a
// few 16-byte chunks per record, for the 8-byte path every item is its own 8-byte chunk.
struct ConvPlan {
    unsigned *status;  // checked build: SPH_DEV_BOUNDS
    int nitems;
    int nchunks;
    int chunk_off[kMaxChunks];  // byte offset of each loaded chunk inside a record
    int item_off[kMaxItems];    // byte offset of the item inside a record
    int item_chunk[kMaxItems];  // which loaded chunk holds the item
    int item_sub[kMaxItems];    // which 8-byte half of that chunk
    int item_pos[kMaxItems];    // -1, or the axis of a position component (FP32 views store it cell-relative)
    int item_pred_chunk[kMaxItems];  // gather only: -1, or the chunk holding the rate the item is predicted with
    int item_pred_sub[kMaxItems];    // ... and its 8-byte half
    double pred_dt;                  // predicted value = item + rate * pred_dt, each operation rounded in FP64
    // scatter only: with kick_dt != 0, the record's v (3 components) and u are kicked by kick_dt times the
    // scattered items kick_item[0..3] (a_x, a_y, a_z, du/dt), after those are written
    double kick_dt;
    int kick_item[4];
    int kick_off[4];
    void *soa[kMaxItems];       // SoA array of the item (n_max elements)
};

// SoA arrays of one view, by member and component.  Element type is double (SPH_F64) or float (SPH_F32).
struct SoaPtrs {
    void *p[SPH_NFIELDS][3];
};

// View-owned scratch of the pair loops (n_max elements each).
struct Scratch {
    float *xf, *yf, *zf;  // FP64 views: cell-relative float copies of the positions (input of the FP32 filter)
    float *hf;            // FP64 views: (float) h, rounded up (filter radius)
    // Per-particle values of the pair loops, in the view's precision.
    //   FP64 density: d[0..4] the cubic-in-r spline coefficients -3/(2h^2), 3/(4h^3), -3/h, 3/(2h^2), -1/(4h^3),
    //         d[5] 1/(pi h^3), d[6] c_s = sqrt(gamma (gamma - 1) u); other kernels / the extended scheme:
    //         d[0] 1/h, d[1] sigma/h^3, d[2] sigma/h^4, d[6] c_s
    //   FP64 force, other kernels / the extended scheme: d[0] h/2, d[1] 1/h, d[2] sigma/h^4, d[3] P/(Omega rho^2),
    //         d[4] alpha c / 2, d[5] the Balsara switch
    //   FP64 force: d[0] s h/2, d[1] -3/(pi h^4), d[2] 3/(pi h^5), d[3] 9/(4 pi h^6), d[4] -3/(4 pi h^6),
    //         d[5] P/rho^2, d[6] alpha c / (2 s), d[7] (h/2)^2, with s = sqrt(eps) for eps > 0, else 1
    //   FP32: d[0] 1/h, d[1] 1/(pi h^5), d[2] P/rho^2
    void *d[8];
};
constexpr int kDerivedF64 = 8;
constexpr int kDerivedF32 = 3;

struct Counters {
    unsigned long long dens_cand, dens_pairs, force_pairs, force_cand;
};

// Leapfrog work fused into a pass (Section 2.1 steps 3-5; on the records, in FP64 for both view precisions): the
// bin kernel first kicks v, u by a dtk, du/dt dtk and drifts x by v dt (the periodic wrap of the grid, or the
// reflecting walls of an open box or patch), then bins the new position; the last scatter of the pass kicks v, u by
// the new a, du/dt it writes.  aos is the records the bin reads, writable.
struct KickDrift {
    uint8_t *aos;
    int off_v, off_a, off_u, off_du;
    double dtk;  // half kick
    double dt;   // drift
};

// Record-order pass of a pass's bin and first gather, fused (and, with kd, the leapfrog's first kick and drift):
// every record is read once, in record order, with coalesced 16-byte chunk loads; its cell is binned from the
// (drifted) position, and the members of the view are written, in record order, to scratch arrays (predicted
// where asked).  A permutation then moves them to the slot order of the SoA view.
struct RecordPlan {
    // chunks loaded per record; items: the staged view members, written to one packed row per record (record
    // order): item k at byte row_off[k] of the row, as a double for FP64 views and for FP32 views' positions (which
    // get their cell-relative cast in the permutation), as a float otherwise; item_pos marks the position items;
    // item_pred_* / pred_dt as for the gather
    ConvPlan conv;
    uint8_t *rows;
    int row_bytes;
    int row_off[kMaxItems];
    int x_ch[3], x_sub[3];  // the position components in the loaded chunks
    int kd;                 // kick and drift first
    int kd_ch[11], kd_sub[11];  // x0..2, v0..2, a0..2, u, du/dt in the loaded chunks
    int kd_off[7];              // record offsets of x0..2, v0..2, u (written back)
    int kd_pred;                // the staged v, u are predicted by dtk (the items then carry no prediction)
    int h_ch, h_sub;            // patch views: h in the loaded chunks (the record pass gathers each patch's max)
    double dtk, dt;
};

// The permutation of a staged gather: dst[k][s] = src[k][perm[s]], positions of FP32 views cast relative to the
// slot's cell origin as the gather does.
struct PermutePlan {
    unsigned *status;  // checked build: SPH_DEV_BOUNDS
    int nitems;
    int item_pos[kMaxItems];
    const uint8_t *rows;  // the record pass's packed rows (RecordPlan)
    int row_bytes;
    int row_off[kMaxItems];
    void *dst[kMaxItems];
};

// ---- launchers: each enqueues on `st`, adds the number of kernels it launched to *nl and returns the first
// CUDA error (cudaGetLastError after the launches). ----
// scan_tmp: scan_tmp_ints(cells) ints of scratch for the multi-CTA scan of large grids (nullptr: one-CTA scan).
int scan_tmp_ints(int ncells_cap);
// kd (may be null): kick and drift every record before binning it (see KickDrift).
cudaError_t launch_bin(const uint8_t *aos, int64_t stride, int off_x, int n, const Grid &g, int ncells,
                       int *cell_of, int *count, int *cell_start, int *fill, int *perm_tmp, int *perm,
                       int *cell_of_slot, int *scan_tmp, unsigned *status, cudaStream_t st, int *nl,
                       const KickDrift *kd = nullptr);

// Patch binning: per-patch grids from the patches' largest h (cells per axis capped at ncap), global cell ids,
// then the same counting sort as launch_bin over at most ncells_cap cells.
cudaError_t launch_bin_patches(const uint8_t *aos, int64_t stride, int off_x, int off_h, int n,
                               const int64_t *patch_start, int npatch, const Grid &box, int ncap, int ncells_cap,
                               int *patch_n, double *patch_edge, int *patch_cells, int *patch_cell_base,
                               int *ncells_dev, int *cell_of,
                               int *count, int *cell_start, int *fill, int *perm_tmp, int *perm, int *cell_of_slot,
                               int *scan_tmp, unsigned *status, cudaStream_t st, int *nl,
                               const KickDrift *kd = nullptr);

// Bin with a record pass (see RecordPlan; records 16-byte aligned, stride a multiple of 16): single grids
// (npatch == 0) or patch views (the per-patch grids of launch_bin_patches first).  f32: the view's precision.
// Patch views gather each patch's largest h in the record pass (hmax: npatch words of scratch), build the patch
// grids from them and bin every patch in one CTA from the staged positions (x_off: byte offset of x in a row).
cudaError_t launch_bin_staged(uint8_t *aos, int64_t stride, int n, const RecordPlan &rp, bool f32, const Grid &g,
                              int ncells, const int64_t *patch_start, int npatch, int ncap, int *patch_n,
                              double *patch_edge, int *patch_cells, int *patch_cell_base, int *ncells_dev,
                              unsigned long long *hmax, int x_off, int *cell_of, int *count,
                              int *cell_start, int *fill, int *perm_tmp, int *perm, int *cell_of_slot, int *scan_tmp,
                              unsigned *status, cudaStream_t st, int *nl);
cudaError_t launch_permute(const int *perm, const int *cell_of_slot, int n, const PermutePlan &pp,
                           const CellSpace &cs, bool f32, cudaStream_t st, int *nl);

cudaError_t launch_gather(const uint8_t *aos, int64_t stride, bool vec16, const int *perm,
                          const int *cell_of_slot, int n, const ConvPlan &plan, const CellSpace &cs, bool f32,
                          cudaStream_t st, int *nl);

cudaError_t launch_scatter(uint8_t *aos, int64_t stride, const int *perm, const int *cell_of_slot, int n,
                           const ConvPlan &plan, const CellSpace &cs, bool f32, cudaStream_t st, int *nl);

// Per-particle preparation of the pair loops (FP64 views: float filter copies of x (and h) and coefficient
// tables, and SPH_DEV_MAGNITUDE in *status for an h or rho outside the FP64 loops' band; FP32 force: 1/h,
// 1/(pi h^5), P/rho^2).
cudaError_t launch_density_prep(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_of_slot, int n,
                                const CellSpace &cs, const sph_params &prm, unsigned *status, cudaStream_t st,
                                int *nl);
cudaError_t launch_force_prep(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_of_slot, int n,
                              const CellSpace &cs, const sph_params &prm, unsigned *status, cudaStream_t st,
                              int *nl);

// Pair-kernel launch shape: active particles staged per tile (0 = default of the path), and for patch views the
// largest-first work list the persistent kernel pulls cells from.
struct PairLaunch {
    int tj;
    int threads;              // 128 or 256 threads per CTA (0 = 128)
    const int *work_order;    // patches: cells in descending cost order (nullptr: one CTA per cell)
    const int *work_count;    // patches: number of entries in work_order (device)
    int *work_next;           // patches: work counter (device, zeroed by the launcher)
    int persistent_ctas;      // patches: CTAs of the persistent launch
    const int *skip;          // device flag: when nonzero the pair kernel returns at once (nullptr: never)
};

// The smoothing-length iteration (sph_hiter.cu): one round's update + bookkeeping, and the final status check.
cudaError_t launch_h_update(bool f32, const SoaPtrs &soa, int n, double eta, double tol, double h_limit,
                            unsigned char *done, int *hstate, unsigned *status, cudaStream_t st, int *nl);
cudaError_t launch_h_finish(const int *hstate, unsigned *status, cudaStream_t st, int *nl);

// The pair kernels.
cudaError_t launch_density_pairs(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_start,
                                 int ncells, int n, const CellSpace &cs, const sph_params &prm, const PairLaunch &pl,
                                 unsigned *status, Counters *counters, cudaStream_t st, int *nl);
cudaError_t launch_force_pairs(bool f32, const SoaPtrs &soa, const Scratch &scr, const int *cell_start,
                               int ncells, int n, const CellSpace &cs, const sph_params &prm, const PairLaunch &pl,
                               unsigned *status, Counters *counters, cudaStream_t st, int *nl);

// Largest-first work list over the non-empty cells (cost = local particles x active particles).
cudaError_t launch_work_list(const CellSpace &cs, const int *cell_start, int ncells_cap, int *cell_bucket,
                             int *bucket_count, int *work_order, int *work_count, cudaStream_t st, int *nl);

cudaError_t launch_reduce(bool f32, const SoaPtrs &soa, int n, double *partials, double *out, cudaStream_t st,
                          int *nl);



}  // namespace sphk
