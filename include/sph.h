/*
 * sph.h -- C ABI of libsph: field-selective AoS<->SoA particle views fused with cell-linked-list SPH density and
 * force loops, on one NVIDIA GB300 (sm_103a).
 *
 * The method is the paper's (arXiv 2502.16517) temporary, local "view" over an array of particle structs:
 *   f(D) = (W_Aout o C_SoA^AoS o f^ o C_AoS^SoA o N_{Ain u Aout})(D)          (Section 4, Eq. 5)
 * N narrows a record to the members a loop reads (A_in) or writes (A_out), C_AoS^SoA transposes the narrowed
 * records into one array per member (the "prologue" of Section 3.1), f^ is the loop body over those arrays, and
 * the "epilogue" C_SoA^AoS + W writes back only A_out; every other byte of every record stays as it was
 * (Section 3.2).  Conversions run on the device (the permuted operator order of Eq. 7), so the AoS never leaves
 * HBM on the hot path.  The loop bodies are the SPH density and force kernels of Section 2.1, evaluated per cell
 * over the local particles of the cell and the active particles of its 3^3 vertex-connected neighbour cells
 * (Section 2.3), local-active loop order, masking instead of branching (Section 5.6), no pair symmetry exploited
 * (Section 5.3).
 *
 * General rules for every call:
 *   - Every call taking a view enqueues its work on the view's CUDA stream and returns without waiting, except
 *     sph_view_sync, sph_reduce, sph_pair_counts, sph_step with stats_out != NULL and sph_step_host, which wait
 *     for the stream.
 *   - Device pointers (suffix _dev) must be device memory of the view's GPU.  Host pointers are plain host
 *     memory.  The caller owns every buffer it passes; the view owns the memory it allocated in
 *     sph_view_create and frees it in sph_view_destroy.  No call other than sph_view_create and
 *     sph_step_host's first staged use allocates device memory.
 *   - Arguments are checked on the host first; a bad argument returns SPH_E_INVAL and enqueues nothing.
 *   - Problems found on the device (a position outside the box, the kernel support kappa h larger than a cell, a
 *     non-finite density)
 *     set bits in the view's device status word; the next waiting call returns SPH_E_DEVICE and
 *     sph_view_status reports the bits.  Kernels never trap and never wait without a bound.
 *   - A view is used from one host thread at a time.
 */
#ifndef LIBSPH_SPH_H_
#define LIBSPH_SPH_H_

#include <stdint.h>

#if defined(__GNUC__)
#define SPH_API __attribute__((visibility("default")))
#else
#define SPH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sph_status {
    SPH_OK = 0,
    SPH_E_INVAL = 1,   /* bad argument: null pointer, bad layout or domain, n > n_max, field absent ...     */
    SPH_E_NOMEM = 2,   /* a device or pinned allocation failed (sph_view_create, first sph_step_host)        */
    SPH_E_CUDA = 3,    /* a CUDA runtime call or a kernel launch failed                                      */
    SPH_E_DEVICE = 4,  /* the device status word has error bits set (see SPH_DEV_*)                          */
    SPH_E_TIMEOUT = 5, /* reserved for a bounded device-side wait; no kernel of this library waits, so no call
                          returns it                                                                         */
    SPH_E_NOTCONV = 6, /* an iteration did not converge                                                      */
    SPH_E_STATE = 7    /* call order: e.g. sph_density before the density view was gathered                   */
} sph_status;

typedef enum sph_prec {
    SPH_F64 = 0, /* SoA views and pair loops in FP64                                                       */
    SPH_F32 = 1  /* SoA views in FP32 (positions relative to their cell's origin), FP32 pair loops with
                    Kahan-compensated sums, global sums with FP64 results (see sph_reduce)                  */
} sph_prec;

/* Particle members known to the library, in the order of sph_layout.off[].  x, v, a and curl v are three
 * contiguous doubles; every other member is one double.  All members are IEEE binary64 in the records.
 * SPH_NNB .. SPH_VSIG are the members of the fuller views (SPH_SCHEME_EXTENDED; the neighbour count, the
 * rotational velocity vector and the derivative properties of Section 2.1, Table 1's larger access sets):
 *   SPH_NNB    neighbours within the support, the particle itself excluded (a count, stored as a double);
 *   SPH_DIVV   velocity divergence  -1/rho_i sum_j m_j v_ij . grad_i W(r_ij, h_i);
 *   SPH_CURLV  velocity curl         1/rho_i sum_j m_j v_ij x grad_i W(r_ij, h_i);
 *   SPH_OMEGA  grad-h term           1 + h_i / (3 rho_i) sum_j m_j dW/dh(r_ij, h_i);
 *   SPH_VSIG   signal velocity       max_j (c_i + c_j - 3 min(v_ij . r_ij / r_ij, 0)) over the force pairs. */
enum {
    SPH_X = 0, SPH_V = 1, SPH_A = 2, SPH_MASS = 3, SPH_H = 4, SPH_RHO = 5, SPH_P = 6, SPH_U = 7, SPH_DUDT = 8,
    SPH_CS = 9, SPH_NNB = 10, SPH_DIVV = 11, SPH_CURLV = 12, SPH_OMEGA = 13, SPH_VSIG = 14, SPH_NFIELDS = 15
};
#define SPH_BIT(f) (1u << (f))

/* The access sets A_in / A_out of the two pair loops (Section 3.1; Table 1 lists the paper's larger sets). */
#define SPH_DENSITY_IN (SPH_BIT(SPH_X) | SPH_BIT(SPH_MASS) | SPH_BIT(SPH_H) | SPH_BIT(SPH_U))
#define SPH_DENSITY_OUT (SPH_BIT(SPH_RHO) | SPH_BIT(SPH_P) | SPH_BIT(SPH_CS))
#define SPH_FORCE_IN                                                                                         \
    (SPH_BIT(SPH_X) | SPH_BIT(SPH_V) | SPH_BIT(SPH_MASS) | SPH_BIT(SPH_H) | SPH_BIT(SPH_RHO) | SPH_BIT(SPH_P) | \
     SPH_BIT(SPH_CS))
#define SPH_FORCE_OUT (SPH_BIT(SPH_A) | SPH_BIT(SPH_DUDT))
/* The access sets of the fuller views (SPH_SCHEME_EXTENDED). */
#define SPH_DENSITY_IN_EXT (SPH_DENSITY_IN | SPH_BIT(SPH_V))
#define SPH_DENSITY_OUT_EXT \
    (SPH_DENSITY_OUT | SPH_BIT(SPH_NNB) | SPH_BIT(SPH_DIVV) | SPH_BIT(SPH_CURLV) | SPH_BIT(SPH_OMEGA))
#define SPH_FORCE_IN_EXT (SPH_FORCE_IN | SPH_BIT(SPH_OMEGA) | SPH_BIT(SPH_DIVV) | SPH_BIT(SPH_CURLV))
#define SPH_FORCE_OUT_EXT (SPH_FORCE_OUT | SPH_BIT(SPH_VSIG))
#define SPH_ALL_FIELDS ((1u << SPH_NFIELDS) - 1u)

/* Device status bits (sph_view_status). */
#define SPH_DEV_POS_RANGE 0x1u  /* a position was outside [0, box] or not finite; it was clamped into a cell */
#define SPH_DEV_H_TOO_BIG 0x2u  /* kappa h exceeded the smallest cell edge: the 3^3 stencil may miss pairs */
#define SPH_DEV_NONFINITE 0x4u  /* a density, pressure or sound speed came out non-finite or <= 0           */
#define SPH_DEV_TIMEOUT 0x8u    /* reserved (as SPH_E_TIMEOUT): no kernel of this library waits             */
#define SPH_DEV_NOTCONV 0x10u   /* a smoothing-length iteration inside sph_step left particles unconverged   */
#define SPH_DEV_BOUNDS 0x20u    /* checked build only (compiled with -DSPH_CHECKED): an index read from device
                                   data (cell, slot range, permutation, work list) was out of range; the access
                                   it guarded was skipped */
#define SPH_DEV_MAGNITUDE 0x40u /* FP64 views: a particle with h outside [2^-50, 2^50) or h^2 rho outside
                                   [2^-105, 2^105) in the caller's units.  The FP64 pair loops refine FP32-seeded
                                   reciprocals and square roots of r^2 and (r^2 + eps hbar^2)(rho_i + rho_j),
                                   which must lie in the float range; outside these bounds the results may be
                                   wrong: rescale the units */

/* Record layout: `stride` bytes per record (a multiple of 8, at most 65536); off[f] is the byte offset of
 * member f inside a record (a multiple of 8), or -1 if the record has no such member.  Present members must
 * lie inside the record and must not overlap.  Records are packed back to back: record k starts at byte
 * k * stride of the AoS buffer, which must be 8-byte aligned (16-byte alignment of the buffer and a stride that
 * is a multiple of 16 enable 128-bit loads). */
typedef struct sph_layout {
    int64_t stride;
    int32_t off[SPH_NFIELDS];
} sph_layout;

/* Domain [0, box[0]) x [0, box[1]) x [0, box[2]), cut into ncell[0] x ncell[1] x ncell[2] equal cells.  The
 * cell edge box[d]/ncell[d] must be at least kappa h of every particle (the interaction radius, Section 2.1:
 * 2h for the cubic spline, 5h/2 for the quartic, see sph_params); this is
 * checked on the device (SPH_DEV_H_TOO_BIG).  periodic != 0 wraps every axis (minimum image) and then needs
 * ncell[d] >= 3; periodic == 0 is an open box.  At most 2^27 cells. */
typedef struct sph_domain {
    double box[3];
    int32_t ncell[3];
    int32_t periodic;
} sph_domain;

/* Smoothing kernels, W(r, h) = sigma f(r/h) / h^3 with support kappa h:
 *   SPH_KERNEL_M4  cubic spline (Monaghan & Lattanzio 1985), kappa = 2;
 *   SPH_KERNEL_M5  quartic spline (Monaghan 1985), kappa = 5/2: the paper's kernel (Section 2.1). */
typedef enum sph_kernel { SPH_KERNEL_M4 = 0, SPH_KERNEL_M5 = 1 } sph_kernel;

/* Equation sets of the two loops:
 *   SPH_SCHEME_MINIMAL   density: rho, P, c_s; force: a, du/dt with the Monaghan viscosity;
 *   SPH_SCHEME_EXTENDED  the fuller views of Section 2.1 / Table 1: the density also writes the neighbour count,
 *                        div v, curl v and Omega (access sets SPH_DENSITY_*_EXT); the force uses
 *                        P / (Omega rho^2) (grad-h terms), scales the viscosity by the pair mean of the Balsara
 *                        switch |div v| / (|div v| + |curl v| + 1e-4 c / h), and writes the signal velocity
 *                        (SPH_FORCE_*_EXT). */
typedef enum sph_scheme { SPH_SCHEME_MINIMAL = 0, SPH_SCHEME_EXTENDED = 1 } sph_scheme;

/* Physics constants: ideal gas gamma; Monaghan viscosity alpha, beta, eps (the softening of mu_ij: finite and
 * >= 0, SPH_E_INVAL otherwise); the kernel and the equation set (zero: the cubic spline and the minimal set).  Any kernel or scheme other than (M4, minimal) needs an FP64
 * single-grid view (SPH_E_INVAL otherwise), cell edges of at least kappa h, and, for the extended scheme, the
 * members of its access sets in the layout. */
typedef struct sph_params {
    double gamma;
    double alpha;
    double beta;
    double eps;
    int32_t kernel; /* sph_kernel */
    int32_t scheme; /* sph_scheme */
} sph_params;

typedef struct sph_view_s *sph_view;

/* Create a view for up to n_max particles of the given record layout, on the CUDA device that is current on the
 * calling thread, enqueueing on `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  Allocates
 * the SoA arrays of every member in the layout at precision `prec`, the cell index (perm, cell_start,
 * cell_of_slot) and the status word once, for n_max particles (the paper's allocation-free prologue, Section
 * 6.3).  Errors: SPH_E_INVAL (null out, bad layout/domain, n_max < 0 or > 2^31-1), SPH_E_NOMEM, SPH_E_CUDA. */
SPH_API sph_status sph_view_create(const sph_layout *layout, sph_prec prec, int64_t n_max, const sph_domain *domain,
                           void *cuda_stream, sph_view *out);

/* Batched form: a view over many independent patches (the paper's per-cell kernels batched into one launch,
 * Section 7.5).  Each patch is an open box [0, patch_box) holding its own particles; particles of different
 * patches never interact.  The records of patch p are records patch_start[p] .. patch_start[p+1]-1 of the AoS,
 * positions patch-local.  Every sph_patches_bin gives each patch its own cell grid with edge >= 2 h_max of that
 * patch (Section 2.1's cells at least as wide as the interaction radius), at most ncell_cap cells per axis, and
 * builds a largest-first work list of the non-empty cells for the persistent pair kernels.  Up to npatch_max
 * patches and n_max particles.  The other calls (sph_aos_to_soa, sph_density, sph_force, sph_soa_to_aos,
 * sph_reduce ...) work on a patch view as on any view; sph_bin and sph_step are rejected (use sph_patches_bin /
 * sph_patches_step).  Errors: SPH_E_INVAL (bad layout, box, npatch_max < 1, ncell_cap outside 1..64, more than
 * 2^27 cells of capacity), SPH_E_NOMEM, SPH_E_CUDA. */
SPH_API sph_status sph_patches_create(const sph_layout *layout, sph_prec prec, int64_t n_max, int32_t npatch_max,
                                      const double patch_box[3], int32_t ncell_cap, void *cuda_stream, sph_view *out);

/* Bin the records [0, n) of a patch view; patch_start_dev: npatch + 1 ascending int64 record offsets in device
 * memory (patch_start[0] = 0, patch_start[npatch] = n), read on the device.  Needs x and h in the layout. */
SPH_API sph_status sph_patches_bin(sph_view view, const void *aos_dev, int64_t n, const int64_t *patch_start_dev,
                                   int32_t npatch);

/* sph_step over all patches: one density + force pass (bin, gather, density, force, scatter), and with dt > 0
 * nsteps leapfrog steps after it, as in sph_step.  Every patch is a closed box [0, patch_box] with reflecting
 * walls: a drift that carries a particle past a wall mirrors its position back through the wall and turns that
 * velocity component (a particle that would still be outside, |v dt| > patch_box, is put on the wall).
 * stats_out as in sph_step. */
SPH_API sph_status sph_patches_step(sph_view view, void *aos_dev, int64_t n, const int64_t *patch_start_dev,
                                    int32_t npatch, const sph_params *params, double dt, int32_t nsteps,
                                    double *stats_out);

/* sph_step / sph_patches_step through a CUDA graph.  A call with a new argument set (aos_dev, n, params, dt,
 * nsteps, patch_start_dev, npatch, the integrator flags) runs the step normally, then captures the same launch
 * sequence into a graph; a call repeating the previous argument set replays that graph (one launch for the whole
 * step, kicks and drifts included).  The records'
 * contents may change between calls; the pointers and sizes may not without a new capture.  The view's stream
 * must not be the legacy default stream (SPH_E_INVAL).  Per-phase event timing is not recorded in replays.  Not
 * on patch views (sph_step_graph) / only on patch views (sph_patches_step_graph). */
SPH_API sph_status sph_step_graph(sph_view view, void *aos_dev, int64_t n, const sph_params *params, double dt,
                                  int32_t nsteps);
SPH_API sph_status sph_patches_step_graph(sph_view view, void *aos_dev, int64_t n, const int64_t *patch_start_dev,
                                          int32_t npatch, const sph_params *params, double dt, int32_t nsteps);

/* Leapfrog options of sph_step, sph_patches_step and their graph forms (flags, OR-ed):
 *   SPH_KDK_PREDICT   the density and force after a drift see predicted values, v_half + a dt/2 and
 *                     u_half + du/dt dt/2 with the a, du/dt of the previous force pass; the second kick starts
 *                     again from the half-step v, u in the records, which replaces the predicted values (the
 *                     paper's second kick that resets the predicted values, Section 2.2).  The predicted values
 *                     exist only in the view: the gather computes them, in FP64, from the record's members.  With
 *                     them the energy error is second order in dt; without, the force sees the half-step v, u and
 *                     the error is first order.  On by default.
 *   SPH_KDK_CONTINUE  a call with dt > 0 skips its initial pass and starts the first kick from the a and du/dt
 *                     already in the records (as a previous call left them), so that successive calls continue one
 *                     run: each call is then exactly nsteps steps.  Off by default.
 * Errors: SPH_E_INVAL (unknown flag bits). */
#define SPH_KDK_PREDICT 0x1
#define SPH_KDK_CONTINUE 0x2
SPH_API sph_status sph_view_set_integrator(sph_view view, int32_t flags);

/* Smoothing-length iteration (Section 2.1, step 1: compute the density, decide whether to grow or shrink the
 * interaction radius, recompute, until every particle meets its termination criterion) on the resident density
 * view.  The paper fixes no update rule; the one used is h_i <- eta (m_i / rho_i)^(1/3) (exact at uniform
 * density rho = m / s^3, where it gives h = eta s) with the termination test |h_new - h| < tol h, evaluated in
 * FP64 for both view precisions; a particle that passes keeps that h_new.  Each round recomputes the density at
 * the current h; at most max_iter rounds run, then the density (and P, c_s) of every particle is recomputed at
 * its final h.  The SoA members h, rho, P, c_s hold the result; scatter SPH_BIT(SPH_H) | SPH_DENSITY_OUT to
 * write it into the records.  Rounds after convergence cost one near-empty launch each; nothing inside waits,
 * then the call waits once and reports *rounds (rounds run) and *unconverged (particles not converged after the
 * last round).  The new h must keep kappa h within the view's cell edge (else SPH_E_DEVICE, SPH_DEV_H_TOO_BIG): create
 * the view with room for h to grow.  Grid views only.  Errors: SPH_E_INVAL (eta <= 0, tol not in (0, 1),
 * max_iter not in 1..1000, patch view), SPH_E_STATE (density view not resident), SPH_E_NOTCONV (particles left
 * unconverged; results are still written), SPH_E_DEVICE. */
SPH_API sph_status sph_density_h(sph_view view, const sph_params *params, double eta, double tol, int32_t max_iter,
                                 int32_t *rounds, int64_t *unconverged);

/* Run the smoothing-length iteration in place of the single density pass inside every sph_step pass
 * (max_iter > 0; 0 switches it off, the default).  h is then scattered with the density outputs.  Nothing waits:
 * a pass that leaves particles unconverged sets SPH_DEV_NOTCONV, and sph_view_h_rounds reports the last
 * iteration.  Errors: SPH_E_INVAL (as sph_density_h, max_iter not in 0..1000). */
SPH_API sph_status sph_view_set_h_iteration(sph_view view, double eta, double tol, int32_t max_iter);

/* Rounds run and particles left unconverged by the view's last smoothing-length iteration.  Waits.  Returns
 * SPH_E_NOTCONV if particles were left, SPH_E_DEVICE if other device status bits are set. */
SPH_API sph_status sph_view_h_rounds(sph_view view, int32_t *rounds, int64_t *unconverged);

/* How sph_step / sph_patches_step convert (Section 8, future work: keep the SoA across loops).  on = 1 (the
 * default): one view serves both loops -- one gather brings in every member either loop reads (x, m, h, u, v),
 * the density outputs stay in SoA for the force, and rho, P, c_s, a, du/dt are scattered together after it.
 * on = 0: one view per loop, converted forth and back around each (scatter the density outputs, gather the full
 * force view), as the paper's annotated loops do.  The records end up byte-identical either way.  Errors:
 * SPH_E_INVAL (on not 0 or 1). */
SPH_API sph_status sph_view_set_union(sph_view view, int32_t on);

/* Staged particles per shared-memory tile of the density and force pair loops (multiples of 64; 0 = the
 * defaults).  Larger tiles stage more neighbours per barrier, smaller ones leave room for more CTAs per SM. */
SPH_API sph_status sph_view_set_tiles(sph_view view, int32_t tile_density, int32_t tile_force);

/* Warps per pair CTA ("warps per cell") of the density and force loops: 4 or 8 (0 = the default: 4, except 8
 * for the FP64 force loop).  One CTA works on one
 * cell at a time; 8 warps split the same staged tile among more local particles (or more candidate streams per
 * particle) and keep more warps per SM resident when registers, not shared memory, bound the CTAs per SM. */
SPH_API sph_status sph_view_set_warps(sph_view view, int32_t warps_density, int32_t warps_force);

/* The view's current pair-loop shapes: out = {tile_density, tile_force, warps_density, warps_force} (tiles 0 =
 * the defaults).  For caching the autotuner's choice and restoring it with sph_view_set_tiles /
 * sph_view_set_warps. */
SPH_API sph_status sph_view_get_tuning(sph_view view, int32_t out[4]);

/* Autotuner: runs one pass on the records (as sph_step / sph_patches_step with the last bin's arguments would,
 * leaving the same outputs in the records), then times the density and the force pair loops at each candidate
 * shape -- tile size x warps per cell (4, 8) -- on this data and keeps the fastest of each in the view.  chosen
 * (may be NULL) receives the two tile sizes, best_ms (may be NULL) their kernel times; sph_view_get_tuning
 * reports the warps as well.  Waits.  For a patch view, call sph_patches_bin first. */
SPH_API sph_status sph_autotune(sph_view view, void *aos_dev, int64_t n, const sph_params *params, int32_t chosen[2],
                                float best_ms[2]);

/* Wait for the view's stream, free everything the view allocated.  NULL is accepted. */
SPH_API sph_status sph_view_destroy(sph_view view);

/* Cell bucketing (Section 2.1; chunk lists of Section 5.2): reads the positions of records [0, n) of aos_dev and
 * builds the cell-major slot order: perm[s] = record held by slot s, cell_start[c] (CSR offsets, ncells + 1
 * entries), cell_of_slot[s].  Inside a cell the slots hold ascending record indices, so the order is
 * deterministic.  Invalidates every SoA member previously gathered.  Needs SPH_X in the layout.
 * Errors: SPH_E_INVAL (null view/aos_dev, n < 0 or n > n_max, misaligned aos_dev), SPH_E_CUDA. */
SPH_API sph_status sph_bin(sph_view view, const void *aos_dev, int64_t n);

/* Prologue (Section 3.1, C_AoS^SoA o N of Eq. 5): for every member in in_mask, copy it from the records in slot
 * order (record perm[s] -> SoA slot s).  FP64 views copy the bits; FP32 views store the round-to-nearest cast,
 * positions as (float)(x - k * box/ncell) relative to the origin of the slot's cell k.  n must equal the n of
 * the last sph_bin.  Errors: SPH_E_INVAL (member absent from the layout, mask outside SPH_ALL_FIELDS, n
 * mismatch), SPH_E_STATE (no sph_bin yet), SPH_E_CUDA. */
SPH_API sph_status sph_aos_to_soa(sph_view view, const void *aos_dev, int64_t n, uint32_t in_mask);

/* Density loop (Section 2.1 step 1; local-active order of Section 5.4): for every particle i,
 * rho_i = sum_j m_j W(|r_ij|, h_i) over the 3^3 neighbour cells of i's cell (self term included; the kernel of
 * params, support kappa h), then P_i = (gamma - 1) rho_i u_i and c_s,i = sqrt(gamma P_i / rho_i), written to the
 * SoA members rho, P, cs; with the extended scheme also nnb, divv, curlv and omega (see the member list).  Needs
 * the scheme's density input set resident (SPH_E_STATE otherwise) and its output set in the layout. */
SPH_API sph_status sph_density(sph_view view, const sph_params *params);

/* Force loop (Section 2.1 step 2): for every particle i and every j != i of the 3^3 neighbour cells with
 * |r_ij| < kappa max(h_i, h_j):
 *   a_i     = -sum_j m_j [P_i/rho_i^2 grad W(r_ij,h_i) + P_j/rho_j^2 grad W(r_ij,h_j) + Pi_ij gradbar]
 *   du_i/dt =  sum_j m_j [P_i/rho_i^2 v_ij . grad W(r_ij,h_i) + Pi_ij v_ij . gradbar / 2]
 * with the Monaghan viscosity Pi_ij (alpha, beta, eps of params) for approaching pairs, written to the SoA
 * members a, dudt.  The extended scheme divides each P_k / rho_k^2 by Omega_k, scales Pi_ij by the Balsara pair
 * mean and writes vsig as well.  Needs the scheme's force input set resident (SPH_E_STATE otherwise). */
SPH_API sph_status sph_force(sph_view view, const sph_params *params);

/* Epilogue (Section 3.1, W o C_SoA^AoS of Eq. 5): for every member in out_mask, write SoA slot s back into record
 * perm[s].  Only those members' bytes change; every other byte of every record is left as it was.  FP32 views
 * widen exactly.  The members must be resident.  n must equal the n of the last sph_bin. */
SPH_API sph_status sph_soa_to_aos(sph_view view, void *aos_dev, int64_t n, uint32_t out_mask);

/* One whole pass on device-resident records: bin, gather SPH_DENSITY_IN, density, scatter SPH_DENSITY_OUT, gather
 * SPH_FORCE_IN, force, scatter SPH_FORCE_OUT.  With dt > 0, nsteps leapfrog kick-drift-kick steps follow the
 * pass (Section 2.1 steps 3-5): kick v, u by dt/2; drift x by dt (periodic wrap; an open box reflects at its
 * walls as patches do, see sph_patches_step); rebin; density; force; kick by dt/2.  Kicks and drifts update the
 * records in FP64, for both view precisions, inside the step's bin kernel (first kick, drift) and its last scatter
 * (second kick); sph_view_set_integrator selects predicted values (the default) and continuation.  Leapfrog steps need x, v, a, u and dudt in the layout; afterwards the view's v and u are no
 * longer resident.  If stats_out is not NULL, waits and writes the eight FP64 sums of sph_reduce of the final
 * state. */
SPH_API sph_status sph_step(sph_view view, void *aos_dev, int64_t n, const sph_params *params, double dt, int32_t nsteps,
                    double *stats_out);

/* sph_step on records in HOST memory, then waits.  By default it copies the n records host->device into a
 * staging buffer that the view allocates on first use (n_max records), runs sph_step (dt, nsteps as there) and
 * copies the records back; aos_host should be page-locked for full copy speed.  With sph_view_set_host_direct
 * on, nothing is copied in bulk: the kernels read the view members from the records and write the written
 * members back across the host link, in place (the views of Section 4 applied to host-resident records).  That
 * needs aos_host page-locked and mapped into the device's address space (cudaHostAlloc, cudaHostRegister);
 * other memory returns SPH_E_INVAL before any launch.  In place, repeated calls with the same records and
 * arguments (and stats_out NULL) replay the step as one captured CUDA graph, as sph_step_graph does (a view with
 * the legacy default stream runs it uncaptured).  In both modes aos_host must hold n records. */
SPH_API sph_status sph_step_host(sph_view view, void *aos_host, int64_t n, const sph_params *params, double dt,
                         int32_t nsteps, double *stats_out);

/* How sph_step_host reaches the host records: 0 = staged bulk copies (the default), 1 = in place (see
 * sph_step_host).  Errors: SPH_E_INVAL (on not 0 or 1). */
SPH_API sph_status sph_view_set_host_direct(sph_view view, int32_t on);

/* FP64 global sums over the SoA members, in a fixed order (deterministic): out[0..2] = sum m v,
 * out[3..5] = sum m a, out[6] = sum m (|v|^2/2 + u), out[7] = sum m (v . a + du/dt).  FP64 views sum in FP64;
 * FP32 views sum their float members in double-float arithmetic (exact products, compensated additions), which
 * agrees with FP64 sums of the same float values to ~1e-14 of the sums of absolute terms.  Needs x, v, a, mass,
 * u, dudt resident.  Waits. */
SPH_API sph_status sph_reduce(sph_view view, double out[8]);

/* Wait for the view's stream; SPH_E_DEVICE if the device status word is non-zero. */
SPH_API sph_status sph_view_sync(sph_view view);

/* Wait, then report (and clear if clear != 0) the device status bits SPH_DEV_*. */
SPH_API sph_status sph_view_status(sph_view view, uint32_t *bits, int32_t clear);

/* Device pointer of SoA member `field`, component `comp` (0..2 for x, v, a; 0 otherwise): n_max elements of
 * 8 bytes (SPH_F64) or 4 bytes (SPH_F32), in slot order.  Owned by the view. */
SPH_API sph_status sph_view_soa(sph_view view, int32_t field, int32_t comp, void **dev_ptr);

/* Device pointers of the cell index: which = 0 perm (int32, n_max), 1 cell_start (int32, ncells + 1),
 * 2 cell_of_slot (int32, n_max).  Owned by the view. */
SPH_API sph_status sph_view_index(sph_view view, int32_t which, void **dev_ptr);

/* Copy `count` elements of SoA member `field`/`comp` (slot order) to dst, which may be host or device memory
 * (unified addressing), then wait.  count <= n_max. */
SPH_API sph_status sph_view_export(sph_view view, int32_t field, int32_t comp, void *dst, int64_t count);

/* Copy `count` int32 entries of index array `which` (as in sph_view_index) to dst (host or device), then wait. */
SPH_API sph_status sph_view_export_index(sph_view view, int32_t which, void *dst, int64_t count);

/* n of the last sph_bin and the number of cells. */
SPH_API sph_status sph_view_info(sph_view view, int64_t *n, int64_t *ncells);

/* Waits, then counts[0] = candidate pairs the density loop visited (local x active of every cell),
 * counts[1] = pairs inside the density support (self included), counts[2] = ordered pairs inside the force
 * support (j != i), counts[3] = candidate pairs of the force loop; all since the last reset (reset != 0
 * clears them after reading). */
SPH_API sph_status sph_pair_counts(sph_view view, uint64_t counts[4], int32_t reset);

/* Phases of the path, for sph_view_phase_times. */
enum {
    SPH_PH_BIN = 0,          /* cell bucketing kernels                                                     */
    SPH_PH_GATHER = 1,       /* prologue: AoS -> SoA                                                       */
    SPH_PH_DENSITY_PREP = 2, /* density loop's per-particle preparation                                    */
    SPH_PH_DENSITY = 3,      /* density pair kernel                                                        */
    SPH_PH_SCATTER = 4,      /* epilogue: SoA -> AoS                                                       */
    SPH_PH_FORCE_PREP = 5,   /* force loop's per-particle preparation                                      */
    SPH_PH_FORCE = 6,        /* force pair kernel                                                          */
    SPH_PH_REDUCE = 7,       /* FP64 global sums                                                           */
    SPH_PH_KDK = 8,          /* reserved: the kicks and the drift run inside a step's bin and scatter kernels */
    SPH_NPHASES = 9
};

/* Enable (enable != 0) or disable per-phase device timing: with timing on, every phase brackets its launches
 * with two CUDA events on the view's stream.  Launch counting is always on. */
SPH_API sph_status sph_view_timing(sph_view view, int32_t enable);

/* Waits, then ms[p] = summed device time of phase p (0 where timing was off) and launches[p] = kernels
 * launched by phase p, since the last reset (reset != 0 clears both after reading). */
SPH_API sph_status sph_view_phase_times(sph_view view, double ms[SPH_NPHASES], int64_t launches[SPH_NPHASES],
                                        int32_t reset);

/* Measured fused multiply-add throughput of the current device, in flops/s (an FMA counts 2): prec SPH_F64 or
 * SPH_F32.  Runs 8 independent FMA chains per thread on 8 CTAs of 256 threads per SM, on a private stream, and
 * waits.  This is the arithmetic peak that the pair kernels' pipe fractions are compared with.  The paper has no
 * counterpart; it reports no hardware peaks. */
SPH_API sph_status sph_probe_fma_rate(int32_t prec, double *flops_per_s);

/* Which build of the library is loaded: *checked = 1 for the checked build (compiled with -DSPH_CHECKED: index
 * checks on the device, see SPH_DEV_BOUNDS), else 0.  Errors: SPH_E_INVAL (checked NULL).  The paper has no
 * counterpart; the checked build stands in for a memory checker where none can run. */
SPH_API sph_status sph_build_info(int32_t *checked);

/* Capacity of sph_bin_static's fixed scratch. */
#define SPH_BIN_STATIC_MAX_PARTICLES 262144
#define SPH_BIN_STATIC_MAX_CELLS 65536

/* Cell bucketing that allocates nothing.  The paper has no counterpart: this entry point exists for callers
 * that may not allocate device memory, such as code running inside an allocator or memory-pool callback, a
 * plug-in whose host framework owns all device allocations, or a loop with a strict no-allocation rule.  Those
 * callers cannot create a view, because sph_view_create allocates.
 * It computes what sph_bin computes, for the records [0, n) of aos_dev (positions at layout->off[SPH_X]) in
 * `domain`, into the caller's device arrays:
 *   perm_dev[n]                record held by each slot;
 *   cell_start_dev[ncells + 1] CSR offsets of the cells;
 *   cell_of_slot_dev[n]        cell of each slot.
 * Inside a cell the slots hold ascending record indices.  status_dev, if not NULL, is a device word into which
 * SPH_DEV_POS_RANGE is OR-ed when a position lies outside the box; the caller clears it.
 * Work is enqueued on cuda_stream; the call does not wait.
 * Intermediate arrays live in one fixed device array of 2.5 MB inside the library.  It exists once per GPU that
 * loads the library and stays allocated until the process exits.  No call allocates or frees memory.  All calls
 * on a device share that array, so calls whose work can overlap on the GPU (other streams, other host threads)
 * race on it and must be ordered by the caller.  Each call clears what must start at zero.
 * The first call on a device looks up the array's address with that device current; make that first call
 * before any stream capture.
 * With n = 0 every cell_start entry becomes 0, and aos_dev, perm_dev and cell_of_slot_dev may be NULL.
 * Errors: SPH_E_INVAL for a null pointer, a bad layout or domain, or a size beyond the fixed capacity
 * (n > SPH_BIN_STATIC_MAX_PARTICLES, an axis or a product of axes above SPH_BIN_STATIC_MAX_CELLS cells);
 * SPH_E_CUDA if the address lookup or a launch fails. */
SPH_API sph_status sph_bin_static(const sph_layout *layout, const sph_domain *domain, const void *aos_dev, int64_t n,
                                  int32_t *perm_dev, int32_t *cell_start_dev, int32_t *cell_of_slot_dev,
                                  uint32_t *status_dev, void *cuda_stream);

/* Human-readable name of a status code (static storage). */
SPH_API const char *sph_strerror(sph_status status);

#ifdef __cplusplus
}
#endif

#endif /* LIBSPH_SPH_H_ */
