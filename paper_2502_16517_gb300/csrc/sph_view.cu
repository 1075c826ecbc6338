// sph_view.cu -- host runtime of libsph: the C ABI of include/sph.h.
//
// A view (paper Concept 5, Section 2.4: a logical object over a struct that knows which members are read, which
// are written and how they are stored) is here a runtime object: the record layout (stride + member offsets),
// the precision of its SoA storage, one SoA array per member the layout has, the cell index of the current
// slot order and a host-side mask of which SoA members currently hold valid data ("resident").  All device
// memory is allocated once at creation for n_max particles (the paper's allocation-free prologue, Section
// 6.3); the hot calls only enqueue kernels on the view's stream (asynchronous map/compute/map of Section 6.5,
// here without host copies since the records stay in device memory).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sph_internal.cuh"

using sphk::ConvPlan;
using sphk::Grid;

namespace {

const int kNcomp[SPH_NFIELDS] = {3, 3, 3, 1, 1, 1, 1, 1, 1, 1, 1, 1, 3, 1, 1};

}  // namespace

struct PendingTiming {
    int phase;
    cudaEvent_t e0, e1;
};

struct sph_view_s {
    sph_layout layout;
    sph_prec prec;
    int64_t n_max;
    sph_domain dom;
    cudaStream_t st;
    Grid g;
    sphk::CellSpace cs;
    int ncells;  // single grid: its cells; patch views: capacity
    size_t esz;

    // patch views
    int npatch_max, npatch, ncap;
    const int64_t *patch_start;  // caller's device array of the last sph_patches_bin
    int *patch_n, *patch_cells, *patch_cell_base;
    double *patch_edge;  // 3 npatch_max edges, then 3 npatch_max inverses
    int *cell_bucket, *bucket_count, *work_order, *work_count, *work_next;
    unsigned long long *hmax;  // per patch: the largest h (bit pattern) of the record pass

    int64_t n;
    bool binned;
    uint32_t resident;
    uint32_t present;

    void *arena;
    sphk::SoaPtrs soa;
    uint8_t *stage_rows;  // record-order packed rows of the staged gather (n_max rows of at most stage_row_max B)
    int stage_row_max;
    sphk::Scratch scr;
    int *cell_of, *count, *cell_start, *fill, *perm_tmp, *perm, *cell_of_slot;
    int *scan_tmp;  // multi-CTA scan scratch
    unsigned *status;
    sphk::Counters *counters;
    double *red_partials, *red_out;

    unsigned *h_status;
    double *h_red;
    sphk::Counters *h_counters;

    void *aos_stage;

    // launch counters and optional per-phase event timing
    int64_t launches[SPH_NPHASES];
    double phase_ms[SPH_NPHASES];
    bool timing;
    std::vector<cudaEvent_t> *ev_free;
    std::vector<PendingTiming> *ev_pending;
    int tile_density, tile_force;  // staged particles per tile (0 = default)
    int warps_density, warps_force;  // warps per pair CTA: 4 or 8 (0 = 4)

    // graph-captured step: the arguments it was captured for, the executable graph, its kernel launches
    bool graph_valid;
    void *g_aos;
    int64_t g_n;
    sph_params g_p;
    double g_dt;
    int32_t g_nsteps;
    const int64_t *g_ps;
    int32_t g_npatch;
    cudaGraphExec_t g_exec;
    int64_t g_launches[SPH_NPHASES];
    int persistent_ctas;           // CTAs of the persistent pair launches (patch views; 0 = as many as fit)
    bool union_view;               // one gather per member and one scatter per pass (sph_view_set_union)
    bool host_direct;              // sph_step_host works on the page-locked records in place (sph_view_set_host_direct)
    // smoothing-length iteration
    unsigned char *hdone;          // per slot: converged
    int *hstate;                   // [left this round, all converged, rounds run, left after the last round]
    int *h_hstate;                 // pinned host copy of hstate
    double h_eta, h_tol;
    int h_max_iter;                // 0: sph_step runs one density pass
    int32_t integrator;            // SPH_KDK_* flags of sph_view_set_integrator
    bool staged_bin;               // a pass bins and gathers in one record pass (do_bin_gather) where it can
    int32_t g_integrator;          // the flags the captured graph was captured with
};

namespace {

sph_status cuda_fail(cudaError_t e) { return e == cudaSuccess ? SPH_OK : SPH_E_CUDA; }

// The access sets of the two loops under the equation set of `p` (include/sph.h).
bool extended(const sph_params *p) { return p->scheme == SPH_SCHEME_EXTENDED; }
uint32_t dens_in(const sph_params *p) { return extended(p) ? SPH_DENSITY_IN_EXT : SPH_DENSITY_IN; }
uint32_t dens_out(const sph_params *p) { return extended(p) ? SPH_DENSITY_OUT_EXT : SPH_DENSITY_OUT; }
uint32_t force_in(const sph_params *p) { return extended(p) ? SPH_FORCE_IN_EXT : SPH_FORCE_IN; }
uint32_t force_out(const sph_params *p) { return extended(p) ? SPH_FORCE_OUT_EXT : SPH_FORCE_OUT; }
// Support radius of the kernel in units of h.
double kappa_of(const sph_params *p) { return p->kernel == SPH_KERNEL_M5 ? 2.5 : 2.0; }

bool layout_valid(const sph_layout *L, uint32_t *present)
{
    if (!L) return false;
    if (L->stride <= 0 || (L->stride % 8) != 0 || L->stride > 65536) return false;
    struct Iv {
        int64_t a, b;
    };
    std::vector<Iv> iv;
    uint32_t pres = 0;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        const int32_t off = L->off[f];
        if (off == -1) continue;
        if (off < 0 || (off % 8) != 0) return false;
        const int64_t len = 8 * kNcomp[f];
        if ((int64_t)off + len > L->stride) return false;
        iv.push_back({off, off + len});
        pres |= SPH_BIT(f);
    }
    std::sort(iv.begin(), iv.end(), [](const Iv &x, const Iv &y) { return x.a < y.a; });
    for (size_t k = 1; k < iv.size(); ++k) {
        if (iv[k].a < iv[k - 1].b) return false;
    }
    *present = pres;
    return true;
}

bool domain_valid(const sph_domain *D)
{
    if (!D) return false;
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(D->box[a] > 0.0) || !(D->box[a] < 1e300)) return false;
        if (D->ncell[a] < 1) return false;
        if (D->periodic && D->ncell[a] < 3) return false;
        cells *= D->ncell[a];
        if (cells > (int64_t(1) << 27)) return false;
    }
    return true;
}

Grid make_grid(const sph_domain &D)
{
    Grid g;
    g.periodic = D.periodic ? 1 : 0;
    g.min_edge = 1e308;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = D.ncell[a];
        g.box[a] = D.box[a];
        g.edge[a] = D.box[a] / (double)D.ncell[a];
        g.inv[a] = (double)D.ncell[a] / D.box[a];
        g.edgef[a] = (float)g.edge[a];
        g.min_edge = std::min(g.min_edge, g.edge[a]);
    }
    return g;
}

// The member whose rate predicts member f after a drift (v from a, u from du/dt), or -1.
int pred_source(int f) { return f == SPH_V ? SPH_A : (f == SPH_U ? SPH_DUDT : -1); }

// Build the conversion plan for the members in `mask`.  vec16: items are served from 16-byte chunks.  pred_dt != 0
// (gathers only): v and u are gathered predicted, v + a pred_dt and u + du/dt pred_dt.
void build_plan(const sph_view_s *v, uint32_t mask, bool vec16, ConvPlan *p, double pred_dt = 0.0)
{
    memset(p, 0, sizeof(*p));
    p->status = v->status;
    std::vector<int> chunks;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(mask & SPH_BIT(f))) continue;
        const int src = pred_dt != 0.0 ? pred_source(f) : -1;
        for (int c = 0; c < kNcomp[f]; ++c) {
            const int off = v->layout.off[f] + 8 * c;
            chunks.push_back(vec16 ? (off / 16) * 16 : off);
            if (src >= 0) {
                const int so = v->layout.off[src] + 8 * c;
                chunks.push_back(vec16 ? (so / 16) * 16 : so);
            }
        }
    }
    std::sort(chunks.begin(), chunks.end());
    chunks.erase(std::unique(chunks.begin(), chunks.end()), chunks.end());
    p->nchunks = (int)chunks.size();
    for (size_t k = 0; k < chunks.size(); ++k) p->chunk_off[k] = chunks[k];
    int k = 0;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(mask & SPH_BIT(f))) continue;
        for (int c = 0; c < kNcomp[f]; ++c, ++k) {
            const int off = v->layout.off[f] + 8 * c;
            p->item_off[k] = off;
            const int ch = vec16 ? (off / 16) * 16 : off;
            p->item_chunk[k] = (int)(std::lower_bound(chunks.begin(), chunks.end(), ch) - chunks.begin());
            p->item_sub[k] = vec16 ? (off - ch) / 8 : 0;
            p->item_pos[k] = (f == SPH_X && v->prec == SPH_F32) ? c : -1;
            p->item_pred_chunk[k] = -1;
            const int src = pred_dt != 0.0 ? pred_source(f) : -1;
            if (src >= 0) {
                const int so = v->layout.off[src] + 8 * c;
                const int sch = vec16 ? (so / 16) * 16 : so;
                p->item_pred_chunk[k] = (int)(std::lower_bound(chunks.begin(), chunks.end(), sch) - chunks.begin());
                p->item_pred_sub[k] = vec16 ? (so - sch) / 8 : 0;
            }
            p->soa[k] = v->soa.p[f][c];
        }
    }
    p->nitems = k;
    p->pred_dt = pred_dt;
}

// Bump allocator over one device allocation, 256-byte aligned pieces.
struct Bump {
    size_t off = 0;
    char *base = nullptr;
    void *take(size_t bytes)
    {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return base ? base + o : nullptr;
    }
};

void carve(sph_view_s *v, Bump &b)
{
    const size_t nm = (size_t)std::max<int64_t>(v->n_max, 1);
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        for (int c = 0; c < 3; ++c) v->soa.p[f][c] = nullptr;
        if (!(v->present & SPH_BIT(f))) continue;
        for (int c = 0; c < kNcomp[f]; ++c) v->soa.p[f][c] = b.take(nm * v->esz);
    }
    int comps = 0;
    for (int f = 0; f < SPH_NFIELDS; ++f)
        if (v->present & SPH_BIT(f)) comps += kNcomp[f];
    v->stage_row_max = 8 * comps;
    v->stage_rows = (uint8_t *)b.take(nm * (size_t)v->stage_row_max);
    memset(&v->scr, 0, sizeof(v->scr));
    if (v->prec == SPH_F64) {
        v->scr.xf = (float *)b.take(nm * 4);
        v->scr.yf = (float *)b.take(nm * 4);
        v->scr.zf = (float *)b.take(nm * 4);
        v->scr.hf = (float *)b.take(nm * 4);
    }
    const int nd = v->prec == SPH_F64 ? sphk::kDerivedF64 : sphk::kDerivedF32;
    for (int k = 0; k < nd; ++k) v->scr.d[k] = b.take(nm * v->esz);
    const size_t nc = (size_t)v->ncells;
    v->cell_of = (int *)b.take(nm * 4);
    v->count = (int *)b.take(nc * 4);
    v->cell_start = (int *)b.take((nc + 1) * 4);
    v->fill = (int *)b.take(nc * 4);
    v->perm_tmp = (int *)b.take(nm * 4);
    v->perm = (int *)b.take(nm * 4);
    v->cell_of_slot = (int *)b.take(nm * 4);
    v->scan_tmp = (int *)b.take((size_t)sphk::scan_tmp_ints((int)nc) * 4);
    if (v->npatch_max > 0) {
        const size_t np = (size_t)v->npatch_max;
        v->patch_n = (int *)b.take(3 * np * 4);
        v->patch_cells = (int *)b.take(np * 4);
        v->patch_cell_base = (int *)b.take((np + 1) * 4);
        v->patch_edge = (double *)b.take(6 * np * 8);
        v->cell_bucket = (int *)b.take(nc * 4);
        v->bucket_count = (int *)b.take(64 * 4);
        v->work_order = (int *)b.take(nc * 4);
        v->work_count = (int *)b.take(4);
        v->work_next = (int *)b.take(4);
        v->hmax = (unsigned long long *)b.take(np * 8);
    }
    v->hdone = (unsigned char *)b.take(nm);
    v->hstate = (int *)b.take(4 * sizeof(int));
    v->status = (unsigned *)b.take(sizeof(unsigned));
    v->counters = (sphk::Counters *)b.take(sizeof(sphk::Counters));
    v->red_partials = (double *)b.take(1024 * 8 * sizeof(double));
    v->red_out = (double *)b.take(8 * sizeof(double));
}

bool aos_aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool mask_present(const sph_view_s *v, uint32_t mask)
{
    return (mask & ~SPH_ALL_FIELDS) == 0 && (mask & ~v->present) == 0;
}

cudaEvent_t take_event(sph_view_s *v)
{
    if (!v->ev_free->empty()) {
        cudaEvent_t e = v->ev_free->back();
        v->ev_free->pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Brackets the launches of one phase: counts them, and with timing on records two events around them.
// One phase of the path (SPH_PH_*): its launches are counted, timed with CUDA events when the view's timing is
// on, and enclosed in an NVTX range named after the phase, so that profilers can select a phase's kernels (the
// ranges cost one function-pointer test when no tool is attached).
const char *const kPhaseRange[SPH_NPHASES] = {"sph bin",   "sph gather",     "sph density prep",
                                              "sph density", "sph scatter",  "sph force prep",
                                              "sph force",   "sph reduce",   "sph kdk"};

struct Phase {
    sph_view_s *v;
    int ph;
    cudaEvent_t e0 = nullptr;
    int nl = 0;
    Phase(sph_view_s *view, int phase) : v(view), ph(phase)
    {
        nvtxRangePushA(kPhaseRange[phase]);
        if (v->timing) {
            e0 = take_event(v);
            if (e0) cudaEventRecord(e0, v->st);
        }
    }
    ~Phase()
    {
        nvtxRangePop();
        v->launches[ph] += nl;
        if (e0) {
            cudaEvent_t e1 = take_event(v);
            if (e1) {
                cudaEventRecord(e1, v->st);
                v->ev_pending->push_back({ph, e0, e1});
            } else {
                v->ev_free->push_back(e0);
            }
        }
    }
};

sph_status drain_timings(sph_view_s *v)
{
    if (v->ev_pending->empty()) return SPH_OK;
    if (cudaStreamSynchronize(v->st) != cudaSuccess) return SPH_E_CUDA;
    for (const PendingTiming &p : *v->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) v->phase_ms[p.phase] += ms;
        v->ev_free->push_back(p.e0);
        v->ev_free->push_back(p.e1);
    }
    v->ev_pending->clear();
    return SPH_OK;
}

// kd (may be null): the leapfrog's first kick and drift, fused into the bin kernel.
sph_status do_bin(sph_view_s *v, const void *aos, int64_t n, const sphk::KickDrift *kd = nullptr)
{
    if (v->npatch_max > 0) return SPH_E_INVAL;  // patch views bin with sph_patches_bin
    if (!aos || n < 0 || n > v->n_max || !aos_aligned(aos, 8)) return SPH_E_INVAL;
    if (!(v->present & SPH_BIT(SPH_X))) return SPH_E_INVAL;
    cudaError_t e;
    {
        Phase ph(v, SPH_PH_BIN);
        e = sphk::launch_bin(static_cast<const uint8_t *>(aos), v->layout.stride, v->layout.off[SPH_X], (int)n, v->g,
                             v->ncells, v->cell_of, v->count, v->cell_start, v->fill, v->perm_tmp, v->perm,
                             v->cell_of_slot, v->scan_tmp, v->status, v->st, &ph.nl, kd);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    v->n = n;
    v->binned = true;
    v->resident = 0;
    return SPH_OK;
}

// Warps per CTA of the force loop: the view's choice, else 8 for FP64 (the register-bound FP64 force keeps more
// warps resident with 256-thread CTAs) and 4 for FP32.
int force_warps(const sph_view_s *v) { return v->warps_force ? v->warps_force : (v->prec == SPH_F64 ? 8 : 4); }

sphk::PairLaunch pair_launch(const sph_view_s *v, int tj, int warps)
{
    sphk::PairLaunch pl;
    pl.tj = tj;
    pl.threads = warps == 8 ? 256 : 128;
    pl.work_order = v->npatch_max > 0 ? v->work_order : nullptr;
    pl.work_count = v->work_count;
    pl.work_next = v->work_next;
    pl.persistent_ctas = v->persistent_ctas;
    pl.skip = nullptr;
    return pl;
}

sph_status do_bin_patches(sph_view_s *v, const void *aos, int64_t n, const int64_t *patch_start, int npatch,
                          const sphk::KickDrift *kd = nullptr)
{
    if (v->npatch_max <= 0) return SPH_E_INVAL;  // not a patch view
    if (!aos || !patch_start || n < 0 || n > v->n_max || !aos_aligned(aos, 8)) return SPH_E_INVAL;
    if (!aos_aligned(patch_start, 8) || npatch < 1 || npatch > v->npatch_max) return SPH_E_INVAL;
    if (!(v->present & SPH_BIT(SPH_X)) || !(v->present & SPH_BIT(SPH_H))) return SPH_E_INVAL;
    v->npatch = npatch;
    v->patch_start = patch_start;
    v->cs.npatch = npatch;
    v->cs.patch_cell_base = v->patch_cell_base;
    v->cs.patch_n = v->patch_n;
    v->cs.patch_edge = v->patch_edge;
    v->cs.ncells_dev = v->patch_cell_base + npatch;
    cudaError_t e;
    {
        Phase ph(v, SPH_PH_BIN);
        e = sphk::launch_bin_patches(static_cast<const uint8_t *>(aos), v->layout.stride, v->layout.off[SPH_X],
                                     v->layout.off[SPH_H], (int)n, patch_start, npatch, v->g, v->ncap, v->ncells,
                                     v->patch_n, v->patch_edge, v->patch_cells, v->patch_cell_base,
                                     v->patch_cell_base + npatch, v->cell_of, v->count, v->cell_start, v->fill,
                                     v->perm_tmp, v->perm, v->cell_of_slot, v->scan_tmp, v->status, v->st,
                                     &ph.nl, kd);
        if (e == cudaSuccess)
            e = sphk::launch_work_list(v->cs, v->cell_start, v->ncells, v->cell_bucket, v->bucket_count,
                                       v->work_order, v->work_count, v->st, &ph.nl);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    v->n = n;
    v->binned = true;
    v->resident = 0;
    return SPH_OK;
}

// The bin of a pass fused with its first gather (sphk::launch_bin_staged + launch_permute): one coalesced pass over
// the records in record order bins them (after the leapfrog's first kick and drift when kd is given) and stages
// the members of `mask` (v and u predicted by pred_dt when it is not 0); a permutation moves them to slot order.
// Returns SPH_E_INVAL when the layout does not suit the record pass (16-byte aligned records with at most 12 loaded
// chunks): the caller then bins and gathers separately.
sph_status do_bin_gather(sph_view_s *v, void *aos, int64_t n, uint32_t mask, const sphk::KickDrift *kd,
                         double pred_dt)
{
    if (!aos || n < 0 || n > v->n_max || !mask_present(v, mask | SPH_BIT(SPH_X))) return SPH_E_INVAL;
    if ((v->layout.stride % 16) != 0 || !aos_aligned(aos, 16) || v->layout.stride > 16 * sphk::kMaxChunks)
        return SPH_E_INVAL;
    if (v->npatch_max > 0 && (!v->patch_start || !(v->present & SPH_BIT(SPH_H)))) return SPH_E_INVAL;
    sphk::RecordPlan rp;
    memset(&rp, 0, sizeof(rp));
    // chunks: the staged items (with their prediction sources), the position, the leapfrog's members
    std::vector<int> chunks;
    auto chunk_of = [&](int off) { return (off / 16) * 16; };
    uint32_t need = mask | SPH_BIT(SPH_X);
    if (kd) need |= SPH_BIT(SPH_V) | SPH_BIT(SPH_A) | SPH_BIT(SPH_U) | SPH_BIT(SPH_DUDT);
    if (v->npatch_max > 0) need |= SPH_BIT(SPH_H);
    // the patch bin reads the staged positions: x is staged whatever the mask
    if (v->npatch_max > 0 && !(mask & SPH_BIT(SPH_X))) return SPH_E_INVAL;
    if (pred_dt != 0.0 && (mask & (SPH_BIT(SPH_V) | SPH_BIT(SPH_U)))) need |= SPH_BIT(SPH_A) | SPH_BIT(SPH_DUDT);
    if (!mask_present(v, need)) return SPH_E_INVAL;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(need & SPH_BIT(f))) continue;
        for (int c = 0; c < kNcomp[f]; ++c) chunks.push_back(chunk_of(v->layout.off[f] + 8 * c));
    }
    std::sort(chunks.begin(), chunks.end());
    chunks.erase(std::unique(chunks.begin(), chunks.end()), chunks.end());
    if (chunks.size() > 12) return SPH_E_INVAL;  // shared memory of the record pass: kTile x 12 x 16 B
    auto locate = [&](int off, int *ch, int *sub) {
        const int c0 = chunk_of(off);
        *ch = (int)(std::lower_bound(chunks.begin(), chunks.end(), c0) - chunks.begin());
        *sub = (off - c0) / 8;
    };
    ConvPlan &p = rp.conv;
    p.status = v->status;
    p.nchunks = (int)chunks.size();
    for (size_t k = 0; k < chunks.size(); ++k) p.chunk_off[k] = chunks[k];
    const bool f32 = v->prec == SPH_F32;
    int k = 0;
    sphk::PermutePlan pp;
    memset(&pp, 0, sizeof(pp));
    pp.status = v->status;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(mask & SPH_BIT(f))) continue;
        const int src = pred_dt != 0.0 ? pred_source(f) : -1;
        for (int c = 0; c < kNcomp[f]; ++c, ++k) {
            const int off = v->layout.off[f] + 8 * c;
            p.item_off[k] = off;
            locate(off, &p.item_chunk[k], &p.item_sub[k]);
            p.item_pos[k] = (f == SPH_X && f32) ? c : -1;
            p.item_pred_chunk[k] = -1;
            if (src >= 0) locate(v->layout.off[src] + 8 * c, &p.item_pred_chunk[k], &p.item_pred_sub[k]);
            pp.item_pos[k] = p.item_pos[k];
            pp.dst[k] = v->soa.p[f][c];
        }
    }
    p.nitems = k;
    p.pred_dt = pred_dt;
    pp.nitems = k;
    // the packed row: doubles first (FP64 views: every item; FP32 views: the positions), then floats
    int rb = 0, x_off = -1;
    for (int q = 0; q < k; ++q) {
        if (!f32 || p.item_pos[q] >= 0) {
            rp.row_off[q] = rb;
            if (p.item_off[q] == v->layout.off[SPH_X]) x_off = rb;
            rb += 8;
        }
    }
    for (int q = 0; q < k; ++q) {
        if (f32 && p.item_pos[q] < 0) {
            rp.row_off[q] = rb;
            rb += 4;
        }
    }
    rb = (rb + 7) & ~7;
    if (rb > v->stage_row_max || x_off < 0) return SPH_E_INVAL;
    rp.rows = v->stage_rows;
    rp.row_bytes = rb;
    pp.rows = v->stage_rows;
    pp.row_bytes = rb;
    for (int q = 0; q < k; ++q) pp.row_off[q] = rp.row_off[q];
    for (int d = 0; d < 3; ++d) locate(v->layout.off[SPH_X] + 8 * d, &rp.x_ch[d], &rp.x_sub[d]);
    if (v->npatch_max > 0) locate(v->layout.off[SPH_H], &rp.h_ch, &rp.h_sub);
    if (kd) {
        rp.kd = 1;
        for (int d = 0; d < 3; ++d) {
            locate(v->layout.off[SPH_X] + 8 * d, &rp.kd_ch[d], &rp.kd_sub[d]);
            locate(v->layout.off[SPH_V] + 8 * d, &rp.kd_ch[3 + d], &rp.kd_sub[3 + d]);
            locate(v->layout.off[SPH_A] + 8 * d, &rp.kd_ch[6 + d], &rp.kd_sub[6 + d]);
            rp.kd_off[d] = v->layout.off[SPH_X] + 8 * d;
            rp.kd_off[3 + d] = v->layout.off[SPH_V] + 8 * d;
        }
        locate(v->layout.off[SPH_U], &rp.kd_ch[9], &rp.kd_sub[9]);
        locate(v->layout.off[SPH_DUDT], &rp.kd_ch[10], &rp.kd_sub[10]);
        rp.kd_off[6] = v->layout.off[SPH_U];
        rp.dtk = kd->dtk;
        rp.dt = kd->dt;
        // the pass's prediction is the step's half kick (pred_dt = dt/2 = dtk): the record pass applies it with
        // the kick's own products, and the staged items carry none
        if (pred_dt != 0.0 && pred_dt == kd->dtk) {
            rp.kd_pred = 1;
            for (int k = 0; k < p.nitems; ++k) p.item_pred_chunk[k] = -1;
        }
    }
    const bool patches = v->npatch_max > 0;
    if (patches) {
        v->cs.npatch = v->npatch;
        v->cs.patch_cell_base = v->patch_cell_base;
        v->cs.patch_n = v->patch_n;
        v->cs.patch_edge = v->patch_edge;
        v->cs.ncells_dev = v->patch_cell_base + v->npatch;
    }
    cudaError_t e;
    {
        Phase ph(v, SPH_PH_BIN);
        e = sphk::launch_bin_staged(static_cast<uint8_t *>(aos), v->layout.stride, (int)n, rp, f32, v->g, v->ncells,
                                    patches ? v->patch_start : nullptr, patches ? v->npatch : 0, v->ncap,
                                    v->patch_n, v->patch_edge, v->patch_cells, v->patch_cell_base,
                                    patches ? v->patch_cell_base + v->npatch : nullptr, v->hmax, x_off, v->cell_of,
                                    v->count, v->cell_start, v->fill, v->perm_tmp, v->perm, v->cell_of_slot,
                                    v->scan_tmp, v->status, v->st, &ph.nl);
        if (e == cudaSuccess && patches)
            e = sphk::launch_work_list(v->cs, v->cell_start, v->ncells, v->cell_bucket, v->bucket_count,
                                       v->work_order, v->work_count, v->st, &ph.nl);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    {
        Phase ph(v, SPH_PH_GATHER);
        e = sphk::launch_permute(v->perm, v->cell_of_slot, (int)n, pp, v->cs, f32, v->st, &ph.nl);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    v->n = n;
    v->binned = true;
    v->resident = mask;
    return SPH_OK;
}

// Gather the members of `mask`; pred_dt != 0 gathers v and u predicted by pred_dt (see build_plan).
sph_status do_gather(sph_view_s *v, const void *aos, int64_t n, uint32_t mask, double pred_dt = 0.0)
{
    if (!aos || !aos_aligned(aos, 8) || !mask_present(v, mask)) return SPH_E_INVAL;
    if (!v->binned) return SPH_E_STATE;
    if (n != v->n) return SPH_E_INVAL;
    const bool vec16 = (v->layout.stride % 16) == 0 && aos_aligned(aos, 16) && v->layout.stride <= 16 * sphk::kMaxChunks;
    ConvPlan plan;
    build_plan(v, mask, vec16, &plan, pred_dt);
    cudaError_t e;
    {
        Phase ph(v, SPH_PH_GATHER);
        e = sphk::launch_gather(static_cast<const uint8_t *>(aos), v->layout.stride, vec16, v->perm, v->cell_of_slot,
                                (int)n, plan, v->cs, v->prec == SPH_F32, v->st, &ph.nl);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    v->resident |= mask;
    return SPH_OK;
}

// Scatter the members of `mask`; kick_dt != 0 (the mask holds a and du/dt) also kicks the records' v and u by
// kick_dt times the a, du/dt written (the leapfrog's second kick, fused into the epilogue).
sph_status do_scatter(sph_view_s *v, void *aos, int64_t n, uint32_t mask, double kick_dt = 0.0)
{
    if (!aos || !aos_aligned(aos, 8) || !mask_present(v, mask)) return SPH_E_INVAL;
    if (!v->binned) return SPH_E_STATE;
    if (n != v->n) return SPH_E_INVAL;
    if ((mask & ~v->resident) != 0) return SPH_E_STATE;
    ConvPlan plan;
    build_plan(v, mask, false, &plan);
    if (kick_dt != 0.0) {
        const uint32_t need = SPH_BIT(SPH_A) | SPH_BIT(SPH_DUDT);
        if ((mask & need) != need || !mask_present(v, SPH_BIT(SPH_V) | SPH_BIT(SPH_U))) return SPH_E_INVAL;
        // items are listed member by member in member order: find a's three components and du/dt
        int k = 0, ka = -1, kdu = -1;
        for (int f = 0; f < SPH_NFIELDS; ++f) {
            if (!(mask & SPH_BIT(f))) continue;
            if (f == SPH_A) ka = k;
            if (f == SPH_DUDT) kdu = k;
            k += kNcomp[f];
        }
        plan.kick_dt = kick_dt;
        for (int c = 0; c < 3; ++c) {
            plan.kick_item[c] = ka + c;
            plan.kick_off[c] = v->layout.off[SPH_V] + 8 * c;
        }
        plan.kick_item[3] = kdu;
        plan.kick_off[3] = v->layout.off[SPH_U];
    }
    cudaError_t e;
    {
        Phase ph(v, SPH_PH_SCATTER);
        e = sphk::launch_scatter(static_cast<uint8_t *>(aos), v->layout.stride, v->perm, v->cell_of_slot, (int)n,
                                 plan, v->cs, v->prec == SPH_F32, v->st, &ph.nl);
    }
    return cuda_fail(e);
}

// One density pass; with `skip` (a device flag) every pair CTA returns at once while the flag is set.
sph_status density_launch(sph_view_s *v, const sph_params *p, const int *skip)
{
    const bool f32 = v->prec == SPH_F32;
    cudaError_t e;
    {
        Phase ph(v, SPH_PH_DENSITY_PREP);
        e = sphk::launch_density_prep(f32, v->soa, v->scr, v->cell_of_slot, (int)v->n, v->cs, *p, v->status, v->st,
                                      &ph.nl);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    {
        Phase ph(v, SPH_PH_DENSITY);
        sphk::PairLaunch pl = pair_launch(v, v->tile_density, v->warps_density);
        pl.skip = skip;
        e = sphk::launch_density_pairs(f32, v->soa, v->scr, v->cell_start, v->ncells, (int)v->n, v->cs, *p, pl,
                                       v->status, v->counters, v->st, &ph.nl);
    }
    return cuda_fail(e);
}

// The kernel and equation set of `p`: anything but (cubic, minimal) needs an FP64 single-grid view.
sph_status check_scheme(const sph_view_s *v, const sph_params *p)
{
    if (!p) return SPH_E_INVAL;
    if (!(p->eps >= 0.0) || !(p->eps < 1e300)) return SPH_E_INVAL;  // the softening must be finite and >= 0
    if (p->kernel != SPH_KERNEL_M4 && p->kernel != SPH_KERNEL_M5) return SPH_E_INVAL;
    if (p->scheme != SPH_SCHEME_MINIMAL && p->scheme != SPH_SCHEME_EXTENDED) return SPH_E_INVAL;
    if ((p->kernel != SPH_KERNEL_M4 || p->scheme != SPH_SCHEME_MINIMAL) && (v->prec != SPH_F64 || v->npatch_max > 0))
        return SPH_E_INVAL;
    return SPH_OK;
}

sph_status do_density(sph_view_s *v, const sph_params *p)
{
    sph_status s = check_scheme(v, p);
    if (s != SPH_OK) return s;
    if (!mask_present(v, dens_out(p))) return SPH_E_INVAL;
    if (!v->binned || (v->resident & dens_in(p)) != dens_in(p)) return SPH_E_STATE;
    s = density_launch(v, p, nullptr);
    if (s != SPH_OK) return s;
    v->resident |= dens_out(p);
    return SPH_OK;
}

// Smoothing-length iteration (Section 2.1, step 1) on the resident density view: max_iter rounds of density +
// FP64 update / termination test, rounds after convergence returning at once on the device, then the density
// of every particle at its final h.  Nothing waits.  With flag_status, particles left unconverged set
// SPH_DEV_NOTCONV in the status word.
sph_status do_density_h(sph_view_s *v, const sph_params *p, double eta, double tol, int max_iter, bool flag_status)
{
    if (!p || !(eta > 0.0) || !(eta < 1e6) || !(tol > 0.0) || !(tol < 1.0) || max_iter < 1 || max_iter > 1000)
        return SPH_E_INVAL;
    if (v->npatch_max > 0) return SPH_E_INVAL;  // patch grids are sized once per bin from the patch's h
    if (check_scheme(v, p) != SPH_OK) return SPH_E_INVAL;
    if (!mask_present(v, dens_out(p))) return SPH_E_INVAL;
    if (!v->binned || (v->resident & dens_in(p)) != dens_in(p)) return SPH_E_STATE;
    const int n = (int)v->n;
    cudaError_t e = cudaMemsetAsync(v->hdone, 0, (size_t)std::max(n, 1), v->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->hstate, 0, 4 * sizeof(int), v->st);
    if (e != cudaSuccess) return SPH_E_CUDA;
    for (int r = 0; r < max_iter; ++r) {
        sph_status s = density_launch(v, p, v->hstate + 1);
        if (s != SPH_OK) return s;
        Phase ph(v, SPH_PH_DENSITY);
        e = sphk::launch_h_update(v->prec == SPH_F32, v->soa, n, eta, tol, v->g.min_edge / kappa_of(p), v->hdone,
                                  v->hstate, v->status, v->st, &ph.nl);
        if (e != cudaSuccess) return SPH_E_CUDA;
    }
    sph_status s = density_launch(v, p, nullptr);
    if (s != SPH_OK) return s;
    if (flag_status) {
        Phase ph(v, SPH_PH_DENSITY);
        if (sphk::launch_h_finish(v->hstate, v->status, v->st, &ph.nl) != cudaSuccess) return SPH_E_CUDA;
    }
    v->resident |= dens_out(p);
    return SPH_OK;
}

sph_status do_force(sph_view_s *v, const sph_params *p)
{
    if (check_scheme(v, p) != SPH_OK) return SPH_E_INVAL;
    if (!mask_present(v, force_out(p))) return SPH_E_INVAL;
    if (!v->binned || (v->resident & force_in(p)) != force_in(p)) return SPH_E_STATE;
    const bool f32 = v->prec == SPH_F32;
    cudaError_t e;
    {
        Phase ph(v, SPH_PH_FORCE_PREP);
        e = sphk::launch_force_prep(f32, v->soa, v->scr, v->cell_of_slot, (int)v->n, v->cs, *p, v->status, v->st,
                                    &ph.nl);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    {
        Phase ph(v, SPH_PH_FORCE);
        e = sphk::launch_force_pairs(f32, v->soa, v->scr, v->cell_start, v->ncells, (int)v->n, v->cs, *p,
                                     pair_launch(v, v->tile_force, force_warps(v)), v->status, v->counters, v->st,
                                     &ph.nl);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    v->resident |= force_out(p);
    return SPH_OK;
}

// One density + force pass on the records.  With dt > 0 the pass is one leapfrog step (Section 2.1 steps 3-5):
// the bin kernel first kicks v, u by dt/2 and drifts x by dt, the view gathers v and u predicted by pred_dt with
// the records' a and du/dt (the leapfrog's predicted values, when pred_dt != 0; the records keep theirs), and the
// last scatter kicks the records' v, u by dt/2 with the new a, du/dt.
sph_status do_pass(sph_view_s *v, void *aos, int64_t n, const sph_params *p, double dt = 0.0, double pred_dt = 0.0)
{
    sph_status s = check_scheme(v, p);
    if (s != SPH_OK) return s;
    if (!mask_present(v, dens_out(p) | force_out(p))) return SPH_E_INVAL;
    sphk::KickDrift kd;
    const sphk::KickDrift *kdp = nullptr;
    if (dt > 0.0) {
        kd.aos = static_cast<uint8_t *>(aos);
        kd.off_v = v->layout.off[SPH_V];
        kd.off_a = v->layout.off[SPH_A];
        kd.off_u = v->layout.off[SPH_U];
        kd.off_du = v->layout.off[SPH_DUDT];
        kd.dtk = 0.5 * dt;
        kd.dt = dt;
        kdp = &kd;
    }
    const double kick_dt = 0.5 * dt;
    // union view: one gather of every member either loop reads (each record is read once: its bytes arrive in
    // whole memory sectors, so a second pass for the force's extra member v would read the records again)
    const uint32_t first = v->union_view ? ((dens_in(p) | force_in(p)) & ~dens_out(p)) : dens_in(p);
    // the bin and the first gather in one record pass where the layout allows, else one after the other
    if (v->staged_bin && do_bin_gather(v, aos, n, first, kdp, pred_dt) == SPH_OK) {
        // staged
    } else {
        if (v->npatch_max > 0) {
            if ((s = do_bin_patches(v, aos, n, v->patch_start, v->npatch, kdp)) != SPH_OK) return s;
        } else if ((s = do_bin(v, aos, n, kdp)) != SPH_OK) {
            return s;
        }
        if ((s = do_gather(v, aos, n, first, pred_dt)) != SPH_OK) return s;
    }
    uint32_t d_out = dens_out(p);
    if (v->h_max_iter > 0) {
        if ((s = do_density_h(v, p, v->h_eta, v->h_tol, v->h_max_iter, true)) != SPH_OK) return s;
        d_out |= SPH_BIT(SPH_H);  // the iteration writes h as well
    } else if ((s = do_density(v, p)) != SPH_OK) {
        return s;
    }
    if (!v->union_view) {
        // one view per loop, converted forth and back around each (the paper's prologue / epilogue per loop)
        if ((s = do_scatter(v, aos, n, d_out)) != SPH_OK) return s;
        if ((s = do_gather(v, aos, n, force_in(p), pred_dt)) != SPH_OK) return s;
        if ((s = do_force(v, p)) != SPH_OK) return s;
        return do_scatter(v, aos, n, force_out(p), kick_dt);
    }
    // union view: the force reads its members and the density outputs where they are, in SoA, and every written
    // member is scattered once at the end
    const uint32_t more = force_in(p) & ~v->resident;
    if (more && (s = do_gather(v, aos, n, more, pred_dt)) != SPH_OK) return s;
    if ((s = do_force(v, p)) != SPH_OK) return s;
    return do_scatter(v, aos, n, d_out | force_out(p), kick_dt);
}

sph_status do_reduce(sph_view_s *v, double *out)
{
    const uint32_t need = SPH_BIT(SPH_V) | SPH_BIT(SPH_A) | SPH_BIT(SPH_MASS) | SPH_BIT(SPH_U) | SPH_BIT(SPH_DUDT);
    if (!out) return SPH_E_INVAL;
    if (!v->binned || (v->resident & need) != need) return SPH_E_STATE;
    cudaError_t e;
    {
        Phase ph(v, SPH_PH_REDUCE);
        e = sphk::launch_reduce(v->prec == SPH_F32, v->soa, (int)v->n, v->red_partials, v->red_out, v->st, &ph.nl);
    }
    if (e != cudaSuccess) return SPH_E_CUDA;
    e = cudaMemcpyAsync(v->h_red, v->red_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, v->st);
    if (e != cudaSuccess) return SPH_E_CUDA;
    e = cudaStreamSynchronize(v->st);
    if (e != cudaSuccess) return SPH_E_CUDA;
    memcpy(out, v->h_red, 8 * sizeof(double));
    return SPH_OK;
}

sph_status read_status(sph_view_s *v, uint32_t *bits, bool clear)
{
    cudaError_t e = cudaMemcpyAsync(v->h_status, v->status, sizeof(unsigned), cudaMemcpyDeviceToHost, v->st);
    if (e != cudaSuccess) return SPH_E_CUDA;
    if (clear) {
        e = cudaMemsetAsync(v->status, 0, sizeof(unsigned), v->st);
        if (e != cudaSuccess) return SPH_E_CUDA;
    }
    e = cudaStreamSynchronize(v->st);
    if (e != cudaSuccess) return SPH_E_CUDA;
    *bits = *v->h_status;
    return SPH_OK;
}

// sph_step: a pass (unless SPH_KDK_CONTINUE), then nsteps leapfrog steps (Section 2.1 steps 3-5), each one pass
// that kicks by dt/2, drifts by dt, re-bins, gathers (with the predicted v, u under SPH_KDK_PREDICT), computes the
// density and the force, scatters and kicks by dt/2.  Kicks and drift act on the records in FP64, inside the
// pass's bin and last scatter kernels.
sph_status do_step(sph_view_s *v, void *aos, int64_t n, const sph_params *p, double dt, int32_t nsteps,
                   double *stats_out)
{
    if (!p || !aos || nsteps < 0 || !(dt >= 0.0) || !(dt < 1e300)) return SPH_E_INVAL;
    const bool kdk = dt > 0.0 && nsteps > 0;
    const uint32_t need = SPH_BIT(SPH_X) | SPH_BIT(SPH_V) | SPH_BIT(SPH_A) | SPH_BIT(SPH_U) | SPH_BIT(SPH_DUDT);
    if (kdk && !mask_present(v, need)) return SPH_E_INVAL;
    const bool cont = kdk && (v->integrator & SPH_KDK_CONTINUE);
    const double pred_dt = (v->integrator & SPH_KDK_PREDICT) ? 0.5 * dt : 0.0;
    sph_status s;
    if (!cont && (s = do_pass(v, aos, n, p)) != SPH_OK) return s;
    for (int32_t k = 0; kdk && k < nsteps; ++k) {
        if ((s = do_pass(v, aos, n, p, dt, pred_dt)) != SPH_OK) return s;
    }
    if (kdk) {
        // the view's v and u are the predicted (or half-step) values: stale against the kicked records
        v->resident &= ~(SPH_BIT(SPH_V) | SPH_BIT(SPH_U));
        if (stats_out && (s = do_gather(v, aos, n, SPH_BIT(SPH_V) | SPH_BIT(SPH_U))) != SPH_OK) return s;
    }
    if (stats_out) return do_reduce(v, stats_out);
    return SPH_OK;
}

void graph_drop(sph_view_s *v)
{
    if (v->graph_valid && v->g_exec) cudaGraphExecDestroy(v->g_exec);
    v->g_exec = nullptr;
    v->graph_valid = false;
}

// One step through a CUDA graph: on a new argument set, run the step normally (this call's result), then capture
// the same sequence into a graph; on a repeated argument set, replay the graph.  The host-side view state after a
// replay is the state the captured run left.
sph_status do_step_graph(sph_view_s *v, void *aos, int64_t n, const sph_params *p, double dt, int32_t nsteps)
{
    if (!p || !aos) return SPH_E_INVAL;
    if (v->st == nullptr) return SPH_E_INVAL;  // the legacy default stream cannot be captured
    const bool same = v->graph_valid && v->g_aos == aos && v->g_n == n && memcmp(&v->g_p, p, sizeof(*p)) == 0 &&
                      v->g_dt == dt && v->g_nsteps == nsteps && v->g_ps == v->patch_start &&
                      v->g_npatch == v->npatch && v->g_integrator == v->integrator;
    if (same) {
        if (cudaGraphLaunch(v->g_exec, v->st) != cudaSuccess) return SPH_E_CUDA;
        for (int k = 0; k < SPH_NPHASES; ++k) v->launches[k] += v->g_launches[k];
        return SPH_OK;
    }
    graph_drop(v);
    sph_status s = do_step(v, aos, n, p, dt, nsteps, nullptr);  // this call's step, uncaptured
    if (s != SPH_OK) return s;
    const bool timing = v->timing;
    v->timing = false;  // no event nodes in the graph
    int64_t before[SPH_NPHASES];
    memcpy(before, v->launches, sizeof(before));
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(v->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        v->timing = timing;
        return SPH_E_CUDA;
    }
    s = do_step(v, aos, n, p, dt, nsteps, nullptr);
    const cudaError_t ec = cudaStreamEndCapture(v->st, &graph);
    v->timing = timing;
    for (int k = 0; k < SPH_NPHASES; ++k) {
        v->g_launches[k] = v->launches[k] - before[k];
        v->launches[k] = before[k];  // captured, not executed
    }
    if (s != SPH_OK || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        return s != SPH_OK ? s : SPH_E_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&v->g_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        v->g_exec = nullptr;
        return SPH_E_CUDA;
    }
    v->graph_valid = true;
    v->g_aos = aos;
    v->g_n = n;
    v->g_p = *p;
    v->g_dt = dt;
    v->g_nsteps = nsteps;
    v->g_ps = v->patch_start;
    v->g_npatch = v->npatch;
    v->g_integrator = v->integrator;
    return SPH_OK;
}

// Median-free minimum of a few timed repetitions of one pair loop at one tile size.
float time_loop(sph_view_s *v, const sph_params *p, bool force, int tj, int warps, int reps, cudaEvent_t e0,
                cudaEvent_t e1)
{
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        if (force) {
            v->tile_force = tj;
            v->warps_force = warps;
        } else {
            v->tile_density = tj;
            v->warps_density = warps;
        }
        cudaEventRecord(e0, v->st);
        const sph_status s = force ? do_force(v, p) : do_density(v, p);
        cudaEventRecord(e1, v->st);
        if (s != SPH_OK || cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;  // the first repetition warms up
    }
    return best;
}

}  // namespace

extern "C" {

sph_status sph_step_graph(sph_view v, void *aos_dev, int64_t n, const sph_params *params, double dt, int32_t nsteps)
{
    if (!v || v->npatch_max > 0) return SPH_E_INVAL;
    return do_step_graph(v, aos_dev, n, params, dt, nsteps);
}

sph_status sph_patches_step_graph(sph_view v, void *aos_dev, int64_t n, const int64_t *patch_start_dev,
                                  int32_t npatch, const sph_params *params, double dt, int32_t nsteps)
{
    if (!v || v->npatch_max <= 0 || !patch_start_dev || npatch < 1 || npatch > v->npatch_max) return SPH_E_INVAL;
    v->patch_start = patch_start_dev;
    v->npatch = npatch;
    return do_step_graph(v, aos_dev, n, params, dt, nsteps);
}

sph_status sph_view_set_integrator(sph_view v, int32_t flags)
{
    if (!v || (flags & ~(SPH_KDK_PREDICT | SPH_KDK_CONTINUE)) != 0) return SPH_E_INVAL;
    v->integrator = flags;
    return SPH_OK;
}

sph_status sph_density_h(sph_view v, const sph_params *params, double eta, double tol, int32_t max_iter,
                         int32_t *rounds, int64_t *unconverged)
{
    if (!v) return SPH_E_INVAL;
    sph_status s = do_density_h(v, params, eta, tol, max_iter, false);
    if (s != SPH_OK) return s;
    return sph_view_h_rounds(v, rounds, unconverged);
}

sph_status sph_view_h_rounds(sph_view v, int32_t *rounds, int64_t *unconverged)
{
    if (!v) return SPH_E_INVAL;
    if (cudaMemcpyAsync(v->h_hstate, v->hstate, 4 * sizeof(int), cudaMemcpyDeviceToHost, v->st) != cudaSuccess)
        return SPH_E_CUDA;
    uint32_t bits = 0;
    sph_status s = read_status(v, &bits, false);  // waits
    if (s != SPH_OK) return s;
    if (rounds) *rounds = v->h_hstate[2];
    if (unconverged) *unconverged = v->h_hstate[3];
    if (bits & ~SPH_DEV_NOTCONV) return SPH_E_DEVICE;
    return v->h_hstate[3] > 0 ? SPH_E_NOTCONV : SPH_OK;
}

sph_status sph_view_set_h_iteration(sph_view v, double eta, double tol, int32_t max_iter)
{
    if (!v || max_iter < 0 || max_iter > 1000) return SPH_E_INVAL;
    if (max_iter > 0 && (!(eta > 0.0) || !(eta < 1e6) || !(tol > 0.0) || !(tol < 1.0) || v->npatch_max > 0))
        return SPH_E_INVAL;
    v->h_eta = eta;
    v->h_tol = tol;
    v->h_max_iter = max_iter;
    graph_drop(v);
    return SPH_OK;
}

sph_status sph_view_set_warps(sph_view v, int32_t warps_density, int32_t warps_force)
{
    const auto ok = [](int32_t w) { return w == 0 || w == 4 || w == 8; };
    if (!v || !ok(warps_density) || !ok(warps_force)) return SPH_E_INVAL;
    v->warps_density = warps_density;
    v->warps_force = warps_force;
    graph_drop(v);
    return SPH_OK;
}

sph_status sph_view_get_tuning(sph_view v, int32_t out[4])
{
    if (!v || !out) return SPH_E_INVAL;
    out[0] = v->tile_density;
    out[1] = v->tile_force;
    out[2] = v->warps_density == 8 ? 8 : 4;
    out[3] = force_warps(v);
    return SPH_OK;
}

sph_status sph_view_set_union(sph_view v, int32_t on)
{
    if (!v || (on != 0 && on != 1)) return SPH_E_INVAL;
    v->union_view = on != 0;
    graph_drop(v);
    return SPH_OK;
}

sph_status sph_view_set_host_direct(sph_view v, int32_t on)
{
    if (!v || (on != 0 && on != 1)) return SPH_E_INVAL;
    v->host_direct = on != 0;
    return SPH_OK;
}

sph_status sph_view_set_tiles(sph_view v, int32_t tile_density, int32_t tile_force)
{
    if (!v || tile_density < 0 || tile_force < 0 || tile_density > 4096 || tile_force > 4096) return SPH_E_INVAL;
    if (tile_density % 64 != 0 || tile_force % 64 != 0) return SPH_E_INVAL;
    const size_t esz = v->esz;
    // shared memory per staged particle of each loop (FP64: 48 / 140 bytes, FP32: 16 / 56 bytes)
    const size_t dens_b = esz == 8 ? 48 : 16, force_b = esz == 8 ? 140 : 56;
    if (tile_density * dens_b > 200 * 1024 || tile_force * force_b > 200 * 1024) return SPH_E_INVAL;
    v->tile_density = tile_density;
    v->tile_force = tile_force;
    graph_drop(v);
    return SPH_OK;
}

sph_status sph_autotune(sph_view v, void *aos_dev, int64_t n, const sph_params *params, int32_t chosen[2],
                        float best_ms[2])
{
    if (!v || !params || !aos_dev) return SPH_E_INVAL;
    // a full pass first: every member the loops read becomes resident (the records get this pass's outputs)
    sph_status s = do_pass(v, aos_dev, n, params);
    if (s != SPH_OK) return s;
    static const int cand_d64[] = {256, 384, 448, 512, 768, 1024, 1536};
    static const int cand_f64[] = {128, 192, 256, 384, 448, 512, 768};
    static const int cand_d32[] = {256, 512, 1024, 2048, 4096};
    static const int cand_f32[] = {256, 384, 512, 1024, 2048};
    const bool f32 = v->prec == SPH_F32;
    const int *cd = f32 ? cand_d32 : cand_d64;
    const int *cf = f32 ? cand_f32 : cand_f64;
    const int nd = f32 ? 5 : 7, nf = f32 ? 5 : 7;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool timing = v->timing;
    v->timing = false;
    // tile size x warps per cell, each loop on its own
    int bd = 0, bf = 0, wd = 4, wf = 4;
    float td = 1e30f, tf = 1e30f;
    for (int w = 4; w <= 8; w += 4) {
        for (int k = 0; k < nd; ++k) {
            const float t = time_loop(v, params, false, cd[k], w, 4, e0, e1);
            if (t < td) {
                td = t;
                bd = cd[k];
                wd = w;
            }
        }
    }
    v->tile_density = bd;
    v->warps_density = wd;
    for (int w = 4; w <= 8; w += 4) {
        for (int k = 0; k < nf; ++k) {
            const float t = time_loop(v, params, true, cf[k], w, 4, e0, e1);
            if (t < tf) {
                tf = t;
                bf = cf[k];
                wf = w;
            }
        }
    }
    v->tile_force = bf;
    v->warps_force = wf;
    v->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    graph_drop(v);
    if (bd == 0 || bf == 0) return SPH_E_CUDA;
    // leave the records as one pass leaves them: the timed loops rewrote only SoA members, so scatter them again
    if ((s = do_scatter(v, aos_dev, n, dens_out(params) | force_out(params))) != SPH_OK) return s;
    if (chosen) {
        chosen[0] = bd;
        chosen[1] = bf;
    }
    if (best_ms) {
        best_ms[0] = td;
        best_ms[1] = tf;
    }
    return sph_view_sync(v);
}

sph_status sph_view_create(const sph_layout *layout, sph_prec prec, int64_t n_max, const sph_domain *domain,
                           void *cuda_stream, sph_view *out)
{
    if (!out) return SPH_E_INVAL;
    *out = nullptr;
    uint32_t present = 0;
    if (!layout_valid(layout, &present) || !domain_valid(domain)) return SPH_E_INVAL;
    if (prec != SPH_F64 && prec != SPH_F32) return SPH_E_INVAL;
    if (n_max < 0 || n_max > 0x7fffffffLL) return SPH_E_INVAL;
    sph_view_s *v = new (std::nothrow) sph_view_s;
    if (!v) return SPH_E_NOMEM;
    memset(v, 0, sizeof(*v));
    v->layout = *layout;
    v->prec = prec;
    v->n_max = n_max;
    v->dom = *domain;
    v->st = static_cast<cudaStream_t>(cuda_stream);
    v->g = make_grid(*domain);
    v->cs.g = v->g;
    v->cs.npatch = 0;
    v->ncells = domain->ncell[0] * domain->ncell[1] * domain->ncell[2];
    v->esz = prec == SPH_F64 ? 8 : 4;
    v->present = present;
    v->union_view = true;
    v->host_direct = false;
    v->h_max_iter = 0;
    v->integrator = SPH_KDK_PREDICT;
    v->staged_bin = true;
    v->h_eta = 1.2;
    v->h_tol = 1e-6;
    v->ev_free = new (std::nothrow) std::vector<cudaEvent_t>();
    v->ev_pending = new (std::nothrow) std::vector<PendingTiming>();
    if (!v->ev_free || !v->ev_pending) {
        delete v->ev_free;
        delete v->ev_pending;
        delete v;
        return SPH_E_NOMEM;
    }
    Bump sizing;
    carve(v, sizing);
    if (cudaMalloc(&v->arena, sizing.off) != cudaSuccess) {
        v->arena = nullptr;
        sph_view_destroy(v);
        return SPH_E_NOMEM;
    }
    Bump real;
    real.base = static_cast<char *>(v->arena);
    carve(v, real);
    if (cudaMallocHost(&v->h_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&v->h_red, 8 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&v->h_counters, sizeof(sphk::Counters)) != cudaSuccess ||
        cudaMallocHost(&v->h_hstate, 4 * sizeof(int)) != cudaSuccess) {
        sph_view_destroy(v);
        return SPH_E_NOMEM;
    }
    if (cudaMemsetAsync(v->status, 0, sizeof(unsigned), v->st) != cudaSuccess ||
        cudaMemsetAsync(v->counters, 0, sizeof(sphk::Counters), v->st) != cudaSuccess ||
        cudaStreamSynchronize(v->st) != cudaSuccess) {
        sph_view_destroy(v);
        return SPH_E_CUDA;
    }
    *out = v;
    return SPH_OK;
}

sph_status sph_patches_create(const sph_layout *layout, sph_prec prec, int64_t n_max, int32_t npatch_max,
                              const double patch_box[3], int32_t ncell_cap, void *cuda_stream, sph_view *out)
{
    if (!out || !patch_box) return SPH_E_INVAL;
    *out = nullptr;
    if (npatch_max < 1 || npatch_max > (1 << 24) || ncell_cap < 1 || ncell_cap > 64) return SPH_E_INVAL;
    const int64_t cells = (int64_t)npatch_max * ncell_cap * ncell_cap * ncell_cap;
    if (cells > (int64_t(1) << 27)) return SPH_E_INVAL;
    uint32_t present = 0;
    if (!layout_valid(layout, &present)) return SPH_E_INVAL;
    if (prec != SPH_F64 && prec != SPH_F32) return SPH_E_INVAL;
    if (n_max < 0 || n_max > 0x7fffffffLL) return SPH_E_INVAL;
    sph_domain dom;
    for (int a = 0; a < 3; ++a) {
        if (!(patch_box[a] > 0.0) || !(patch_box[a] < 1e300)) return SPH_E_INVAL;
        dom.box[a] = patch_box[a];
        dom.ncell[a] = 1;
    }
    dom.periodic = 0;
    sph_view_s *v = new (std::nothrow) sph_view_s;
    if (!v) return SPH_E_NOMEM;
    memset(v, 0, sizeof(*v));
    v->layout = *layout;
    v->prec = prec;
    v->n_max = n_max;
    v->dom = dom;
    v->st = static_cast<cudaStream_t>(cuda_stream);
    v->g = make_grid(dom);
    v->g.min_edge = 1e308;  // patch grids are sized so that every cell edge is at least 2 h_max of its patch
    v->cs.g = v->g;
    v->cs.npatch = 0;
    v->npatch_max = npatch_max;
    v->ncap = ncell_cap;
    v->ncells = (int)std::max<int64_t>(cells, npatch_max);
    v->esz = prec == SPH_F64 ? 8 : 4;
    v->present = present;
    v->persistent_ctas = 0;  // sized from the pair kernels' occupancy at launch
    v->union_view = true;
    v->host_direct = false;
    v->h_max_iter = 0;
    v->integrator = SPH_KDK_PREDICT;
    v->staged_bin = true;
    v->h_eta = 1.2;
    v->h_tol = 1e-6;
    v->ev_free = new (std::nothrow) std::vector<cudaEvent_t>();
    v->ev_pending = new (std::nothrow) std::vector<PendingTiming>();
    if (!v->ev_free || !v->ev_pending) {
        delete v->ev_free;
        delete v->ev_pending;
        delete v;
        return SPH_E_NOMEM;
    }
    Bump sizing;
    carve(v, sizing);
    if (cudaMalloc(&v->arena, sizing.off) != cudaSuccess) {
        v->arena = nullptr;
        sph_view_destroy(v);
        return SPH_E_NOMEM;
    }
    Bump real;
    real.base = static_cast<char *>(v->arena);
    carve(v, real);
    if (cudaMallocHost(&v->h_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&v->h_red, 8 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&v->h_counters, sizeof(sphk::Counters)) != cudaSuccess ||
        cudaMallocHost(&v->h_hstate, 4 * sizeof(int)) != cudaSuccess) {
        sph_view_destroy(v);
        return SPH_E_NOMEM;
    }
    if (cudaMemsetAsync(v->status, 0, sizeof(unsigned), v->st) != cudaSuccess ||
        cudaMemsetAsync(v->counters, 0, sizeof(sphk::Counters), v->st) != cudaSuccess ||
        cudaStreamSynchronize(v->st) != cudaSuccess) {
        sph_view_destroy(v);
        return SPH_E_CUDA;
    }
    *out = v;
    return SPH_OK;
}

sph_status sph_patches_bin(sph_view v, const void *aos_dev, int64_t n, const int64_t *patch_start_dev,
                           int32_t npatch)
{
    if (!v) return SPH_E_INVAL;
    return do_bin_patches(v, aos_dev, n, patch_start_dev, npatch);
}

sph_status sph_patches_step(sph_view v, void *aos_dev, int64_t n, const int64_t *patch_start_dev, int32_t npatch,
                            const sph_params *params, double dt, int32_t nsteps, double *stats_out)
{
    if (!v) return SPH_E_INVAL;
    if (v->npatch_max <= 0 || !patch_start_dev || npatch < 1 || npatch > v->npatch_max) return SPH_E_INVAL;
    v->patch_start = patch_start_dev;
    v->npatch = npatch;
    return do_step(v, aos_dev, n, params, dt, nsteps, stats_out);
}

sph_status sph_view_destroy(sph_view v)
{
    if (!v) return SPH_OK;
    cudaStreamSynchronize(v->st);
    if (v->arena) cudaFree(v->arena);
    if (v->aos_stage) cudaFree(v->aos_stage);
    if (v->h_status) cudaFreeHost(v->h_status);
    if (v->h_red) cudaFreeHost(v->h_red);
    if (v->h_counters) cudaFreeHost(v->h_counters);
    if (v->h_hstate) cudaFreeHost(v->h_hstate);
    graph_drop(v);
    if (v->ev_pending) {
        for (const PendingTiming &p : *v->ev_pending) {
            cudaEventDestroy(p.e0);
            cudaEventDestroy(p.e1);
        }
        delete v->ev_pending;
    }
    if (v->ev_free) {
        for (cudaEvent_t e : *v->ev_free) cudaEventDestroy(e);
        delete v->ev_free;
    }
    delete v;
    return SPH_OK;
}

sph_status sph_bin(sph_view v, const void *aos_dev, int64_t n)
{
    if (!v) return SPH_E_INVAL;
    return do_bin(v, aos_dev, n);
}

sph_status sph_aos_to_soa(sph_view v, const void *aos_dev, int64_t n, uint32_t in_mask)
{
    if (!v) return SPH_E_INVAL;
    return do_gather(v, aos_dev, n, in_mask);
}

sph_status sph_density(sph_view v, const sph_params *params)
{
    if (!v) return SPH_E_INVAL;
    return do_density(v, params);
}

sph_status sph_force(sph_view v, const sph_params *params)
{
    if (!v) return SPH_E_INVAL;
    return do_force(v, params);
}

sph_status sph_soa_to_aos(sph_view v, void *aos_dev, int64_t n, uint32_t out_mask)
{
    if (!v) return SPH_E_INVAL;
    return do_scatter(v, aos_dev, n, out_mask);
}

sph_status sph_step(sph_view v, void *aos_dev, int64_t n, const sph_params *params, double dt, int32_t nsteps,
                    double *stats_out)
{
    if (!v) return SPH_E_INVAL;
    return do_step(v, aos_dev, n, params, dt, nsteps, stats_out);
}

sph_status sph_step_host(sph_view v, void *aos_host, int64_t n, const sph_params *params, double dt,
                         int32_t nsteps, double *stats_out)
{
    if (!v || !aos_host || !params || n < 0 || n > v->n_max) return SPH_E_INVAL;
    if (v->host_direct) {
        // the pass reads and writes the records where they are: only page-locked memory mapped into the device's
        // address space qualifies (anything else is rejected before a launch)
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, aos_host) != cudaSuccess) {
            cudaGetLastError();
            return SPH_E_INVAL;
        }
        if (at.type != cudaMemoryTypeHost || !at.devicePointer) return SPH_E_INVAL;
        // the step's launches replay as one captured graph when the records and the arguments repeat (as
        // sph_step_graph); with stats_out, or on the legacy default stream, the step runs uncaptured
        sph_status s = stats_out || !v->st ? do_step(v, at.devicePointer, n, params, dt, nsteps, stats_out)
                                           : do_step_graph(v, at.devicePointer, n, params, dt, nsteps);
        if (s != SPH_OK) return s;
        return sph_view_sync(v);
    }
    if (!v->aos_stage) {
        const size_t bytes = (size_t)std::max<int64_t>(v->n_max, 1) * (size_t)v->layout.stride;
        if (cudaMalloc(&v->aos_stage, bytes) != cudaSuccess) {
            v->aos_stage = nullptr;
            return SPH_E_NOMEM;
        }
    }
    const size_t bytes = (size_t)n * (size_t)v->layout.stride;
    if (bytes && cudaMemcpyAsync(v->aos_stage, aos_host, bytes, cudaMemcpyHostToDevice, v->st) != cudaSuccess)
        return SPH_E_CUDA;
    sph_status s = do_step(v, v->aos_stage, n, params, dt, nsteps, stats_out);
    if (s != SPH_OK) return s;
    if (bytes && cudaMemcpyAsync(aos_host, v->aos_stage, bytes, cudaMemcpyDeviceToHost, v->st) != cudaSuccess)
        return SPH_E_CUDA;
    return sph_view_sync(v);
}

sph_status sph_reduce(sph_view v, double out[8])
{
    if (!v) return SPH_E_INVAL;
    return do_reduce(v, out);
}

sph_status sph_view_sync(sph_view v)
{
    if (!v) return SPH_E_INVAL;
    uint32_t bits = 0;
    sph_status s = read_status(v, &bits, false);
    if (s != SPH_OK) return s;
    if (bits & SPH_DEV_TIMEOUT) return SPH_E_TIMEOUT;
    return bits ? SPH_E_DEVICE : SPH_OK;
}

sph_status sph_view_status(sph_view v, uint32_t *bits, int32_t clear)
{
    if (!v || !bits) return SPH_E_INVAL;
    return read_status(v, bits, clear != 0);
}

sph_status sph_view_soa(sph_view v, int32_t field, int32_t comp, void **dev_ptr)
{
    if (!v || !dev_ptr || field < 0 || field >= SPH_NFIELDS || comp < 0 || comp >= kNcomp[field]) return SPH_E_INVAL;
    if (!(v->present & SPH_BIT(field))) return SPH_E_INVAL;
    *dev_ptr = v->soa.p[field][comp];
    return SPH_OK;
}

sph_status sph_view_index(sph_view v, int32_t which, void **dev_ptr)
{
    if (!v || !dev_ptr) return SPH_E_INVAL;
    switch (which) {
    case 0: *dev_ptr = v->perm; return SPH_OK;
    case 1: *dev_ptr = v->cell_start; return SPH_OK;
    case 2: *dev_ptr = v->cell_of_slot; return SPH_OK;
    default: return SPH_E_INVAL;
    }
}

sph_status sph_view_export(sph_view v, int32_t field, int32_t comp, void *dst, int64_t count)
{
    void *src = nullptr;
    sph_status s = sph_view_soa(v, field, comp, &src);
    if (s != SPH_OK) return s;
    if (!dst || count < 0 || count > v->n_max) return SPH_E_INVAL;
    if (count && cudaMemcpyAsync(dst, src, (size_t)count * v->esz, cudaMemcpyDefault, v->st) != cudaSuccess)
        return SPH_E_CUDA;
    return cudaStreamSynchronize(v->st) == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}

sph_status sph_view_export_index(sph_view v, int32_t which, void *dst, int64_t count)
{
    void *src = nullptr;
    sph_status s = sph_view_index(v, which, &src);
    if (s != SPH_OK) return s;
    const int64_t cap = which == 1 ? (int64_t)v->ncells + 1 : v->n_max;
    if (!dst || count < 0 || count > cap) return SPH_E_INVAL;
    if (count && cudaMemcpyAsync(dst, src, (size_t)count * 4, cudaMemcpyDefault, v->st) != cudaSuccess)
        return SPH_E_CUDA;
    return cudaStreamSynchronize(v->st) == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}

sph_status sph_view_info(sph_view v, int64_t *n, int64_t *ncells)
{
    if (!v) return SPH_E_INVAL;
    if (n) *n = v->n;
    if (ncells) *ncells = v->ncells;
    return SPH_OK;
}

sph_status sph_pair_counts(sph_view v, uint64_t counts[4], int32_t reset)
{
    if (!v || !counts) return SPH_E_INVAL;
    cudaError_t e = cudaMemcpyAsync(v->h_counters, v->counters, sizeof(sphk::Counters), cudaMemcpyDeviceToHost, v->st);
    if (e != cudaSuccess) return SPH_E_CUDA;
    if (reset && cudaMemsetAsync(v->counters, 0, sizeof(sphk::Counters), v->st) != cudaSuccess) return SPH_E_CUDA;
    if (cudaStreamSynchronize(v->st) != cudaSuccess) return SPH_E_CUDA;
    counts[0] = v->h_counters->dens_cand;
    counts[1] = v->h_counters->dens_pairs;
    counts[2] = v->h_counters->force_pairs;
    counts[3] = v->h_counters->force_cand;
    return SPH_OK;
}

sph_status sph_view_timing(sph_view v, int32_t enable)
{
    if (!v) return SPH_E_INVAL;
    v->timing = enable != 0;
    return SPH_OK;
}

sph_status sph_view_phase_times(sph_view v, double ms[SPH_NPHASES], int64_t launches[SPH_NPHASES], int32_t reset)
{
    if (!v) return SPH_E_INVAL;
    sph_status s = drain_timings(v);
    if (s != SPH_OK) return s;
    for (int p = 0; p < SPH_NPHASES; ++p) {
        if (ms) ms[p] = v->phase_ms[p];
        if (launches) launches[p] = v->launches[p];
        if (reset) {
            v->phase_ms[p] = 0.0;
            v->launches[p] = 0;
        }
    }
    return SPH_OK;
}

const char *sph_strerror(sph_status s)
{
    switch (s) {
    case SPH_OK: return "ok";
    case SPH_E_INVAL: return "invalid argument";
    case SPH_E_NOMEM: return "out of memory";
    case SPH_E_CUDA: return "CUDA error";
    case SPH_E_DEVICE: return "device status word set";
    case SPH_E_TIMEOUT: return "bounded device wait timed out";
    case SPH_E_NOTCONV: return "iteration did not converge";
    case SPH_E_STATE: return "call order (view member not resident or not binned)";
    default: return "unknown status";
    }
}

}  // extern "C"
