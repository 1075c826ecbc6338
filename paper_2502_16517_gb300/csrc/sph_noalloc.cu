// sph_noalloc.cu -- cell bucketing that allocates nothing: sph_bin_static.
//
// Some callers cannot allocate device memory at all.  Examples are code running inside a custom allocator or
// memory-pool callback (a cudaMalloc there would re-enter the pool), plug-ins hosted by a framework that owns
// every device allocation and forbids others, and real-time loops with a hard no-allocation rule.  Such a
// caller cannot create a view, because sph_view_create allocates its arrays.  sph_bin_static gives it the cell
// bucketing with no view: it takes the caller's records and output arrays, and keeps its own intermediate
// arrays in one fixed device array defined below.
//
// That array exists once per GPU that loads this library and stays allocated until the process exits.  Every
// call shares it, so two calls whose work overlaps on the GPU (different streams, or different host threads
// on one device) race on it; callers must order such calls, for example by issuing them on one stream.  Each
// call clears the parts that must start at zero before its kernels run, so leftovers of the previous call do
// not matter.
//
// The first call on each device looks up the array's device address (cudaGetSymbolAddress) with that device
// current and caches it; make that first call before any stream capture begins.
#include <mutex>

#include "sph_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;

// Scratch layout (int32): cell_of[P] | perm_tmp[P] | count[C] | fill[C] | status[1] | scan[64], P = max
// particles, C = max cells; scan is the scratch of the multi-CTA scan.  2 * 262,144 + 2 * 65,536 + 65 ints =
// 2.5 MB.
constexpr int64_t kMaxP = SPH_BIN_STATIC_MAX_PARTICLES;
constexpr int64_t kMaxC = SPH_BIN_STATIC_MAX_CELLS;
constexpr int64_t kScanInts = 64;
constexpr int64_t kScratchInts = 2 * kMaxP + 2 * kMaxC + 1 + kScanInts;

static __device__ __align__(256) int g_bin_scratch[kScratchInts];

std::mutex g_lock;
int *g_scratch_dev[kMaxDevices] = {};

// Device address of g_bin_scratch on the current device (looked up once per device).
int *scratch_address(int device)
{
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_dev[device]) {
        int *p = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_bin_scratch) != cudaSuccess || !p) return nullptr;
        g_scratch_dev[device] = p;
    }
    return g_scratch_dev[device];
}

}  // namespace

extern "C" sph_status sph_bin_static(const sph_layout *layout, const sph_domain *domain, const void *aos_dev,
                                     int64_t n, int32_t *perm_dev, int32_t *cell_start_dev,
                                     int32_t *cell_of_slot_dev, uint32_t *status_dev, void *cuda_stream)
{
    if (!layout || !domain || !cell_start_dev) return SPH_E_INVAL;
    // the per-particle arrays may be NULL only when there are no particles
    if (n != 0 && (!aos_dev || !perm_dev || !cell_of_slot_dev)) return SPH_E_INVAL;
    if (layout->stride <= 0 || layout->stride % 8 != 0 || layout->stride > 65536) return SPH_E_INVAL;
    const int32_t off_x = layout->off[SPH_X];
    if (off_x < 0 || off_x % 8 != 0 || (int64_t)off_x + 24 > layout->stride) return SPH_E_INVAL;
    if (reinterpret_cast<uintptr_t>(aos_dev) % 8 != 0) return SPH_E_INVAL;
    // the fixed capacity of the static scratch, checked axis by axis so that the running product of the cell
    // counts stays within kMaxC * kMaxC and cannot overflow
    int64_t ncells = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(domain->box[a] > 0.0) || !(domain->box[a] < 1e300) || domain->ncell[a] < 1) return SPH_E_INVAL;
        if (domain->periodic && domain->ncell[a] < 3) return SPH_E_INVAL;
        if (domain->ncell[a] > kMaxC) return SPH_E_INVAL;
        ncells *= domain->ncell[a];
        if (ncells > kMaxC) return SPH_E_INVAL;
    }
    if (n < 0 || n > kMaxP) return SPH_E_INVAL;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return SPH_E_CUDA;
    int *s = scratch_address(device);
    if (!s) return SPH_E_CUDA;
    int *cell_of = s;
    int *perm_tmp = s + kMaxP;
    int *count = s + 2 * kMaxP;
    int *fill = s + 2 * kMaxP + kMaxC;
    unsigned *status = status_dev ? reinterpret_cast<unsigned *>(status_dev)
                                  : reinterpret_cast<unsigned *>(s + 2 * kMaxP + 2 * kMaxC);
    int *scan_tmp = s + 2 * kMaxP + 2 * kMaxC + 1;
    static_assert(kScanInts >= 3 * ((kMaxC + 4095) / 4096) + 4, "scan scratch too small");

    sphk::Grid g;
    g.periodic = domain->periodic ? 1 : 0;
    g.min_edge = 1e308;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = domain->ncell[a];
        g.box[a] = domain->box[a];
        g.edge[a] = domain->box[a] / (double)domain->ncell[a];
        g.inv[a] = (double)domain->ncell[a] / domain->box[a];
        g.edgef[a] = (float)g.edge[a];
        g.min_edge = g.min_edge < g.edge[a] ? g.min_edge : g.edge[a];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (!status_dev && cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return SPH_E_CUDA;
    int launched = 0;
    // launch_bin clears the histogram (count) itself; fill, perm_tmp and cell_of are fully rewritten
    cudaError_t e = sphk::launch_bin(static_cast<const uint8_t *>(aos_dev), layout->stride, off_x, (int)n, g,
                                     (int)ncells, cell_of, count, cell_start_dev, fill, perm_tmp, perm_dev,
                                     cell_of_slot_dev, scan_tmp, status, st, &launched);
    return e == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}
