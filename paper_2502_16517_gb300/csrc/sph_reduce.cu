// sph_reduce.cu -- FP64 global momentum / energy sums and the leapfrog kick-drift-kick updates.
//
// Sums (kept in FP64 on the GPU for both precisions):
//   out[0..2] = sum m v, out[3..5] = sum m a, out[6] = sum m (|v|^2/2 + u), out[7] = sum m (v . a + du/dt).
// Deterministic: a fixed grid (from n only), each CTA sums a fixed contiguous slot range with a fixed
// thread-stride order and a fixed shared-memory tree, then one CTA adds the CTA partials in order.
//
// Leapfrog (paper Section 2.1 steps 3-5): kicks and drifts update v, u and x in place in the AoS records, in FP64
// (positions change cells, so the next pass re-bins from the records).
#include "sph_internal.cuh"

namespace sphk {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_reduce_part(SoaPtrs s, int n, int per_block,
                                                             double *__restrict__ partials)
{
    __shared__ double sh[8][kRedThreads];
    const T *m = (const T *)s.p[SPH_MASS][0];
    const T *vx = (const T *)s.p[SPH_V][0], *vy = (const T *)s.p[SPH_V][1], *vz = (const T *)s.p[SPH_V][2];
    const T *ax = (const T *)s.p[SPH_A][0], *ay = (const T *)s.p[SPH_A][1], *az = (const T *)s.p[SPH_A][2];
    const T *u = (const T *)s.p[SPH_U][0], *du = (const T *)s.p[SPH_DUDT][0];
    const int b0 = blockIdx.x * per_block;
    const int b1 = min(n, b0 + per_block);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = b0 + threadIdx.x; i < b1; i += kRedThreads) {
        const double mm = (double)m[i];
        const double v0 = (double)vx[i], v1 = (double)vy[i], v2 = (double)vz[i];
        const double a0 = (double)ax[i], a1 = (double)ay[i], a2 = (double)az[i];
        acc[0] += mm * v0;
        acc[1] += mm * v1;
        acc[2] += mm * v2;
        acc[3] += mm * a0;
        acc[4] += mm * a1;
        acc[5] += mm * a2;
        acc[6] += mm * (0.5 * (v0 * v0 + v1 * v1 + v2 * v2) + (double)u[i]);
        acc[7] += mm * ((v0 * a0 + v1 * a1 + v2 * a2) + (double)du[i]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) partials[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const double *__restrict__ partials, int nblocks,
                                                              double *__restrict__ out)
{
    __shared__ double sh[8][kRedThreads];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kRedThreads) {
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += partials[b * 8 + k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) out[threadIdx.x] = sh[threadIdx.x][0];
}

// v + a dt, each operation rounded on its own (no contraction), as the leapfrog is written.
__device__ __forceinline__ double kick1(double v, double a, double d) { return __dadd_rn(v, __dmul_rn(a, d)); }

// Kicks and drift on the records, in FP64 for both view precisions (the records are the state; the SoA views are
// temporary, Section 4).  Per record: nkick half kicks v += a dtk, u += du/dt dtk (two when the second kick of one
// step and the first kick of the next meet), then, with drift, x += v dt, wrapped into [0, box) on a periodic
// grid, or mirrored at the walls of an open box (the velocity component turns; a position still outside after
// one mirror is put on the wall).  One thread per record.
__global__ void k_kick_drift_aos(uint8_t *__restrict__ aos, int64_t stride, int off_x, int off_v, int off_a,
                                 int off_u, int off_du, int n, Grid g, double dtk, int nkick, double dt, int drift)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t *rec = aos + (int64_t)i * stride;
    double *xp = reinterpret_cast<double *>(rec + off_x);
    double *vp = reinterpret_cast<double *>(rec + off_v);
    double v[3] = {vp[0], vp[1], vp[2]};
    if (nkick > 0) {
        const double *ap = reinterpret_cast<const double *>(rec + off_a);
        double *up = reinterpret_cast<double *>(rec + off_u);
        const double a[3] = {ap[0], ap[1], ap[2]};
        const double du = *reinterpret_cast<const double *>(rec + off_du);
        double u = *up;
        for (int k = 0; k < nkick; ++k) {
#pragma unroll
            for (int d = 0; d < 3; ++d) v[d] = kick1(v[d], a[d], dtk);
            u = kick1(u, du, dtk);
        }
        *up = u;
    }
    if (drift) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double xn = __dadd_rn(xp[d], __dmul_rn(v[d], dt));
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
            xp[d] = xn;
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) vp[d] = v[d];
}

}  // namespace

cudaError_t launch_reduce(bool f32, const SoaPtrs &soa, int n, double *partials, double *out, cudaStream_t st,
                          int *nl)
{
    *nl += 2;
    int nblocks = (n + 2047) / 2048;
    if (nblocks < 1) nblocks = 1;
    if (nblocks > kRedMaxBlocks) nblocks = kRedMaxBlocks;
    const int per_block = (n + nblocks - 1) / nblocks;
    if (f32) {
        k_reduce_part<float><<<nblocks, kRedThreads, 0, st>>>(soa, n, per_block, partials);
    } else {
        k_reduce_part<double><<<nblocks, kRedThreads, 0, st>>>(soa, n, per_block, partials);
    }
    k_reduce_final<<<1, kRedThreads, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_kick_drift_aos(uint8_t *aos, int64_t stride, const int off[5], int n, const Grid &g, double dtk,
                                  int nkick, double dt, bool drift, cudaStream_t st, int *nl)
{
    if (n <= 0) return cudaSuccess;
    ++*nl;
    k_kick_drift_aos<<<(n + 255) / 256, 256, 0, st>>>(aos, stride, off[0], off[1], off[2], off[3], off[4], n, g, dtk,
                                                      nkick, dt, drift ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace sphk
