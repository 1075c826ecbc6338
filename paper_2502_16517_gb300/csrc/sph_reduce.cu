// sph_reduce.cu -- FP64 global momentum / energy sums.
//
// Sums (kept in FP64 on the GPU for both precisions):
//   out[0..2] = sum m v, out[3..5] = sum m a, out[6] = sum m (|v|^2/2 + u), out[7] = sum m (v . a + du/dt).
// Deterministic: a fixed grid (from n only), each CTA sums a fixed contiguous slot range with a fixed
// thread-stride order and a fixed shared-memory tree, then one CTA adds the CTA partials in order.
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

}  // namespace sphk
