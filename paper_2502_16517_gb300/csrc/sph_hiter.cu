// sph_hiter.cu -- the smoothing-length iteration of Section 2.1, step 1: per particle, compute the density,
// decide whether to grow or shrink the interaction radius, recompute, until every particle meets its
// termination criterion.  The paper gives no update rule; the one used is h <- eta (m / rho)^(1/3) (at uniform
// density rho = m / s^3 it gives h = eta s), with the termination test |h_new - h| < tol h.  Update and test run
// in FP64 for both view precisions; a particle that passes is frozen at h_new.
//
// Device state of one iteration (int hstate[4]): [0] particles left unconverged by the current round,
// [1] all converged (set by the round that left none; later rounds' kernels return at once -- the density
// launches read it through their skip pointer), [2] rounds run, [3] particles unconverged after the last round
// run.  The host enqueues max_iter rounds and a final density pass without waiting in between, so the whole
// iteration can be captured in a CUDA graph.
#include "sph_internal.cuh"

namespace sphk {

namespace {

template <typename T>
__global__ void k_h_update(T *__restrict__ h, const T *__restrict__ m, const T *__restrict__ rho, int n, double eta,
                           double tol, double h_limit, unsigned char *__restrict__ done, int *__restrict__ hstate,
                           unsigned *__restrict__ status)
{
    if (hstate[1]) return;  // converged in an earlier round (block-uniform)
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    bool open = false;
    if (s < n && !done[s]) {
        const double hv = (double)h[s];
        const double hn = eta * cbrt((double)m[s] / (double)rho[s]);
        if (fabs(hn - hv) < tol * hv) {
            done[s] = 1;
        } else {
            open = true;
        }
        h[s] = (T)hn;
        // the 3^3 stencil needs every 2h within a cell edge
        if (!(hn <= h_limit)) atomicOr(status, SPH_DEV_H_TOO_BIG);
    }
    const unsigned b = __ballot_sync(0xffffffffu, open);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&hstate[0], __popc(b));
}

__global__ void k_h_round_end(int *hstate)
{
    if (hstate[1]) return;
    hstate[2] += 1;
    hstate[3] = hstate[0];
    if (hstate[0] == 0) hstate[1] = 1;
    hstate[0] = 0;
}

__global__ void k_h_finish(const int *hstate, unsigned *status)
{
    if (hstate[3] > 0) atomicOr(status, SPH_DEV_NOTCONV);
}

}  // namespace

cudaError_t launch_h_update(bool f32, const SoaPtrs &soa, int n, double eta, double tol, double h_limit,
                            unsigned char *done, int *hstate, unsigned *status, cudaStream_t st, int *nl)
{
    const int nb = n > 0 ? (n + 255) / 256 : 1;
    if (f32) {
        k_h_update<float><<<nb, 256, 0, st>>>((float *)soa.p[SPH_H][0], (const float *)soa.p[SPH_MASS][0],
                                              (const float *)soa.p[SPH_RHO][0], n, eta, tol, h_limit, done, hstate,
                                              status);
    } else {
        k_h_update<double><<<nb, 256, 0, st>>>((double *)soa.p[SPH_H][0], (const double *)soa.p[SPH_MASS][0],
                                               (const double *)soa.p[SPH_RHO][0], n, eta, tol, h_limit, done,
                                               hstate, status);
    }
    k_h_round_end<<<1, 1, 0, st>>>(hstate);
    *nl += 2;
    return cudaGetLastError();
}

cudaError_t launch_h_finish(const int *hstate, unsigned *status, cudaStream_t st, int *nl)
{
    k_h_finish<<<1, 1, 0, st>>>(hstate, status);
    *nl += 1;
    return cudaGetLastError();
}

}  // namespace sphk
