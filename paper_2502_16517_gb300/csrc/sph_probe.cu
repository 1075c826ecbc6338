// sph_probe.cu -- FMA throughput probe: the measured FP64 / FP32 arithmetic peak that the pair kernels'
// roofline fractions are quoted against (the GB300's FP64 rate is not in the generated peaks file).
//
// Each thread runs 8 independent fused multiply-add chains for `iters` iterations (enough independent work per
// warp to hide the pipe latency), 8 CTAs of 256 threads per SM.  flops = 2 x threads x iters x 8.
#include "sph_internal.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T a, T b)
{
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int k = 0; k < iters; ++k) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live, never taken
}

}  // namespace

extern "C" sph_status sph_probe_fma_rate(int32_t prec, double *flops_per_s)
{
    if (!flops_per_s || (prec != SPH_F64 && prec != SPH_F32)) return SPH_E_INVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_E_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPH_E_CUDA;
    const int blocks = sms * 8, threads = 256;
    const int iters = prec == SPH_F64 ? 2048 : 65536;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SPH_E_CUDA;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_ms = 1e30;
    for (int rep = 0; rep < 4; ++rep) {  // first repetition warms up
        cudaEventRecord(e0, st);
        if (prec == SPH_F64) {
            k_fma_probe<double><<<blocks, threads, 0, st>>>(nullptr, iters, 0.999999, 1e-7);
        } else {
            k_fma_probe<float><<<blocks, threads, 0, st>>>(nullptr, iters, 0.999999f, 1e-7f);
        }
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best_ms) best_ms = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (err != cudaSuccess || !(best_ms < 1e30)) return SPH_E_CUDA;
    *flops_per_s = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads / (best_ms * 1e-3);
    return SPH_OK;
}

extern "C" sph_status sph_build_info(int32_t *checked)
{
    if (!checked) return SPH_E_INVAL;
#ifdef SPH_CHECKED
    *checked = 1;
#else
    *checked = 0;
#endif
    return SPH_OK;
}
