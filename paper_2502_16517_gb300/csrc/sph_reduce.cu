// sph_reduce.cu -- FP64 global momentum / energy sums.
//
// Sums (FP64 results for both precisions):
//   out[0..2] = sum m v, out[3..5] = sum m a, out[6] = sum m (|v|^2/2 + u), out[7] = sum m (v . a + du/dt).
// Deterministic: a fixed grid (from n only), each CTA sums a fixed contiguous slot range with a fixed
// thread-stride order and a fixed shared-memory tree, then one CTA adds the CTA partials in order.
// FP64 views: every operation in FP64.  FP32 views: the per-particle terms and the per-thread and per-CTA sums in
// double-float arithmetic on the FP32 pipes (k_reduce_part_f32), each CTA's sums converted to FP64 once.
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

// ---- FP32 views: double-float arithmetic ----
// A value is carried as the unevaluated sum hi + lo of two floats (|lo| <= half an ulp of hi).  FP64 operations run
// at 1/64 of the FP32 rate on this part, and the FP64 form of the sums below (about 30 operations per particle with
// the conversions) made the reduction of a 14.6 M-particle FP32 view compute-bound at ~0.7 ms; in double-float
// it is a pass over the members.  The product of two floats is exact as two_prod's pair (Dekker, with one FMA);
// two_sum's pair is the exact sum of two floats (Knuth); additions of pairs round once in the low part, an error
// of at most ~2^-46 of the magnitudes added.  So the eight sums agree with FP64 sums of the same float values
// within ~1e-14 of the sums of the absolute terms, for terms inside the float range (products of the FP32 view's
// members, which its own kernels form too).  The intrinsics below are never contracted into FMAs.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// s + e = a + b exactly when |a| >= |b| (Dekker); used below where the second operand is a rounding-error term
__device__ __forceinline__ DF fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_add_f(DF a, float b)
{
    const DF s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ DF df_mul_f(DF a, float b)
{
    const DF p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_part_f32(SoaPtrs s, int n, int per_block,
                                                                 double *__restrict__ partials)
{
    __shared__ float sh_hi[8][kRedThreads], sh_lo[8][kRedThreads];
    const float *m = (const float *)s.p[SPH_MASS][0];
    const float *vx = (const float *)s.p[SPH_V][0], *vy = (const float *)s.p[SPH_V][1],
                *vz = (const float *)s.p[SPH_V][2];
    const float *ax = (const float *)s.p[SPH_A][0], *ay = (const float *)s.p[SPH_A][1],
                *az = (const float *)s.p[SPH_A][2];
    const float *u = (const float *)s.p[SPH_U][0], *du = (const float *)s.p[SPH_DUDT][0];
    const int b0 = blockIdx.x * per_block;
    const int b1 = min(n, b0 + per_block);
    DF acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = {0.f, 0.f};
    // kGroup particles per trip (i, i + kRedThreads, ...): their loads are issued together, then they are added in
    // the same order as one at a time
    constexpr int kGroup = 4;
    for (int i0 = b0 + threadIdx.x; i0 < b1; i0 += kGroup * kRedThreads) {
        float r[kGroup][9];
#pragma unroll
        for (int g = 0; g < kGroup; ++g) {
            const int i = i0 + g * kRedThreads;
            const bool in = i < b1;
            r[g][0] = in ? m[i] : 0.f;
            r[g][1] = in ? vx[i] : 0.f;
            r[g][2] = in ? vy[i] : 0.f;
            r[g][3] = in ? vz[i] : 0.f;
            r[g][4] = in ? ax[i] : 0.f;
            r[g][5] = in ? ay[i] : 0.f;
            r[g][6] = in ? az[i] : 0.f;
            r[g][7] = in ? u[i] : 0.f;
            r[g][8] = in ? du[i] : 0.f;
        }
#pragma unroll
        for (int g = 0; g < kGroup; ++g) {
            if (i0 + g * kRedThreads >= b1) break;
            const float mm = r[g][0], v0 = r[g][1], v1 = r[g][2], v2 = r[g][3];
            const float a0 = r[g][4], a1 = r[g][5], a2 = r[g][6];
            acc[0] = df_add(acc[0], two_prod(mm, v0));
            acc[1] = df_add(acc[1], two_prod(mm, v1));
            acc[2] = df_add(acc[2], two_prod(mm, v2));
            acc[3] = df_add(acc[3], two_prod(mm, a0));
            acc[4] = df_add(acc[4], two_prod(mm, a1));
            acc[5] = df_add(acc[5], two_prod(mm, a2));
            // m (|v|^2 / 2 + u): the halving is exact
            DF e = df_add(df_add(two_prod(v0, v0), two_prod(v1, v1)), two_prod(v2, v2));
            e.hi = __fmul_rn(0.5f, e.hi);
            e.lo = __fmul_rn(0.5f, e.lo);
            acc[6] = df_add(acc[6], df_mul_f(df_add_f(e, r[g][7]), mm));
            // m (v . a + du/dt)
            const DF w = df_add(df_add(two_prod(v0, a0), two_prod(v1, a1)), two_prod(v2, a2));
            acc[7] = df_add(acc[7], df_mul_f(df_add_f(w, r[g][8]), mm));
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        sh_hi[k][threadIdx.x] = acc[k].hi;
        sh_lo[k][threadIdx.x] = acc[k].lo;
    }
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const DF r = df_add({sh_hi[k][threadIdx.x], sh_lo[k][threadIdx.x]},
                                    {sh_hi[k][threadIdx.x + w], sh_lo[k][threadIdx.x + w]});
                sh_hi[k][threadIdx.x] = r.hi;
                sh_lo[k][threadIdx.x] = r.lo;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 8)
        partials[blockIdx.x * 8 + threadIdx.x] = (double)sh_hi[threadIdx.x][0] + (double)sh_lo[threadIdx.x][0];
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
        k_reduce_part_f32<<<nblocks, kRedThreads, 0, st>>>(soa, n, per_block, partials);
    } else {
        k_reduce_part<double><<<nblocks, kRedThreads, 0, st>>>(soa, n, per_block, partials);
    }
    k_reduce_final<<<1, kRedThreads, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace sphk
