// Kernels of the adjoint gradient (ws_adjoint_gradient).
//
// The forward step is u^{n+1} = G (2 u^n - G u^{n-1} + W L u^n) + W_s h^2 s_n
// at the source, W = (V dt / h)^2, L the stencil sum (without 1/h^2), G the
// taper; the traces sample u^{n+1} at the receivers and the misfit is
// J = 1/2 sum (traces - d_obs)^2. With lambda the multipliers of the step
// equations, rho = W G lambda obeys the forward recurrence itself, run
// backwards:
//     rho^k = G (2 rho^{k+1} - G rho^{k+2} + W L rho^{k+1}) + W G r^k,
// r^k the residual at the receivers for the trace sample of u^k; so the
// step kernels advance rho, and these kernels add W G r^k at the receivers
// and accumulate the gradient with respect to m = 1/V^2,
//     dJ/dm_i = -V_i^2 sum_n rho^{n+1}_i (L u^n)_i
//               - [i = s] V_s^2 sum_n rho^{n+1}_s h^2 s_n / G_s.
#include "ws_internal.h"

namespace ws {
namespace {

constexpr int kRedThreads = 256;

// r = traces - d_obs over n entries (r = traces when d_obs is null); per-block
// FP64 partial sums of r^2 / 2.
__global__ void __launch_bounds__(kRedThreads) residual_kernel(const float *__restrict__ traces,
                                                               const float *d_obs,
                                                               long long n, float *__restrict__ r,
                                                               double *__restrict__ partials) {
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const float d = d_obs ? traces[t] - d_obs[t] : traces[t];
        r[t] = d;
        acc += 0.5 * (double)d * (double)d;
    }
    __shared__ double ws[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < kRedThreads / 32 ? ws[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

__global__ void __launch_bounds__(kRedThreads) sum_kernel(const double *__restrict__ partials,
                                                          int n, double *__restrict__ out) {
    double acc = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) acc += partials[q];
    __shared__ double ws[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < kRedThreads / 32 ? ws[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) out[0] = acc;
    }
}

// rho[rec_r] += W G r[r][col] (atomic: receivers may share a cell).
__global__ void inject_kernel(float *__restrict__ rho, const float *__restrict__ w,
                              const float *__restrict__ gx, const float *__restrict__ gy,
                              const float *__restrict__ gz, Geom g,
                              const int *__restrict__ rec_ijk, int nrec,
                              const float *__restrict__ r, int nt, int col) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nrec) return;
    const int i = rec_ijk[3 * q], j = rec_ijk[3 * q + 1], k = rec_ijk[3 * q + 2];
    const long long p = pidx(g, i, j, k);
    const float gd = gx[i] * gy[j] * gz[k];
    atomicAdd(&rho[p], w[p] * gd * r[(long long)q * nt + col]);
}

// acc += rho * (L u) with L u the stencil sum the step kernel stored while
// recomputing u^{n+1} (the same float value the step used), and at source
// cells rho * (h^2 s_n) / G. The accumulator is a compensated FP32 sum
// (Kahan): per cell a float2 {sum, correction} in the padded layout, so a
// thread's 4 consecutive x cells are one float4 of rho, one of L u and two
// of acc. GB300 runs FP64 at a small fraction of FP32, which made an FP64
// accumulator the bottleneck of this pass; the compensated sum keeps the
// rounding of 800 additions at the level of one. A block covers 128 x 8
// cells of one plane; one thread finds the block's sources first.
__device__ __forceinline__ void kahan_add(float &sum, float &corr, float x) {
    const float y = x - corr;
    const float t = sum + y;
    corr = (t - sum) - y;
    sum = t;
}

__global__ void __launch_bounds__(256) imaging_kernel(const float *__restrict__ rho,
                                                      const float *__restrict__ lapu, Geom g,
                                                      Sources src, const float *__restrict__ gx,
                                                      const float *__restrict__ gy,
                                                      const float *__restrict__ gz,
                                                      float2 *__restrict__ acc) {
    const int i = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    __shared__ unsigned mask;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        unsigned m = 0;
        const int i0 = 4 * blockIdx.x * blockDim.x, j0 = blockIdx.y * blockDim.y;
        for (int q = 0; q < src.n; ++q) {
            const SourceSample &ss = src.s[q];
            if (ss.k == k && ss.j >= j0 && ss.j < j0 + (int)blockDim.y && ss.i >= i0 &&
                ss.i < i0 + 4 * (int)blockDim.x)
                m |= 1u << q;
        }
        mask = m;
    }
    __syncthreads();
    if (i >= g.nx || j >= g.ny) return;
    const long long p = pidx(g, i, j, k);   // a multiple of 4: rows start on 32-cell lines
    const float4 r4 = *reinterpret_cast<const float4 *>(rho + p);
    const float4 l4 = __ldcs(reinterpret_cast<const float4 *>(lapu + p));
    float4 a01 = *reinterpret_cast<const float4 *>(acc + p);       // {s0, c0, s1, c1}
    float4 a23 = *reinterpret_cast<const float4 *>(acc + p + 2);   // {s2, c2, s3, c3}
    float t[4] = {r4.x * l4.x, r4.y * l4.y, r4.z * l4.z, r4.w * l4.w};
    const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
    for (unsigned m = mask; m; m &= m - 1) {
        const SourceSample &ss = src.s[__ffs(m) - 1];
        const int l = ss.i - i;
        if (ss.j == j && l >= 0 && l < 4)
            t[l] = fmaf(rv[l], ss.amp / (gx[ss.i] * gy[j] * gz[k]), t[l]);
    }
    // cells past nx (x padding: zero in rho and in L u) accumulate zeros
    kahan_add(a01.x, a01.y, t[0]);
    kahan_add(a01.z, a01.w, t[1]);
    kahan_add(a23.x, a23.y, t[2]);
    kahan_add(a23.z, a23.w, t[3]);
    *reinterpret_cast<float4 *>(acc + p) = a01;
    *reinterpret_cast<float4 *>(acc + p + 2) = a23;
}

// grad_m = -V^2 (sum - correction), V^2 = W (h/dt)^2; acc padded, unpadded
// float output.
__global__ void finalize_kernel(const float2 *__restrict__ acc, const float *__restrict__ w,
                                Geom g, double h_over_dt2, float *__restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= g.nx) return;
    const long long o = ((long long)k * g.ny + j) * g.nx + i;
    const long long p = pidx(g, i, j, k);
    const float2 a = acc[p];
    grad[o] = -w[p] * (float)h_over_dt2 * (a.x - a.y);
}

// out = sum over shots s = 0 .. n-1 of src[s] (FP64 sum in shot order, rounded
// once); out may be src[0].
__global__ void sum_fields_kernel(FieldList src, int n, long long count, float *out) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < n; ++q) acc += (double)src.p[q][t];
        out[t] = (float)acc;
    }
}

// Per-block FP64 partial sums of x^2 (a fixed grid: the same blocks sum the
// same elements on every call).
__global__ void __launch_bounds__(kRedThreads) norm2_partials_kernel(const float *__restrict__ x,
                                                                     long long n,
                                                                     double *__restrict__ partials) {
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        acc = fma((double)x[t], (double)x[t], acc);
    __shared__ double ws[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < kRedThreads / 32 ? ws[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

__global__ void sqrt_kernel(double *x) { x[0] = sqrt(x[0]); }

}  // namespace

int residual_partial_count() { return 1024; }

cudaError_t launch_sum_fields(const FieldList &src, int n, long long count, float *out,
                              cudaStream_t s) {
    if (n < 1 || n > kMaxFieldList) return cudaErrorInvalidValue;
    sum_fields_kernel<<<1216, 256, 0, s>>>(src, n, count, out);
    return cudaGetLastError();
}

cudaError_t launch_norm2(const float *x, long long n, double *partials, double *out,
                         cudaStream_t s) {
    const int blocks = residual_partial_count();
    norm2_partials_kernel<<<blocks, kRedThreads, 0, s>>>(x, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_kernel<<<1, kRedThreads, 0, s>>>(partials, blocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sqrt_kernel<<<1, 1, 0, s>>>(out);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float *traces, const float *d_obs, long long n, float *r,
                            double *partials, double *misfit, cudaStream_t s) {
    const int blocks = residual_partial_count();
    residual_kernel<<<blocks, kRedThreads, 0, s>>>(traces, d_obs, n, r, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_kernel<<<1, kRedThreads, 0, s>>>(partials, blocks, misfit);
    return cudaGetLastError();
}

cudaError_t launch_inject(float *rho, const float *w, const float *gx, const float *gy,
                          const float *gz, const Geom &g, const int *rec_ijk, int nrec,
                          const float *r, int nt, int col, cudaStream_t s) {
    inject_kernel<<<(nrec + 255) / 256, 256, 0, s>>>(rho, w, gx, gy, gz, g, rec_ijk, nrec, r, nt,
                                                     col);
    return cudaGetLastError();
}

cudaError_t launch_imaging(const float *rho, const float *lapu, const Geom &g, const Sources &src,
                           const float *gx, const float *gy, const float *gz, float2 *acc,
                           cudaStream_t s) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 127) / 128, (g.ny + 7) / 8, g.nz);
    imaging_kernel<<<grid, block, 0, s>>>(rho, lapu, g, src, gx, gy, gz, acc);
    return cudaGetLastError();
}

cudaError_t launch_finalize_gradient(const float2 *acc, const float *w, const Geom &g,
                                     double h_over_dt2, float *grad, cudaStream_t s) {
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    finalize_kernel<<<grid, 128, 0, s>>>(acc, w, g, h_over_dt2, grad);
    return cudaGetLastError();
}

}  // namespace ws
