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

// acc += rho * L u (the steppers' zero-sum float stencil), and at source
// cells rho * (h^2 s_n) / G; acc unpadded FP64.
__global__ void __launch_bounds__(256) imaging_kernel(const float *__restrict__ rho,
                                                      const float *__restrict__ u, Geom g,
                                                      Coeffs c, Sources src,
                                                      const float *__restrict__ gx,
                                                      const float *__restrict__ gy,
                                                      const float *__restrict__ gz,
                                                      double *__restrict__ acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long p = pidx(g, i, j, k);
    const long long sy = g.pnx, sz = g.plane;
    const float uc = u[p];
    float s[5];
#pragma unroll
    for (int m = 1; m <= 4; ++m)
        s[m] = ((u[p + m] + u[p - m]) + (u[p + m * sy] + u[p - m * sy])) + (u[p + m * sz] + u[p - m * sz]);
    float lap = c.c4 * fmaf(-6.0f, uc, s[4]);
    lap = fmaf(c.c3, fmaf(-6.0f, uc, s[3]), lap);
    lap = fmaf(c.c2, fmaf(-6.0f, uc, s[2]), lap);
    lap = fmaf(c.c1, fmaf(-6.0f, uc, s[1]), lap);
    const float rv = rho[p];
    double term = (double)rv * (double)lap;
    for (int q = 0; q < src.n; ++q) {
        const SourceSample &ss = src.s[q];
        if (ss.i == i && ss.j == j && ss.k == k)
            term += (double)rv * (double)ss.amp / ((double)gx[i] * gy[j] * gz[k]);
    }
    acc[((long long)k * g.ny + j) * g.nx + i] += term;
}

// grad_m = -V^2 acc, V^2 = W (h/dt)^2; unpadded float output.
__global__ void finalize_kernel(const double *__restrict__ acc, const float *__restrict__ w,
                                Geom g, double h_over_dt2, float *__restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= g.nx) return;
    const long long o = ((long long)k * g.ny + j) * g.nx + i;
    grad[o] = (float)(-(double)w[pidx(g, i, j, k)] * h_over_dt2 * acc[o]);
}

}  // namespace

int residual_partial_count() { return 1024; }

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

cudaError_t launch_imaging(const float *rho, const float *u, const Geom &g, const Coeffs &c,
                           const Sources &src, const float *gx, const float *gy, const float *gz,
                           double *acc, cudaStream_t s) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    imaging_kernel<<<grid, block, 0, s>>>(rho, u, g, c, src, gx, gy, gz, acc);
    return cudaGetLastError();
}

cudaError_t launch_finalize_gradient(const double *acc, const float *w, const Geom &g,
                                     double h_over_dt2, float *grad, cudaStream_t s) {
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    finalize_kernel<<<grid, 128, 0, s>>>(acc, w, g, h_over_dt2, grad);
    return cudaGetLastError();
}

}  // namespace ws
