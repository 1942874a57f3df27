// Direct step kernel (one thread per cell, neighbours read from global
// memory through L1/L2) and the small helper kernels of the library.
//
// The direct kernel is the plain form of the fused step: it is used for
// grids smaller than a streaming tile and as a second, independent CUDA path
// in the parity tests. The hot path is the streaming kernel.
#include "ws_internal.h"

namespace ws {

// One fused step at one cell: Laplacian (Section II, 25-point formula),
// leapfrog of Eq. 2, absorbing taper, source (right-hand side of Eq. 2).
// u: u^n, up: u^{n-1} on entry and u^{n+1} on exit (same cell only),
// w: (V dt / h)^2.
__global__ void __launch_bounds__(256) step_direct_kernel(const float *__restrict__ u,
                                                          const float *up, float *out,
                                                          const float *__restrict__ w,
                                                          const __grid_constant__ StepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const Geom &g = a.g;
    if (i >= g.nx || j >= g.ny) return;
    const long long p = pidx(g, i, j, k);
    const long long sy = g.pnx, sz = g.plane;

    const float uc = u[p];
    float s[5];
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
        s[m] = ((u[p + m] + u[p - m]) + (u[p + m * sy] + u[p - m * sy])) +
               (u[p + m * sz] + u[p - m * sz]);
    }
    // sum_m c_m (s_m - 6 u): exactly zero on constants (see Coeffs)
    float d[5];
#pragma unroll
    for (int m = 1; m <= 4; ++m) d[m] = fmaf(-6.0f, uc, s[m]);
    float lap = a.c.c4 * d[4];
    lap = fmaf(a.c.c3, d[3], lap);
    lap = fmaf(a.c.c2, d[2], lap);
    lap = fmaf(a.c.c1, d[1], lap);

    if (a.lap) a.lap[p] = lap;
    const float wc = w[p];
    const float gd = a.gx[i] * a.gy[j] * a.gz[k];
    float un = gd * fmaf(wc, lap, fmaf(2.0f, uc, -gd * up[p]));
    for (int q = 0; q < a.src.n; ++q) {
        const SourceSample &ss = a.src.s[q];
        if (ss.i == i && ss.j == j && ss.k == k) un = fmaf(wc, ss.amp, un);
    }
    out[p] = un;
}

cudaError_t launch_step_direct(const float *u, const float *up, float *out, const float *w,
                               const StepArgs &a, cudaStream_t s) {
    dim3 block(32, 8, 1);
    dim3 grid((a.g.nx + 31) / 32, (a.g.ny + 7) / 8, a.g.nz);
    step_direct_kernel<<<grid, block, 0, s>>>(u, up, out, w, a);
    return cudaGetLastError();
}

// traces[r][step] = u^{n+1} at receiver r (the direct kernel's receiver pass).
__global__ void gather_receivers_kernel(const float *__restrict__ u_next,
                                        const long long *__restrict__ rec_pidx, int nrec,
                                        float *__restrict__ traces, int nt_max,
                                        long long trace_step) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    traces[(long long)r * nt_max + trace_step] = u_next[rec_pidx[r]];
}

cudaError_t launch_gather_receivers(const float *u_next, const long long *rec_pidx, int nrec,
                                    float *traces, int nt_max, long long trace_step,
                                    cudaStream_t s) {
    if (nrec <= 0) return cudaSuccess;
    gather_receivers_kernel<<<(nrec + 255) / 256, 256, 0, s>>>(u_next, rec_pidx, nrec, traces,
                                                               nt_max, trace_step);
    return cudaGetLastError();
}

// In place over the interior of the padded buffer: V -> (V dt / h)^2,
// computed in double and rounded once. extrema[0] collects max(V) and
// extrema[1] min(V) as float bit patterns (their unsigned order is the float
// order for V >= 0). A value that is not finite and > 0 contributes 0 to the
// minimum, which the host rejects.
__global__ void velocity_to_w_kernel(float *__restrict__ w, Geom g, double dt_over_h,
                                     unsigned *__restrict__ extrema) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int k = blockIdx.z;
    unsigned vmax = 0u, vmin = 0x7f800000u;
    if (i < g.nx) {
        const long long p = pidx(g, i, j, k);
        const float v = w[p];
        if (v > 0.0f && isfinite(v)) {
            vmax = __float_as_uint(v);
            vmin = vmax;
        } else {
            vmin = 0u;
        }
        const double r = __dmul_rn((double)v, dt_over_h);   // as ws_energy_noalloc forms it
        w[p] = (float)__dmul_rn(r, r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&extrema[0], vmax);
        atomicMin(&extrema[1], vmin);
    }
}

// In place: m (squared slowness, s^2/m^2) -> (V dt / h)^2 = (dt / h)^2 / m,
// in double, rounded once. extrema[0] / extrema[1] collect max(m) / min(m)
// as float bits; a value that is not finite and > 0 contributes 0 to the
// minimum, which the host rejects.
__global__ void slowness2_to_w_kernel(float *__restrict__ w, Geom g, double dt_over_h2,
                                      unsigned *__restrict__ extrema) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int k = blockIdx.z;
    unsigned mmax = 0u, mmin = 0x7f800000u;
    if (i < g.nx) {
        const long long p = pidx(g, i, j, k);
        const float m = w[p];
        if (m > 0.0f && isfinite(m)) {
            mmax = __float_as_uint(m);
            mmin = mmax;
        } else {
            mmin = 0u;
        }
        w[p] = (float)(dt_over_h2 / (double)m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mmax = max(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
        mmin = min(mmin, __shfl_xor_sync(0xffffffffu, mmin, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&extrema[0], mmax);
        atomicMin(&extrema[1], mmin);
    }
}

cudaError_t launch_slowness2_to_w(float *w, const Geom &g, double dt_over_h2, unsigned *extrema,
                                  cudaStream_t s) {
    dim3 block(128, 1, 1);
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    slowness2_to_w_kernel<<<grid, block, 0, s>>>(w, g, dt_over_h2, extrema);
    return cudaGetLastError();
}

cudaError_t launch_velocity_to_w(float *w, const Geom &g, double dt_over_h, unsigned *extrema,
                                 cudaStream_t s) {
    dim3 block(128, 1, 1);
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    velocity_to_w_kernel<<<grid, block, 0, s>>>(w, g, dt_over_h, extrema);
    return cudaGetLastError();
}

}  // namespace ws
