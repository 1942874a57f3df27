// FP64 reduction of the discrete energy of the leapfrog scheme.
//
// With M = 1/(V dt)^2 and L the 25-point Laplacian (zero outside the grid),
// the recurrence of Eq. 2 without source or damping is
// M (u^{n+1} - 2 u^n + u^{n-1}) = L u^n; multiplying by u^{n+1} - u^{n-1}
// and summing over the grid telescopes (L is symmetric), so
//     E^{n-1/2} = sum (u^n - u^{n-1})^2 / (V dt)^2 - sum u^n (L u^{n-1})
// is the same for every n. The kernels evaluate it in double precision from
// the float fields: each block sums a fixed set of rows into one partial,
// and one block adds the partials in a fixed order, so the result does not
// depend on scheduling.
#include "ws_internal.h"

namespace ws {
namespace {

constexpr int kThreads = 256;

// Scratch of the allocation-free entry point: the per-block partial sums,
// one array per device that loads the library, held until the process exits.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

// u^n / u^{n-1} / (V dt / h)^2 of the handle's padded layout (halo is zero).
struct PaddedFields {
    const float *u, *p, *w;
    Geom g;
    __device__ float u_at(int i, int j, int k) const { return u[pidx(g, i, j, k)]; }
    __device__ float p_at(int i, int j, int k) const { return p[pidx(g, i, j, k)]; }
    __device__ float w_at(int i, int j, int k) const { return w[pidx(g, i, j, k)]; }
};

// Unpadded [nz][ny][nx] caller arrays; (V dt / h)^2 is formed from the
// velocity exactly as the stepper stores it (double, rounded once to float),
// and cells outside the grid read as zero, so every cell's term is the one
// the padded variant computes.
struct DenseFields {
    const float *u, *p, *v;
    int nx, ny, nz;
    double dt_over_h;
    __device__ long long at(int i, int j, int k) const { return ((long long)k * ny + j) * nx + i; }
    __device__ float u_at(int i, int j, int k) const { return u[at(i, j, k)]; }
    __device__ float p_at(int i, int j, int k) const {
        const bool in = i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz;
        return in ? p[at(i, j, k)] : 0.0f;
    }
    __device__ float w_at(int i, int j, int k) const {
        const double r = __dmul_rn((double)v[at(i, j, k)], dt_over_h);
        return (float)__dmul_rn(r, r);
    }
};

// Block (x = row block jb, y = plane k) sums rows [jb*rows, jb*rows+rows) of
// plane k into partials[k * gridDim.x + jb].
template <class F>
__global__ void __launch_bounds__(kThreads) energy_partials_kernel(F f, int nx, int ny, int rows,
                                                                   double h2, Coeffs64 c,
                                                                   double *__restrict__ partials) {
    const int k = blockIdx.y;
    const int j0 = blockIdx.x * rows;
    const int j1 = min(j0 + rows, ny);
    double acc = 0.0;
    for (int j = j0; j < j1; ++j) {
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            // every operation explicitly rounded (no contraction left to the
            // compiler), so each field layout gives the same bits
            const double pc = f.p_at(i, j, k);
            double lx = __dmul_rn(c.c0, pc), ly = lx, lz = lx;
#pragma unroll
            for (int m = 1; m <= 4; ++m) {
                const double cm = m == 1 ? c.c1 : m == 2 ? c.c2 : m == 3 ? c.c3 : c.c4;
                lx = __fma_rn(cm, __dadd_rn(f.p_at(i + m, j, k), f.p_at(i - m, j, k)), lx);
                ly = __fma_rn(cm, __dadd_rn(f.p_at(i, j + m, k), f.p_at(i, j - m, k)), ly);
                lz = __fma_rn(cm, __dadd_rn(f.p_at(i, j, k + m), f.p_at(i, j, k - m)), lz);
            }
            const double lap = __ddiv_rn(__dadd_rn(__dadd_rn(lx, ly), lz), h2);
            const double uc = f.u_at(i, j, k);
            const double d = __dsub_rn(uc, pc);
            const double vdt2 = __dmul_rn((double)f.w_at(i, j, k), h2);   // (V dt)^2
            acc = __dadd_rn(acc, __fma_rn(-uc, lap, __ddiv_rn(__dmul_rn(d, d), vdt2)));
        }
    }
    // fixed-order block reduction: warp shuffles, then warp 0
    __shared__ double warp_sum[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < kThreads / 32 ? warp_sum[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) partials[(long long)k * gridDim.x + blockIdx.x] = acc;
    }
}

// One block: out[0] = sum of partials[0 .. n), in a fixed order.
__global__ void __launch_bounds__(kThreads) sum_partials_kernel(const double *__restrict__ partials,
                                                                int n, double *__restrict__ out) {
    double acc = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) acc += partials[q];
    __shared__ double warp_sum[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < kThreads / 32 ? warp_sum[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) out[0] = acc;
    }
}

template <class F>
cudaError_t launch_energy(const F &f, int nx, int ny, int nz, double h, const Coeffs64 &c,
                          double *partials, double *out, cudaStream_t s) {
    const int rows = energy_rows_per_block();
    dim3 grid((ny + rows - 1) / rows, nz, 1);
    energy_partials_kernel<F><<<grid, kThreads, 0, s>>>(f, nx, ny, rows, h * h, c, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_kernel<<<1, kThreads, 0, s>>>(partials, (int)(grid.x * grid.y), out);
    return cudaGetLastError();
}

}  // namespace

int energy_rows_per_block() { return 32; }

long long energy_partial_count(int ny, int nz) {
    const int rows = energy_rows_per_block();
    return (long long)((ny + rows - 1) / rows) * nz;
}

cudaError_t launch_energy_padded(const float *u, const float *p, const float *w, const Geom &g,
                                 double h, const Coeffs64 &c, double *partials, double *out,
                                 cudaStream_t s) {
    PaddedFields f{u, p, w, g};
    return launch_energy(f, g.nx, g.ny, g.nz, h, c, partials, out, s);
}

cudaError_t launch_energy_noalloc(const float *u, const float *p, const float *v, int nx, int ny,
                                  int nz, double h, double dt, const Coeffs64 &c, double *out,
                                  cudaStream_t s) {
    // Host code cannot pass g_noalloc_partials itself (in host code the name
    // is a stand-in, not a device address): look its address up on the
    // current device. This is done on every call, so an address never
    // outlives the context it belongs to (a device reset may move it).
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    double *partials = static_cast<double *>(ptr);
    DenseFields f{u, p, v, nx, ny, nz, dt / h};
    return launch_energy(f, nx, ny, nz, h, c, partials, out, s);
}

}  // namespace ws
