// Host-side internals shared by the translation units of the C ABI
// (include/wavestep.h): the handle, the adjoint scratch and the helpers
// that the core entry points (ws_api.cu), the adjoint driver
// (ws_api_adjoint.cu) and the tuner and batches (ws_api_batch.cu) share.
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <type_traits>
#include <vector>

#include "ws_internal.h"

namespace wsh {

int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define WS_CUDA(call, what)                              \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return wsh::cuda_fail(e_, what); \
    } while (0)

// The 1D weights of the 8th-order second difference, offsets 0..4.
constexpr double kW0 = -205.0 / 72.0, kW1 = 8.0 / 5.0, kW2 = -1.0 / 5.0, kW3 = 8.0 / 315.0,
                 kW4 = -1.0 / 560.0;

// Leapfrog stability limit of V dt / h for the 3D 25-point Laplacian.
double cfl_limit();
// Ricker wavelet amp (1 - 2 a^2) exp(-a^2), a = pi f0 (t - t0).
double ricker(double t, double f0, double t0, double amp);
// Cerjan factor of cell idx on an axis of n cells.
double taper(int idx, int n, int nb, double a);

struct SourceDef {
    int i, j, k;
    double f0, t0, amp;
};

// The CUDA driver API's cuTensorMapEncodeTiled (null when unavailable).
PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn();

}  // namespace wsh

struct ws_handle {
    ws::Geom g{};
    double h = 0, dt = 0;
    float *buf[2] = {nullptr, nullptr};  // the two wavefield levels
    int cur = 0;                         // buf[cur] = u^n, buf[1-cur] = u^{n-1}
    float *w = nullptr;                  // (V dt / h)^2, padded
    float *gx = nullptr, *gy = nullptr, *gz = nullptr;
    unsigned *status = nullptr;          // [0] status bits, [1] vmax bits, [2] vmin bits
    double *energy = nullptr;            // energy partial sums, then the total
    cudaStream_t stream = nullptr;
    bool vel_ok = false;
    int nb = 0;
    double a = 0;
    long long step = 0;
    std::vector<wsh::SourceDef> src;

    int nrec = 0, nt_max = 0;
    long long trace_start = 0;
    std::vector<int> rec_ijk;
    float *traces = nullptr;
    long long *rec_pidx = nullptr;       // direct path
    int *rec_ptr = nullptr;              // streaming path: per-tile ranges
    ws::RecEntry *rec_entries = nullptr;
    int rec_tiling_tx = 0, rec_tiling_ty = 0, rec_tiling_rows = 0;

    int kernel = WS_KERNEL_AUTO;
    ws::StreamTiling tiling{64, 8, 0};
    CUtensorMap tmap_halo[2];  // buf[b] with the (tx+8, ty+8, 1) box
    CUtensorMap tmap_tile[2];  // buf[b] with the (tx, ty, 1) box
    CUtensorMap tmap_w;        // w with the (tx, ty, 1) box
    bool tmap_ok = false;
    long long launches = 0;

    // 16-bit storage (WS_STORAGE_BF16 / WS_STORAGE_FP16): the state lives in
    // buf16[cur] (u^n) and d16 (u^n - u^{n-1}), the model in w16 as well as
    // w; buf then serves as FP32 scratch copies.
    int storage = WS_STORAGE_FP32;
    uint16_t *buf16[2] = {nullptr, nullptr};
    uint16_t *d16 = nullptr, *w16 = nullptr;
    bool w16_ok = false;       // w16 holds the current model
    ws::Scale16 *scale = nullptr;
    CUtensorMap t16_halo[2], t16_d, t16_w;
    double wmax = 0.0;         // max (V dt / h)^2 of the model
    ws::Free16 free16{};       // cells whose taper is exactly 1, per axis
    int tile16_y = 0;          // 16-bit tile height chosen by ws_set_kernel (0: default)
    int t16_ty = 0;            // tile height the 16-bit tensor maps are encoded for

    // device scratch of ws_adjoint_gradient, kept for the next call
    struct AdjointCache *adj = nullptr;
    // bumped by every call that changes what a forward run from rest computes
    // (model, taper, sources, receivers, storage)
    unsigned long long model_version = 0;
    int stall_item = -1;       // test hook (ws_test_stall), consumed by the next FP32 step
};

// A padded FP32 field with the streaming kernel's two boxes on it.
struct MappedField {
    float *p = nullptr;
    CUtensorMap halo, tile;
};

// Scratch of ws_adjoint_gradient: checkpoint pairs, the states of one
// segment, the two adjoint levels, the gradient accumulator and the trace
// arrays. Reused while the step count, receivers and tiling stay the same.
struct AdjointCache {
    int N = -1, nrec = -1, kern = -1, tx = 0, ty = 0;
    // the checkpoints hold the forward run of this model version (ws_forward)
    bool fwd_valid = false;
    unsigned long long fwd_version = 0;
    std::vector<void *> mem;        // everything below, for cudaFree
    std::vector<float *> ck;
    std::vector<float *> lap;       // L u^n of the segment's steps
    MappedField ring[2], rho[2];    // recomputed u^n / u^{n-1}; rho^{k+1} / rho^{k+2}
    float2 *acc = nullptr;          // compensated FP32 gradient sums, padded layout
    double *partials = nullptr;     // residual partial sums, then the misfit
    double *norm = nullptr;         // gradient-norm partial sums, then the norm
    float *r = nullptr, *dd = nullptr, *grad = nullptr;
    int *rec = nullptr;
    ~AdjointCache() {
        for (void *p : mem) cudaFree(p);
    }
};

namespace wsh {

size_t field_bytes(const ws::Geom &g);
// A tensor map of a padded field over its interior (cells outside read as
// zeros) with a (bx, by, 1) box.
int encode_map(CUtensorMap *map, void *base, const ws::Geom &g, int bx, int by,
               int elem_bytes = 4);
// The handle's maps for its current tiling.
int encode_maps(ws_t ws);
bool stream_fits(const ws_t ws, const ws::StreamTiling &t);
// Planes per work item: the default for nz planes, and the default shortened
// to about two full waves of items on small grids.
int default_zblock(int nz);
int default_zblock(const ws::Geom &g, int tx, int ty);
// Choose the kernel for the next steps; fills *tiling for the streaming one.
int pick_kernel(ws_t ws, ws::StreamTiling *tiling);
void free_receivers(ws_t ws);
// Receiver table of the streaming kernels for tile t, whose consumer threads
// own 4 x-cells of `rows` consecutive rows (FP32 kernels 1, 16-bit kernel 2).
int build_rec_tiles(ws_t ws, const ws::StreamTiling &t, int rows = 1);
// Unpadded [nz][ny][nx] user array <-> interior of a padded field.
int copy_in(ws_t ws, float *dst, const float *src, int on_device);
int copy_out(ws_t ws, float *dst, const float *src, int on_device);
int upload_profiles(ws_t ws);
// The tile of the 16-bit streaming kernel (64 x ty) and the rows each of its
// threads computes. The default tile height is the first of kTile16Ys that
// the grid holds: 24 (two CTAs of 6 warps per SM) measured fastest on the
// 1024^3 survey (FP16 434.7, BF16 436.5 Gcell/s, against 418 for 48 and 395
// for 16); 48 is selectable with ws_set_kernel.
constexpr int kTile16X = 64, kRows16 = 2;
constexpr int kTile16Ys[] = {24, 16};
constexpr int kNumTile16Ys = 2;
int pick_tile16(const ws_t ws);
int default_zblock16(const ws::Geom &g, int ty);
int encode_maps16(ws_t ws, int ty);
int encode_state16(ws_t ws);
int decode_state16(ws_t ws);
// Point sources of step n (amp = h^2 s(t_n)).
void sources_of_step(const ws_t ws, long long n, ws::Sources *out);
// Step arguments common to every step of the handle's model.
ws::StepArgs base_args(const ws_t ws);
// One FP32 step: out = u^{n+1} from un = u^n and unm1 = u^{n-1} (out may be unm1).
int step_fp32(ws_t ws, ws::StepArgs &a, int kern, const ws::StreamTiling &tiling, const float *un,
              const CUtensorMap *un_halo, const float *unm1, const CUtensorMap *unm1_tile,
              float *out, long long n, bool sources, bool record);
// Select the FP32 kernel and bring maps and receiver table in line with it.
int prepare_fp32(ws_t ws, int *kern, ws::StreamTiling *tiling);
void destroy(ws_t ws);

// Device scratch of one call: freed, after the stream drains, on every return.
struct Scratch {
    cudaStream_t stream;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t s) : stream(s) {}
    ~Scratch() {
        cudaStreamSynchronize(stream);
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T **p, size_t bytes) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return e;
        ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return cudaSuccess;
    }
};

}  // namespace wsh
