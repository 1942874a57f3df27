// Host side of the C ABI declared in include/wavestep.h.
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

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(WS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(WS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define WS_CUDA(call, what)                              \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// The 1D weights of the 8th-order second difference, offsets 0..4.
constexpr double kW0 = -205.0 / 72.0, kW1 = 8.0 / 5.0, kW2 = -1.0 / 5.0, kW3 = 8.0 / 315.0,
                 kW4 = -1.0 / 560.0;

// Leapfrog stability limit of V dt / h for the 3D 25-point Laplacian: the
// largest |eigenvalue| times h^2 is 3 (|w0| + 2 sum |wm|) (the checkerboard
// mode), and the recurrence needs (V dt / h)^2 * that <= 4.
double cfl_limit() {
    const double s = std::fabs(kW0) + 2.0 * (std::fabs(kW1) + std::fabs(kW2) + std::fabs(kW3) +
                                             std::fabs(kW4));
    return 2.0 / std::sqrt(3.0 * s);
}

double ricker(double t, double f0, double t0, double amp) {
    const double pi = 3.14159265358979323846;
    const double a = pi * f0 * (t - t0);
    const double a2 = a * a;
    return amp * (1.0 - 2.0 * a2) * std::exp(-a2);
}

// Cerjan factor of cell idx on an axis of n cells.
double taper(int idx, int n, int nb, double a) {
    const int d = std::min(idx, n - 1 - idx);
    if (nb <= 0 || d >= nb) return 1.0;
    const double x = a * double(nb - d);
    return std::exp(-x * x);
}

struct SourceDef {
    int i, j, k;
    double f0, t0, amp;
};

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn) return fn;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return fn;
}

}  // namespace

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
    std::vector<SourceDef> src;

    int nrec = 0, nt_max = 0;
    long long trace_start = 0;
    std::vector<int> rec_ijk;
    float *traces = nullptr;
    long long *rec_pidx = nullptr;       // direct path
    int *rec_ptr = nullptr;              // streaming path: per-tile ranges
    ws::RecEntry *rec_entries = nullptr;
    int rec_tiling_tx = 0, rec_tiling_ty = 0;

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

    // device scratch of ws_adjoint_gradient, kept for the next call
    struct AdjointCache *adj = nullptr;
    // bumped by every call that changes what a forward run from rest computes
    // (model, taper, sources, receivers, storage)
    unsigned long long model_version = 0;
    int stall_item = -1;       // test hook (ws_test_stall), consumed by the next FP32 step
};

// A group of handles advanced together: one launch per step
// covers every shot's items; runs of steps are replayed as CUDA graphs.
struct ws_batch {
    std::vector<ws_t> shots;
    cudaStream_t stream = nullptr;     // the batch's own stream (graphs need one)
    cudaEvent_t ev = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr;
    int tx = 0, ty = 0;                // current tile (0: none yet)
    std::vector<int> zb;               // per shot
    ws::BatchShot *d_shots = nullptr;
    int2 *d_items = nullptr;
    int nitems = 0;
    ws::SourceSample *d_src = nullptr;
    size_t src_cap = 0;
    unsigned *status = nullptr;
    std::map<int, cudaGraphExec_t> graphs;   // by number of steps
    // online tuning: candidates still to time, and the best so far
    struct Cand {
        int tx, ty, m;                 // m: target items = m x resident CTAs (0: default z-blocks)
    };
    std::vector<Cand> todo;
    bool tuned = false, fixed = false;
    Cand best{0, 0, 0};
    Cand cfg{0, 0, -1};                // what the item table was built for
    float best_ms = 1e30f;
    long long launches = 0;
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
    double *partials = nullptr;
    float *r = nullptr, *dd = nullptr, *grad = nullptr;
    int *rec = nullptr;
    ~AdjointCache() {
        for (void *p : mem) cudaFree(p);
    }
};

namespace {

size_t field_bytes(const ws::Geom &g) {
    return size_t(g.pnx) * size_t(g.pny) * size_t(g.pnz) * sizeof(float);
}

int encode_map(CUtensorMap *map, void *base, const ws::Geom &g, int bx, int by,
               int elem_bytes = 4) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode_fn();
    if (!enc) return fail(WS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[3] = {(cuuint64_t)g.pnx, (cuuint64_t)g.pny, (cuuint64_t)g.pnz};
    cuuint64_t strides[2] = {(cuuint64_t)g.pnx * elem_bytes, (cuuint64_t)g.plane * elem_bytes};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    CUresult r = enc(map, dt, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(WS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return WS_OK;
}

int encode_maps(ws_t ws) {
    const ws::Geom &g = ws->g;
    const int tx = ws->tiling.tx, ty = ws->tiling.ty;
    int rc = WS_OK;
    for (int b = 0; b < 2 && rc == WS_OK; ++b) {
        rc = encode_map(&ws->tmap_halo[b], ws->buf[b], g, tx + 2 * ws::kHalo, ty + 2 * ws::kHalo);
        if (rc == WS_OK) rc = encode_map(&ws->tmap_tile[b], ws->buf[b], g, tx, ty);
    }
    if (rc == WS_OK) rc = encode_map(&ws->tmap_w, ws->w, g, tx, ty);
    ws->tmap_ok = rc == WS_OK;
    return rc;
}

bool stream_fits(const ws_t ws, const ws::StreamTiling &t) {
    return ws::stream_tiling_supported(t.tx, t.ty) && ws->g.nx >= t.tx && ws->g.ny >= t.ty;
}

// Planes per work item: long blocks re-read fewer 4-plane halos at their
// ends, short ones give the in-order dispatch more, smaller items; about 200
// planes measured best on the 1024^3 survey (five blocks of 205: 389.6
// Gcell/s against 387.2 at 342 and 376.7 at 64, 64 x 8 tiles).
int default_zblock(int nz) {
    const int blocks = std::max(1, (int)std::lround(nz / 200.0));
    return (nz + blocks - 1) / blocks;
}

// The default, shortened on small grids to about two full waves of items
// over the resident CTAs (a 256^3 grid in 64 x 8 tiles has 128 tiles for 456
// CTAs: one 256-plane block per tile ran at 139 Gcell/s, short blocks at
// more than twice that); the count is rounded down so the last wave is full.
int default_zblock(const ws::Geom &g, int tx, int ty) {
    int zb = default_zblock(g.nz), slots = 0;
    if (ws::stream_slots(tx, ty, false, &slots) != cudaSuccess) return zb;
    const long long tiles = (long long)((g.nx + tx - 1) / tx) * ((g.ny + ty - 1) / ty);
    const long long blocks = std::max<long long>(1, 2LL * slots / tiles);
    const int zs = (int)std::max<long long>(8, (g.nz + blocks - 1) / blocks);
    return std::min(zb, std::min(zs, g.nz));
}

// Choose the kernel for the next steps; fills *tiling for the streaming one.
int pick_kernel(ws_t ws, ws::StreamTiling *tiling) {
    if (ws->kernel == WS_KERNEL_DIRECT) return WS_KERNEL_DIRECT;
    ws::StreamTiling t = ws->tiling;
    if (ws->kernel == WS_KERNEL_AUTO && !stream_fits(ws, t)) {
        const ws::StreamTiling cands[3] = {{32, 16, 0}, {32, 8, 0}, {64, 16, 0}};
        bool found = false;
        for (const auto &c : cands)
            if (stream_fits(ws, c)) {
                t.tx = c.tx;
                t.ty = c.ty;
                found = true;
                break;
            }
        if (!found) return WS_KERNEL_DIRECT;
    }
    if (t.zb <= 0) t.zb = default_zblock(ws->g, t.tx, t.ty);
    *tiling = t;
    return WS_KERNEL_STREAM;
}

void free_receivers(ws_t ws) {
    cudaFree(ws->traces);
    cudaFree(ws->rec_pidx);
    cudaFree(ws->rec_ptr);
    cudaFree(ws->rec_entries);
    ws->traces = nullptr;
    ws->rec_pidx = nullptr;
    ws->rec_ptr = nullptr;
    ws->rec_entries = nullptr;
    ws->rec_tiling_tx = ws->rec_tiling_ty = 0;
}

// Receiver table of the streaming kernels for tile t: per (tile, consumer
// warp) a range of entries sorted by k.
int build_rec_tiles(ws_t ws, const ws::StreamTiling &t) {
    if (ws->nrec == 0) return WS_OK;
    if (ws->rec_tiling_tx == t.tx && ws->rec_tiling_ty == t.ty) return WS_OK;
    const int tiles_x = (ws->g.nx + t.tx - 1) / t.tx;
    const int tiles_y = (ws->g.ny + t.ty - 1) / t.ty;
    const int warps = t.tx / 4 * t.ty / 32;   // consumer warps of a CTA
    const int ntiles = tiles_x * tiles_y * warps;   // (tile, warp) ranges
    std::vector<std::pair<int, ws::RecEntry>> e(ws->nrec);
    for (int r = 0; r < ws->nrec; ++r) {
        const int i = ws->rec_ijk[3 * r], j = ws->rec_ijk[3 * r + 1], k = ws->rec_ijk[3 * r + 2];
        const int tile = (j / t.ty) * tiles_x + (i / t.tx);
        const int li = i - (i / t.tx) * t.tx, lj = j - (j / t.ty) * t.ty;
        const int owner = lj * (t.tx / 4) + li / 4;
        e[r] = {tile * warps + owner / 32, ws::RecEntry{k, owner, li % 4, r}};
    }
    std::stable_sort(e.begin(), e.end(), [](const auto &x, const auto &y) {
        return x.first != y.first ? x.first < y.first : x.second.k < y.second.k;
    });
    std::vector<int> ptr(ntiles + 1, 0);
    std::vector<ws::RecEntry> ent(ws->nrec);
    for (int r = 0; r < ws->nrec; ++r) {
        ptr[e[r].first + 1]++;
        ent[r] = e[r].second;
    }
    for (int tt = 0; tt < ntiles; ++tt) ptr[tt + 1] += ptr[tt];
    cudaFree(ws->rec_ptr);
    cudaFree(ws->rec_entries);
    ws->rec_ptr = nullptr;
    ws->rec_entries = nullptr;
    WS_CUDA(cudaMalloc(&ws->rec_ptr, sizeof(int) * (ntiles + 1)), "cudaMalloc receiver table");
    WS_CUDA(cudaMalloc(&ws->rec_entries, sizeof(ws::RecEntry) * ws->nrec),
            "cudaMalloc receiver table");
    WS_CUDA(cudaMemcpyAsync(ws->rec_ptr, ptr.data(), sizeof(int) * (ntiles + 1),
                            cudaMemcpyHostToDevice, ws->stream),
            "upload receiver table");
    WS_CUDA(cudaMemcpyAsync(ws->rec_entries, ent.data(), sizeof(ws::RecEntry) * ws->nrec,
                            cudaMemcpyHostToDevice, ws->stream),
            "upload receiver table");
    // the host vectors die here: wait for the copies
    WS_CUDA(cudaStreamSynchronize(ws->stream), "upload receiver table");
    ws->rec_tiling_tx = t.tx;
    ws->rec_tiling_ty = t.ty;
    return WS_OK;
}

// Copy an unpadded [nz][ny][nx] array into the interior of a padded buffer.
int copy_in(ws_t ws, float *dst, const float *src, int on_device) {
    const ws::Geom &g = ws->g;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int k = 0; k < g.nz; ++k) {
        WS_CUDA(cudaMemcpy2DAsync(dst + ws::pidx(g, 0, 0, k), size_t(g.pnx) * 4,
                                  src + size_t(k) * g.ny * g.nx, size_t(g.nx) * 4,
                                  size_t(g.nx) * 4, g.ny, kind, ws->stream),
                "copy into the padded field");
    }
    return WS_OK;
}

int copy_out(ws_t ws, float *dst, const float *src, int on_device) {
    const ws::Geom &g = ws->g;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k = 0; k < g.nz; ++k) {
        WS_CUDA(cudaMemcpy2DAsync(dst + size_t(k) * g.ny * g.nx, size_t(g.nx) * 4,
                                  src + ws::pidx(g, 0, 0, k), size_t(g.pnx) * 4,
                                  size_t(g.nx) * 4, g.ny, kind, ws->stream),
                "copy out of the padded field");
    }
    return WS_OK;
}

int upload_profiles(ws_t ws) {
    const ws::Geom &g = ws->g;
    std::vector<float> px(g.nx), py(g.ny), pz(g.nz);
    for (int i = 0; i < g.nx; ++i) px[i] = (float)taper(i, g.nx, ws->nb, ws->a);
    for (int j = 0; j < g.ny; ++j) py[j] = (float)taper(j, g.ny, ws->nb, ws->a);
    for (int k = 0; k < g.nz; ++k) pz[k] = (float)taper(k, g.nz, ws->nb, ws->a);
    WS_CUDA(cudaMemcpyAsync(ws->gx, px.data(), 4 * px.size(), cudaMemcpyHostToDevice, ws->stream),
            "upload taper");
    WS_CUDA(cudaMemcpyAsync(ws->gy, py.data(), 4 * py.size(), cudaMemcpyHostToDevice, ws->stream),
            "upload taper");
    WS_CUDA(cudaMemcpyAsync(ws->gz, pz.data(), 4 * pz.size(), cudaMemcpyHostToDevice, ws->stream),
            "upload taper");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "upload taper");
    return WS_OK;
}

// The tile of the 16-bit streaming kernel.
constexpr int kTile16X = 64, kTile16Y = 8;

int encode_maps16(ws_t ws) {
    const ws::Geom &g = ws->g;
    int rc = WS_OK;
    for (int b = 0; b < 2 && rc == WS_OK; ++b)
        rc = encode_map(&ws->t16_halo[b], ws->buf16[b], g, kTile16X + 16, kTile16Y + 2 * ws::kHalo, 2);
    if (rc == WS_OK) rc = encode_map(&ws->t16_d, ws->d16, g, kTile16X, kTile16Y, 2);
    if (rc == WS_OK) rc = encode_map(&ws->t16_w, ws->w16, g, kTile16X, kTile16Y, 2);
    return rc;
}

// FP32 buffers -> the 16-bit state (U = u^n, D = u^n - u^{n-1}), exponents
// in the step's slot.
int encode_state16(ws_t ws) {
    const int sn = (int)(ws->step & 3), so = (int)((ws->step + 1) & 3);
    WS_CUDA(ws::launch_encode16(ws->storage, ws->buf[ws->cur], ws->buf[1 - ws->cur],
                                ws->buf16[ws->cur], ws->d16, ws->g, ws->scale, sn, ws->stream),
            "encode field");
    // the next step accumulates max |u^{n+1}| into slot (step + 1) & 3
    WS_CUDA(cudaMemsetAsync(&ws->scale->amax[so], 0, sizeof(unsigned), ws->stream), "encode field");
    ws->launches += 2;
    return WS_OK;
}

// The 16-bit state -> FP32 buffers (u^n, u^{n-1}).
int decode_state16(ws_t ws) {
    const int sn = (int)(ws->step & 3);
    WS_CUDA(ws::launch_decode16(ws->storage, ws->buf16[ws->cur], ws->d16, ws->buf[ws->cur],
                                ws->buf[1 - ws->cur], ws->g, ws->scale, sn, ws->stream),
            "decode field");
    ws->launches += 1;
    return WS_OK;
}

// Point sources of step n: (V_s dt)^2 s(t_n) is added at each source cell,
// i.e. amp = h^2 s(t_n) times the stored (V dt / h)^2.
void sources_of_step(const ws_t ws, long long n, ws::Sources *out) {
    out->n = (int)ws->src.size();
    const double t = double(n) * ws->dt;
    for (int q = 0; q < out->n; ++q) {
        const SourceDef &d = ws->src[q];
        out->s[q] = ws::SourceSample{d.i, d.j, d.k,
                                     (float)(ws->h * ws->h * ricker(t, d.f0, d.t0, d.amp))};
    }
}

// Step arguments common to every step of the handle's model.
ws::StepArgs base_args(const ws_t ws) {
    ws::StepArgs a{};
    a.stall_item = -1;
    a.g = ws->g;
    a.c.c1 = (float)kW1;
    a.c.c2 = (float)kW2;
    a.c.c3 = (float)kW3;
    a.c.c4 = (float)kW4;
    a.gx = ws->gx;
    a.gy = ws->gy;
    a.gz = ws->gz;
    a.traces = ws->traces;
    a.nt_max = ws->nt_max;
    a.status = ws->status;
    return a;
}

// One FP32 step of the handle's model (Eq. 1 discretised): out = u^{n+1}
// from un = u^n (with its halo box map) and unm1 = u^{n-1} (with its tile box
// map); out may be unm1. Adds the sources of step n when `sources`, records
// the receivers' trace column n - trace_start when `record`.
int step_fp32(ws_t ws, ws::StepArgs &a, int kern, const ws::StreamTiling &tiling, const float *un,
              const CUtensorMap *un_halo, const float *unm1, const CUtensorMap *unm1_tile,
              float *out, long long n, bool sources, bool record) {
    if (sources)
        sources_of_step(ws, n, &a.src);
    else
        a.src.n = 0;
    a.trace_step = n - ws->trace_start;
    cudaError_t e;
    if (kern == WS_KERNEL_STREAM) {
        e = ws::launch_step_stream(un_halo, unm1_tile, &ws->tmap_w, out, a, tiling,
                                   record ? ws->rec_ptr : nullptr, ws->rec_entries, ws->stream);
        ws->launches++;
    } else {
        e = ws::launch_step_direct(un, unm1, out, ws->w, a, ws->stream);
        ws->launches++;
        if (e == cudaSuccess && record) {
            e = ws::launch_gather_receivers(out, ws->rec_pidx, ws->nrec, ws->traces, ws->nt_max,
                                            a.trace_step, ws->stream);
            ws->launches++;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
    return WS_OK;
}

// Select the FP32 kernel for the next steps and bring the tensor maps and
// the receiver table in line with its tiling.
int prepare_fp32(ws_t ws, int *kern, ws::StreamTiling *tiling) {
    *kern = pick_kernel(ws, tiling);
    if (*kern != WS_KERNEL_STREAM) return WS_OK;
    if (tiling->tx != ws->tiling.tx || tiling->ty != ws->tiling.ty) {
        ws->tiling.tx = tiling->tx;
        ws->tiling.ty = tiling->ty;
        int rc = encode_maps(ws);
        if (rc != WS_OK) return rc;
    }
    return build_rec_tiles(ws, *tiling);
}

void destroy(ws_t ws) {
    if (!ws) return;
    cudaStreamSynchronize(ws->stream);
    cudaFree(ws->buf[0]);
    cudaFree(ws->buf[1]);
    cudaFree(ws->w);
    cudaFree(ws->gx);
    cudaFree(ws->gy);
    cudaFree(ws->gz);
    cudaFree(ws->status);
    cudaFree(ws->energy);
    cudaFree(ws->buf16[0]);
    cudaFree(ws->buf16[1]);
    cudaFree(ws->d16);
    cudaFree(ws->w16);
    cudaFree(ws->scale);
    free_receivers(ws);
    delete ws->adj;
    delete ws;
}


// Tiles of the streaming kernel, in the order the tuners try them.
constexpr int kTileCands[5][2] = {{64, 8}, {32, 8}, {32, 16}, {64, 16}, {64, 32}};

// z-block candidates for a grid of nz planes cut into `tiles` xy tiles: the
// default, and for m = 1 .. 8 the z blocks whose item count comes closest to
// m waves of the resident CTAs from below and from above (a wave that is only
// partly filled leaves SMs idle at the end of every step on small grids).
std::vector<int> zblock_candidates(int nz, long long tiles, int slots) {
    std::vector<int> z{default_zblock(nz)};
    for (int m = 1; m <= 8; ++m) {
        const long long target = (long long)m * slots;
        for (long long blocks : {target / tiles, (target + tiles - 1) / tiles}) {
            blocks = std::max<long long>(1, blocks);
            const int zb = (int)std::max<long long>(8, (nz + blocks - 1) / blocks);
            z.push_back(std::min(zb, nz));
        }
    }
    std::sort(z.begin(), z.end());
    z.erase(std::unique(z.begin(), z.end()), z.end());
    return z;
}

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, ws::StreamTiling> g_tune_cache;



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


}  // namespace

extern "C" {

const char *ws_last_error(void) { return g_err; }

int ws_create(ws_t *out, int nx, int ny, int nz, double h, double dt) {
    if (!out) return fail(WS_ERR_BADARG, "ws_create: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 65535 || ny > 65535 || nz > 65535)
        return fail(WS_ERR_BADARG, "ws_create: sizes must be in [1, 65535], got %d x %d x %d", nx,
                    ny, nz);
    if (!(h > 0.0) || !(dt > 0.0) || !std::isfinite(h) || !std::isfinite(dt))
        return fail(WS_ERR_BADARG, "ws_create: h and dt must be finite and > 0");
    ws_t ws = new (std::nothrow) ws_handle();
    if (!ws) return fail(WS_ERR_OOM, "ws_create: host allocation failed");
    ws::Geom &g = ws->g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.pnx = (ws::kXOff + nx + ws::kHalo + ws::kRowAlign - 1) / ws::kRowAlign * ws::kRowAlign;
    g.pny = ny + 2 * ws::kHalo;
    g.pnz = nz + 2 * ws::kHalo;
    g.plane = (long long)g.pnx * g.pny;
    ws->h = h;
    ws->dt = dt;
    const size_t fb = field_bytes(g);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&ws->buf[b], fb);
    if (e == cudaSuccess) e = cudaMalloc(&ws->w, fb);
    if (e == cudaSuccess) e = cudaMalloc(&ws->gx, sizeof(float) * nx);
    if (e == cudaSuccess) e = cudaMalloc(&ws->gy, sizeof(float) * ny);
    if (e == cudaSuccess) e = cudaMalloc(&ws->gz, sizeof(float) * nz);
    if (e == cudaSuccess) e = cudaMalloc(&ws->status, sizeof(unsigned) * 4);
    if (e == cudaSuccess)
        e = cudaMalloc(&ws->energy, sizeof(double) * (ws::energy_partial_count(ny, nz) + 1));
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMemsetAsync(ws->buf[b], 0, fb, ws->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws->w, 0, fb, ws->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws->status, 0, sizeof(unsigned) * 4, ws->stream);
    if (e != cudaSuccess) {
        destroy(ws);
        return cuda_fail(e, "ws_create");
    }
    int rc = upload_profiles(ws);
    if (rc == WS_OK) rc = encode_maps(ws);
    if (rc == WS_OK && cudaStreamSynchronize(ws->stream) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "ws_create");
    if (rc != WS_OK) {
        destroy(ws);
        return rc;
    }
    *out = ws;
    return WS_OK;
}

int ws_destroy(ws_t ws) {
    destroy(ws);
    return WS_OK;
}

int ws_set_stream(ws_t ws, void *cuda_stream) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_set_stream: NULL handle");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_set_stream");
    ws->stream = static_cast<cudaStream_t>(cuda_stream);
    return WS_OK;
}

int ws_set_velocity(ws_t ws, const float *v, int on_device) {
    if (!ws || !v) return fail(WS_ERR_BADARG, "ws_set_velocity: NULL argument");
    ws->model_version++;
    ws->vel_ok = false;
    int rc = copy_in(ws, ws->w, v, on_device);
    if (rc != WS_OK) return rc;
    static const unsigned init[2] = {0u, 0x7f800000u};
    WS_CUDA(cudaMemcpyAsync(ws->status + 1, init, sizeof init, cudaMemcpyHostToDevice, ws->stream),
            "ws_set_velocity");
    WS_CUDA(ws::launch_velocity_to_w(ws->w, ws->g, ws->dt / ws->h, ws->status + 1, ws->stream),
            "velocity conversion kernel");
    ws->launches++;
    unsigned ext[2];
    WS_CUDA(cudaMemcpyAsync(ext, ws->status + 1, sizeof ext, cudaMemcpyDeviceToHost, ws->stream),
            "ws_set_velocity");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_set_velocity");
    float vmax, vmin;
    std::memcpy(&vmax, &ext[0], 4);
    std::memcpy(&vmin, &ext[1], 4);
    if (ext[1] == 0u) return fail(WS_ERR_BADARG, "ws_set_velocity: every value must be finite and > 0");
    const double c = double(vmax) * ws->dt / ws->h;
    if (c > cfl_limit())
        return fail(WS_ERR_CFL, "ws_set_velocity: max(V) dt / h = %.6f exceeds the limit %.6f", c,
                    cfl_limit());
    ws->wmax = c * c;
    ws->vel_ok = true;
    ws->w16_ok = false;
    return WS_OK;
}

int ws_set_slowness2(ws_t ws, const float *m, int on_device) {
    if (!ws || !m) return fail(WS_ERR_BADARG, "ws_set_slowness2: NULL argument");
    ws->model_version++;
    ws->vel_ok = false;
    int rc = copy_in(ws, ws->w, m, on_device);
    if (rc != WS_OK) return rc;
    static const unsigned init[2] = {0u, 0x7f800000u};
    WS_CUDA(cudaMemcpyAsync(ws->status + 1, init, sizeof init, cudaMemcpyHostToDevice, ws->stream),
            "ws_set_slowness2");
    const double r = ws->dt / ws->h;
    WS_CUDA(ws::launch_slowness2_to_w(ws->w, ws->g, r * r, ws->status + 1, ws->stream),
            "slowness conversion kernel");
    ws->launches++;
    unsigned ext[2];
    WS_CUDA(cudaMemcpyAsync(ext, ws->status + 1, sizeof ext, cudaMemcpyDeviceToHost, ws->stream),
            "ws_set_slowness2");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_set_slowness2");
    float mmin;
    std::memcpy(&mmin, &ext[1], 4);
    if (ext[1] == 0u)
        return fail(WS_ERR_BADARG, "ws_set_slowness2: every value must be finite and > 0");
    const double c = ws->dt / (ws->h * std::sqrt(double(mmin)));   // max V dt / h
    if (c > cfl_limit())
        return fail(WS_ERR_CFL, "ws_set_slowness2: max(V) dt / h = %.6f exceeds the limit %.6f", c,
                    cfl_limit());
    ws->wmax = c * c;
    ws->vel_ok = true;
    ws->w16_ok = false;
    return WS_OK;
}

int ws_set_sponge(ws_t ws, int nb, double a) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_set_sponge: NULL handle");
    if (nb < 0 || !(a >= 0.0) || !std::isfinite(a))
        return fail(WS_ERR_BADARG, "ws_set_sponge: need nb >= 0 and finite a >= 0");
    ws->nb = nb;
    ws->a = a;
    ws->model_version++;
    return upload_profiles(ws);
}

int ws_add_source(ws_t ws, int ix, int iy, int iz, double f0, double t0, double amp) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_add_source: NULL handle");
    const ws::Geom &g = ws->g;
    if (ix < 0 || ix >= g.nx || iy < 0 || iy >= g.ny || iz < 0 || iz >= g.nz)
        return fail(WS_ERR_BADARG, "ws_add_source: cell (%d, %d, %d) outside the grid", ix, iy, iz);
    if (!(f0 > 0.0) || !std::isfinite(f0) || !std::isfinite(t0) || !std::isfinite(amp))
        return fail(WS_ERR_BADARG, "ws_add_source: need finite t0, amp and f0 > 0");
    if ((int)ws->src.size() >= ws::kMaxSources)
        return fail(WS_ERR_BADARG, "ws_add_source: at most %d sources", ws::kMaxSources);
    ws->src.push_back({ix, iy, iz, f0, t0, amp});
    ws->model_version++;
    return WS_OK;
}

int ws_clear_sources(ws_t ws) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_clear_sources: NULL handle");
    ws->src.clear();
    ws->model_version++;
    return WS_OK;
}

int ws_set_receivers(ws_t ws, int nrec, const int *ijk, int nt_max) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_set_receivers: NULL handle");
    if (nrec < 0 || (nrec > 0 && (!ijk || nt_max < 1)))
        return fail(WS_ERR_BADARG, "ws_set_receivers: need nrec >= 0, ijk and nt_max >= 1");
    const ws::Geom &g = ws->g;
    for (int r = 0; r < nrec; ++r) {
        const int i = ijk[3 * r], j = ijk[3 * r + 1], k = ijk[3 * r + 2];
        if (i < 0 || i >= g.nx || j < 0 || j >= g.ny || k < 0 || k >= g.nz)
            return fail(WS_ERR_BADARG, "ws_set_receivers: receiver %d at (%d, %d, %d) outside the grid",
                        r, i, j, k);
    }
    if (nrec > 0 && (long long)nrec * nt_max > (1ll << 40))
        return fail(WS_ERR_BADARG, "ws_set_receivers: trace buffer too large");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_set_receivers");
    ws->model_version++;
    free_receivers(ws);
    ws->nrec = 0;
    ws->nt_max = 0;
    ws->rec_ijk.assign(ijk, ijk + 3 * size_t(nrec));
    ws->trace_start = ws->step;
    if (nrec == 0) return WS_OK;
    WS_CUDA(cudaMalloc(&ws->traces, sizeof(float) * size_t(nrec) * nt_max), "cudaMalloc traces");
    WS_CUDA(cudaMemsetAsync(ws->traces, 0, sizeof(float) * size_t(nrec) * nt_max, ws->stream),
            "zero traces");
    std::vector<long long> pid(nrec);
    for (int r = 0; r < nrec; ++r) pid[r] = ws::pidx(g, ijk[3 * r], ijk[3 * r + 1], ijk[3 * r + 2]);
    WS_CUDA(cudaMalloc(&ws->rec_pidx, sizeof(long long) * nrec), "cudaMalloc receivers");
    WS_CUDA(cudaMemcpyAsync(ws->rec_pidx, pid.data(), sizeof(long long) * nrec,
                            cudaMemcpyHostToDevice, ws->stream),
            "upload receivers");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "upload receivers");
    ws->nrec = nrec;
    ws->nt_max = nt_max;
    return WS_OK;
}

int ws_set_storage(ws_t ws, int storage) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_set_storage: NULL handle");
    if (storage != WS_STORAGE_FP32 && storage != WS_STORAGE_BF16 && storage != WS_STORAGE_FP16)
        return fail(WS_ERR_BADARG, "ws_set_storage: unknown storage %d", storage);
    if (storage == ws->storage) return WS_OK;
    ws->model_version++;
    if (storage != WS_STORAGE_FP32 && (ws->g.nx < kTile16X || ws->g.ny < kTile16Y))
        return fail(WS_ERR_BADARG,
                    "ws_set_storage: 16-bit storage needs nx >= %d and ny >= %d (grid %d x %d)",
                    kTile16X, kTile16Y, ws->g.nx, ws->g.ny);
    // bring the state to FP32 first
    if (ws->storage != WS_STORAGE_FP32) {
        int rc = decode_state16(ws);
        if (rc != WS_OK) return rc;
    }
    if (storage != WS_STORAGE_FP32) {
        const size_t hb = size_t(ws->g.pnx) * ws->g.pny * ws->g.pnz * sizeof(uint16_t);
        for (uint16_t **f : {&ws->buf16[0], &ws->buf16[1], &ws->d16, &ws->w16})
            if (!*f) {
                WS_CUDA(cudaMalloc(f, hb), "cudaMalloc 16-bit field");
                WS_CUDA(cudaMemsetAsync(*f, 0, hb, ws->stream), "zero 16-bit field");
            }
        ws->w16_ok = false;
        if (!ws->scale) {
            WS_CUDA(cudaMalloc(&ws->scale, sizeof(ws::Scale16)), "cudaMalloc scales");
            WS_CUDA(cudaMemsetAsync(ws->scale, 0, sizeof(ws::Scale16), ws->stream), "zero scales");
        }
        int rc = encode_maps16(ws);
        if (rc != WS_OK) return rc;
        ws->storage = storage;
        rc = encode_state16(ws);
        if (rc != WS_OK) return rc;
    } else {
        ws->storage = storage;
    }
    return WS_OK;
}

int ws_set_kernel(ws_t ws, int kernel, int tile_x, int tile_y, int zblock) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_set_kernel: NULL handle");
    if (kernel != WS_KERNEL_AUTO && kernel != WS_KERNEL_DIRECT && kernel != WS_KERNEL_STREAM)
        return fail(WS_ERR_BADARG, "ws_set_kernel: unknown kernel %d", kernel);
    if (zblock < 0) return fail(WS_ERR_BADARG, "ws_set_kernel: zblock must be >= 0");
    ws::StreamTiling t = ws->tiling;
    if (tile_x != 0 || tile_y != 0) {
        if (!ws::stream_tiling_supported(tile_x, tile_y))
            return fail(WS_ERR_BADARG, "ws_set_kernel: unsupported tile %d x %d", tile_x, tile_y);
        t.tx = tile_x;
        t.ty = tile_y;
    }
    t.zb = zblock;
    if (kernel == WS_KERNEL_STREAM && !stream_fits(ws, t))
        return fail(WS_ERR_BADARG, "ws_set_kernel: grid %d x %d is smaller than the tile %d x %d",
                    ws->g.nx, ws->g.ny, t.tx, t.ty);
    const bool box_changed = t.tx != ws->tiling.tx || t.ty != ws->tiling.ty;
    ws->kernel = kernel;
    ws->tiling = t;
    if (box_changed) return encode_maps(ws);
    return WS_OK;
}

int ws_step(ws_t ws, int nsteps) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_step: NULL handle");
    if (nsteps < 0) return fail(WS_ERR_BADARG, "ws_step: nsteps must be >= 0");
    if (!ws->vel_ok) return fail(WS_ERR_STATE, "ws_step: no valid velocity model");
    if (ws->nrec > 0) {
        const long long col = ws->step - ws->trace_start;
        if (col < 0 || col + nsteps > ws->nt_max)
            return fail(WS_ERR_STATE,
                        "ws_step: receivers hold %d steps from step %lld; cannot record steps "
                        "%lld..%lld",
                        ws->nt_max, ws->trace_start, ws->step, ws->step + nsteps - 1);
    }
    ws::StreamTiling tiling{};
    int kern = WS_KERNEL_STREAM;
    if (ws->storage != WS_STORAGE_FP32) {
        tiling.tx = kTile16X;
        tiling.ty = kTile16Y;
        tiling.zb = ws->tiling.zb > 0 ? ws->tiling.zb : default_zblock(ws->g.nz);
        int rc = build_rec_tiles(ws, tiling);
        if (rc != WS_OK) return rc;
        if (!ws->w16_ok) {
            WS_CUDA(ws::launch_model16(ws->w, ws->w16, ws->g, ws->stream), "16-bit model");
            ws->launches++;
            ws->w16_ok = true;
        }
    } else {
        int rc = prepare_fp32(ws, &kern, &tiling);
        if (rc != WS_OK) return rc;
    }
    ws::StepArgs a = base_args(ws);
    for (int s = 0; s < nsteps; ++s) {
        if (ws->storage != WS_STORAGE_FP32) {
            sources_of_step(ws, ws->step, &a.src);
            a.trace_step = ws->step - ws->trace_start;
            double hint = 0.0;
            for (int q = 0; q < a.src.n; ++q)
                hint = std::max(hint, std::fabs((double)a.src.s[q].amp) * ws->wmax);
            cudaError_t e = ws::launch_step_stream16(
                ws->storage, &ws->t16_halo[ws->cur], &ws->t16_d, &ws->t16_w,
                ws->buf16[1 - ws->cur], ws->d16, a, ws->scale, ws->step, (float)hint, tiling,
                ws->nrec > 0 ? ws->rec_ptr : nullptr, ws->rec_entries, ws->stream);
            ws->launches++;
            if (e != cudaSuccess) return cuda_fail(e, "ws_step launch");
        } else {
            const int c = ws->cur;
            a.stall_item = kern == WS_KERNEL_STREAM ? ws->stall_item : -1;
            ws->stall_item = -1;
            int rc = step_fp32(ws, a, kern, tiling, ws->buf[c], &ws->tmap_halo[c], ws->buf[1 - c],
                               &ws->tmap_tile[1 - c], ws->buf[1 - c], ws->step, true,
                               ws->nrec > 0);
            a.stall_item = -1;
            if (rc != WS_OK) return rc;
        }
        ws->cur = 1 - ws->cur;
        ws->step++;
    }
    return WS_OK;
}

int ws_read_traces(ws_t ws, float *out, int on_device) {
    if (!ws || !out) return fail(WS_ERR_BADARG, "ws_read_traces: NULL argument");
    if (ws->nrec == 0) return WS_OK;
    WS_CUDA(cudaMemcpyAsync(out, ws->traces, sizeof(float) * size_t(ws->nrec) * ws->nt_max,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            ws->stream),
            "ws_read_traces");
    if (!on_device) WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_read_traces");
    return WS_OK;
}

int ws_read_field(ws_t ws, float *u, float *u_prev, int on_device) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_read_field: NULL handle");
    int rc = WS_OK;
    if (ws->storage != WS_STORAGE_FP32) {
        rc = decode_state16(ws);
        if (rc != WS_OK) return rc;
    }
    if (u) rc = copy_out(ws, u, ws->buf[ws->cur], on_device);
    if (rc == WS_OK && u_prev) rc = copy_out(ws, u_prev, ws->buf[1 - ws->cur], on_device);
    if (rc != WS_OK) return rc;
    if (!on_device) WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_read_field");
    return WS_OK;
}

int ws_write_field(ws_t ws, const float *u, const float *u_prev, long long step, int on_device) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_write_field: NULL handle");
    if (step < 0) return fail(WS_ERR_BADARG, "ws_write_field: step must be >= 0");
    const size_t fb = field_bytes(ws->g);
    float *dst[2] = {ws->buf[ws->cur], ws->buf[1 - ws->cur]};
    const float *srcs[2] = {u, u_prev};
    for (int b = 0; b < 2; ++b) {
        WS_CUDA(cudaMemsetAsync(dst[b], 0, fb, ws->stream), "ws_write_field");
        if (srcs[b]) {
            int rc = copy_in(ws, dst[b], srcs[b], on_device);
            if (rc != WS_OK) return rc;
        }
    }
    ws->step = step;
    if (ws->storage != WS_STORAGE_FP32) {
        int rc = encode_state16(ws);
        if (rc != WS_OK) return rc;
    }
    if (!on_device) WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_write_field");
    return WS_OK;
}

int ws_get_step(ws_t ws, long long *step) {
    if (!ws || !step) return fail(WS_ERR_BADARG, "ws_get_step: NULL argument");
    *step = ws->step;
    return WS_OK;
}

int ws_synchronize(ws_t ws) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_synchronize: NULL handle");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_synchronize");
    unsigned st = 0;
    WS_CUDA(cudaMemcpy(&st, ws->status, sizeof st, cudaMemcpyDeviceToHost), "ws_synchronize");
    if (st & ws::kStatusTimeout) {
        WS_CUDA(cudaMemset(ws->status, 0, sizeof(unsigned)), "ws_synchronize");
        return fail(WS_ERR_TIMEOUT, "a bounded device wait ran out in a step kernel");
    }
    return WS_OK;
}

int ws_energy(ws_t ws, double *e) {
    if (!ws || !e) return fail(WS_ERR_BADARG, "ws_energy: NULL argument");
    if (!ws->vel_ok) return fail(WS_ERR_STATE, "ws_energy: no valid velocity model");
    if (ws->storage != WS_STORAGE_FP32) {
        int rc = decode_state16(ws);
        if (rc != WS_OK) return rc;
    }
    const ws::Coeffs64 c{kW0, kW1, kW2, kW3, kW4};
    const long long np = ws::energy_partial_count(ws->g.ny, ws->g.nz);
    WS_CUDA(ws::launch_energy_padded(ws->buf[ws->cur], ws->buf[1 - ws->cur], ws->w, ws->g, ws->h, c,
                                     ws->energy, ws->energy + np, ws->stream),
            "energy kernels");
    ws->launches += 2;
    WS_CUDA(cudaMemcpyAsync(e, ws->energy + np, sizeof(double), cudaMemcpyDeviceToHost, ws->stream),
            "ws_energy");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_energy");
    return WS_OK;
}

int ws_energy_noalloc(const float *u, const float *u_prev, const float *v, int nx, int ny, int nz,
                      double h, double dt, double *e, void *cuda_stream) {
    if (!u || !u_prev || !v || !e) return fail(WS_ERR_BADARG, "ws_energy_noalloc: NULL argument");
    if (nx < 1 || ny < 1 || nz < 1 || nx > 65535 || ny > 65535 || nz > 65535)
        return fail(WS_ERR_BADARG, "ws_energy_noalloc: sizes must be in [1, 65535], got %d x %d x %d",
                    nx, ny, nz);
    if (!(h > 0.0) || !(dt > 0.0) || !std::isfinite(h) || !std::isfinite(dt))
        return fail(WS_ERR_BADARG, "ws_energy_noalloc: h and dt must be finite and > 0");
    const long long np = ws::energy_partial_count(ny, nz);
    if (np > ws::kNoAllocMaxPartials)
        return fail(WS_ERR_BADARG,
                    "ws_energy_noalloc: %d x %d x %d needs %lld partial sums, ceil(ny/%d)*nz, but "
                    "the static scratch holds %d",
                    nx, ny, nz, np, ws::energy_rows_per_block(), ws::kNoAllocMaxPartials);
    const ws::Coeffs64 c{kW0, kW1, kW2, kW3, kW4};
    WS_CUDA(ws::launch_energy_noalloc(u, u_prev, v, nx, ny, nz, h, dt, c, e,
                                      static_cast<cudaStream_t>(cuda_stream)),
            "ws_energy_noalloc");
    return WS_OK;
}

}  // extern "C"

namespace {

// Checks shared by ws_forward and ws_adjoint_gradient; selects the kernel and
// makes sure the handle's adjoint scratch matches the run (N = nt_max steps).
int adjoint_prepare(ws_t ws, const char *who, int *kern_out, ws::StreamTiling *tiling_out,
                    AdjointCache **acp) {
    if (!ws->vel_ok) return fail(WS_ERR_STATE, "%s: no valid velocity model", who);
    if (ws->nrec == 0) return fail(WS_ERR_STATE, "%s: no receivers", who);
    if (ws->storage != WS_STORAGE_FP32) return fail(WS_ERR_STATE, "%s: needs FP32 field storage", who);
    const ws::Geom &g = ws->g;
    const int N = ws->nt_max;
    const int C = (int)std::ceil(std::sqrt((double)N));    // states per segment
    const int nck = (N + C - 1) / C;                        // segments
    int kern = WS_KERNEL_STREAM;
    ws::StreamTiling tiling{};
    int rc = prepare_fp32(ws, &kern, &tiling);
    if (rc != WS_OK) return rc;
    const bool maps = kern == WS_KERNEL_STREAM;
    const size_t fb = field_bytes(g);
    const size_t ncell = size_t(g.nx) * g.ny * g.nz;
    const size_t ntr = size_t(ws->nrec) * N;
    const cudaStream_t st = ws->stream;
    AdjointCache *ac = ws->adj;
    if (!ac || ac->N != N || ac->nrec != ws->nrec || ac->kern != kern ||
        (maps && (ac->tx != ws->tiling.tx || ac->ty != ws->tiling.ty))) {
        WS_CUDA(cudaStreamSynchronize(st), "ws_adjoint_gradient");
        delete ws->adj;
        ws->adj = nullptr;
        ac = new (std::nothrow) AdjointCache();
        if (!ac) return fail(WS_ERR_OOM, "ws_adjoint_gradient: host allocation failed");
        ws->adj = ac;
        auto grab = [&](auto **p, size_t bytes) -> cudaError_t {
            void *q = nullptr;
            cudaError_t e = cudaMalloc(&q, bytes);
            if (e == cudaSuccess) {
                ac->mem.push_back(q);
                *p = static_cast<std::remove_reference_t<decltype(**p)> *>(q);
            }
            return e;
        };
        auto field = [&](MappedField *f) -> int {
            WS_CUDA(grab(&f->p, fb), "cudaMalloc adjoint field");
            WS_CUDA(cudaMemsetAsync(f->p, 0, fb, st), "zero adjoint field");
            if (!maps) return WS_OK;
            const int tx = ws->tiling.tx, ty = ws->tiling.ty;
            int r2 = encode_map(&f->halo, f->p, g, tx + 2 * ws::kHalo, ty + 2 * ws::kHalo);
            if (r2 == WS_OK) r2 = encode_map(&f->tile, f->p, g, tx, ty);
            return r2;
        };
        // checkpoints (u^{jC}, u^{jC-1}), j = 1 .. nck-1; segment states; rho
        ac->ck.assign(2 * size_t(nck - 1), nullptr);
        for (auto &c : ac->ck) {
            cudaError_t e = grab(&c, fb);
            if (e != cudaSuccess) {
                delete ws->adj;
                ws->adj = nullptr;
                return cuda_fail(e, "cudaMalloc checkpoint");
            }
        }
        ac->lap.assign(C, nullptr);
        cudaError_t e = cudaSuccess;
        for (auto &f : ac->lap) {   // zeroed: the steps write the interior only
            if (e == cudaSuccess) e = grab(&f, fb);
            if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, fb, st);
        }
        int r3 = e == cudaSuccess ? WS_OK : cuda_fail(e, "cudaMalloc adjoint field");
        for (auto &f : ac->ring)
            if (r3 == WS_OK) r3 = field(&f);
        for (auto &f : ac->rho)
            if (r3 == WS_OK) r3 = field(&f);
        if (r3 == WS_OK) e = grab(&ac->acc, 2 * fb);   // float2 per cell, padded layout
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->partials, sizeof(double) * (ws::residual_partial_count() + 1));
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->r, sizeof(float) * ntr);
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->dd, sizeof(float) * ntr);
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->grad, sizeof(float) * ncell);
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->rec, sizeof(int) * 3 * ws->nrec);
        if (r3 != WS_OK || e != cudaSuccess) {
            delete ws->adj;
            ws->adj = nullptr;
            return r3 != WS_OK ? r3 : cuda_fail(e, "cudaMalloc adjoint scratch");
        }
        ac->N = N;
        ac->nrec = ws->nrec;
        ac->kern = kern;
        ac->tx = ws->tiling.tx;
        ac->ty = ws->tiling.ty;
    } else {
    }
    *kern_out = kern;
    *tiling_out = tiling;
    *acp = ac;
    return WS_OK;
}

// The forward run from rest over N steps: traces recorded, checkpoint pairs
// (u^{jC}, u^{jC-1}) saved; the cache then holds this model version's run.
int adjoint_forward(ws_t ws, AdjointCache *ac, int kern, const ws::StreamTiling &tiling) {
    const ws::Geom &g = ws->g;
    const int N = ws->nt_max;
    const int C = (int)std::ceil(std::sqrt((double)N));
    const size_t fb = field_bytes(g);
    const size_t ntr = size_t(ws->nrec) * N;
    const cudaStream_t st = ws->stream;
    std::vector<float *> &ck = ac->ck;
    int rc = WS_OK;
    ac->fwd_valid = false;
    for (int b = 0; b < 2; ++b) WS_CUDA(cudaMemsetAsync(ws->buf[b], 0, fb, st), "zero fields");
    WS_CUDA(cudaMemsetAsync(ws->traces, 0, sizeof(float) * ntr, st), "zero traces");
    ws->step = 0;
    ws->trace_start = 0;
    ws::StepArgs a = base_args(ws);
    for (int n = 0; n < N; ++n) {
        if (n > 0 && n % C == 0) {
            const int j = n / C;
            WS_CUDA(cudaMemcpyAsync(ck[2 * (j - 1)], ws->buf[ws->cur], fb, cudaMemcpyDeviceToDevice, st),
                    "save checkpoint");
            WS_CUDA(cudaMemcpyAsync(ck[2 * (j - 1) + 1], ws->buf[1 - ws->cur], fb,
                                    cudaMemcpyDeviceToDevice, st),
                    "save checkpoint");
        }
        const int c = ws->cur;
        rc = step_fp32(ws, a, kern, tiling, ws->buf[c], &ws->tmap_halo[c], ws->buf[1 - c],
                       &ws->tmap_tile[1 - c], ws->buf[1 - c], n, true, true);
        if (rc != WS_OK) return rc;
        ws->cur = 1 - c;
        ws->step++;
    }

    ac->fwd_valid = true;
    ac->fwd_version = ws->model_version;
    return WS_OK;
}

}  // namespace

extern "C" {

int ws_forward(ws_t ws) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_forward: NULL handle");
    int kern = WS_KERNEL_STREAM;
    ws::StreamTiling tiling{};
    AdjointCache *ac = nullptr;
    int rc = adjoint_prepare(ws, "ws_forward", &kern, &tiling, &ac);
    if (rc != WS_OK) return rc;
    return adjoint_forward(ws, ac, kern, tiling);
}

int ws_adjoint_gradient(ws_t ws, const float *data, int mode, float *grad_m, double *misfit,
                        int on_device) {
    if (!ws || !data || !grad_m) return fail(WS_ERR_BADARG, "ws_adjoint_gradient: NULL argument");
    if (mode != WS_ADJ_DATA && mode != WS_ADJ_RESIDUAL)
        return fail(WS_ERR_BADARG, "ws_adjoint_gradient: unknown mode %d", mode);
    int kern = WS_KERNEL_STREAM;
    ws::StreamTiling tiling{};
    AdjointCache *ac = nullptr;
    int rc = adjoint_prepare(ws, "ws_adjoint_gradient", &kern, &tiling, &ac);
    if (rc != WS_OK) return rc;
    const ws::Geom &g = ws->g;
    const int N = ws->nt_max;
    const int C = (int)std::ceil(std::sqrt((double)N));    // states per segment
    const int nck = (N + C - 1) / C;                        // segments
    const size_t fb = field_bytes(g);
    const size_t ncell = size_t(g.nx) * g.ny * g.nz;
    const size_t ntr = size_t(ws->nrec) * N;
    const cudaStream_t st = ws->stream;
    for (auto &f : ac->rho) WS_CUDA(cudaMemsetAsync(f.p, 0, fb, st), "zero adjoint field");
    std::vector<float *> &ck = ac->ck;
    std::vector<float *> &lap = ac->lap;
    MappedField *ring = ac->ring;
    MappedField *rho = ac->rho;
    float2 *acc = ac->acc;
    double *partials = ac->partials;
    float *r = ac->r, *grad = on_device ? grad_m : ac->grad;
    const float *d = data;
    int *rec = ac->rec;
    const int np = ws::residual_partial_count();
    WS_CUDA(cudaMemsetAsync(acc, 0, 2 * fb, st), "zero gradient accumulator");
    WS_CUDA(cudaMemcpyAsync(rec, ws->rec_ijk.data(), sizeof(int) * 3 * ws->nrec,
                            cudaMemcpyHostToDevice, st),
            "upload receivers");
    if (!on_device) {
        WS_CUDA(cudaMemcpyAsync(ac->dd, data, sizeof(float) * ntr, cudaMemcpyHostToDevice, st),
                "upload observed data");
        d = ac->dd;
    }

    // 1. forward from rest, recording the traces and the checkpoints; a
    // residual given for the run that ws_forward left in the cache (same
    // model version) needs no new forward run
    if (!(mode == WS_ADJ_RESIDUAL && ac->fwd_valid && ac->fwd_version == ws->model_version)) {
        rc = adjoint_forward(ws, ac, kern, tiling);
        if (rc != WS_OK) return rc;
    }
    ws::StepArgs a = base_args(ws);

    // 2. residual and misfit
    WS_CUDA(ws::launch_residual(mode == WS_ADJ_DATA ? ws->traces : d,
                                mode == WS_ADJ_DATA ? d : nullptr, (long long)ntr, r, partials,
                                partials + np, st),
            "residual kernels");
    ws->launches += 2;

    // 3. backward: rho^k, k = N .. 1, segment by segment, the segment's
    // states recomputed from its checkpoint
    int rc_cur = 0;   // rho[rc_cur] = rho^{k+1}, rho[1 - rc_cur] = rho^{k+2}
    for (int j = nck - 1; j >= 0; --j) {
        const int n0 = j * C, n1 = std::min(n0 + C, N);
        // u^{n0}, u^{n0-1} into the ring, then steps n0 .. n1-1, each storing
        // L u^n into lap[n - n0] (u^{n1} itself is not needed)
        if (j == 0) {
            WS_CUDA(cudaMemsetAsync(ring[0].p, 0, fb, st), "zero initial state");
            WS_CUDA(cudaMemsetAsync(ring[1].p, 0, fb, st), "zero initial state");
        } else {
            WS_CUDA(cudaMemcpyAsync(ring[0].p, ck[2 * (j - 1)], fb, cudaMemcpyDeviceToDevice, st),
                    "restore checkpoint");
            WS_CUDA(cudaMemcpyAsync(ring[1].p, ck[2 * (j - 1) + 1], fb, cudaMemcpyDeviceToDevice, st),
                    "restore checkpoint");
        }
        int uc = 0;   // ring[uc] = u^n
        for (int t = 0; t < n1 - n0; ++t) {
            MappedField &un = ring[uc], &um = ring[1 - uc];
            a.lap = lap[t];
            rc = step_fp32(ws, a, kern, tiling, un.p, &un.halo, um.p, &um.tile, um.p, n0 + t, true,
                           false);
            a.lap = nullptr;
            if (rc != WS_OK) return rc;
            uc = 1 - uc;
        }
        for (int k = n1; k > n0; --k) {
            MappedField &r1 = rho[rc_cur], &r2 = rho[1 - rc_cur];
            rc = step_fp32(ws, a, kern, tiling, r1.p, &r1.halo, r2.p, &r2.tile, r2.p, k, false,
                           false);
            if (rc != WS_OK) return rc;
            rc_cur = 1 - rc_cur;   // rho[rc_cur] = rho^k
            WS_CUDA(ws::launch_inject(rho[rc_cur].p, ws->w, ws->gx, ws->gy, ws->gz, g, rec,
                                      ws->nrec, r, N, k - 1, st),
                    "adjoint injection kernel");
            ws::Sources src{};
            sources_of_step(ws, k - 1, &src);
            WS_CUDA(ws::launch_imaging(rho[rc_cur].p, lap[k - 1 - n0], g, src, ws->gx, ws->gy,
                                       ws->gz, acc, st),
                    "gradient imaging kernel");
            ws->launches += 2;
        }
    }
    const double hdt = ws->h / ws->dt;
    WS_CUDA(ws::launch_finalize_gradient(acc, ws->w, g, hdt * hdt, grad, st),
            "gradient finalize kernel");
    ws->launches++;
    if (!on_device)
        WS_CUDA(cudaMemcpyAsync(grad_m, grad, sizeof(float) * ncell, cudaMemcpyDeviceToHost, st),
                "copy gradient");
    double J = 0.0;
    WS_CUDA(cudaMemcpyAsync(&J, partials + np, sizeof(double), cudaMemcpyDeviceToHost, st),
            "copy misfit");
    WS_CUDA(cudaStreamSynchronize(st), "ws_adjoint_gradient");
    if (misfit) *misfit = J;
    unsigned status = 0;
    WS_CUDA(cudaMemcpy(&status, ws->status, sizeof status, cudaMemcpyDeviceToHost),
            "ws_adjoint_gradient");
    if (status & ws::kStatusTimeout) {
        WS_CUDA(cudaMemset(ws->status, 0, sizeof(unsigned)), "ws_adjoint_gradient");
        return fail(WS_ERR_TIMEOUT, "a bounded device wait ran out in a step kernel");
    }
    return WS_OK;
}

int ws_autotune(ws_t ws, int *tile_x, int *tile_y, int *zblock) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_autotune: NULL handle");
    if (!ws->vel_ok) return fail(WS_ERR_STATE, "ws_autotune: no valid velocity model");
    if (ws->storage != WS_STORAGE_FP32)
        return fail(WS_ERR_STATE, "ws_autotune: tunes the FP32 streaming kernel only");
    const ws::Geom &g = ws->g;
    ws::StreamTiling best{0, 0, 0};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(std::make_tuple(g.nx, g.ny, g.nz));
        if (it != g_tune_cache.end()) best = it->second;
    }
    if (best.tx == 0) {
        Scratch sc(ws->stream);
        float *out = nullptr;
        WS_CUDA(sc.alloc(&out, field_bytes(g)), "cudaMalloc tuning field");
        cudaEvent_t e0, e1;
        WS_CUDA(cudaEventCreate(&e0), "ws_autotune");
        WS_CUDA(cudaEventCreate(&e1), "ws_autotune");
        ws::StepArgs a = base_args(ws);
        a.src.n = 0;
        float best_ms = 1e30f;
        const ws::StreamTiling keep = ws->tiling;
        int rc = WS_OK;
        for (const auto &tc : kTileCands) {
            ws::StreamTiling t{tc[0], tc[1], 0};
            if (!stream_fits(ws, t)) continue;
            int slots = 0;
            cudaError_t e = ws::stream_slots(t.tx, t.ty, false, &slots);
            if (e != cudaSuccess) { rc = cuda_fail(e, "ws_autotune"); break; }
            ws->tiling = t;
            if ((rc = encode_maps(ws)) != WS_OK) break;
            const long long tiles =
                (long long)((g.nx + t.tx - 1) / t.tx) * ((g.ny + t.ty - 1) / t.ty);
            for (int zb : zblock_candidates(g.nz, tiles, slots)) {
                t.zb = zb;
                const int c = ws->cur;
                float ms = 0.f;
                for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                    if (rep == 1) e = cudaEventRecord(e0, ws->stream);
                    if (e == cudaSuccess)
                        e = ws::launch_step_stream(&ws->tmap_halo[c], &ws->tmap_tile[1 - c],
                                                   &ws->tmap_w, out, a, t, nullptr, nullptr,
                                                   ws->stream);
                    ws->launches++;
                }
                if (e == cudaSuccess) e = cudaEventRecord(e1, ws->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) { rc = cuda_fail(e, "ws_autotune"); break; }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
            if (rc != WS_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ws->tiling = keep;
        if (rc != WS_OK) {
            encode_maps(ws);
            return rc;
        }
        if (best.tx != 0) {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            g_tune_cache[std::make_tuple(g.nx, g.ny, g.nz)] = best;
        }
    }
    if (best.tx == 0) {   // no tile fits: the direct kernel
        ws->kernel = WS_KERNEL_DIRECT;
    } else {
        ws->kernel = WS_KERNEL_STREAM;
        ws->tiling = best;
        int rc = encode_maps(ws);
        if (rc != WS_OK) return rc;
    }
    if (tile_x) *tile_x = best.tx;
    if (tile_y) *tile_y = best.ty;
    if (zblock) *zblock = best.zb;
    return WS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches

namespace {

void batch_drop_graphs(ws_batch_t b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

void batch_free(ws_batch_t b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    cudaFree(b->d_shots);
    cudaFree(b->d_items);
    cudaFree(b->d_src);
    cudaFree(b->status);
    for (cudaEvent_t e : {b->ev, b->t0, b->t1, b->t2})
        if (e) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Configure every shot for tile tx x ty with z-blocks for m x slots items
// (m = 0: each shot's default) and rebuild the item table: shots in order
// of decreasing size, each shot's items block-major.
int batch_configure(ws_batch_t b, int tx, int ty, int m) {
    int slots = 0;
    WS_CUDA(ws::stream_slots(tx, ty, true, &slots), "ws_batch_step");
    const int n = (int)b->shots.size();
    long long cells = 0;
    for (ws_t ws : b->shots) cells += (long long)ws->g.nx * ws->g.ny * ws->g.nz;
    std::vector<int> order(n);
    for (int q = 0; q < n; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const ws::Geom &gx = b->shots[x]->g, &gy = b->shots[y]->g;
        return (long long)gx.nx * gx.ny * gx.nz > (long long)gy.nx * gy.ny * gy.nz;
    });
    std::vector<int2> items;
    b->zb.assign(n, 0);
    for (int q : order) {
        ws_t ws = b->shots[q];
        const ws::Geom &g = ws->g;
        const long long tiles = (long long)((g.nx + tx - 1) / tx) * ((g.ny + ty - 1) / ty);
        int zb = default_zblock(g.nz);
        if (m > 0) {   // this shot's share of m waves, rounded down to whole blocks
            const double share = double(g.nx) * g.ny * g.nz / double(cells);
            const long long want = std::max<long long>(1, std::llround(m * slots * share));
            const long long blocks = std::max<long long>(1, want / tiles);
            zb = (int)std::min<long long>(g.nz, std::max<long long>(8, (g.nz + blocks - 1) / blocks));
        }
        b->zb[q] = zb;
        if (ws->tiling.tx != tx || ws->tiling.ty != ty) {
            ws->tiling.tx = tx;
            ws->tiling.ty = ty;
            int rc = encode_maps(ws);
            if (rc != WS_OK) return rc;
        }
        int rc = build_rec_tiles(ws, ws::StreamTiling{tx, ty, zb});
        if (rc != WS_OK) return rc;
        const long long nit = tiles * ((g.nz + zb - 1) / zb);
        for (long long l = 0; l < nit; ++l) items.push_back(make_int2(q, (int)l));
    }
    if ((long long)items.size() > INT32_MAX / 2)
        return fail(WS_ERR_BADARG, "ws_batch_step: too many work items");
    batch_drop_graphs(b);
    cudaFree(b->d_items);
    b->d_items = nullptr;
    WS_CUDA(cudaMalloc(&b->d_items, sizeof(int2) * items.size()), "cudaMalloc batch items");
    WS_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(int2) * items.size(),
                            cudaMemcpyHostToDevice, b->stream),
            "upload batch items");
    WS_CUDA(cudaStreamSynchronize(b->stream), "upload batch items");
    b->nitems = (int)items.size();
    b->tx = tx;
    b->ty = ty;
    b->cfg = ws_batch::Cand{tx, ty, m};
    return WS_OK;
}

// Descriptors and source samples of the next nsteps steps.
int batch_upload(ws_batch_t b, int nsteps) {
    const int n = (int)b->shots.size();
    // a shot may have been used on its own since the table was built: its
    // tensor-map boxes and receiver table must match the batch's tile (a
    // box larger than the kernel's ring slot would overrun shared memory)
    for (int q = 0; q < n; ++q) {
        ws_t ws = b->shots[q];
        if (ws->tiling.tx != b->tx || ws->tiling.ty != b->ty) {
            ws->tiling.tx = b->tx;
            ws->tiling.ty = b->ty;
            int rc = encode_maps(ws);
            if (rc != WS_OK) return rc;
        }
        int rc = build_rec_tiles(ws, ws::StreamTiling{b->tx, b->ty, b->zb[q]});
        if (rc != WS_OK) return rc;
    }
    size_t total = 0;
    for (ws_t ws : b->shots) total += ws->src.size() * size_t(nsteps);
    if (total > b->src_cap) {
        cudaFree(b->d_src);
        b->d_src = nullptr;
        b->src_cap = 0;
        WS_CUDA(cudaMalloc(&b->d_src, sizeof(ws::SourceSample) * std::max<size_t>(total, 1)),
                "cudaMalloc batch sources");
        b->src_cap = total;
    }
    std::vector<ws::SourceSample> src(total);
    std::vector<ws::BatchShot> d(n);
    size_t off = 0;
    for (int q = 0; q < n; ++q) {
        ws_t ws = b->shots[q];
        ws::BatchShot &x = d[q];
        for (int p = 0; p < 2; ++p) {
            x.halo[p] = ws->tmap_halo[p];
            x.tile[p] = ws->tmap_tile[p];
            x.buf[p] = ws->buf[p];
        }
        x.w = ws->tmap_w;
        x.gx = ws->gx;
        x.gy = ws->gy;
        x.gz = ws->gz;
        x.nsrc = (int)ws->src.size();
        x.src = b->d_src + off;
        ws::Sources one{};
        for (int t = 0; t < nsteps; ++t) {
            sources_of_step(ws, ws->step + t, &one);
            for (int k = 0; k < one.n; ++k) src[off + size_t(t) * one.n + k] = one.s[k];
        }
        off += size_t(x.nsrc) * nsteps;
        const bool rec = ws->nrec > 0;
        x.traces = rec ? ws->traces : nullptr;
        x.rec_ptr = rec ? ws->rec_ptr : nullptr;
        x.rec = rec ? ws->rec_entries : nullptr;
        x.g = ws->g;
        x.trace_col0 = ws->step - ws->trace_start;
        x.nt_max = ws->nt_max;
        x.cur0 = ws->cur;
        x.zb = b->zb[q];
        x.tiles_x = (ws->g.nx + b->tx - 1) / b->tx;
        x.ntiles = x.tiles_x * ((ws->g.ny + b->ty - 1) / b->ty);
    }
    if (!b->d_shots)
        WS_CUDA(cudaMalloc(&b->d_shots, sizeof(ws::BatchShot) * n), "cudaMalloc batch shots");
    WS_CUDA(cudaMemcpyAsync(b->d_shots, d.data(), sizeof(ws::BatchShot) * n,
                            cudaMemcpyHostToDevice, b->stream),
            "upload batch shots");
    if (total)
        WS_CUDA(cudaMemcpyAsync(b->d_src, src.data(), sizeof(ws::SourceSample) * total,
                                cudaMemcpyHostToDevice, b->stream),
                "upload batch sources");
    // the host vectors die here
    WS_CUDA(cudaStreamSynchronize(b->stream), "upload batch shots");
    return WS_OK;
}

ws::Coeffs step_coeffs() { return ws::Coeffs{(float)kW1, (float)kW2, (float)kW3, (float)kW4}; }

// Run nsteps steps from the uploaded descriptors, as a CUDA graph.
int batch_run(ws_batch_t b, int nsteps) {
    const ws::Coeffs c = step_coeffs();
    auto it = b->graphs.find(nsteps);
    if (it == b->graphs.end()) {
        int slots = 0;
        WS_CUDA(ws::stream_slots(b->tx, b->ty, true, &slots), "ws_batch_step");
        WS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
                "ws_batch_step capture");
        cudaError_t e = cudaSuccess;
        for (int t = 0; t < nsteps && e == cudaSuccess; ++t)
            e = ws::launch_step_batch(b->d_shots, b->d_items, b->nitems, t, c, b->status, b->tx,
                                      b->ty, b->stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "ws_batch_step graph");
        it = b->graphs.emplace(nsteps, exec).first;
    }
    WS_CUDA(cudaGraphLaunch(it->second, b->stream), "ws_batch_step graph launch");
    b->launches += nsteps;
    return WS_OK;
}

void batch_advance(ws_batch_t b, int nsteps) {
    for (ws_t ws : b->shots) {
        if (nsteps & 1) ws->cur = 1 - ws->cur;
        ws->step += nsteps;
    }
}

}  // namespace

extern "C" {

int ws_batch_create(ws_batch_t *out, int nshots, const ws_t *shots) {
    if (!out) return fail(WS_ERR_BADARG, "ws_batch_create: out is NULL");
    *out = nullptr;
    if (nshots < 1 || !shots) return fail(WS_ERR_BADARG, "ws_batch_create: need nshots >= 1 handles");
    for (int q = 0; q < nshots; ++q) {
        if (!shots[q]) return fail(WS_ERR_BADARG, "ws_batch_create: handle %d is NULL", q);
        for (int r = 0; r < q; ++r)
            if (shots[r] == shots[q])
                return fail(WS_ERR_BADARG, "ws_batch_create: handle %d appears twice", q);
    }
    ws_batch_t b = new (std::nothrow) ws_batch();
    if (!b) return fail(WS_ERR_OOM, "ws_batch_create: host allocation failed");
    b->shots.assign(shots, shots + nshots);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&b->ev, &b->t0, &b->t1, &b->t2})
        if (e == cudaSuccess) e = cudaEventCreate(ev);
    if (e == cudaSuccess) e = cudaMalloc(&b->status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "ws_batch_create");
    }
    // online tuning candidates: every tile that fits every shot, z-blocks
    // for 1, 2, 4, 8 x the resident CTAs and the per-shot default
    for (const auto &tc : kTileCands) {
        bool fits = true;
        for (ws_t ws : b->shots) fits = fits && ws->g.nx >= tc[0] && ws->g.ny >= tc[1];
        if (!fits) continue;
        for (int m : {0, 1, 2, 3, 4, 6}) b->todo.push_back(ws_batch::Cand{tc[0], tc[1], m});
    }
    if (b->todo.empty()) {
        batch_free(b);
        return fail(WS_ERR_BADARG, "ws_batch_create: some shot is smaller than every tile "
                                   "(needs nx >= 32 and ny >= 8)");
    }
    *out = b;
    return WS_OK;
}

int ws_batch_destroy(ws_batch_t b) {
    batch_free(b);
    return WS_OK;
}

int ws_batch_set_tiling(ws_batch_t b, int tile_x, int tile_y, int zmul) {
    if (!b) return fail(WS_ERR_BADARG, "ws_batch_set_tiling: NULL batch");
    if (tile_x == 0 && tile_y == 0) {   // back to tuning
        b->fixed = false;
        return WS_OK;
    }
    if (!ws::stream_tiling_supported(tile_x, tile_y) || zmul < 0)
        return fail(WS_ERR_BADARG, "ws_batch_set_tiling: unsupported tile %d x %d or zmul %d", tile_x,
                    tile_y, zmul);
    for (ws_t ws : b->shots)
        if (ws->g.nx < tile_x || ws->g.ny < tile_y)
            return fail(WS_ERR_BADARG, "ws_batch_set_tiling: a shot is smaller than the tile");
    b->fixed = true;
    b->best = ws_batch::Cand{tile_x, tile_y, zmul};
    return WS_OK;
}

int ws_batch_get_tiling(ws_batch_t b, int *tile_x, int *tile_y, int *zmul) {
    if (!b) return fail(WS_ERR_BADARG, "ws_batch_get_tiling: NULL batch");
    if (tile_x) *tile_x = b->best.tx;
    if (tile_y) *tile_y = b->best.ty;
    if (zmul) *zmul = b->best.m;
    return WS_OK;
}

int ws_batch_step(ws_batch_t b, int nsteps) {
    if (!b) return fail(WS_ERR_BADARG, "ws_batch_step: NULL batch");
    if (nsteps < 0) return fail(WS_ERR_BADARG, "ws_batch_step: nsteps must be >= 0");
    for (size_t q = 0; q < b->shots.size(); ++q) {
        ws_t ws = b->shots[q];
        if (!ws->vel_ok) return fail(WS_ERR_STATE, "ws_batch_step: shot %zu has no velocity model", q);
        if (ws->storage != WS_STORAGE_FP32)
            return fail(WS_ERR_STATE, "ws_batch_step: shot %zu does not use FP32 storage", q);
        if (ws->nrec > 0) {
            const long long col = ws->step - ws->trace_start;
            if (col < 0 || col + nsteps > ws->nt_max)
                return fail(WS_ERR_STATE, "ws_batch_step: shot %zu can record %d steps from step "
                                          "%lld, not steps %lld..%lld",
                            q, ws->nt_max, ws->trace_start, ws->step, ws->step + nsteps - 1);
        }
    }
    if (nsteps == 0) return WS_OK;
    // order after the shots' own pending work
    for (ws_t ws : b->shots) {
        WS_CUDA(cudaEventRecord(b->ev, ws->stream), "ws_batch_step");
        WS_CUDA(cudaStreamWaitEvent(b->stream, b->ev, 0), "ws_batch_step");
    }
    int done = 0, rc = WS_OK;
    const ws::Coeffs c = step_coeffs();
    // online tuning: each untried candidate takes two real steps (every
    // tiling computes the same values); the second one is timed
    while (!b->fixed && !b->tuned && nsteps - done >= 2 && rc == WS_OK) {
        const ws_batch::Cand cd = b->todo.back();
        b->todo.pop_back();
        if ((rc = batch_configure(b, cd.tx, cd.ty, cd.m)) != WS_OK) break;
        if ((rc = batch_upload(b, 2)) != WS_OK) break;
        cudaError_t e = cudaEventRecord(b->t0, b->stream);
        if (e == cudaSuccess)
            e = ws::launch_step_batch(b->d_shots, b->d_items, b->nitems, 0, c, b->status, b->tx,
                                      b->ty, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->stream);
        if (e == cudaSuccess)
            e = ws::launch_step_batch(b->d_shots, b->d_items, b->nitems, 1, c, b->status, b->tx,
                                      b->ty, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->t2, b->stream);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventSynchronize(b->t2);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->t1, b->t2);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "ws_batch_step tuning");
            break;
        }
        b->launches += 2;
        batch_advance(b, 2);
        done += 2;
        if (ms < b->best_ms) {
            b->best_ms = ms;
            b->best = cd;
        }
        if (b->todo.empty()) b->tuned = true;
    }
    if (rc == WS_OK && done < nsteps) {
        // the best candidate; while tuning is incomplete, 64 x 8 with 2 x CTAs items
        const ws_batch::Cand want = b->best.tx ? b->best : ws_batch::Cand{64, 8, 2};
        if (b->cfg.tx != want.tx || b->cfg.ty != want.ty || b->cfg.m != want.m)
            rc = batch_configure(b, want.tx, want.ty, want.m);
        if (rc == WS_OK) rc = batch_upload(b, nsteps - done);
        if (rc == WS_OK) rc = batch_run(b, nsteps - done);
        if (rc == WS_OK) batch_advance(b, nsteps - done);
    }
    // later work on each shot's stream follows the batch
    cudaError_t e = cudaEventRecord(b->ev, b->stream);
    for (ws_t ws : b->shots)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ws->stream, b->ev, 0);
    if (rc == WS_OK && e != cudaSuccess) rc = cuda_fail(e, "ws_batch_step");
    return rc;
}

int ws_batch_synchronize(ws_batch_t b) {
    if (!b) return fail(WS_ERR_BADARG, "ws_batch_synchronize: NULL batch");
    WS_CUDA(cudaStreamSynchronize(b->stream), "ws_batch_synchronize");
    unsigned st = 0;
    WS_CUDA(cudaMemcpy(&st, b->status, sizeof st, cudaMemcpyDeviceToHost), "ws_batch_synchronize");
    if (st & ws::kStatusTimeout) {
        WS_CUDA(cudaMemset(b->status, 0, sizeof(unsigned)), "ws_batch_synchronize");
        return fail(WS_ERR_TIMEOUT, "a bounded device wait ran out in a batched step");
    }
    return WS_OK;
}

long long ws_batch_launch_count(ws_batch_t b) { return b ? b->launches : -1; }

int ws_test_stall(ws_t ws, int item) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_test_stall: NULL handle");
    if (item < -1) return fail(WS_ERR_BADARG, "ws_test_stall: item must be >= -1");
    ws->stall_item = item;
    return WS_OK;
}

long long ws_launch_count(ws_t ws) { return ws ? ws->launches : -1; }

}  // extern "C"
