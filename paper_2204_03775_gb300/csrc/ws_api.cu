// Host side of the C ABI declared in include/wavestep.h: the handle, its
// buffers and tensor maps, and the entry points of the forward stepper.
#include "ws_host.h"

namespace wsh {

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

size_t field_bytes(const ws::Geom &g) {
    return size_t(g.pnx) * size_t(g.pny) * size_t(g.pnz) * sizeof(float);
}

// A tensor map of a padded field over its interior only: origin at interior
// cell (0, 0, 0) (a 128-byte aligned address), extent nx x ny x nz, the
// padded pitches. The kernels' boxes that reach past the interior (the 4-cell
// halo of the edge tiles, the ragged end of the last tiles) are filled with
// zeros by the copy engine without reading memory: exactly the zero halo,
// and no DRAM traffic for halo or row padding.
int encode_map(CUtensorMap *map, void *base, const ws::Geom &g, int bx, int by,
               int elem_bytes) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode_fn();
    if (!enc) return fail(WS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    cuuint64_t strides[2] = {(cuuint64_t)g.pnx * elem_bytes, (cuuint64_t)g.plane * elem_bytes};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    void *origin = static_cast<char *>(base) + ws::pidx(g, 0, 0, 0) * elem_bytes;
    CUresult r = enc(map, dt, 3, origin, dims, strides, box, estr,
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
// Gcell/s against 387.2 at 342 and 376.7 at 64, 64 x 8 tiles). The blocks
// are cut so that the last one is about a quarter as long as the others:
// items run in block order, so the launch ends on short items and its tail,
// when fewer CTAs than SM slots remain, is short (1024^3, four blocks of 241
// and one of 60: FP32 393.5 against 390.9 Gcell/s for five of 205; 16-bit
// storage 493 against 485 with equal blocks, 64 x 24 tiles).
int default_zblock(int nz) {
    const int blocks = std::max(1, (int)std::lround(nz / 200.0));
    if (blocks == 1) return nz;
    return (4 * nz + 4 * blocks - 4) / (4 * blocks - 3);   // ceil(nz / (blocks - 3/4))
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
    ws->rec_tiling_tx = ws->rec_tiling_ty = ws->rec_tiling_rows = 0;
}

// Receiver table of the streaming kernels for tile t: per (tile, consumer
// warp) a range of entries sorted by k. Thread owner = (row pair) * tx/4 + x
// quad, lane = 4 * (row within the thread's rows) + x cell.
int build_rec_tiles(ws_t ws, const ws::StreamTiling &t, int rows) {
    if (ws->nrec == 0) return WS_OK;
    if (ws->rec_tiling_tx == t.tx && ws->rec_tiling_ty == t.ty && ws->rec_tiling_rows == rows)
        return WS_OK;
    const int tiles_x = (ws->g.nx + t.tx - 1) / t.tx;
    const int tiles_y = (ws->g.ny + t.ty - 1) / t.ty;
    const int warps = t.tx / 4 * (t.ty / rows) / 32;   // consumer warps of a CTA
    const int ntiles = tiles_x * tiles_y * warps;   // (tile, warp) ranges
    std::vector<std::pair<int, ws::RecEntry>> e(ws->nrec);
    for (int r = 0; r < ws->nrec; ++r) {
        const int i = ws->rec_ijk[3 * r], j = ws->rec_ijk[3 * r + 1], k = ws->rec_ijk[3 * r + 2];
        const int tile = (j / t.ty) * tiles_x + (i / t.tx);
        const int li = i - (i / t.tx) * t.tx, lj = j - (j / t.ty) * t.ty;
        const int owner = (lj / rows) * (t.tx / 4) + li / 4;
        e[r] = {tile * warps + owner / 32, ws::RecEntry{k, owner, (lj % rows) * 4 + li % 4, r}};
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
    ws->rec_tiling_rows = rows;
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
    // the cells of each axis whose factor is exactly 1 (a contiguous middle
    // range: the profile rises monotonically from both faces)
    auto ones = [](const std::vector<float> &p, int *lo, int *hi) {
        const int n = (int)p.size();
        int a = 0;
        while (a < n && p[a] != 1.0f) ++a;
        int b = a;
        while (b < n && p[b] == 1.0f) ++b;
        *lo = a;
        *hi = b;
    };
    ones(px, &ws->free16.x0, &ws->free16.x1);
    ones(py, &ws->free16.y0, &ws->free16.y1);
    ones(pz, &ws->free16.z0, &ws->free16.z1);
    WS_CUDA(cudaMemcpyAsync(ws->gx, px.data(), 4 * px.size(), cudaMemcpyHostToDevice, ws->stream),
            "upload taper");
    WS_CUDA(cudaMemcpyAsync(ws->gy, py.data(), 4 * py.size(), cudaMemcpyHostToDevice, ws->stream),
            "upload taper");
    WS_CUDA(cudaMemcpyAsync(ws->gz, pz.data(), 4 * pz.size(), cudaMemcpyHostToDevice, ws->stream),
            "upload taper");
    WS_CUDA(cudaStreamSynchronize(ws->stream), "upload taper");
    return WS_OK;
}

int encode_maps16(ws_t ws, int ty) {
    const ws::Geom &g = ws->g;
    int rc = WS_OK;
    for (int b = 0; b < 2 && rc == WS_OK; ++b)
        rc = encode_map(&ws->t16_halo[b], ws->buf16[b], g, kTile16X + 16, ty + 2 * ws::kHalo, 2);
    if (rc == WS_OK) rc = encode_map(&ws->t16_d, ws->d16, g, kTile16X, ty, 2);
    if (rc == WS_OK) rc = encode_map(&ws->t16_w, ws->w16, g, kTile16X, ty, 2);
    ws->t16_ty = rc == WS_OK ? ty : 0;
    return rc;
}

// The 16-bit kernel's tile height for this grid: the one ws_set_kernel chose
// if the grid holds it, else the first of kTile16Ys that the grid holds.
int pick_tile16(const ws_t ws) {
    if (ws->tile16_y > 0 && ws->g.ny >= ws->tile16_y) return ws->tile16_y;
    for (int ty : kTile16Ys)
        if (ws->g.ny >= ty) return ty;
    return 0;
}

// Planes per work item of the 16-bit kernel: the FP32 kernel's default,
// shortened on small grids to about two full waves of the resident CTAs.
int default_zblock16(const ws::Geom &g, int ty) {
    int zb = default_zblock(g.nz), slots = 0;
    if (ws::stream16_slots(ty, &slots) != cudaSuccess) return zb;
    const long long tiles = (long long)((g.nx + kTile16X - 1) / kTile16X) * ((g.ny + ty - 1) / ty);
    const long long blocks = std::max<long long>(1, 2LL * slots / tiles);
    const int zs = (int)std::max<long long>(8, (g.nz + blocks - 1) / blocks);
    return std::min(zb, std::min(zs, g.nz));
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

}  // namespace wsh

using namespace wsh;

namespace {

// Padding canaries (test hooks). A padded field is the interior, the 4-cell
// zero halo around it, and the row padding beyond the halo in x; no kernel
// may write outside the interior, and nothing read beyond the halo may reach
// a result.
__device__ __forceinline__ int pad_class(const ws::Geom &g, long long idx) {
    const int x = (int)(idx % g.pnx);
    const long long r = idx / g.pnx;
    const int y = (int)(r % g.pny), z = (int)(r / g.pny);
    const bool ix = x >= ws::kXOff && x < ws::kXOff + g.nx;
    const bool iy = y >= ws::kHalo && y < g.ny + ws::kHalo;
    const bool iz = z >= ws::kHalo && z < g.nz + ws::kHalo;
    if (ix && iy && iz) return 0;                                     // interior
    const bool hx = x >= ws::kXOff - ws::kHalo && x < ws::kXOff + g.nx + ws::kHalo;
    return (hx && y < g.ny + 2 * ws::kHalo && z < g.nz + 2 * ws::kHalo) ? 1 : 2;   // halo : padding
}

template <class T>
__global__ void fill_pad_kernel(T *f, ws::Geom g, T canary) {
    const long long n = (long long)g.pnx * g.pny * g.pnz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x)
        if (pad_class(g, idx) == 2) f[idx] = canary;
}

// Cells that differ from what they must hold: 0 in the halo, the canary in
// the padding (bit patterns).
template <class T>
__global__ void check_pad_kernel(const T *f, ws::Geom g, T canary, unsigned long long *bad) {
    const long long n = (long long)g.pnx * g.pny * g.pnz;
    unsigned long long c = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = pad_class(g, idx);
        if ((k == 1 && f[idx] != T(0)) || (k == 2 && f[idx] != canary)) ++c;
    }
    if (c) atomicAdd(bad, c);
}

constexpr uint32_t kCanary32 = 0x7fc00000u;   // FP32 quiet NaN
constexpr uint16_t kCanaryF16 = 0x7e00u;      // FP16 quiet NaN
constexpr uint16_t kCanaryBf16 = 0x7fc0u;     // BF16 quiet NaN

// Every field buffer of the handle with its canary: the FP32 state and
// model, and with 16-bit storage the 16-bit state and model too.
template <class F>
int for_each_field(ws_t ws, F &&fn) {
    const uint16_t c16 = ws->storage == WS_STORAGE_BF16 ? kCanaryBf16 : kCanaryF16;
    for (float *f : {ws->buf[0], ws->buf[1], ws->w}) {
        int rc = fn(reinterpret_cast<uint32_t *>(f), kCanary32);
        if (rc != WS_OK) return rc;
    }
    if (ws->storage != WS_STORAGE_FP32) {
        for (uint16_t *f : {ws->buf16[0], ws->buf16[1], ws->d16}) {
            int rc = fn(f, c16);
            if (rc != WS_OK) return rc;
        }
        return fn(ws->w16, kCanaryF16);
    }
    return WS_OK;
}

constexpr int kPadGrid = 1216, kPadBlock = 256;

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
    if (storage != WS_STORAGE_FP32 && (ws->g.nx < kTile16X || pick_tile16(ws) == 0))
        return fail(WS_ERR_BADARG,
                    "ws_set_storage: 16-bit storage needs nx >= %d and ny >= %d (grid %d x %d)",
                    kTile16X, kTile16Ys[kNumTile16Ys - 1], ws->g.nx, ws->g.ny);
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
        int rc = encode_maps16(ws, pick_tile16(ws));
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
        const bool fp32 = ws::stream_tiling_supported(tile_x, tile_y);
        const bool t16 = ws::stream16_tiling_supported(tile_x, tile_y);
        if (!fp32 && !t16)
            return fail(WS_ERR_BADARG, "ws_set_kernel: unsupported tile %d x %d", tile_x, tile_y);
        if (t16) {   // the 16-bit kernel's tile; the FP32 tile only if that kernel has it too
            if (ws->g.nx < tile_x || ws->g.ny < tile_y)
                return fail(WS_ERR_BADARG,
                            "ws_set_kernel: grid %d x %d is smaller than the tile %d x %d",
                            ws->g.nx, ws->g.ny, tile_x, tile_y);
            ws->tile16_y = tile_y;
        }
        if (fp32) {
            t.tx = tile_x;
            t.ty = tile_y;
        }
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
        tiling.ty = pick_tile16(ws);
        tiling.zb = ws->tiling.zb > 0 ? ws->tiling.zb : default_zblock16(ws->g, tiling.ty);
        if (tiling.ty != ws->t16_ty) {
            int rc = encode_maps16(ws, tiling.ty);
            if (rc != WS_OK) return rc;
        }
        int rc = build_rec_tiles(ws, tiling, kRows16);
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
            a.stall_item = ws->stall_item;
            ws->stall_item = -1;
            const ws::Maps16In maps{&ws->t16_halo[ws->cur], &ws->t16_d, &ws->t16_w,
                                    ws->buf16[1 - ws->cur], ws->d16};
            cudaError_t e = ws::launch_step_stream16(
                ws->storage, maps, a, ws->scale, ws->step, (float)hint, ws->free16, tiling,
                ws->nrec > 0 ? ws->rec_ptr : nullptr, ws->rec_entries, ws->stream);
            a.stall_item = -1;
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

int ws_test_stall(ws_t ws, int item) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_test_stall: NULL handle");
    if (item < -1) return fail(WS_ERR_BADARG, "ws_test_stall: item must be >= -1");
    ws->stall_item = item;
    return WS_OK;
}

long long ws_launch_count(ws_t ws) { return ws ? ws->launches : -1; }

int ws_test_fill_padding(ws_t ws) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_test_fill_padding: NULL handle");
    int rc = for_each_field(ws, [&](auto *f, auto canary) {
        fill_pad_kernel<<<kPadGrid, kPadBlock, 0, ws->stream>>>(f, ws->g, canary);
        ws->launches++;
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? WS_OK : cuda_fail(e, "ws_test_fill_padding");
    });
    if (rc != WS_OK) return rc;
    WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_test_fill_padding");
    return WS_OK;
}

int ws_test_check_padding(ws_t ws, long long *bad) {
    if (!ws || !bad) return fail(WS_ERR_BADARG, "ws_test_check_padding: NULL argument");
    unsigned long long *d = nullptr;
    WS_CUDA(cudaMalloc(&d, sizeof *d), "ws_test_check_padding");
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof *d, ws->stream);
    int rc = e == cudaSuccess ? WS_OK : cuda_fail(e, "ws_test_check_padding");
    if (rc == WS_OK)
        rc = for_each_field(ws, [&](auto *f, auto canary) {
            check_pad_kernel<<<kPadGrid, kPadBlock, 0, ws->stream>>>(f, ws->g, canary, d);
            ws->launches++;
            cudaError_t e2 = cudaGetLastError();
            return e2 == cudaSuccess ? WS_OK : cuda_fail(e2, "ws_test_check_padding");
        });
    unsigned long long h = 0;
    if (rc == WS_OK) {
        e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, ws->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ws->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "ws_test_check_padding");
    }
    cudaFree(d);
    if (rc == WS_OK) *bad = (long long)h;
    return rc;
}

}  // extern "C"
