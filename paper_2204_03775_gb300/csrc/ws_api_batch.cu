// Host side of the tiling autotuner (ws_autotune) and of batched shots
// (ws_batch_*): one launch per step over every shot's items, runs of steps
// replayed as CUDA graphs, the tile and z-block rule tuned online.
#include <sys/stat.h>
#include <unistd.h>

#include <cstdlib>
#include <string>

#include "ws_host.h"

using namespace wsh;

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

namespace {

// Tiles of the streaming kernel, in the order the tuners try them. 64 x 16
// and 64 x 32 are left out: with 9 and 17 warps per CTA one SM sub-partition
// holds 5 of their warps, which caps them at 96 registers per thread, and
// they spill (measured at less than half the speed of these three).
constexpr int kTileCands[3][2] = {{64, 8}, {32, 8}, {32, 16}};

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

// Tilings chosen by ws_autotune, keyed by (GPU name, storage, nx, ny, nz):
// kept in memory and in a text file (one "gpu|storage|nx|ny|nz|tx|ty|zb"
// line per entry) at $WS_TUNE_CACHE, else $XDG_CACHE_HOME/wavestep/tune.txt,
// else $HOME/.cache/wavestep/tune.txt, so a later process on the same GPU
// model reuses them. Lines that do not parse are ignored; a file that cannot
// be written leaves the in-memory cache only.
using TuneKey = std::tuple<std::string, int, int, int, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, ws::StreamTiling> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_cache_path() {
    if (const char *p = std::getenv("WS_TUNE_CACHE")) return p;
    if (const char *x = std::getenv("XDG_CACHE_HOME")) return std::string(x) + "/wavestep/tune.txt";
    if (const char *h = std::getenv("HOME")) return std::string(h) + "/.cache/wavestep/tune.txt";
    return std::string();
}

// Call with g_tune_mutex held.
void tune_cache_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char *bar = std::strchr(line, '|');
        if (!bar) continue;
        int st, nx, ny, nz, tx, ty, zb;
        if (std::sscanf(bar + 1, "%d|%d|%d|%d|%d|%d|%d", &st, &nx, &ny, &nz, &tx, &ty, &zb) != 7)
            continue;
        if (!ws::stream_tiling_supported(tx, ty) || zb < 1) continue;
        g_tune_cache[TuneKey(std::string(line, bar - line), st, nx, ny, nz)] =
            ws::StreamTiling{tx, ty, zb};
    }
    std::fclose(f);
}

// Rewrite the file with every entry (a temporary file renamed over it).
// Call with g_tune_mutex held.
void tune_cache_save() {
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos && slash > 0) {
        const std::string dir = path.substr(0, slash);
        const size_t s2 = dir.rfind('/');
        if (s2 != std::string::npos && s2 > 0) mkdir(dir.substr(0, s2).c_str(), 0755);
        mkdir(dir.c_str(), 0755);
    }
    const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const auto &kv : g_tune_cache)
        std::fprintf(f, "%s|%d|%d|%d|%d|%d|%d|%d\n", std::get<0>(kv.first).c_str(),
                     std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
                     std::get<4>(kv.first), kv.second.tx, kv.second.ty, kv.second.zb);
    const bool ok = std::fclose(f) == 0;
    if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) std::remove(tmp.c_str());
}

// The name of the current device ("" if it cannot be read), '|' replaced.
std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return std::string();
    std::string n(prop.name);
    for (char &c : n)
        if (c == '|' || c == '\n') c = '_';
    return n;
}

}  // namespace

extern "C" {

int ws_autotune(ws_t ws, int *tile_x, int *tile_y, int *zblock) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_autotune: NULL handle");
    if (!ws->vel_ok) return fail(WS_ERR_STATE, "ws_autotune: no valid velocity model");
    if (ws->storage != WS_STORAGE_FP32)
        return fail(WS_ERR_STATE, "ws_autotune: tunes the FP32 streaming kernel only");
    const ws::Geom &g = ws->g;
    ws::StreamTiling best{0, 0, 0};
    const TuneKey key(device_name(), ws->storage, g.nx, g.ny, g.nz);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_cache_load();
        auto it = g_tune_cache.find(key);
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
            g_tune_cache[key] = best;
            tune_cache_save();
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
// (m = 0: each shot's default) and rebuild the item table: longest items
// (most planes) first, so the last wave of the launch holds the shortest
// ones; among equal lengths, shots in order of decreasing size and each
// shot's items block-major (neighbouring tiles run together).
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
    std::vector<int> planes;   // z extent of each item
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
        for (long long l = 0; l < nit; ++l) {
            items.push_back(make_int2(q, (int)l));
            planes.push_back((int)std::min<long long>(zb, g.nz - (l / tiles) * zb));
        }
    }
    std::vector<int> perm(items.size());
    for (size_t x = 0; x < perm.size(); ++x) perm[x] = (int)x;
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return planes[x] > planes[y]; });
    std::vector<int2> sorted(items.size());
    for (size_t x = 0; x < perm.size(); ++x) sorted[x] = items[perm[x]];
    items.swap(sorted);
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
        x.stall_item = ws->stall_item;   // test hook, for the first step of this run only
        ws->stall_item = -1;
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
    // for about 1, 2, 3, 4, 6 x the resident CTAs in items and the per-shot
    // default (0)
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

}  // extern "C"
