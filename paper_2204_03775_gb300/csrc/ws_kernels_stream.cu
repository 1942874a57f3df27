// Streaming step kernel for sm_103a: the hot path of the library.
//
// The grid is cut into work items: a TX x TY tile of (x, y) columns over a
// block of zb planes, walked in increasing z. The paper keeps a whole z
// column in a processing element's memory and receives x/y neighbours from 4
// PEs per direction over the fabric (Section III-B, III-C); here the column
// lives in a per-thread register queue of 9 planes (k-4 .. k+4), and the x/y
// neighbours come from a shared-memory copy of plane k with its 4-cell halo.
//
// Warp-specialized CTAs, one per work item, which the hardware dispatches in
// item order as resident CTAs finish. (A persistent grid of SMs x CTAs-per-SM
// looping over the items measured 2-5% slower on the 1024^3 survey: its CTAs
// drift apart, so a tile's halo rows leave L2 before the neighbouring tile
// reads them; in-order dispatch keeps the tiles in flight a contiguous range
// of items. The item loop is kept, so a smaller grid still works.)
//  - one producer lane issues every TMA copy (cp.async.bulk.tensor) into two
//    shared-memory rings, ring A (u^n tile with halo, (TX+8) x (TY+8)) and
//    ring B (u^{n-1} and (V dt/h)^2 tiles, TX x TY), each slot guarded by a
//    "full" mbarrier (transaction count) and an "empty" mbarrier;
//  - the consumer warps compute: each thread owns 4 consecutive x cells of
//    one row, waits on "full", reads the slot, and arrives on "empty" -- no
//    atomics, fences or divergent code in the steady state. The producer
//    runs ahead by the ring depth, across item boundaries too.
// u^{n+1} is written in place of u^{n-1} with 128-bit streaming stores.
// Taper, source injection and receiver sampling are fused into the pass.
// The z loop is unrolled by 3 with the queue indices rotated at compile time.
//
// Each thread's 4 cells are processed as two pairs with the packed FP32x2
// instructions of sm_100+ (add/mul/fma .rn .f32x2), which halves the
// floating-point instruction count. Each lane is rounded exactly as the
// scalar instruction, so the arithmetic per cell is the same expression, in
// the same order, as the direct kernel, and the two CUDA paths agree bit for
// bit.
//
// Every wait is bounded (kWaitLimitNs); on a timeout the kernel records
// kStatusTimeout, all warps leave their loops, and the CTA waits (bounded)
// for its copies in flight before it exits.
//
// The same pipeline serves two sources of work items: one grid whose maps
// and arguments are kernel parameters (OneGrid), and a batch of independent
// shots on grids of different sizes (ShotBatch), whose per-shot tensor maps,
// geometry, sources and receivers sit in a descriptor table in global memory
// and whose items from every shot share one launch.
#include <climits>

#include "ws_ptx.cuh"

namespace ws {
namespace {

#ifndef WS_STREAM_UNROLL
#define WS_STREAM_UNROLL 3
#endif
constexpr int kUnroll = WS_STREAM_UNROLL;  // planes per loop trip: 3 or 9 (divides the queue rotation)
static_assert(kUnroll == 3 || kUnroll == 9, "the 9-plane queue rotation needs 3 or 9");
#ifndef WS_RING_A
#define WS_RING_A 8
#endif

// Tile geometry and ring sizes of one streaming-kernel instantiation.
template <int TX, int TY, int NA, int NB>
struct StreamCfg {
    static constexpr int kConsumers = (TX / 4) * TY;   // compute threads
    static constexpr int kThreads = kConsumers + 32;   // + one producer warp
    static constexpr int kRowW = TX + 2 * kHalo;       // floats per ring-A row
    static constexpr int kRows = TY + 2 * kHalo;
    static constexpr int kSlotA = kRowW * kRows;       // floats per ring-A slot
    static constexpr unsigned kSlotABytes = kSlotA * 4u;
    static constexpr int kTile = TX * TY;              // floats per field in a ring-B slot
    static constexpr unsigned kSlotBBytes = 2u * kTile * 4u;
    static_assert(kConsumers % 32 == 0, "whole consumer warps");
    static_assert((NA & (NA - 1)) == 0 && NA >= 8, "ring A: power of two, >= 8 planes");
    static_assert((NB & (NB - 1)) == 0 && NB >= 2, "ring B: power of two, >= 2 planes");
    static_assert(kSlotABytes % 128 == 0 && kSlotBBytes % 128 == 0, "slots stay 128-byte aligned");
    static constexpr size_t kSmem = size_t(NA) * kSlotABytes + size_t(NB) * kSlotBBytes;
};

// The tensor maps of one launch: u^n with the halo box, u^{n-1} and
// (V dt/h)^2 with the interior box.
struct StreamMaps {
    CUtensorMap u, up, w;
};

// What the producer needs of an item: its extent and the three maps;
// stall (a test hook) withholds the item's first copy.
struct Job {
    Item it;
    const CUtensorMap *u, *up, *w;
    bool stall;
};

// What the consumers need of an item's grid: fields read at the start of an
// item or on every plane, and accessors for what only source injection and
// receiver recording use.
struct View {
    Geom g;
    const float *gx, *gy, *gz;
    float *out;                // u^{n+1} field (padded)
    long long lap_delta;       // L u^n goes to out + lap_delta (0: not stored)
    const int *rec_ptr;        // per-tile receiver ranges, or null
    const RecEntry *rec_;
    const SourceSample *src_;  // this step's source samples
    int nsrc_;
    float *traces_;            // [nrec][nt_max]
    int nt_max_;
    long long trace_step_;
    __device__ __forceinline__ const SourceSample *src() const { return src_; }
    __device__ __forceinline__ int nsrc() const { return nsrc_; }
    __device__ __forceinline__ const RecEntry *rec() const { return rec_; }
    __device__ __forceinline__ float *traces() const { return traces_; }
    __device__ __forceinline__ int nt_max() const { return nt_max_; }
    __device__ __forceinline__ long long trace_step() const { return trace_step_; }
};

// Items of one grid; everything comes from kernel parameters. kLap: the
// launch also stores the stencil sum L u^n (into a.lap).
template <int TX, int TY, bool kLap>
struct OneGrid {
    static constexpr bool kStoreLap = kLap;
    using V = View;
    const StreamMaps &mp;
    const StepArgs &a;
    float *up;
    int zb, tiles_x, ntiles, n;
    const int *rec_ptr;
    const RecEntry *rec;

    __device__ __forceinline__ int nitems() const { return n; }
    __device__ __forceinline__ Job job(int item) const {
        return Job{item_of(item, tiles_x, ntiles, zb, a.g.nz, TX, TY), &mp.u, &mp.up, &mp.w,
                   item == a.stall_item};
    }
    __device__ __forceinline__ Item view(int item, View *v) const {
        v->g = a.g;
        v->gx = a.gx;
        v->gy = a.gy;
        v->gz = a.gz;
        v->src_ = a.src.s;
        v->nsrc_ = a.src.n;
        v->traces_ = a.traces;
        v->nt_max_ = a.nt_max;
        v->trace_step_ = a.trace_step;
        v->out = up;
        v->lap_delta = kLap ? a.lap - up : 0;
        v->rec_ptr = rec_ptr;
        v->rec_ = rec;
        return item_of(item, tiles_x, ntiles, zb, a.g.nz, TX, TY);
    }
};

// The view of a batch item: the fields of every plane in registers, the rest
// read from the shot's descriptor where they are used (held in registers for
// the whole item they would not fit the batched kernel's register budget).
struct BatchView {
    Geom g;
    const float *gx, *gy, *gz;
    float *out;
    const int *rec_ptr;
    const BatchShot *shot;
    int t;
    __device__ __forceinline__ const SourceSample *src() const {
        return shot->src + (long long)t * shot->nsrc;
    }
    __device__ __forceinline__ int nsrc() const { return shot->nsrc; }
    __device__ __forceinline__ const RecEntry *rec() const { return shot->rec; }
    __device__ __forceinline__ float *traces() const { return shot->traces; }
    __device__ __forceinline__ int nt_max() const { return shot->nt_max; }
    __device__ __forceinline__ long long trace_step() const { return shot->trace_col0 + t; }
};

// Items of a batch of shots: items[q] = (shot, item of that shot), step t of
// the run; shot s reads u^n from buf[cur0 ^ (t & 1)].
template <int TX, int TY>
struct ShotBatch {
    static constexpr bool kStoreLap = false;
    using V = BatchView;
    const BatchShot *shots;
    const int2 *items;
    int n, t;

    __device__ __forceinline__ int nitems() const { return n; }
    __device__ __forceinline__ Job job(int item) const {
        const int2 e = items[item];
        const BatchShot &s = shots[e.x];
        const int p = s.cur0 ^ (t & 1);
        return Job{item_of(e.y, s.tiles_x, s.ntiles, s.zb, s.g.nz, TX, TY), &s.halo[p],
                   &s.tile[1 - p], &s.w, t == 0 && e.y == s.stall_item};
    }
    __device__ __forceinline__ Item view(int item, BatchView *v) const {
        const int2 e = items[item];
        const BatchShot &s = shots[e.x];
        const int p = s.cur0 ^ (t & 1);
        v->g = s.g;
        v->gx = s.gx;
        v->gy = s.gy;
        v->gz = s.gz;
        v->out = s.buf[1 - p];
        v->rec_ptr = s.rec_ptr;
        v->shot = &s;
        v->t = t;
        return item_of(e.y, s.tiles_x, s.ntiles, s.zb, s.g.nz, TX, TY);
    }
};

// Per-thread state of a consumer thread's walk down one item.
struct Walk {
    float4 q[9];            // u^n of planes k-4 .. k+4 (rotated: see plane_step)
    float gzb[3];           // z taper of planes k, k+1, k+2 (rotated)
    float4 gxy;             // gx * gy of this thread's 4 columns
    float *out_k;           // u^{n+1} of plane k
    int nvalid;             // cells of the 4 inside the grid (0 when the row is outside)
    int rcur, rend, rnext_k;
    unsigned src_mask;
    unsigned gAw, gAr, gB;  // ring-A planes waited for / released, ring-B planes used
    bool ok;
};

template <int TX, int TY, int NA, int NB>
struct Kern {
    using Cfg = StreamCfg<TX, TY, NA, NB>;
    using R = Rings<NA, NB>;

    // ---------------------------------------------------------------- producer

    // Copy relative plane pr of the item (interior plane z0 - 4 + pr, with
    // its halo) into the g-th ring-A slot use, once its previous plane is
    // released. The maps cover the interior only (origin at interior cell 0):
    // the box corner is (i0 - 4, j0 - 4, z0 - 4 + pr), and whatever of the
    // box lies outside the grid arrives as zeros without a memory read (the
    // zero halo). x is a multiple of 4 elements (16 bytes).
    static __device__ __forceinline__ bool produce_a(R &rg, float *ringA, const Job &jb, unsigned g,
                                                     int pr, unsigned *status) {
        const int slot = g & (NA - 1);
        if (!wait_phase(&rg.emptyA[slot], ((g / NA) & 1u) ^ 1u, &rg.abort, status)) return false;
        rg.issuedA[slot]++;
        mbar_arrive_expect_tx(&rg.fullA[slot], Cfg::kSlotABytes);
        tma_load_3d(ringA + slot * Cfg::kSlotA, jb.u, &rg.fullA[slot], jb.it.i0 - kHalo,
                    jb.it.j0 - kHalo, jb.it.z0 - kHalo + pr);
        return true;
    }

    // u^{n-1} and (V dt/h)^2 of interior plane z0 + b into the g-th ring-B use.
    static __device__ __forceinline__ bool produce_b(R &rg, float *ringB, const Job &jb, unsigned g,
                                                     int b, unsigned *status) {
        const int slot = g & (NB - 1);
        if (!wait_phase(&rg.emptyB[slot], ((g / NB) & 1u) ^ 1u, &rg.abort, status)) return false;
        rg.issuedB[slot]++;
        float *dst = ringB + slot * (2 * Cfg::kTile);
        mbar_arrive_expect_tx(&rg.fullB[slot], Cfg::kSlotBBytes);
        tma_load_3d(dst, jb.up, &rg.fullB[slot], jb.it.i0, jb.it.j0, jb.it.z0 + b);
        tma_load_3d(dst + Cfg::kTile, jb.w, &rg.fullB[slot], jb.it.i0, jb.it.j0, jb.it.z0 + b);
        return true;
    }

    // One lane issues every copy of every item of this CTA, in the order the
    // consumers need them: the 8 planes of the queue prologue, then for each
    // plane k of the block its u^{n-1} / (V dt/h)^2 and the u^n plane k + 8.
    template <class S>
    static __device__ void producer(R &rg, float *ringA, float *ringB, const S &src,
                                    unsigned *status) {
        unsigned gA = 0, gB = 0;
        for (int item = blockIdx.x; item < src.nitems(); item += gridDim.x) {
            const Job jb = src.job(item);
            const int nb = jb.it.z1 - jb.it.z0, nplanes = nb + 2 * kHalo;
            for (int pr = 0; pr < 2 * kHalo; ++pr) {
                if (pr == 0 && jb.stall) {   // never filled: the consumers' bounded waits run out
                    ++gA;
                    continue;
                }
                if (!produce_a(rg, ringA, jb, gA++, pr, status)) return;
            }
            for (int b = 0; b < nb; ++b) {
                if (!produce_b(rg, ringB, jb, gB++, b, status)) return;
                if (b + 2 * kHalo < nplanes && !produce_a(rg, ringA, jb, gA++, b + 2 * kHalo, status))
                    return;
            }
        }
    }

    // ---------------------------------------------------------------- consumers

    static __device__ __forceinline__ const float *wait_a(Walk &wk, R &rg, const float *ringA,
                                                          unsigned g, unsigned *status) {
        const int slot = g & (NA - 1);
        wk.ok = wk.ok && wait_phase(&rg.fullA[slot], (g / NA) & 1u, &rg.abort, status);
        return ringA + slot * Cfg::kSlotA;
    }

    // Plane k of the item, with the rotation R = (k - z0) mod 9 fixed at
    // compile time.
    template <int RQ, bool kLap, class VT>
    static __device__ __forceinline__ void plane_step(Walk &wk, R &rg, const float *ringA,
                                                      const float *ringB, const VT &v,
                                                      const Coeffs &c, unsigned *status,
                                                      const Item &it, int k, int i, int j,
                                                      int offA, int offB) {
#define QI(m) ((RQ + (m)) % 9)
#define BI(d) ((RQ + (d)) % 3)
        // u^n of plane k + 4 into the queue
        const float *sa = wait_a(wk, rg, ringA, wk.gAw, status);
        wk.q[QI(8)] = lds4(sa + offA);
        ++wk.gAw;

        // u^{n-1} and (V dt/h)^2 of plane k
        const int sb = wk.gB & (NB - 1);
        wk.ok = wk.ok && wait_phase(&rg.fullB[sb], (wk.gB / NB) & 1u, &rg.abort, status);
        const float *tb = ringB + sb * (2 * Cfg::kTile) + offB;
        const float4 upc = lds4(tb);
        const float4 wc = lds4(tb + Cfg::kTile);
        warp_arrive(&rg.emptyB[sb]);
        ++wk.gB;

        if (k + 2 < it.z1) wk.gzb[BI(2)] = __ldg(v.gz + k + 2);

        // u^n of plane k with its halo (waited for four planes ago)
        const float *row = ringA + (wk.gAr & (NA - 1)) * Cfg::kSlotA + offA;
        const float4 xl = lds4(row - 4);   // cells x-4 .. x-1 of lane 0
        const float4 xc = wk.q[QI(4)];
        const float4 xr = lds4(row + 4);   // cells x+4 .. x+7 of lane 0
        float4 yp[4], ym[4];
#pragma unroll
        for (int m = 1; m <= 4; ++m) {
            yp[m - 1] = lds4(row + m * Cfg::kRowW);
            ym[m - 1] = lds4(row - m * Cfg::kRowW);
        }
        warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
        ++wk.gAr;

        // x pairs: offsets +-2 and +-4 are aligned float2 pairs of (xl, xc, xr);
        // offsets +-1 and +-3 straddle pairs and are summed per lane.
        const float e[12] = {xl.x, xl.y, xl.z, xl.w, xc.x, xc.y, xc.z, xc.w,
                             xr.x, xr.y, xr.z, xr.w};
        float2 sx[2][5];
        sx[0][2] = add2(hi2(xc), hi2(xl));
        sx[1][2] = add2(lo2(xr), lo2(xc));
        sx[0][4] = add2(lo2(xr), lo2(xl));
        sx[1][4] = add2(hi2(xr), hi2(xl));
#pragma unroll
        for (int p = 0; p < 2; ++p) {
#pragma unroll
            for (int m = 1; m <= 3; m += 2) {
                const int l0 = 2 * p, l1 = 2 * p + 1;
                sx[p][m] = make_float2(e[4 + l0 + m] + e[4 + l0 - m], e[4 + l1 + m] + e[4 + l1 - m]);
            }
        }

        const float gzk = wk.gzb[BI(0)];
        float2 o[2], lp[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            float2 s[5];
#pragma unroll
            for (int m = 1; m <= 4; ++m) {
                const float2 sy = add2(pair(yp[m - 1], p), pair(ym[m - 1], p));
                const float2 sz = add2(pair(wk.q[QI(4 + m)], p), pair(wk.q[QI(4 - m)], p));
                s[m] = add2(add2(sx[p][m], sy), sz);
            }
            const float2 uc = pair(xc, p);
            // sum_m c_m (s_m - 6 u): exactly zero on constants (see Coeffs)
            float2 lap = mul2(splat(c.c4), fma2(splat(-6.0f), uc, s[4]));
            lap = fma2(splat(c.c3), fma2(splat(-6.0f), uc, s[3]), lap);
            lap = fma2(splat(c.c2), fma2(splat(-6.0f), uc, s[2]), lap);
            lap = fma2(splat(c.c1), fma2(splat(-6.0f), uc, s[1]), lap);
            lp[p] = lap;
            const float2 gd = mul2(pair(wk.gxy, p), splat(gzk));
            const float2 ngd = mul2(pair(wk.gxy, p), splat(-gzk));   // -gd, exactly
            const float2 t = fma2(pair(wc, p), lap, fma2(splat(2.0f), uc, mul2(ngd, pair(upc, p))));
            o[p] = mul2(gd, t);
        }
        float4 out = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        if (wk.src_mask) {
            const SourceSample *srcs = v.src();
            for (int qs = 0, ns = v.nsrc(); qs < ns; ++qs) {
                const SourceSample ss = srcs[qs];
                if (((wk.src_mask >> qs) & 1u) && ss.k == k && ss.j == j) {
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        if (ss.i == i + l) set_comp(out, l, fmaf(comp(wc, l), ss.amp, comp(out, l)));
                }
            }
        }
        if (wk.nvalid == 4) {
            __stcs(reinterpret_cast<float4 *>(wk.out_k), out);
        } else if (wk.nvalid > 0) {
            wk.out_k[0] = out.x;
            if (wk.nvalid > 1) wk.out_k[1] = out.y;
            if (wk.nvalid > 2) wk.out_k[2] = out.z;
        }
        if constexpr (kLap) {   // the stencil sum, for the adjoint's imaging
            float *lk = wk.out_k + v.lap_delta;
            const float4 l4 = make_float4(lp[0].x, lp[0].y, lp[1].x, lp[1].y);
            if (wk.nvalid == 4) {
                __stcs(reinterpret_cast<float4 *>(lk), l4);
            } else if (wk.nvalid > 0) {
                lk[0] = l4.x;
                if (wk.nvalid > 1) lk[1] = l4.y;
                if (wk.nvalid > 2) lk[2] = l4.z;
            }
        }
        wk.out_k += v.g.plane;
        if (k == wk.rnext_k)
            record_plane(out, 1.0f, k, &wk.rcur, wk.rend, &wk.rnext_k, v.rec(), v.traces(),
                         v.nt_max(), v.trace_step());
#undef QI
#undef BI
    }

    // After kUnroll planes the queue is rotated by kUnroll; rename it back.
    static __device__ __forceinline__ void rotate_queue(Walk &wk) {
        if constexpr (kUnroll % 9 != 0) {
            float4 t[9];
#pragma unroll
            for (int m = 0; m < 9; ++m) t[m] = wk.q[(m + kUnroll) % 9];
#pragma unroll
            for (int m = 0; m < 9; ++m) wk.q[m] = t[m];
        }
    }

    template <class S>
    static __device__ void consumer(R &rg, const float *ringA, const float *ringB, const S &src,
                                    const Coeffs &c, unsigned *status) {
        const int tid = threadIdx.x;
        const int tx = tid % (TX / 4);
        const int ty = tid / (TX / 4);
        const int offA = (kHalo + ty) * Cfg::kRowW + kHalo + 4 * tx;
        const int offB = ty * TX + 4 * tx;
        Walk wk;
        wk.gAw = wk.gAr = wk.gB = 0;
        wk.ok = true;
        for (int item = blockIdx.x; item < src.nitems() && wk.ok; item += gridDim.x) {
            typename S::V v;
            const Item it = src.view(item, &v);
            const Geom &g = v.g;
            const int i = it.i0 + 4 * tx;
            const int j = it.j0 + ty;
            const bool col_ok = (j < g.ny) && (i < g.nx);
            wk.nvalid = col_ok ? min(4, g.nx - i) : 0;
            wk.gxy = make_float4(0.f, 0.f, 0.f, 0.f);
            if (col_ok) {
                const float gyj = v.gy[j];
                wk.gxy.x = v.gx[i] * gyj;
                if (wk.nvalid > 1) wk.gxy.y = v.gx[i + 1] * gyj;
                if (wk.nvalid > 2) wk.gxy.z = v.gx[i + 2] * gyj;
                if (wk.nvalid > 3) wk.gxy.w = v.gx[i + 3] * gyj;
            }
            wk.src_mask = 0u;
            const SourceSample *srcs = v.src();
            for (int qs = 0, ns = v.nsrc(); qs < ns; ++qs) {
                const SourceSample ss = srcs[qs];
                if (ss.i >= it.i0 && ss.i < it.i0 + TX && ss.j >= it.j0 && ss.j < it.j0 + TY &&
                    ss.k >= it.z0 && ss.k < it.z1)
                    wk.src_mask |= 1u << qs;
            }
            wk.rcur = wk.rend = 0;
            if (v.rec_ptr != nullptr) {
                const int r = it.tile * (Cfg::kConsumers / 32) + (tid >> 5);
                wk.rend = v.rec_ptr[r + 1];
                wk.rcur = first_entry(v.rec(), v.rec_ptr[r], wk.rend, it.z0);
            }
            wk.rnext_k = wk.rcur < wk.rend ? v.rec()[wk.rcur].k : INT_MAX;
            wk.out_k = v.out + pidx(g, col_ok ? i : 0, col_ok ? j : 0, it.z0);
#pragma unroll
            for (int d = 0; d < 2; ++d)
                wk.gzb[d] = (it.z0 + d < it.z1) ? __ldg(v.gz + it.z0 + d) : 1.0f;

            // queue prologue: planes z0-4 .. z0+3; the first four are only
            // needed here and are released at once
#pragma unroll
            for (int m = 0; m < 2 * kHalo; ++m) {
                const float *sa = wait_a(wk, rg, ringA, wk.gAw, status);
                wk.q[m] = lds4(sa + offA);
                ++wk.gAw;
            }
#pragma unroll
            for (int m = 0; m < kHalo; ++m) {
                warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
                ++wk.gAr;
            }
            if (!warp_all_ok(wk)) break;

            for (int kb = it.z0; kb < it.z1; kb += kUnroll) {
#define WS_PLANE(RQ)                                                                         \
    if (kb + (RQ) >= it.z1) break;                                                           \
    plane_step<RQ, S::kStoreLap>(wk, rg, ringA, ringB, v, c, status, it, kb + (RQ), i, j, offA, \
                                 offB);                                                     \
    if (!warp_all_ok(wk)) break;
                WS_PLANE(0)
                WS_PLANE(1)
                WS_PLANE(2)
                if constexpr (kUnroll == 9) {
                    WS_PLANE(3)
                    WS_PLANE(4)
                    WS_PLANE(5)
                    WS_PLANE(6)
                    WS_PLANE(7)
                    WS_PLANE(8)
                }
#undef WS_PLANE
                rotate_queue(wk);
            }
            // the last four planes (z1 .. z1+3) were needed only for the queue
#pragma unroll
            for (int m = 0; m < kHalo; ++m) {
                warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
                ++wk.gAr;
            }
        }
    }
};

// The body of a launch: ring set-up, the warp roles, and the drain.
template <int TX, int TY, int NA, int NB, class S>
__device__ __forceinline__ void stream_body(const S &src, const Coeffs &c, unsigned *status) {
    using K = Kern<TX, TY, NA, NB>;
    using Cfg = typename K::Cfg;
    extern __shared__ __align__(128) float smem[];
    __shared__ Rings<NA, NB> rg;
    float *ringA = smem;
    float *ringB = smem + NA * Cfg::kSlotA;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(&rg.fullA[s], 1);
            mbar_init(&rg.emptyA[s], Cfg::kConsumers / 32);
            rg.issuedA[s] = 0;
        }
        for (int s = 0; s < NB; ++s) {
            mbar_init(&rg.fullB[s], 1);
            mbar_init(&rg.emptyB[s], Cfg::kConsumers / 32);
            rg.issuedB[s] = 0;
        }
        rg.abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (threadIdx.x >= Cfg::kConsumers) {
        if (threadIdx.x == Cfg::kConsumers) K::producer(rg, ringA, ringB, src, status);
    } else {
        K::consumer(rg, ringA, ringB, src, c, status);
    }

    // After an abort, wait (bounded) for the last copy issued into each slot
    // to land before the CTA exits.
    __syncthreads();
    if (rg.abort && threadIdx.x == 0) {
        for (int s = 0; s < NA + NB; ++s) {
            const int cnt = s < NA ? rg.issuedA[s] : rg.issuedB[s - NA];
            uint64_t *bar = s < NA ? &rg.fullA[s] : &rg.fullB[s - NA];
            if (cnt == 0) continue;
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(bar, (unsigned)(cnt - 1) & 1u) && global_ns() - t0 < kWaitLimitNs) {
            }
        }
    }
}

template <int TX, int TY, int NA, int NB, int MINB, bool kLap>
__global__ void __launch_bounds__(StreamCfg<TX, TY, NA, NB>::kThreads, MINB)
    step_stream_kernel(const __grid_constant__ StreamMaps maps, float *__restrict__ up,
                       const __grid_constant__ StepArgs a, const int zb, const int tiles_x,
                       const int ntiles, const int nitems, const int *__restrict__ rec_ptr,
                       const RecEntry *__restrict__ rec) {
    const OneGrid<TX, TY, kLap> src{maps, a, up, zb, tiles_x, ntiles, nitems, rec_ptr, rec};
    stream_body<TX, TY, NA, NB>(src, a.c, a.status);
}

template <int TX, int TY, int NA, int NB, int MINB>
__global__ void __launch_bounds__(StreamCfg<TX, TY, NA, NB>::kThreads, MINB)
    step_batch_kernel(const BatchShot *__restrict__ shots, const int2 *__restrict__ items,
                      const int nitems, const int t, const Coeffs c, unsigned *status) {
    const ShotBatch<TX, TY> src{shots, items, nitems, t};
    stream_body<TX, TY, NA, NB>(src, c, status);
}

// Resident CTAs per SM and SM count of a kernel on the current device,
// looked up (and the kernel's shared-memory limit set) the first time the
// kernel runs on each device.
template <class KernFn>
cudaError_t occupancy(KernFn kern, int threads, size_t smem, LaunchFacts &lf, int *ctas_per_sm,
                      int *sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= LaunchFacts::kMaxDevices) return cudaErrorInvalidDevice;
    if (lf.ctas[dev] == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int n = 0, c = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kern, threads, smem);
        if (e != cudaSuccess) return e;
        if (c < 1) return cudaErrorInvalidConfiguration;
        lf.sms[dev] = n;
        lf.ctas[dev] = c;
    }
    *ctas_per_sm = lf.ctas[dev];
    *sms = lf.sms[dev];
    return cudaSuccess;
}

template <int TX, int TY, int NA, int NB, int MINB, bool kLap>
cudaError_t launch_tile_as(const StreamMaps &maps, float *up, const StepArgs &a, int zb,
                           const int *rec_ptr, const RecEntry *rec, cudaStream_t s) {
    using Cfg = StreamCfg<TX, TY, NA, NB>;
    auto kern = step_stream_kernel<TX, TY, NA, NB, MINB, kLap>;
    static LaunchFacts lf;
    int ctas_per_sm = 0, sms = 0;
    cudaError_t e = occupancy(kern, Cfg::kThreads, Cfg::kSmem, lf, &ctas_per_sm, &sms);
    if (e != cudaSuccess) return e;
    const int tiles_x = (a.g.nx + TX - 1) / TX;
    const int ntiles = tiles_x * ((a.g.ny + TY - 1) / TY);
    const int nitems = ntiles * ((a.g.nz + zb - 1) / zb);
    // one CTA per item (see the header: in-order dispatch keeps neighbours' halos in L2)
    kern<<<nitems, Cfg::kThreads, Cfg::kSmem, s>>>(maps, up, a, zb, tiles_x, ntiles, nitems, rec_ptr,
                                                   rec);
    return cudaGetLastError();
}

template <int TX, int TY, int NA, int NB, int MINB>
cudaError_t launch_tile(const StreamMaps &maps, float *up, const StepArgs &a, int zb,
                        const int *rec_ptr, const RecEntry *rec, cudaStream_t s) {
    if (a.lap) return launch_tile_as<TX, TY, NA, NB, MINB, true>(maps, up, a, zb, rec_ptr, rec, s);
    return launch_tile_as<TX, TY, NA, NB, MINB, false>(maps, up, a, zb, rec_ptr, rec, s);
}

template <int TX, int TY, int NA, int NB, int MINB>
cudaError_t slots_of(bool batch, int *slots) {
    using Cfg = StreamCfg<TX, TY, NA, NB>;
    static LaunchFacts lf_grid, lf_batch;
    int c = 0, n = 0;
    cudaError_t e = batch ? occupancy(step_batch_kernel<TX, TY, NA, NB, MINB>, Cfg::kThreads,
                                      Cfg::kSmem, lf_batch, &c, &n)
                          : occupancy(step_stream_kernel<TX, TY, NA, NB, MINB, false>,
                                      Cfg::kThreads, Cfg::kSmem, lf_grid, &c, &n);
    if (e == cudaSuccess) *slots = c * n;
    return e;
}

template <int TX, int TY, int NA, int NB, int MINB>
cudaError_t launch_batch_tile(const BatchShot *shots, const int2 *items, int nitems, int t,
                              const Coeffs &c, unsigned *status, cudaStream_t s) {
    using Cfg = StreamCfg<TX, TY, NA, NB>;
    auto kern = step_batch_kernel<TX, TY, NA, NB, MINB>;
    static LaunchFacts lf;
    int ctas_per_sm = 0, sms = 0;
    cudaError_t e = occupancy(kern, Cfg::kThreads, Cfg::kSmem, lf, &ctas_per_sm, &sms);
    if (e != cudaSuccess) return e;
    kern<<<nitems, Cfg::kThreads, Cfg::kSmem, s>>>(shots, items, nitems, t, c, status);
    return cudaGetLastError();
}

}  // namespace

bool stream_tiling_supported(int tx, int ty) {
    return (tx == 64 && (ty == 8 || ty == 16 || ty == 32)) || (tx == 32 && (ty == 8 || ty == 16));
}

cudaError_t launch_step_stream(const CUtensorMap *tmap_u, const CUtensorMap *tmap_up,
                               const CUtensorMap *tmap_w, float *up, const StepArgs &a,
                               const StreamTiling &t, const int *rec_ptr, const RecEntry *rec,
                               cudaStream_t s) {
    StreamMaps maps;
    maps.u = *tmap_u;
    maps.up = *tmap_up;
    maps.w = *tmap_w;
    // ring sizes chosen so that the CTAs of one SM fit in its shared memory
    if (t.tx == 64 && t.ty == 32) return launch_tile<64, 32, 8, 4, 1>(maps, up, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 64 && t.ty == 16) return launch_tile<64, 16, 8, 4, 2>(maps, up, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 64 && t.ty == 8) return launch_tile<64, 8, 8, 4, 3>(maps, up, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 32 && t.ty == 16)
        return launch_tile<32, 16, WS_RING_A, 4, 3>(maps, up, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 32 && t.ty == 8) return launch_tile<32, 8, 8, 4, 4>(maps, up, a, t.zb, rec_ptr, rec, s);
    return cudaErrorInvalidValue;
}

}  // namespace ws

namespace ws {

cudaError_t stream_slots(int tx, int ty, bool batch, int *slots) {
    if (tx == 64 && ty == 32) return slots_of<64, 32, 8, 4, 1>(batch, slots);
    if (tx == 64 && ty == 16) return slots_of<64, 16, 8, 4, 2>(batch, slots);
    if (tx == 64 && ty == 8) return slots_of<64, 8, 8, 4, 3>(batch, slots);
    if (tx == 32 && ty == 16) return slots_of<32, 16, WS_RING_A, 4, 3>(batch, slots);
    if (tx == 32 && ty == 8) return slots_of<32, 8, 8, 4, 4>(batch, slots);
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_batch(const BatchShot *shots, const int2 *items, int nitems, int t,
                              const Coeffs &c, unsigned *status, int tx, int ty, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    if (tx == 64 && ty == 32) return launch_batch_tile<64, 32, 8, 4, 1>(shots, items, nitems, t, c, status, s);
    if (tx == 64 && ty == 16) return launch_batch_tile<64, 16, 8, 4, 2>(shots, items, nitems, t, c, status, s);
    if (tx == 64 && ty == 8) return launch_batch_tile<64, 8, 8, 4, 3>(shots, items, nitems, t, c, status, s);
    if (tx == 32 && ty == 16)
        return launch_batch_tile<32, 16, WS_RING_A, 4, 3>(shots, items, nitems, t, c, status, s);
    if (tx == 32 && ty == 8) return launch_batch_tile<32, 8, 8, 4, 4>(shots, items, nitems, t, c, status, s);
    return cudaErrorInvalidValue;
}

}  // namespace ws
