// Streaming step kernel for sm_103a: the hot path of the library.
//
// Each CTA owns a TX x TY tile of (x, y) columns and a block of zb planes,
// which it walks in increasing z. The paper keeps a whole z column in a
// processing element's memory and receives x/y neighbours from 4 PEs per
// direction over the fabric (Section III-B, III-C); here the column lives in
// a per-thread register queue of 9 planes (k-4 .. k+4), and the x/y
// neighbours come from a shared-memory copy of plane k with its 4-cell halo.
//
// All three input streams arrive by TMA (cp.async.bulk.tensor) into two
// shared-memory rings, so no register is spent on prefetching:
//   ring A (kRingA slots): u^n tile with halo, (TX+8) x (TY+8), runs up to
//     kRingA - 5 planes ahead of the queue;
//   ring B (kRingB slots): u^{n-1} and (V dt/h)^2 tiles, TX x TY each, runs
//     up to kRingB - 1 planes ahead of the plane being computed.
// u^{n+1} is written in place of u^{n-1} with 128-bit streaming stores.
// Taper, source injection and receiver sampling are fused into the pass.
// Each thread owns 4 consecutive x cells of one row.
//
// There is no CTA-wide barrier in the z loop. Every warp counts itself out of
// a ring slot once it has read it (a shared-memory counter per slot); the
// warp that completes the count refills the slot with the plane one ring
// length further on. Warps drift apart by up to the ring depth instead of
// meeting at every plane. The z loop is unrolled by 3 with the queue indices
// rotated at compile time.
//
// Each thread's 4 cells are processed as two pairs with the packed FP32x2
// instructions of sm_100+ (add/mul/fma .rn .f32x2), which halves the
// floating-point instruction count. Each lane is rounded exactly as the
// scalar instruction, so the arithmetic per cell is the same expression, in
// the same order, as the direct kernel, and the two CUDA paths agree bit for
// bit.
#include <climits>

#include "ws_internal.h"

namespace ws {
namespace {

constexpr int kRingA = 8;   // u^n tile slots (power of two, >= 8)
constexpr int kRingALog2 = 3;
constexpr int kRingB = 4;   // u^{n-1} / (V dt/h)^2 slots (power of two)
constexpr int kRingBLog2 = 2;
constexpr int kUnroll = 3;  // planes per loop trip; divides the 9-plane queue rotation

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ float4 lds4(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
}

__device__ __forceinline__ float comp(const float4 &v, int l) {
    return l == 0 ? v.x : (l == 1 ? v.y : (l == 2 ? v.z : v.w));
}

__device__ __forceinline__ void set_comp(float4 &v, int l, float x) {
    if (l == 0) v.x = x;
    else if (l == 1) v.y = x;
    else if (l == 2) v.z = x;
    else v.w = x;
}

// Packed FP32x2 arithmetic (two independent IEEE round-to-nearest lanes).
__device__ __forceinline__ unsigned long long as_u64(float2 v) {
    return (static_cast<unsigned long long>(__float_as_uint(v.y)) << 32) | __float_as_uint(v.x);
}
__device__ __forceinline__ float2 as_f2(unsigned long long v) {
    return make_float2(__uint_as_float(static_cast<unsigned>(v)),
                       __uint_as_float(static_cast<unsigned>(v >> 32)));
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
    return as_f2(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
    return as_f2(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)), "l"(as_u64(c)));
    return as_f2(r);
}
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 pair(const float4 &v, int p) { return p == 0 ? lo2(v) : hi2(v); }
__device__ __forceinline__ float2 splat(float x) { return make_float2(x, x); }

template <int TX, int TY>
struct StreamCfg {
    static constexpr int kThreads = (TX / 4) * TY;
    static constexpr int kWarps = kThreads / 32;
    static constexpr int kRowW = TX + 2 * kHalo;   // floats per ring-A row
    static constexpr int kRows = TY + 2 * kHalo;
    static constexpr int kSlotA = kRowW * kRows;   // floats per ring-A slot
    static constexpr unsigned kSlotABytes = kSlotA * 4u;
    static constexpr int kTile = TX * TY;          // floats per field in a ring-B slot
    static constexpr unsigned kSlotBBytes = 2u * kTile * 4u;
    static_assert(kThreads % 32 == 0, "whole warps");
    static_assert(kSlotABytes % 128 == 0 && kSlotBBytes % 128 == 0, "slots stay 128-byte aligned");
    static constexpr size_t kSmem = size_t(kRingA) * kSlotABytes + size_t(kRingB) * kSlotBBytes;
};

// The tensor maps of one launch: u^n with the halo box, u^{n-1} and
// (V dt/h)^2 with the interior box.
struct StreamMaps {
    CUtensorMap u, up, w;
};

// Per-thread state of the z walk.
struct Walk {
    float4 q[9];            // u of planes k-4 .. k+4 (rotated: see plane_step)
    float gzb[3];           // z taper of planes k, k+1, k+2 (rotated)
    float4 gxy;             // gx * gy of this thread's 4 columns
    float *out_k;           // u^{n+1} of plane k
    long long plane;        // elements per padded plane
    int offA;               // this thread's first cell in a ring-A row (row of plane k)
    int offB;               // this thread's first cell in a ring-B tile
    int z0, z1, nplanes, nvalid;
    bool col_ok;
    int rcur, rend, rnext_k;
    unsigned src_mask;
    bool aborted;
};

struct Rings {
    uint64_t *fullA, *fullB;
    int *arrivedA, *arrivedB;  // warps done with each slot, over all its uses
    int *issuedA, *issuedB;    // copies issued into each slot
    int *abort;
    float *ringA, *ringB;
};

template <int TX, int TY>
struct Kern {
    using Cfg = StreamCfg<TX, TY>;

    // Wait for a phase of a ring barrier; bounded, and gives up early once
    // another warp has aborted. The outcome is made uniform across the warp.
    static __device__ __forceinline__ void wait_bar(Walk &wk, const Rings &rg, uint64_t *bar,
                                                    unsigned par, unsigned *status) {
        bool fail = false;
        if (!mbar_try_wait(bar, par)) {
            const unsigned long long t0 = global_ns();
            unsigned n = 0;
            while (!mbar_try_wait(bar, par)) {
                if ((++n & 63u) == 0) {
                    if (*reinterpret_cast<volatile int *>(rg.abort)) {
                        fail = true;
                        break;
                    }
                    if (global_ns() - t0 > kWaitLimitNs) {
                        atomicOr(status, kStatusTimeout);
                        *reinterpret_cast<volatile int *>(rg.abort) = 1;
                        fail = true;
                        break;
                    }
                }
            }
        }
        wk.aborted = __any_sync(0xffffffffu, fail);
    }

    // Refill of ring-A slot with relative plane pr (interior plane z0-4+pr).
    static __device__ __forceinline__ void issue_a(const Rings &rg, const StreamMaps &mp, int pr,
                                                   int i0, int j0, int z0) {
        const int slot = pr & (kRingA - 1);
        rg.issuedA[slot]++;
        mbar_arrive_expect_tx(&rg.fullA[slot], Cfg::kSlotABytes);
        // box corner at interior (i0 - 4, j0 - 4, z0 - 4 + pr): padded
        // (i0 + kXOff - 4, j0, z0 + pr); x is a multiple of 4 elements
        tma_load_3d(rg.ringA + slot * Cfg::kSlotA, &mp.u, &rg.fullA[slot], i0 + kXOff - kHalo, j0,
                    z0 + pr);
    }

    // Refill of ring-B slot with plane index b (interior plane z0 + b).
    static __device__ __forceinline__ void issue_b(const Rings &rg, const StreamMaps &mp, int b,
                                                   int i0, int j0, int z0) {
        const int slot = b & (kRingB - 1);
        float *dst = rg.ringB + slot * (2 * Cfg::kTile);
        rg.issuedB[slot]++;
        mbar_arrive_expect_tx(&rg.fullB[slot], Cfg::kSlotBBytes);
        tma_load_3d(dst, &mp.up, &rg.fullB[slot], i0 + kXOff, j0 + kHalo, z0 + b + kHalo);
        tma_load_3d(dst + Cfg::kTile, &mp.w, &rg.fullB[slot], i0 + kXOff, j0 + kHalo,
                    z0 + b + kHalo);
    }

    // This warp is done reading a slot for its use-th time. True for the warp
    // that completes the count, which then refills the slot.
    static __device__ __forceinline__ bool last_reader(int *arrived, int slot, int use) {
        __threadfence_block();
        const int old = atomicAdd(&arrived[slot], 1);
        return old == Cfg::kWarps * (use + 1) - 1;
    }

    static __device__ __forceinline__ void release_a(const Rings &rg, const StreamMaps &mp, int pr,
                                                     int nplanes, int i0, int j0, int z0) {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            if (last_reader(rg.arrivedA, pr & (kRingA - 1), pr >> kRingALog2) &&
                pr + kRingA < nplanes) {
                __threadfence_block();
                fence_proxy_async_smem();
                issue_a(rg, mp, pr + kRingA, i0, j0, z0);
            }
        }
    }

    static __device__ __forceinline__ void release_b(const Rings &rg, const StreamMaps &mp, int b,
                                                     int nb, int i0, int j0, int z0) {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            if (last_reader(rg.arrivedB, b & (kRingB - 1), b >> kRingBLog2) && b + kRingB < nb) {
                __threadfence_block();
                fence_proxy_async_smem();
                issue_b(rg, mp, b + kRingB, i0, j0, z0);
            }
        }
    }

    // Plane k, with the rotation R = (k - z0) mod 9 fixed at compile time.
    template <int R>
    static __device__ __forceinline__ void plane_step(Walk &wk, const Rings &rg,
                                                      const StreamMaps &mp, const StepArgs &a,
                                                      int k, int i, int j, int i0, int j0,
                                                      const RecEntry *rec) {
#define QI(m) ((R + (m)) % 9)
#define BI(d) ((R + (d)) % 3)
        const int b = k - wk.z0;        // ring-B plane index
        const int pc = b + kHalo;       // ring-A relative index of plane k

        // u^n of plane k + 4 into the queue
        wait_bar(wk, rg, &rg.fullA[(pc + kHalo) & (kRingA - 1)],
                 (unsigned)((pc + kHalo) >> kRingALog2) & 1u, a.status);
        if (wk.aborted) return;
        wk.q[QI(8)] = lds4(rg.ringA + ((pc + kHalo) & (kRingA - 1)) * Cfg::kSlotA + wk.offA);

        // u^{n-1} and (V dt/h)^2 of plane k
        wait_bar(wk, rg, &rg.fullB[b & (kRingB - 1)], (unsigned)(b >> kRingBLog2) & 1u, a.status);
        if (wk.aborted) return;
        const float *tb = rg.ringB + (b & (kRingB - 1)) * (2 * Cfg::kTile) + wk.offB;
        const float4 upc = lds4(tb);
        const float4 wc = lds4(tb + Cfg::kTile);
        release_b(rg, mp, b, wk.z1 - wk.z0, i0, j0, wk.z0);

        if (k + 2 < wk.z1) wk.gzb[BI(2)] = __ldg(a.gz + k + 2);

        const float *row = rg.ringA + (pc & (kRingA - 1)) * Cfg::kSlotA + wk.offA;
        const float4 xl = lds4(row - 4);   // cells x-4 .. x-1 of lane 0
        const float4 xc = wk.q[QI(4)];
        const float4 xr = lds4(row + 4);   // cells x+4 .. x+7 of lane 0
        float4 yp[4], ym[4];
#pragma unroll
        for (int m = 1; m <= 4; ++m) {
            yp[m - 1] = lds4(row + m * Cfg::kRowW);
            ym[m - 1] = lds4(row - m * Cfg::kRowW);
        }
        release_a(rg, mp, pc, wk.nplanes, i0, j0, wk.z0);

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
        float2 o[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            float2 s[5];
#pragma unroll
            for (int m = 1; m <= 4; ++m) {
                const float2 sy = add2(pair(yp[m - 1], p), pair(ym[m - 1], p));
                const float2 sz = add2(pair(wk.q[QI(4 + m)], p), pair(wk.q[QI(4 - m)], p));
                s[m] = add2(add2(sx[p][m], sy), sz);
            }
            float2 lap = mul2(splat(a.c.c4), s[4]);
            lap = fma2(splat(a.c.c3), s[3], lap);
            lap = fma2(splat(a.c.c2), s[2], lap);
            lap = fma2(splat(a.c.c1), s[1], lap);
            const float2 uc = pair(xc, p);
            lap = fma2(splat(a.c.c0x3), uc, lap);
            const float2 gd = mul2(pair(wk.gxy, p), splat(gzk));
            const float2 ngd = mul2(pair(wk.gxy, p), splat(-gzk));   // -gd, exactly
            const float2 t = fma2(pair(wc, p), lap, fma2(splat(2.0f), uc, mul2(ngd, pair(upc, p))));
            o[p] = mul2(gd, t);
        }
        float4 out = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        if (wk.src_mask) {
            for (int qs = 0; qs < a.src.n; ++qs) {
                const SourceSample &ss = a.src.s[qs];
                if (((wk.src_mask >> qs) & 1u) && ss.k == k && ss.j == j) {
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        if (ss.i == i + l) set_comp(out, l, fmaf(comp(wc, l), ss.amp, comp(out, l)));
                }
            }
        }
        if (wk.col_ok) {
            float *dst = wk.out_k;
            if (wk.nvalid == 4) {
                __stcs(reinterpret_cast<float4 *>(dst), out);
            } else {
                dst[0] = out.x;
                if (wk.nvalid > 1) dst[1] = out.y;
                if (wk.nvalid > 2) dst[2] = out.z;
            }
        }
        wk.out_k += wk.plane;
        if (k == wk.rnext_k) {
            while (wk.rcur < wk.rend && rec[wk.rcur].k == k) {
                const RecEntry er = rec[wk.rcur];
                if (er.owner == (int)threadIdx.x)
                    a.traces[(long long)er.r * a.nt_max + a.trace_step] = comp(out, er.lane);
                ++wk.rcur;
            }
            wk.rnext_k = wk.rcur < wk.rend ? rec[wk.rcur].k : INT_MAX;
        }
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
};

template <int TX, int TY>
__global__ void __launch_bounds__((TX / 4) * TY, 2)
    step_stream_kernel(const __grid_constant__ StreamMaps maps, float *__restrict__ up,
                       const __grid_constant__ StepArgs a, const int zb,
                       const int *__restrict__ rec_ptr, const RecEntry *__restrict__ rec) {
    using K = Kern<TX, TY>;
    using Cfg = typename K::Cfg;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t fullA[kRingA], fullB[kRingB];
    __shared__ int arrivedA[kRingA], arrivedB[kRingB], issuedA[kRingA], issuedB[kRingB];
    __shared__ int s_abort;

    const Geom &g = a.g;
    const int tiles_x = (g.nx + TX - 1) / TX;
    const int tile = blockIdx.x;
    const int i0 = (tile % tiles_x) * TX;
    const int j0 = (tile / tiles_x) * TY;
    const int tid = threadIdx.x;
    const int tx = tid % (TX / 4);
    const int ty = tid / (TX / 4);
    const int i = i0 + 4 * tx;
    const int j = j0 + ty;

    Walk wk;
    wk.z0 = blockIdx.y * zb;
    wk.z1 = min(wk.z0 + zb, g.nz);
    wk.nplanes = (wk.z1 - wk.z0) + 2 * kHalo;  // ring-A planes: k in [z0-4, z1+4)
    wk.col_ok = (j < g.ny) && (i < g.nx);
    wk.nvalid = wk.col_ok ? min(4, g.nx - i) : 0;
    wk.aborted = false;
    const Rings rg{fullA, fullB, arrivedA, arrivedB, issuedA, issuedB, &s_abort, smem,
                   smem + kRingA * Cfg::kSlotA};
    const int nb = wk.z1 - wk.z0;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < kRingA; ++s) {
            mbar_init(&fullA[s], 1);
            arrivedA[s] = 0;
            issuedA[s] = 0;
        }
#pragma unroll
        for (int s = 0; s < kRingB; ++s) {
            mbar_init(&fullB[s], 1);
            arrivedB[s] = 0;
            issuedB[s] = 0;
        }
        fence_mbar_init();
        s_abort = 0;
        for (int pr = 0; pr < min(kRingA, wk.nplanes); ++pr) K::issue_a(rg, maps, pr, i0, j0, wk.z0);
        for (int bb = 0; bb < min(kRingB, nb); ++bb) K::issue_b(rg, maps, bb, i0, j0, wk.z0);
    }
    __syncthreads();

    wk.gxy = make_float4(0.f, 0.f, 0.f, 0.f);
    if (wk.col_ok) {
        const float gyj = a.gy[j];
        wk.gxy.x = a.gx[i] * gyj;
        if (wk.nvalid > 1) wk.gxy.y = a.gx[i + 1] * gyj;
        if (wk.nvalid > 2) wk.gxy.z = a.gx[i + 2] * gyj;
        if (wk.nvalid > 3) wk.gxy.w = a.gx[i + 3] * gyj;
    }

    // Sources inside this CTA's tile and planes.
    wk.src_mask = 0u;
    for (int qs = 0; qs < a.src.n; ++qs) {
        const SourceSample &ss = a.src.s[qs];
        if (ss.i >= i0 && ss.i < i0 + TX && ss.j >= j0 && ss.j < j0 + TY && ss.k >= wk.z0 &&
            ss.k < wk.z1)
            wk.src_mask |= 1u << qs;
    }

    // Receivers of this tile with k in [z0, z1), sorted by k.
    wk.rcur = wk.rend = 0;
    if (rec_ptr != nullptr) {
        wk.rcur = rec_ptr[tile];
        wk.rend = rec_ptr[tile + 1];
        while (wk.rcur < wk.rend && rec[wk.rcur].k < wk.z0) ++wk.rcur;
    }
    wk.rnext_k = wk.rcur < wk.rend ? rec[wk.rcur].k : INT_MAX;

    wk.offA = (kHalo + ty) * Cfg::kRowW + kHalo + 4 * tx;
    wk.offB = ty * TX + 4 * tx;
    wk.plane = g.plane;
    wk.out_k = up + pidx(g, i, j, 0) + (long long)wk.z0 * g.plane;

    // Prologue: queue planes z0-4 .. z0+3; z taper of planes z0, z0+1.
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        K::wait_bar(wk, rg, &fullA[m], 0u, a.status);
        if (wk.aborted) break;
        wk.q[m] = lds4(rg.ringA + m * Cfg::kSlotA + wk.offA);
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) wk.gzb[d] = (wk.z0 + d < wk.z1) ? __ldg(a.gz + wk.z0 + d) : 1.0f;

    if (!wk.aborted) {
        // planes z0-4 .. z0-1 were read only for the queue
#pragma unroll
        for (int pr = 0; pr < kHalo; ++pr) K::release_a(rg, maps, pr, wk.nplanes, i0, j0, wk.z0);

        for (int kb = wk.z0; kb < wk.z1; kb += kUnroll) {
#define WS_PLANE(R)                                                                  \
    if (kb + (R) >= wk.z1) break;                                                    \
    K::template plane_step<R>(wk, rg, maps, a, kb + (R), i, j, i0, j0, rec);         \
    if (wk.aborted) break;
            WS_PLANE(0)
            WS_PLANE(1)
            WS_PLANE(2)
#undef WS_PLANE
            K::rotate_queue(wk);
        }
    }

    // Every warp is past the loop: no more refills. After an abort, wait
    // (bounded) for the last copy issued into each slot to land before the
    // CTA exits.
    __syncthreads();
    if (s_abort && tid == 0) {
        for (int s = 0; s < kRingA + kRingB; ++s) {
            const int c = s < kRingA ? issuedA[s] : issuedB[s - kRingA];
            uint64_t *bar = s < kRingA ? &fullA[s] : &fullB[s - kRingA];
            if (c == 0) continue;
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(bar, (unsigned)(c - 1) & 1u) && global_ns() - t0 < kWaitLimitNs) {
            }
        }
    }
}

template <int TX, int TY>
cudaError_t launch_tile(const StreamMaps &maps, float *up, const StepArgs &a, int zb,
                        const int *rec_ptr, const RecEntry *rec, cudaStream_t s) {
    using Cfg = StreamCfg<TX, TY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_stream_kernel<TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::kSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((a.g.nx + TX - 1) / TX) * ((a.g.ny + TY - 1) / TY);
    const int chunks = (a.g.nz + zb - 1) / zb;
    dim3 grid(tiles, chunks, 1);
    step_stream_kernel<TX, TY><<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(maps, up, a, zb, rec_ptr, rec);
    return cudaGetLastError();
}

}  // namespace

bool stream_tiling_supported(int tx, int ty) {
    return (tx == 32 || tx == 64) && (ty == 8 || ty == 16);
}

size_t stream_smem_bytes(const StreamTiling &t) {
    return size_t(kRingA) * size_t(t.tx + 2 * kHalo) * size_t(t.ty + 2 * kHalo) * 4u +
           size_t(kRingB) * 2u * size_t(t.tx) * size_t(t.ty) * 4u;
}

cudaError_t launch_step_stream(const CUtensorMap *tmap_u, const CUtensorMap *tmap_up,
                               const CUtensorMap *tmap_w, float *up, const StepArgs &a,
                               const StreamTiling &t, const int *rec_ptr, const RecEntry *rec,
                               cudaStream_t s) {
    StreamMaps maps;
    maps.u = *tmap_u;
    maps.up = *tmap_up;
    maps.w = *tmap_w;
    if (t.tx == 64 && t.ty == 16) return launch_tile<64, 16>(maps, up, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 64 && t.ty == 8) return launch_tile<64, 8>(maps, up, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 32 && t.ty == 16) return launch_tile<32, 16>(maps, up, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 32 && t.ty == 8) return launch_tile<32, 8>(maps, up, a, t.zb, rec_ptr, rec, s);
    return cudaErrorInvalidValue;
}

}  // namespace ws
