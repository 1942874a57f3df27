// Inline-PTX helpers shared by the streaming kernels (sm_100+): mbarriers,
// TMA tensor copies, whole 128/64-bit shared loads, packed FP32x2 arithmetic.
#pragma once

#include <climits>

#include "ws_internal.h"

namespace ws {

// Per-device launch facts of one kernel (see occupancy()).
struct LaunchFacts {
    static constexpr int kMaxDevices = 64;
    int ctas[kMaxDevices] = {};
    int sms[kMaxDevices] = {};
};

static __device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

static __device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

static __device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

static __device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

static __device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
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

static __device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

static __device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// 128-bit shared-memory load, kept whole: a warp reading 16-byte cells at
// 16-byte stride is conflict-free only as one 128-bit access per thread (two
// 64-bit halves would each hit every bank twice). Volatile, so it stays after
// the barrier wait that guards the data.
static __device__ __forceinline__ float4 lds4(const float *p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(smem_addr(p)));
    return v;
}

static __device__ __forceinline__ float comp(const float4 &v, int l) {
    return l == 0 ? v.x : (l == 1 ? v.y : (l == 2 ? v.z : v.w));
}

static __device__ __forceinline__ void set_comp(float4 &v, int l, float x) {
    if (l == 0) v.x = x;
    else if (l == 1) v.y = x;
    else if (l == 2) v.z = x;
    else v.w = x;
}

// Packed FP32x2 arithmetic (two independent IEEE round-to-nearest lanes).
static __device__ __forceinline__ unsigned long long as_u64(float2 v) {
    return (static_cast<unsigned long long>(__float_as_uint(v.y)) << 32) | __float_as_uint(v.x);
}
static __device__ __forceinline__ float2 as_f2(unsigned long long v) {
    return make_float2(__uint_as_float(static_cast<unsigned>(v)),
                       __uint_as_float(static_cast<unsigned>(v >> 32)));
}
static __device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
    return as_f2(r);
}
static __device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
    return as_f2(r);
}
static __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)), "l"(as_u64(c)));
    return as_f2(r);
}
static __device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
static __device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
static __device__ __forceinline__ float2 pair(const float4 &v, int p) { return p == 0 ? lo2(v) : hi2(v); }
static __device__ __forceinline__ float2 splat(float x) { return make_float2(x, x); }

// A warp is done with a ring slot: after __syncwarp orders every lane's
// reads, lane 0 alone arrives (release semantics at CTA scope) on the slot's
// "empty" barrier, whose expected count is the number of consumer warps.
static __device__ __forceinline__ void warp_arrive(uint64_t *bar) {
    __syncwarp();
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .u32 l;\n\t"
        "mov.u32 l, %%laneid;\n\t"
        "setp.eq.u32 p, l, 0;\n\t"
        "@p mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}


// A work item: one tile of columns over one block of planes. Items are
// numbered block-major (all tiles of block 0, then block 1, ...), so the
// CTAs that run at the same time work on neighbouring tiles at similar
// depths and the halo of one tile is still in L2 when its neighbour reads it.
struct Item {
    int i0, j0, z0, z1, tile;
};

static __device__ __forceinline__ Item item_of(int item, int tiles_x, int ntiles, int zb, int nz, int TX,
                                        int TY) {
    Item it;
    const int blk = item / ntiles;
    it.tile = item - blk * ntiles;
    const int ty = it.tile / tiles_x;
    it.i0 = (it.tile - ty * tiles_x) * TX;
    it.j0 = ty * TY;
    it.z0 = blk * zb;
    it.z1 = min(it.z0 + zb, nz);
    return it;
}

// Receivers: each warp of a streaming CTA owns a range of the receiver
// table sorted by plane k (the receivers whose cell one of its threads
// computes). first_entry skips to the first entry at or below plane z0 by
// binary search; record_plane stores the values of plane k: lane q takes
// entry cur + q, fetches the owning thread's cell by shuffle, and stores it.
// Every lane of the warp calls both with the same range.
static __device__ __forceinline__ int first_entry(const RecEntry *rec, int lo, int hi, int z0) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rec[mid].k < z0)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

static __device__ __forceinline__ void record_plane(const float4 &out, float scale, int k,
                                                    int *rcur, int rend, int *rnext_k,
                                                    const RecEntry *rec, float *traces, int nt_max,
                                                    long long trace_step) {
    const int lane = threadIdx.x & 31;
    int cur = *rcur;
    for (;;) {
        const int idx = cur + lane;
        RecEntry e{INT_MAX, 0, 0, 0};
        if (idx < rend) e = rec[idx];
        const bool take = e.k == k;
        const int src = e.owner & 31;
        const float v0 = __shfl_sync(0xffffffffu, out.x, src);
        const float v1 = __shfl_sync(0xffffffffu, out.y, src);
        const float v2 = __shfl_sync(0xffffffffu, out.z, src);
        const float v3 = __shfl_sync(0xffffffffu, out.w, src);
        if (take) {
            const float v = e.lane == 0 ? v0 : e.lane == 1 ? v1 : e.lane == 2 ? v2 : v3;
            traces[(long long)e.r * nt_max + trace_step] = v * scale;
        }
        const int n = __popc(__ballot_sync(0xffffffffu, take));
        cur += n;
        if (n < 32) break;
    }
    *rcur = cur;
    *rnext_k = cur < rend ? rec[cur].k : INT_MAX;
}

// A consumer leaves its loops only together with its whole warp (the
// receiver shuffles and the warp-wide arrives need every lane): after a
// failed wait in any lane, every lane's walk stops.
template <class W>
static __device__ __forceinline__ bool warp_all_ok(W &wk) {
    wk.ok = __all_sync(0xffffffffu, wk.ok);
    return wk.ok;
}

// Shared-memory state of one CTA.
template <int NA, int NB>
struct Rings {
    uint64_t fullA[NA], emptyA[NA], fullB[NB], emptyB[NB];
    int issuedA[NA], issuedB[NB];   // copies issued into each slot (for the drain)
    int abort;
};

// Bounded wait for a phase of an mbarrier. Gives up after kWaitLimitNs, or
// early once another warp has aborted; returns false then.
static __device__ __forceinline__ bool wait_phase(uint64_t *bar, unsigned parity, volatile int *abort,
                                           unsigned *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    unsigned n = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++n & 63u) == 0) {
            if (*abort) return false;
            if (global_ns() - t0 > kWaitLimitNs) {
                atomicOr(status, kStatusTimeout);
                *abort = 1;
                return false;
            }
        }
    }
    return true;
}

}  // namespace ws
