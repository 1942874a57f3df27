// Streaming step kernel with 16-bit field storage (BF16 or FP16), velocity form.
//
// Same pipeline as the FP32 streaming kernel (one CTA per work item in item
// order, one TMA producer lane, 9-plane register queue, fused
// taper/source/receivers), but the state is stored as
//     U = u^n   and   D = u^n - u^{n-1}   (16 bits each),
// and the model as FP16 of (V dt/h)^2 * 2^kW16Exp: 10 bytes per cell update
// (read U, D, W; write U', D'). All arithmetic is FP32; the step computes
// u^{n-1} = U - D and the same tapered leapfrog update as the FP32 kernels.
//
// Why the velocity form: rounding u^{n+1} and keeping it as the next step's
// u^{n-1} makes every rounding error a kick to the discrete velocity
// u^n - u^{n-1}, and kicks integrate (relative error ~ N^1.5 eps over N
// steps). Storing D' = u~^{n+1} - u^n (from the unrounded new value) leaves
// the rounding of U' in the displacement only, and the velocity carries just
// the rounding of D', which is an order of magnitude smaller than |u|.
//
// Ring A holds U of plane k with its halo ((TX+16) x (TY+8), 16-bit), ring B
// the D and W tiles of plane k. U is double-buffered (U' goes to the other
// buffer: neighbours still read U); D is updated in place (only the thread
// that computes a cell reads its D).
//
// Instruction issue, not memory, limits a 16-bit stencil, so every value is
// decoded once: a thread decodes its own cells of plane k+4 into its register
// queue, and at plane k writes them (FP32) into a double-buffered staging
// tile; the cells around the tile that the star stencil reads (not the
// corners) are decoded into the same tile, 4 cells per consumer thread above
// and below the tile and 4 per lane of the last warp beside it. The consumer
// warps then agree at a named barrier that also ANDs their "no
// wait failed" flags (so a bounded wait that gives up stops every consumer
// warp at the same plane) and read their x/y neighbours from the staging tile
// with 128-bit loads. Each thread computes 4 x-cells of two rows.
//
// One power-of-two scale per step for U' and D' (|d| <= |u^{n+1}| + |u^n|,
// so the same exponent bounds both): stored values are value * 2^e, with e
// chosen on the device from max |u^n| (accumulated by the previous step) and
// a host bound on the source term, putting the field's largest value near
// 2^12, 16x below the FP16 maximum; exponents and maxima live in a 4-slot
// ring (Scale16) indexed by step, so no host synchronization is needed.
//
// Decoding is exact and cheap: both formats go through the hardware
// conversion, one instruction per value (for FP16 measured 6% faster than
// rebuilding the FP32 bits with integer logic; for BF16, whose bits are the
// upper half of an FP32, the same speed as shifts and masks but 2 registers
// fewer, which removed a spill). The kernel computes on the stored values:
// every input of one field carries the same power-of-two factor, the model's
// factor 2^kW16Exp is folded into the stencil weights, and the factors meet
// in exact power-of-two multiplies. Results are rounded to 16 bits once,
// when stored.
#include <climits>

#include "ws_ptx.cuh"

namespace ws {
namespace {

// 64-bit shared load (4 x 16-bit), kept whole.
__device__ __forceinline__ uint2 lds2u(const uint16_t *p) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(smem_addr(p)));
    return v;
}

// FP16 -> FP32 of the two halves of a word (exact, subnormals included).
__device__ __forceinline__ float2 f16x2_to_f32(unsigned w) {
    float2 r;
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "cvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "r"(w));
    return r;
}

struct Bf16Fmt {
    static __device__ __forceinline__ float2 two(unsigned w) {
        float2 r;
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
            "cvt.f32.bf16 %0, l;\n\tcvt.f32.bf16 %1, h;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "r"(w));
        return r;
    }
    static __device__ __forceinline__ float4 decode(uint2 v) {
        const float2 a = two(v.x), b = two(v.y);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ uint2 encode(float4 f) {
        uint2 r;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r.x) : "f"(f.y), "f"(f.x));
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r.y) : "f"(f.w), "f"(f.z));
        return r;
    }
};

struct Fp16Fmt {
    static __device__ __forceinline__ float4 decode(uint2 v) {
        const float2 a = f16x2_to_f32(v.x), b = f16x2_to_f32(v.y);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ uint2 encode(float4 f) {
        uint2 r;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r.x) : "f"(f.y), "f"(f.x));
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r.y) : "f"(f.w), "f"(f.z));
        return r;
    }
};

// Two rows per thread: a consumer thread computes the 4 x-cells i..i+3 of the
// rows j and j+1, so the per-plane costs of a thread (ring waits, barrier,
// loads of the x neighbours, bookkeeping) are spread over 8 cells and the y
// neighbours rows j-4..j-1 and j+2..j+5 serve both rows.
template <int TX, int TY, int NA, int NB>
struct Cfg16 {
    static constexpr int kCols = TX / 4;               // threads across a row
    static constexpr int kConsumers = kCols * (TY / 2);
    static constexpr int kThreads = kConsumers + 32;
    static constexpr int kLead = 8;                    // halo box starts 8 cells left: 16-byte x
    static constexpr int kRowW = TX + 2 * kLead;       // elements per ring-A row
    static constexpr int kRows = TY + 2 * kHalo;
    static constexpr int kSlotA = kRowW * kRows;       // elements per ring-A slot
    static constexpr unsigned kSlotABytes = kSlotA * 2u;
    static constexpr int kTile = TX * TY;
    static constexpr int kSlotB = 2 * kTile;           // D tile, then W tile (16-bit elements)
    static constexpr unsigned kSlotBBytes = kSlotB * 2u;
    // FP32 staging tile: columns i0-4 .. i0+TX+3, rows j0-4 .. j0+TY+3 (the
    // four corner blocks are never read by the star stencil and stay unset)
    static constexpr int kSW = TX + 2 * kHalo;
    static constexpr int kStage = kSW * kRows;
    // halo cells decoded per plane, in units of 4 cells: 2*TX units in the 8
    // rows above and below the tile (one per consumer thread), 2*TY = 32
    // units beside it (the last consumer warp, one per lane)
    static constexpr int kSideWarp = kConsumers / 32 - 1;
    static_assert(kConsumers % 32 == 0, "whole consumer warps");
    static_assert(TX % 64 == 0 && TY == 16, "64-wide tiles of 16 rows (8 row pairs)");
    static_assert(2 * TX == kConsumers && 2 * TY == 32, "one band unit per thread, one side warp");
    static_assert((NA & (NA - 1)) == 0 && NA >= 8 && (NB & (NB - 1)) == 0 && NB >= 2, "rings");
    static_assert(kSlotABytes % 128 == 0 && kSlotBBytes % 128 == 0 && (kStage * 4) % 128 == 0,
                  "slots stay 128-byte aligned");
    static constexpr size_t kSmem =
        size_t(2 * kStage) * 4u + size_t(NA) * kSlotABytes + size_t(NB) * kSlotBBytes;
};

// 128-bit shared store.
__device__ __forceinline__ void sts4(float *p, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(smem_addr(p)), "f"(v.x),
                 "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Named barrier 1 over the consumer threads that also ANDs their flags.
__device__ __forceinline__ bool consumers_all(bool ok, int nthreads) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)ok), "r"(nthreads)
        : "memory");
    return r != 0;
}

struct Maps16 {
    CUtensorMap u, d, w;
};

// 2^e as a float, e clamped to the normal range.
__device__ __forceinline__ float pow2f(int e) {
    e = max(-126, min(127, e));
    return __int_as_float((e + 127) << 23);
}

// x * 2^e for e beyond one float's exponent range, in two exact steps.
__device__ __forceinline__ float scale2(float x, int e) {
    const int h = e / 2;
    return x * pow2f(h) * pow2f(e - h);
}

// Exponent that puts a maximum magnitude a near 2^12 (a * 2^e in [2^11, 2^12)).
__device__ __forceinline__ int scale_exponent(float a) {
    if (!(a > 0.0f) || !isfinite(a)) return 0;
    int k;
    frexpf(a, &k);
    return max(-100, min(100, 12 - k));
}

// Receivers of a two-row thread: RecEntry.lane = 4 * row + x cell. Lane q of
// the warp takes entry cur + q, fetches the owner's 8 values by shuffle and
// stores the one it names.
__device__ __forceinline__ void record_plane2(const float4 (&out)[2], float scale, int k, int *rcur,
                                              int rend, int *rnext_k, const RecEntry *rec,
                                              float *traces, int nt_max, long long trace_step) {
    const int lane = threadIdx.x & 31;
    int cur = *rcur;
    for (;;) {
        const int idx = cur + lane;
        RecEntry e{INT_MAX, 0, 0, 0};
        if (idx < rend) e = rec[idx];
        const bool take = e.k == k;
        const int src = e.owner & 31;
        float v[8];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            v[4 * r + 0] = __shfl_sync(0xffffffffu, out[r].x, src);
            v[4 * r + 1] = __shfl_sync(0xffffffffu, out[r].y, src);
            v[4 * r + 2] = __shfl_sync(0xffffffffu, out[r].z, src);
            v[4 * r + 3] = __shfl_sync(0xffffffffu, out[r].w, src);
        }
        if (take) {
            float x = v[0];
#pragma unroll
            for (int l = 1; l < 8; ++l)
                if (e.lane == l) x = v[l];
            traces[(long long)e.r * nt_max + trace_step] = x * scale;
        }
        const int n = __popc(__ballot_sync(0xffffffffu, take));
        cur += n;
        if (n < 32) break;
    }
    *rcur = cur;
    *rnext_k = cur < rend ? rec[cur].k : INT_MAX;
}

// Rarely taken paths of a plane. (Moving them out of line, as calls, to
// shrink the unrolled loop measured 2 % slower: the calls cost registers.)

// Sources of this plane inside the thread's 8 cells: u~ += (W h^2 s) in
// stored units (src_mask: the CTA's sources).
__device__ __forceinline__ void inject_sources(float4 *un, const float4 *wr, unsigned src_mask,
                                            const Sources &src, int i, int j, int k, float wtrue,
                                            float amp2r) {
    for (int qs = 0; qs < src.n; ++qs) {
        const SourceSample &ss = src.s[qs];
        if (((src_mask >> qs) & 1u) && ss.k == k) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (ss.j != j + r) continue;
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    if (ss.i == i + l)
                        set_comp(un[r], l, fmaf(comp(wr[r], l) * wtrue, ss.amp * amp2r,
                                                comp(un[r], l)));
            }
        }
    }
}

// Stores of a thread with cells outside the grid (nvalid < 4 or no row j+1).
__device__ __forceinline__ void store_partial(uint16_t *p, long long d_delta, int pitch, uint2 su0,
                                           uint2 sd0, uint2 su1, uint2 sd1, int nvalid,
                                           bool row1) {
    const uint2 su[2] = {su0, su1}, sd[2] = {sd0, sd1};
    for (int r = 0; r < (row1 ? 2 : 1); ++r) {
        uint16_t *o = p + r * pitch;
        for (int l = 0; l < nvalid; ++l) {
            const unsigned wu = l < 2 ? su[r].x : su[r].y, wd = l < 2 ? sd[r].x : sd[r].y;
            o[l] = (uint16_t)((l & 1) ? (wu >> 16) : (wu & 0xffffu));
            o[l + d_delta] = (uint16_t)((l & 1) ? (wd >> 16) : (wd & 0xffffu));
        }
    }
}

// Receivers of plane k (see record_plane2), values in true units; returns
// the new (cursor, next plane).
__device__ __forceinline__ int2 record16(float4 u0, float4 u1, int r2t, int k, int rcur, int rend,
                                      const RecEntry *rec, float *traces, int nt_max,
                                      long long trace_step) {
    const float4 ut[2] = {make_float4(scale2(u0.x, r2t), scale2(u0.y, r2t), scale2(u0.z, r2t),
                                      scale2(u0.w, r2t)),
                          make_float4(scale2(u1.x, r2t), scale2(u1.y, r2t), scale2(u1.z, r2t),
                                      scale2(u1.w, r2t))};
    int next = INT_MAX;
    record_plane2(ut, 1.0f, k, &rcur, rend, &next, rec, traces, nt_max, trace_step);
    return make_int2(rcur, next);
}

struct Walk16 {
    float4 q[9][2];     // u^n (stored units) of planes k-4 .. k+4, rows j and j+1 (rotated)
    float gzb[3];       // z taper of planes k, k+1, k+2 (rotated)
    float4 gxy[2];
    uint16_t *out_k;    // U' of (i, j, k); D of it at out_k + d_delta, row j+1 one pitch on
    int nvalid;         // valid x cells of the rows (0: none)
    bool row1;          // row j+1 inside the grid
    bool full;          // all 8 cells inside the grid
    int rcur, rend, rnext_k;
    unsigned src_mask;
    unsigned gAw, gAr, gB;
    float amax;         // running max |u~| in stored units
    bool ok;
};

// A thread's halo units: ring-A element offset and staging offset of its 4
// cells above or below the tile, and (last consumer warp) of its 4 cells
// beside the tile.
struct Halo {
    int band_src, band_dst, side_src, side_dst;
};

template <class Fmt, int TX, int TY, int NA, int NB, int NU>
struct Kern16 {
    using Cfg = Cfg16<TX, TY, NA, NB>;
    using R = Rings<NA, NB>;

    // factors of one launch (uniform)
    struct Factors {
        Coeffs c;       // stencil weights times 2^-kW16Exp: absorbs the model's factor
        float wtrue;    // stored W -> (V dt/h)^2
        float amp2r;    // source amplitude (h^2 s) -> stored U units
        float ro;       // u~ and u~ - u (stored U units) -> stored U' and D' values
        int r2t;        // stored U units -> true units: times 2^r2t
    };

    static __device__ __forceinline__ bool produce_a(R &rg, uint16_t *ringA, const Maps16 &mp,
                                                     unsigned g, const Item &it, int pr,
                                                     unsigned *status) {
        const int slot = g & (NA - 1);
        if (!wait_phase(&rg.emptyA[slot], ((g / NA) & 1u) ^ 1u, &rg.abort, status)) return false;
        rg.issuedA[slot]++;
        mbar_arrive_expect_tx(&rg.fullA[slot], Cfg::kSlotABytes);
        // box corner at interior (i0 - 8, j0 - 4, z0 - 4 + pr): padded (i0 + kXOff - 8, j0, z0 + pr)
        tma_load_3d(ringA + slot * Cfg::kSlotA, &mp.u, &rg.fullA[slot], it.i0 + kXOff - Cfg::kLead,
                    it.j0, it.z0 + pr);
        return true;
    }

    static __device__ __forceinline__ bool produce_b(R &rg, uint16_t *ringB, const Maps16 &mp,
                                                     unsigned g, const Item &it, int b,
                                                     unsigned *status) {
        const int slot = g & (NB - 1);
        if (!wait_phase(&rg.emptyB[slot], ((g / NB) & 1u) ^ 1u, &rg.abort, status)) return false;
        rg.issuedB[slot]++;
        uint16_t *dst = ringB + slot * Cfg::kSlotB;
        mbar_arrive_expect_tx(&rg.fullB[slot], Cfg::kSlotBBytes);
        tma_load_3d(dst, &mp.d, &rg.fullB[slot], it.i0 + kXOff, it.j0 + kHalo, it.z0 + b + kHalo);
        tma_load_3d(dst + Cfg::kTile, &mp.w, &rg.fullB[slot], it.i0 + kXOff, it.j0 + kHalo,
                    it.z0 + b + kHalo);
        return true;
    }

    static __device__ void producer(R &rg, uint16_t *ringA, uint16_t *ringB, const Maps16 &mp,
                                    const StepArgs &a, int zb, int tiles_x, int ntiles,
                                    int nitems) {
        unsigned gA = 0, gB = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            const Item it = item_of(item, tiles_x, ntiles, zb, a.g.nz, TX, TY);
            const int nb = it.z1 - it.z0, nplanes = nb + 2 * kHalo;
            for (int pr = 0; pr < 2 * kHalo; ++pr) {
                if (pr == 0 && item == a.stall_item) {   // test hook: never filled, so the
                    ++gA;                                 // consumers' bounded waits run out
                    continue;
                }
                if (!produce_a(rg, ringA, mp, gA++, it, pr, a.status)) return;
            }
            for (int b = 0; b < nb; ++b) {
                if (!produce_b(rg, ringB, mp, gB++, it, b, a.status)) return;
                if (b + 2 * kHalo < nplanes &&
                    !produce_a(rg, ringA, mp, gA++, it, b + 2 * kHalo, a.status))
                    return;
            }
        }
    }

    // 4 stored values (8 bytes), streaming store.
    static __device__ __forceinline__ void store16(uint16_t *p, const uint2 st) {
        asm volatile("st.global.cs.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(st.x), "r"(st.y)
                     : "memory");
    }

    static __device__ __forceinline__ Halo halo_units(int tid) {
        Halo h;
        const int band = tid / Cfg::kCols, n = tid - band * Cfg::kCols;
        int y = band < kHalo ? band : TY + band;            // rows 0..3, TY+4..TY+7
        int c = kHalo + 4 * n;                                // staging column
        h.band_src = y * Cfg::kRowW + c + (Cfg::kLead - kHalo);
        h.band_dst = y * Cfg::kSW + c;
        const int v = tid & 31;
        y = kHalo + (v >> 1);
        c = (v & 1) ? TX + kHalo : 0;
        h.side_src = y * Cfg::kRowW + c + (Cfg::kLead - kHalo);
        h.side_dst = y * Cfg::kSW + c;
        return h;
    }

    // u~ (stored units) of one row's 4 cells: the tapered leapfrog update of the FP32
    // kernels, in their operation order. yp/ym: rows j+m / j-m of this row.
    template <int RQ>
    static __device__ __forceinline__ float4 update_row(const Walk16 &wk, int r, const float4 &xl,
                                                        const float4 &xr, const float4 (&yp)[4],
                                                        const float4 (&ym)[4], const float4 &dc,
                                                        const float4 &wr, float gzk,
                                                        const Factors &fc) {
        const float4 xc = wk.q[(RQ + 4) % 9][r];
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
        float2 o[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            float2 s[5];
#pragma unroll
            for (int m = 1; m <= 4; ++m) {
                const float2 sy = add2(pair(yp[m - 1], p), pair(ym[m - 1], p));
                const float2 sz = add2(pair(wk.q[(RQ + 4 + m) % 9][r], p),
                                       pair(wk.q[(RQ + 4 - m + 9) % 9][r], p));
                s[m] = add2(add2(sx[p][m], sy), sz);
            }
            const float2 uc = pair(xc, p);
            // sum_m c_m (s_m - 6 u): exactly zero on constants (see Coeffs)
            float2 lap = mul2(splat(fc.c.c4), fma2(splat(-6.0f), uc, s[4]));
            lap = fma2(splat(fc.c.c3), fma2(splat(-6.0f), uc, s[3]), lap);
            lap = fma2(splat(fc.c.c2), fma2(splat(-6.0f), uc, s[2]), lap);
            lap = fma2(splat(fc.c.c1), fma2(splat(-6.0f), uc, s[1]), lap);
            const float2 um = add2(uc, mul2(splat(-1.0f), pair(dc, p)));     // u^{n-1}
            const float2 gd = mul2(pair(wk.gxy[r], p), splat(gzk));
            const float2 ngd = mul2(pair(wk.gxy[r], p), splat(-gzk));        // -gd, exactly
            const float2 t = fma2(pair(wr, p), lap, fma2(splat(2.0f), uc, mul2(ngd, um)));
            o[p] = mul2(gd, t);                                              // u~
        }
        return make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
    }

    template <int RQ>
    static __device__ __forceinline__ void plane_step(Walk16 &wk, R &rg, const uint16_t *ringA,
                                                      const uint16_t *ringB, float *stage,
                                                      const StepArgs &a, const Factors &fc,
                                                      long long d_delta, const Halo &hu, int k,
                                                      int i, int j, int offA, int offB, int offS,
                                                      const RecEntry *rec) {
        constexpr int Q8 = (RQ + 8) % 9, Q4 = (RQ + 4) % 9;
        // plane k+4 of this thread's two rows -> the queue
        {
            const int slot = wk.gAw & (NA - 1);
            wk.ok = wait_phase(&rg.fullA[slot], (wk.gAw / NA) & 1u, &rg.abort, a.status) && wk.ok;
            const uint16_t *p = ringA + slot * Cfg::kSlotA + offA;
            wk.q[Q8][0] = Fmt::decode(lds2u(p));
            wk.q[Q8][1] = Fmt::decode(lds2u(p + Cfg::kRowW));
            ++wk.gAw;
        }
        const int sb = wk.gB & (NB - 1);
        wk.ok = wait_phase(&rg.fullB[sb], (wk.gB / NB) & 1u, &rg.abort, a.status) && wk.ok;
        const uint16_t *tb = ringB + sb * Cfg::kSlotB + offB;
        const float4 dc0 = Fmt::decode(lds2u(tb)), dc1 = Fmt::decode(lds2u(tb + TX));
        const float4 wr0 = Fp16Fmt::decode(lds2u(tb + Cfg::kTile));
        const float4 wr1 = Fp16Fmt::decode(lds2u(tb + Cfg::kTile + TX));
        warp_arrive(&rg.emptyB[sb]);
        ++wk.gB;

        wk.gzb[(RQ + 2) % 3] = __ldg(a.gz + min(k + 2, a.g.nz - 1));   // past nz: unused

        // staging tile of plane k: this thread's own two rows (decoded four
        // planes ago), and its halo unit from the ring; then every consumer
        // agrees before anyone reads a neighbour
        float *st = stage + (k & 1) * Cfg::kStage;
        sts4(st + offS, wk.q[Q4][0]);
        sts4(st + offS + Cfg::kSW, wk.q[Q4][1]);
        {
            const uint16_t *src = ringA + (wk.gAr & (NA - 1)) * Cfg::kSlotA;
            sts4(st + hu.band_dst, Fmt::decode(lds2u(src + hu.band_src)));
            if ((threadIdx.x >> 5) == Cfg::kSideWarp)
                sts4(st + hu.side_dst, Fmt::decode(lds2u(src + hu.side_src)));
        }
        wk.ok = consumers_all(wk.ok, Cfg::kConsumers);
        warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
        ++wk.gAr;

        const float *row = st + offS;
        const float4 xl0 = lds4(row - 4), xr0 = lds4(row + 4);
        const float4 xl1 = lds4(row + Cfg::kSW - 4), xr1 = lds4(row + Cfg::kSW + 4);
        // rows j-4..j-1 and j+2..j+5
        float4 lm[4], lp[4];
#pragma unroll
        for (int m = 1; m <= 4; ++m) {
            lm[m - 1] = lds4(row - m * Cfg::kSW);
            lp[m - 1] = lds4(row + (m + 1) * Cfg::kSW);
        }
        const float gzk = wk.gzb[RQ % 3];
        float4 un[2];
        {
            const float4 yp[4] = {wk.q[Q4][1], lp[0], lp[1], lp[2]};
            un[0] = update_row<RQ>(wk, 0, xl0, xr0, yp, lm, dc0, wr0, gzk, fc);
        }
        {
            const float4 ym[4] = {wk.q[Q4][0], lm[0], lm[1], lm[2]};
            un[1] = update_row<RQ>(wk, 1, xl1, xr1, lp, ym, dc1, wr1, gzk, fc);
        }
        if (wk.src_mask) {
            float4 t[2] = {un[0], un[1]};
            const float4 w[2] = {wr0, wr1};
            inject_sources(t, w, wk.src_mask, a.src, i, j, k, fc.wtrue, fc.amp2r);
            un[0] = t[0];
            un[1] = t[1];
        }
        // cells outside the grid have zero taper, so zero u~: no guard needed
        wk.amax = fmaxf(wk.amax, fmaxf(fmaxf(fmaxf(fabsf(un[0].x), fabsf(un[0].y)),
                                             fmaxf(fabsf(un[0].z), fabsf(un[0].w))),
                                       fmaxf(fmaxf(fabsf(un[1].x), fabsf(un[1].y)),
                                             fmaxf(fabsf(un[1].z), fabsf(un[1].w)))));
        // increments u~ - u, then the stored values of both rows
        uint2 su[2], sd[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float4 xc = wk.q[Q4][r];
            const float2 d0 = add2(lo2(un[r]), make_float2(-xc.x, -xc.y));
            const float2 d1 = add2(hi2(un[r]), make_float2(-xc.z, -xc.w));
            const float2 u0 = mul2(lo2(un[r]), splat(fc.ro)), u1 = mul2(hi2(un[r]), splat(fc.ro));
            const float2 e0 = mul2(d0, splat(fc.ro)), e1 = mul2(d1, splat(fc.ro));
            su[r] = Fmt::encode(make_float4(u0.x, u0.y, u1.x, u1.y));
            sd[r] = Fmt::encode(make_float4(e0.x, e0.y, e1.x, e1.y));
        }
        if (wk.full) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                store16(wk.out_k + r * a.g.pnx, su[r]);
                store16(wk.out_k + r * a.g.pnx + d_delta, sd[r]);
            }
        } else if (wk.nvalid > 0) {
            store_partial(wk.out_k, d_delta, a.g.pnx, su[0], sd[0], su[1], sd[1], wk.nvalid,
                          wk.row1);
        }
        wk.out_k += a.g.plane;
        if (k == wk.rnext_k) {
            const int2 rc = record16(un[0], un[1], fc.r2t, k, wk.rcur, wk.rend, rec, a.traces,
                                     a.nt_max, a.trace_step);
            wk.rcur = rc.x;
            wk.rnext_k = rc.y;
        }
    }

    // planes kb + RQ .. kb + NU - 1 of a group; false once the item ends
    template <int RQ>
    static __device__ __forceinline__ bool planes(Walk16 &wk, R &rg, const uint16_t *ringA,
                                                  const uint16_t *ringB, float *stage,
                                                  const StepArgs &a, const Factors &fc,
                                                  long long d_delta, const Halo &hu,
                                                  const Item &it, int kb, int i, int j, int offA,
                                                  int offB, int offS, const RecEntry *rec) {
        if constexpr (RQ < NU) {
            // wk.ok is the same in every consumer after a staging barrier
            if (kb + RQ >= it.z1 || !wk.ok) return false;
            plane_step<RQ>(wk, rg, ringA, ringB, stage, a, fc, d_delta, hu, kb + RQ, i, j, offA,
                           offB, offS, rec);
            return planes<RQ + 1>(wk, rg, ringA, ringB, stage, a, fc, d_delta, hu, it, kb, i, j,
                                  offA, offB, offS, rec);
        }
        return true;
    }

    static __device__ __forceinline__ void rotate_queue(Walk16 &wk) {
        if constexpr (NU % 9 != 0) {
            float4 t[9][2];
#pragma unroll
            for (int m = 0; m < 9; ++m) {
                t[m][0] = wk.q[(m + NU) % 9][0];
                t[m][1] = wk.q[(m + NU) % 9][1];
            }
#pragma unroll
            for (int m = 0; m < 9; ++m) {
                wk.q[m][0] = t[m][0];
                wk.q[m][1] = t[m][1];
            }
        }
        if constexpr (NU % 3 != 0) {
            const float t0 = wk.gzb[NU % 3], t1 = wk.gzb[(NU + 1) % 3], t2 = wk.gzb[(NU + 2) % 3];
            wk.gzb[0] = t0;
            wk.gzb[1] = t1;
            wk.gzb[2] = t2;
        }
    }

    static __device__ __forceinline__ void consumer(R &rg, const uint16_t *ringA,
                                                    const uint16_t *ringB, float *stage,
                                                    uint16_t *u_out, long long d_delta,
                                    const StepArgs &a, const Factors &fc, int zb, int tiles_x,
                                    int ntiles, int nitems, const int *rec_ptr,
                                    const RecEntry *rec, unsigned *amax_out) {
        const Geom &g = a.g;
        const int tid = threadIdx.x;
        const int tx = tid % Cfg::kCols;
        const int py = tid / Cfg::kCols;
        const int offA = (kHalo + 2 * py) * Cfg::kRowW + Cfg::kLead + 4 * tx;
        const int offB = 2 * py * TX + 4 * tx;
        const int offS = (kHalo + 2 * py) * Cfg::kSW + kHalo + 4 * tx;
        const Halo hu = halo_units(tid);
        Walk16 wk;
        wk.gAw = wk.gAr = wk.gB = 0;
        wk.ok = true;
        wk.amax = 0.0f;
        for (int item = blockIdx.x; item < nitems && wk.ok; item += gridDim.x) {
            const Item it = item_of(item, tiles_x, ntiles, zb, g.nz, TX, TY);
            const int i = it.i0 + 4 * tx;
            const int j = it.j0 + 2 * py;
            const bool col_ok = (j < g.ny) && (i < g.nx);
            wk.nvalid = col_ok ? min(4, g.nx - i) : 0;
            wk.row1 = j + 1 < g.ny;
            wk.full = wk.nvalid == 4 && wk.row1;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                wk.gxy[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (col_ok && j + r < g.ny) {
                    const float gyj = a.gy[j + r];
                    wk.gxy[r].x = a.gx[i] * gyj;
                    if (wk.nvalid > 1) wk.gxy[r].y = a.gx[i + 1] * gyj;
                    if (wk.nvalid > 2) wk.gxy[r].z = a.gx[i + 2] * gyj;
                    if (wk.nvalid > 3) wk.gxy[r].w = a.gx[i + 3] * gyj;
                }
            }
            wk.src_mask = 0u;
            for (int qs = 0; qs < a.src.n; ++qs) {
                const SourceSample &ss = a.src.s[qs];
                if (ss.i >= it.i0 && ss.i < it.i0 + TX && ss.j >= it.j0 && ss.j < it.j0 + TY &&
                    ss.k >= it.z0 && ss.k < it.z1)
                    wk.src_mask |= 1u << qs;
            }
            wk.rcur = wk.rend = 0;
            if (rec_ptr != nullptr) {
                const int r = it.tile * (Cfg::kConsumers / 32) + (tid >> 5);
                wk.rend = rec_ptr[r + 1];
                wk.rcur = first_entry(rec, rec_ptr[r], wk.rend, it.z0);
            }
            wk.rnext_k = wk.rcur < wk.rend ? rec[wk.rcur].k : INT_MAX;
            wk.out_k = u_out + pidx(g, col_ok ? i : 0, col_ok ? j : 0, it.z0);
#pragma unroll
            for (int d = 0; d < 2; ++d)
                wk.gzb[d] = (it.z0 + d < g.nz) ? __ldg(a.gz + it.z0 + d) : 1.0f;

#pragma unroll
            for (int m = 0; m < 2 * kHalo; ++m) {
                const int slot = wk.gAw & (NA - 1);
                wk.ok = wk.ok && wait_phase(&rg.fullA[slot], (wk.gAw / NA) & 1u, &rg.abort, a.status);
                const uint16_t *p = ringA + slot * Cfg::kSlotA + offA;
                wk.q[m][0] = Fmt::decode(lds2u(p));
                wk.q[m][1] = Fmt::decode(lds2u(p + Cfg::kRowW));
                ++wk.gAw;
            }
#pragma unroll
            for (int m = 0; m < kHalo; ++m) {
                warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
                ++wk.gAr;
            }
            // every consumer leaves together (the staging barrier needs all)
            wk.ok = consumers_all(wk.ok, Cfg::kConsumers);
            if (!wk.ok) break;

            for (int kb = it.z0; kb < it.z1; kb += NU) {
                if (!planes<0>(wk, rg, ringA, ringB, stage, a, fc, d_delta, hu, it, kb, i, j,
                               offA, offB, offS, rec))
                    break;
                rotate_queue(wk);
            }
            if (!wk.ok) break;
#pragma unroll
            for (int m = 0; m < kHalo; ++m) {
                warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
                ++wk.gAr;
            }
        }
        // max |u^{n+1}| of this warp, in true units, into the next step's slot
        float m = scale2(wk.amax, fc.r2t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMax(amax_out, __float_as_uint(m));
    }
};

template <class Fmt, int TX, int TY, int NA, int NB, int NU, int MINB>
__global__ void __launch_bounds__(Cfg16<TX, TY, NA, NB>::kThreads, MINB)
    step_stream16_kernel(const __grid_constant__ Maps16 maps, uint16_t *__restrict__ u_out,
                         uint16_t *d_io, const __grid_constant__ StepArgs a,
                         Scale16 *__restrict__ sc, const long long step, const float src_hint,
                         const int zb, const int tiles_x, const int ntiles, const int nitems,
                         const int *__restrict__ rec_ptr, const RecEntry *__restrict__ rec) {
    using K = Kern16<Fmt, TX, TY, NA, NB, NU>;
    using Cfg = typename K::Cfg;
    extern __shared__ __align__(128) float smem16[];
    __shared__ Rings<NA, NB> rg;
    float *stage = smem16;
    uint16_t *ringA = reinterpret_cast<uint16_t *>(smem16 + 2 * Cfg::kStage);
    uint16_t *ringB = ringA + NA * Cfg::kSlotA;

    // scale of this step: U, D of step n have e; U', D' get e_o
    const int sn = (int)(step & 3), so = (int)((step + 1) & 3);
    const int e = sc->e[sn];
    const int e_o = scale_exponent(fmaxf(__uint_as_float(sc->amax[sn]), src_hint));
    typename K::Factors fc;
    const float cw = pow2f(-kW16Exp);
    fc.c = Coeffs{a.c.c1 * cw, a.c.c2 * cw, a.c.c3 * cw, a.c.c4 * cw};
    fc.wtrue = cw;
    fc.amp2r = scale2(1.0f, e);
    fc.ro = pow2f(e_o - e);
    fc.r2t = -e;

    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) {
            sc->e[so] = e_o;
            sc->amax[(step + 2) & 3] = 0u;  // accumulated by the next step
        }
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
        if (threadIdx.x == Cfg::kConsumers)
            K::producer(rg, ringA, ringB, maps, a, zb, tiles_x, ntiles, nitems);
    } else {
        K::consumer(rg, ringA, ringB, stage, u_out, d_io - u_out, a, fc, zb, tiles_x, ntiles,
                    nitems, rec_ptr, rec, &sc->amax[so]);
    }

    __syncthreads();
    if (rg.abort && threadIdx.x == 0) {
        for (int s = 0; s < NA + NB; ++s) {
            const int c = s < NA ? rg.issuedA[s] : rg.issuedB[s - NA];
            uint64_t *bar = s < NA ? &rg.fullA[s] : &rg.fullB[s - NA];
            if (c == 0) continue;
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(bar, (unsigned)(c - 1) & 1u) && global_ns() - t0 < kWaitLimitNs) {
            }
        }
    }
}

template <class Fmt, int TX, int TY, int NA, int NB, int NU, int MINB>
cudaError_t launch16(const Maps16 &maps, uint16_t *u_out, uint16_t *d_io, const StepArgs &a,
                     Scale16 *sc, long long step, float src_hint, int zb, const int *rec_ptr,
                     const RecEntry *rec, cudaStream_t s) {
    using Cfg = Cfg16<TX, TY, NA, NB>;
    auto kern = step_stream16_kernel<Fmt, TX, TY, NA, NB, NU, MINB>;
    // the shared-memory limit is a per-device property of the kernel
    static LaunchFacts lf;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= LaunchFacts::kMaxDevices) return cudaErrorInvalidDevice;
    if (lf.ctas[dev] == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg::kSmem);
        int c = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kern, Cfg::kThreads, Cfg::kSmem);
        if (e != cudaSuccess) return e;
        if (c < 1) return cudaErrorInvalidConfiguration;
        lf.ctas[dev] = c;
    }
    const int tiles_x = (a.g.nx + TX - 1) / TX;
    const int ntiles = tiles_x * ((a.g.ny + TY - 1) / TY);
    const int nitems = ntiles * ((a.g.nz + zb - 1) / zb);
    kern<<<nitems, Cfg::kThreads, Cfg::kSmem, s>>>(maps, u_out, d_io, a, sc, step, src_hint, zb,
                                                   tiles_x, ntiles, nitems, rec_ptr, rec);
    return cudaGetLastError();
}

template <class Fmt>
cudaError_t dispatch16(const Maps16 &maps, uint16_t *u_out, uint16_t *d_io, const StepArgs &a,
                       Scale16 *sc, long long step, float src_hint, const StreamTiling &t,
                       const int *rec_ptr, const RecEntry *rec, cudaStream_t s) {
    // planes 3 at a time (the queue rotates every 3 planes), 2 CTAs per SM
    // at <= 168 registers: unrolling 9 planes (no rotation) ran 4-27% slower
    // (instruction cache), a 128-register cap for 3 CTAs per SM spilled and
    // ran at half speed, and no cap (188 registers) at 60%
    if (t.tx == 64 && t.ty == 16)
        return launch16<Fmt, 64, 16, 8, 4, 3, 2>(
            maps, u_out, d_io, a, sc, step, src_hint, t.zb, rec_ptr, rec, s);
    return cudaErrorInvalidValue;
}

}  // namespace

bool stream16_tiling_supported(int tx, int ty) { return tx == 64 && ty == 16; }

cudaError_t launch_step_stream16(int storage, const CUtensorMap *tmap_u, const CUtensorMap *tmap_d,
                                 const CUtensorMap *tmap_w, uint16_t *u_out, uint16_t *d_io,
                                 const StepArgs &a, Scale16 *sc, long long step, float src_hint,
                                 const StreamTiling &t, const int *rec_ptr, const RecEntry *rec,
                                 cudaStream_t s) {
    Maps16 maps;
    maps.u = *tmap_u;
    maps.d = *tmap_d;
    maps.w = *tmap_w;
    if (storage == WS_STORAGE_BF16)
        return dispatch16<Bf16Fmt>(maps, u_out, d_io, a, sc, step, src_hint, t, rec_ptr, rec, s);
    if (storage == WS_STORAGE_FP16)
        return dispatch16<Fp16Fmt>(maps, u_out, d_io, a, sc, step, src_hint, t, rec_ptr, rec, s);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ conversions

namespace {

// max |u| and max |u - up| over the interior into *amax (float bits).
__global__ void amax2_kernel(const float *__restrict__ u, const float *__restrict__ up, Geom g,
                             unsigned *__restrict__ amax) {
    const int j = blockIdx.y, k = blockIdx.z;
    float m = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nx; i += gridDim.x * blockDim.x) {
        const long long p = pidx(g, i, j, k);
        m = fmaxf(m, fmaxf(fabsf(u[p]), fabsf(u[p] - up[p])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

// FP32 (u^n, u^{n-1}) -> U = u^n, D = u^n - u^{n-1} (16-bit, interior), with
// the exponent from the maximum of slot `slot`; block (0,0,0) records it.
template <class Fmt>
__global__ void encode_kernel(const float *__restrict__ u, const float *__restrict__ up,
                              uint16_t *__restrict__ U, uint16_t *__restrict__ D, Geom g,
                              Scale16 *__restrict__ sc, int slot) {
    const int e = scale_exponent(__uint_as_float(sc->amax[slot]));
    const int j = blockIdx.y, k = blockIdx.z;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && j == 0 && k == 0 && threadIdx.x == 0) sc->e[slot] = e;
    if (i >= g.nx) return;
    const long long p = pidx(g, i, j, k);
    const uint2 v = Fmt::encode(make_float4(scale2(u[p], e), scale2(u[p] - up[p], e), 0.f, 0.f));
    U[p] = (uint16_t)(v.x & 0xffffu);
    D[p] = (uint16_t)(v.x >> 16);
}

// U, D (16-bit) -> FP32 u^n = U, u^{n-1} = U - D (interior).
template <class Fmt>
__global__ void decode_kernel(const uint16_t *__restrict__ U, const uint16_t *__restrict__ D,
                              float *__restrict__ u, float *__restrict__ up, Geom g,
                              const Scale16 *__restrict__ sc, int slot) {
    const int j = blockIdx.y, k = blockIdx.z;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const long long p = pidx(g, i, j, k);
    const float4 v = Fmt::decode(make_uint2((unsigned)U[p] | ((unsigned)D[p] << 16), 0u));
    const float un = scale2(v.x, -sc->e[slot]);
    const float dn = scale2(v.y, -sc->e[slot]);
    u[p] = un;
    up[p] = un - dn;
}

// (V dt/h)^2 (FP32 padded) -> FP16 of value * 2^kW16Exp (interior).
__global__ void model16_kernel(const float *__restrict__ w, uint16_t *__restrict__ w16, Geom g) {
    const int j = blockIdx.y, k = blockIdx.z;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const long long p = pidx(g, i, j, k);
    unsigned short h;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(w[p] * (float)(1 << kW16Exp)));
    w16[p] = h;
}

}  // namespace

cudaError_t launch_encode16(int storage, const float *u, const float *up, uint16_t *U, uint16_t *D,
                            const Geom &g, Scale16 *sc, int slot, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&sc->amax[slot], 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    amax2_kernel<<<dim3((g.nx + 255) / 256, g.ny, g.nz), 256, 0, s>>>(u, up, g, &sc->amax[slot]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    if (storage == WS_STORAGE_BF16)
        encode_kernel<Bf16Fmt><<<grid, 128, 0, s>>>(u, up, U, D, g, sc, slot);
    else
        encode_kernel<Fp16Fmt><<<grid, 128, 0, s>>>(u, up, U, D, g, sc, slot);
    return cudaGetLastError();
}

cudaError_t launch_decode16(int storage, const uint16_t *U, const uint16_t *D, float *u, float *up,
                            const Geom &g, const Scale16 *sc, int slot, cudaStream_t s) {
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    if (storage == WS_STORAGE_BF16)
        decode_kernel<Bf16Fmt><<<grid, 128, 0, s>>>(U, D, u, up, g, sc, slot);
    else
        decode_kernel<Fp16Fmt><<<grid, 128, 0, s>>>(U, D, u, up, g, sc, slot);
    return cudaGetLastError();
}

cudaError_t launch_model16(const float *w, uint16_t *w16, const Geom &g, cudaStream_t s) {
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    model16_kernel<<<grid, 128, 0, s>>>(w, w16, g);
    return cudaGetLastError();
}

}  // namespace ws
