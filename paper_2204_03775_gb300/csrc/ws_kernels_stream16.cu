// Streaming step kernel with 16-bit field storage (BF16 or FP16).
//
// Same pipeline as the FP32 streaming kernel (persistent CTAs, one TMA
// producer lane, ring A for u^n with its halo, ring B for u^{n-1} and the
// model, 9-plane register queue, fused taper/source/receivers), with
// u^n and u^{n-1} stored as 16-bit numbers ((V dt/h)^2 stays FP32): 10 bytes
// per cell update instead of 16. All arithmetic is FP32.
//
// Per-field power-of-two scale. A stored field holds u * 2^e. The exponent
// of the field written by step n is chosen on the device from max|u^n|
// (accumulated while u^n was written) and a host bound on the source term,
// so that the field's largest value sits near 2^12, 16x below the FP16
// maximum; step n also accumulates max|u^{n+1}| for step n+1. Exponents and
// maxima live in a 4-slot ring (Scale16), indexed by step, so no host
// synchronization is needed.
//
// Decoding is exact and cheap: BF16 is the upper half of an FP32; for FP16,
// ((h & 0x7fff) << 13) | (sign << 16) read as an FP32 is the FP16 value times
// 2^-112 (normal and subnormal alike). The kernel computes on these "raw"
// values directly: every input of one field carries the same power-of-two
// factor, so the stencil and update are the FP32 kernel's operations on
// exactly scaled numbers, and the factors meet in two exact power-of-two
// multiplies (rp for u^{n-1}, ro for the output). The result is rounded to
// 16 bits once, when stored.
#include <climits>

#include "ws_ptx.cuh"

namespace ws {
namespace {

constexpr int kUnroll16 = 3;

// 64-bit shared load (4 x 16-bit), kept whole.
__device__ __forceinline__ uint2 lds2u(const uint16_t *p) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(smem_addr(p)));
    return v;
}

struct Bf16Fmt {
    static constexpr int kRawExp = 0;  // raw = stored value * 2^kRawExp
    static __device__ __forceinline__ float4 decode(uint2 v) {
        return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                           __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
    }
    static __device__ __forceinline__ uint2 encode(float4 f) {
        uint2 r;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r.x) : "f"(f.y), "f"(f.x));
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r.y) : "f"(f.w), "f"(f.z));
        return r;
    }
};

struct Fp16Fmt {
    static constexpr int kRawExp = -112;
    static __device__ __forceinline__ float lo(unsigned w) {
        return __uint_as_float(((w & 0x7fffu) << 13) | ((w & 0x8000u) << 16));
    }
    static __device__ __forceinline__ float hi(unsigned w) {
        return __uint_as_float(((w >> 3) & 0x0fffe000u) | (w & 0x80000000u));
    }
    static __device__ __forceinline__ float4 decode(uint2 v) {
        return make_float4(lo(v.x), hi(v.x), lo(v.y), hi(v.y));
    }
    static __device__ __forceinline__ uint2 encode(float4 f) {
        uint2 r;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r.x) : "f"(f.y), "f"(f.x));
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r.y) : "f"(f.w), "f"(f.z));
        return r;
    }
};

template <int TX, int TY, int NA, int NB>
struct Cfg16 {
    static constexpr int kConsumers = (TX / 4) * TY;
    static constexpr int kThreads = kConsumers + 32;
    static constexpr int kLead = 8;                    // halo box starts 8 cells left: 16-byte x
    static constexpr int kRowW = TX + 2 * kLead;       // elements per ring-A row
    static constexpr int kRows = TY + 2 * kHalo;
    static constexpr int kSlotA = kRowW * kRows;       // elements per ring-A slot
    static constexpr unsigned kSlotABytes = kSlotA * 2u;
    static constexpr int kTile = TX * TY;
    // ring-B slot: u^{n-1} tile (16-bit), then the (V dt/h)^2 tile (FP32)
    static constexpr unsigned kSlotBBytes = kTile * 2u + kTile * 4u;
    static constexpr int kSlotB = kSlotBBytes / 2;     // in 16-bit elements
    static_assert(kConsumers % 32 == 0, "whole consumer warps");
    static_assert((NA & (NA - 1)) == 0 && NA >= 8 && (NB & (NB - 1)) == 0 && NB >= 2, "rings");
    static_assert(kSlotABytes % 128 == 0 && kSlotBBytes % 128 == 0, "slots stay 128-byte aligned");
    static constexpr size_t kSmem = size_t(NA) * kSlotABytes + size_t(NB) * kSlotBBytes;
};

struct Maps16 {
    CUtensorMap u, up, w;
};

// 2^e as a float, e clamped to the normal range.
__device__ __forceinline__ float pow2f(int e) {
    e = max(-126, min(127, e));
    return __int_as_float((e + 127) << 23);
}

// Exponent that puts a maximum magnitude a near 2^12 (a * 2^e in [2^11, 2^12)).
__device__ __forceinline__ int scale_exponent(float a) {
    if (!(a > 0.0f) || !isfinite(a)) return 0;
    int k;
    frexpf(a, &k);
    return max(-100, min(100, 12 - k));
}

struct Walk16 {
    float4 q[9];        // raw u^n of planes k-4 .. k+4 (rotated)
    float gzb[3];       // z taper of planes k, k+1, k+2 (rotated)
    float4 gxy;
    uint16_t *out_k;
    int nvalid;
    int rcur, rend, rnext_k;
    unsigned src_mask;
    unsigned gAw, gAr, gB;
    float amax;         // running max |u^{n+1}| in output units
    bool ok;
};

template <class Fmt, int TX, int TY, int NA, int NB>
struct Kern16 {
    using Cfg = Cfg16<TX, TY, NA, NB>;
    using R = Rings<NA, NB>;

    // factors of one launch (uniform)
    struct Factors {
        float rp;     // raw u^{n-1} -> raw u^n units
        float ro;     // raw u^n -> stored u^{n+1} units
        float out2true;  // stored u^{n+1} -> u^{n+1}
        float src2out;   // true source term -> stored u^{n+1} units
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
        tma_load_3d(dst, &mp.up, &rg.fullB[slot], it.i0 + kXOff, it.j0 + kHalo, it.z0 + b + kHalo);
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
            for (int pr = 0; pr < 2 * kHalo; ++pr)
                if (!produce_a(rg, ringA, mp, gA++, it, pr, a.status)) return;
            for (int b = 0; b < nb; ++b) {
                if (!produce_b(rg, ringB, mp, gB++, it, b, a.status)) return;
                if (b + 2 * kHalo < nplanes &&
                    !produce_a(rg, ringA, mp, gA++, it, b + 2 * kHalo, a.status))
                    return;
            }
        }
    }

    template <int RQ>
    static __device__ __forceinline__ void plane_step(Walk16 &wk, R &rg, const uint16_t *ringA,
                                                      const uint16_t *ringB, const StepArgs &a,
                                                      const Factors &fc, const Item &it, int k,
                                                      int i, int j, int offA, int offB,
                                                      const RecEntry *rec) {
#define QI(m) ((RQ + (m)) % 9)
#define BI(d) ((RQ + (d)) % 3)
        {
            const int slot = wk.gAw & (NA - 1);
            wk.ok = wk.ok && wait_phase(&rg.fullA[slot], (wk.gAw / NA) & 1u, &rg.abort, a.status);
            wk.q[QI(8)] = Fmt::decode(lds2u(ringA + slot * Cfg::kSlotA + offA));
            ++wk.gAw;
        }
        const int sb = wk.gB & (NB - 1);
        wk.ok = wk.ok && wait_phase(&rg.fullB[sb], (wk.gB / NB) & 1u, &rg.abort, a.status);
        const uint16_t *tb = ringB + sb * Cfg::kSlotB;
        const float4 upc = Fmt::decode(lds2u(tb + offB));
        const float4 wr = lds4(reinterpret_cast<const float *>(tb + Cfg::kTile) + offB);
        warp_arrive(&rg.emptyB[sb]);
        ++wk.gB;

        if (k + 2 < it.z1) wk.gzb[BI(2)] = __ldg(a.gz + k + 2);

        const uint16_t *row = ringA + (wk.gAr & (NA - 1)) * Cfg::kSlotA + offA;
        const float4 xl = Fmt::decode(lds2u(row - 4));
        const float4 xc = wk.q[QI(4)];
        const float4 xr = Fmt::decode(lds2u(row + 4));
        float4 yp[4], ym[4];
#pragma unroll
        for (int m = 1; m <= 4; ++m) {
            yp[m - 1] = Fmt::decode(lds2u(row + m * Cfg::kRowW));
            ym[m - 1] = Fmt::decode(lds2u(row - m * Cfg::kRowW));
        }
        warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
        ++wk.gAr;

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
        const float gzo = gzk * fc.ro;            // exact: ro is a power of two
        const float ngzp = -gzk * fc.rp;          // exact: rp is a power of two
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
            const float2 uc = pair(xc, p);
            // sum_m c_m (s_m - 6 u): exactly zero on constants (see Coeffs)
            float2 lap = mul2(splat(a.c.c4), fma2(splat(-6.0f), uc, s[4]));
            lap = fma2(splat(a.c.c3), fma2(splat(-6.0f), uc, s[3]), lap);
            lap = fma2(splat(a.c.c2), fma2(splat(-6.0f), uc, s[2]), lap);
            lap = fma2(splat(a.c.c1), fma2(splat(-6.0f), uc, s[1]), lap);
            const float2 wv = pair(wr, p);
            const float2 gdo = mul2(pair(wk.gxy, p), splat(gzo));    // g * ro
            const float2 ngr = mul2(pair(wk.gxy, p), splat(ngzp));   // -g * rp
            const float2 t = fma2(wv, lap, fma2(splat(2.0f), uc, mul2(ngr, pair(upc, p))));
            o[p] = mul2(gdo, t);
        }
        float4 out = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        if (wk.src_mask) {
            for (int qs = 0; qs < a.src.n; ++qs) {
                const SourceSample &ss = a.src.s[qs];
                if (((wk.src_mask >> qs) & 1u) && ss.k == k && ss.j == j) {
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        if (ss.i == i + l)
                            set_comp(out, l, fmaf(comp(wr, l), ss.amp * fc.src2out, comp(out, l)));
                }
            }
        }
        if (wk.nvalid > 0) {
            wk.amax = fmaxf(wk.amax, fmaxf(fmaxf(fabsf(out.x), fabsf(wk.nvalid > 1 ? out.y : 0.f)),
                                           fmaxf(fabsf(wk.nvalid > 2 ? out.z : 0.f),
                                                 fabsf(wk.nvalid > 3 ? out.w : 0.f))));
            const uint2 st = Fmt::encode(out);
            if (wk.nvalid == 4) {
                asm volatile("st.global.cs.v2.u32 [%0], {%1, %2};" ::"l"(wk.out_k), "r"(st.x),
                             "r"(st.y)
                             : "memory");
            } else {
                wk.out_k[0] = (uint16_t)(st.x & 0xffffu);
                if (wk.nvalid > 1) wk.out_k[1] = (uint16_t)(st.x >> 16);
                if (wk.nvalid > 2) wk.out_k[2] = (uint16_t)(st.y & 0xffffu);
            }
        }
        wk.out_k += a.g.plane;
        if (k == wk.rnext_k)
            record_plane(out, fc.out2true, k, &wk.rcur, wk.rend, &wk.rnext_k, rec, a.traces,
                         a.nt_max, a.trace_step);
#undef QI
#undef BI
    }

    static __device__ __forceinline__ void rotate_queue(Walk16 &wk) {
        float4 t[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) t[m] = wk.q[(m + kUnroll16) % 9];
#pragma unroll
        for (int m = 0; m < 9; ++m) wk.q[m] = t[m];
    }

    static __device__ void consumer(R &rg, const uint16_t *ringA, const uint16_t *ringB,
                                    uint16_t *up, const StepArgs &a, const Factors &fc, int zb,
                                    int tiles_x, int ntiles, int nitems, const int *rec_ptr,
                                    const RecEntry *rec, unsigned *amax_out) {
        const Geom &g = a.g;
        const int tid = threadIdx.x;
        const int tx = tid % (TX / 4);
        const int ty = tid / (TX / 4);
        const int offA = (kHalo + ty) * Cfg::kRowW + Cfg::kLead + 4 * tx;
        const int offB = ty * TX + 4 * tx;
        Walk16 wk;
        wk.gAw = wk.gAr = wk.gB = 0;
        wk.ok = true;
        wk.amax = 0.0f;
        for (int item = blockIdx.x; item < nitems && wk.ok; item += gridDim.x) {
            const Item it = item_of(item, tiles_x, ntiles, zb, g.nz, TX, TY);
            const int i = it.i0 + 4 * tx;
            const int j = it.j0 + ty;
            const bool col_ok = (j < g.ny) && (i < g.nx);
            wk.nvalid = col_ok ? min(4, g.nx - i) : 0;
            wk.gxy = make_float4(0.f, 0.f, 0.f, 0.f);
            if (col_ok) {
                const float gyj = a.gy[j];
                wk.gxy.x = a.gx[i] * gyj;
                if (wk.nvalid > 1) wk.gxy.y = a.gx[i + 1] * gyj;
                if (wk.nvalid > 2) wk.gxy.z = a.gx[i + 2] * gyj;
                if (wk.nvalid > 3) wk.gxy.w = a.gx[i + 3] * gyj;
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
            wk.out_k = up + pidx(g, col_ok ? i : 0, col_ok ? j : 0, it.z0);
#pragma unroll
            for (int d = 0; d < 2; ++d)
                wk.gzb[d] = (it.z0 + d < it.z1) ? __ldg(a.gz + it.z0 + d) : 1.0f;

#pragma unroll
            for (int m = 0; m < 2 * kHalo; ++m) {
                const int slot = wk.gAw & (NA - 1);
                wk.ok = wk.ok && wait_phase(&rg.fullA[slot], (wk.gAw / NA) & 1u, &rg.abort, a.status);
                wk.q[m] = Fmt::decode(lds2u(ringA + slot * Cfg::kSlotA + offA));
                ++wk.gAw;
            }
#pragma unroll
            for (int m = 0; m < kHalo; ++m) {
                warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
                ++wk.gAr;
            }
            if (!warp_all_ok(wk)) break;

            for (int kb = it.z0; kb < it.z1; kb += kUnroll16) {
#define WS_PLANE(RQ)                                                                           \
    if (kb + (RQ) >= it.z1) break;                                                             \
    plane_step<RQ>(wk, rg, ringA, ringB, a, fc, it, kb + (RQ), i, j, offA, offB, rec);         \
    if (!warp_all_ok(wk)) break;
                WS_PLANE(0)
                WS_PLANE(1)
                WS_PLANE(2)
#undef WS_PLANE
                rotate_queue(wk);
            }
#pragma unroll
            for (int m = 0; m < kHalo; ++m) {
                warp_arrive(&rg.emptyA[wk.gAr & (NA - 1)]);
                ++wk.gAr;
            }
        }
        // max |u^{n+1}| of this warp, in true units, into the next step's slot
        float m = wk.amax * fc.out2true;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMax(amax_out, __float_as_uint(m));
    }
};

template <class Fmt, int TX, int TY, int NA, int NB, int MINB>
__global__ void __launch_bounds__(Cfg16<TX, TY, NA, NB>::kThreads, MINB)
    step_stream16_kernel(const __grid_constant__ Maps16 maps, uint16_t *__restrict__ up,
                         const __grid_constant__ StepArgs a, Scale16 *__restrict__ sc,
                         const long long step, const float src_hint, const int zb,
                         const int tiles_x, const int ntiles, const int nitems,
                         const int *__restrict__ rec_ptr, const RecEntry *__restrict__ rec) {
    using K = Kern16<Fmt, TX, TY, NA, NB>;
    using Cfg = typename K::Cfg;
    extern __shared__ __align__(128) uint16_t smem16[];
    __shared__ Rings<NA, NB> rg;
    uint16_t *ringA = smem16;
    uint16_t *ringB = smem16 + NA * Cfg::kSlotA;

    // scales of this step: u^n has e_n, u^{n-1} e_p; u^{n+1} gets e_o
    const int sn = (int)(step & 3), sp = (int)((step + 3) & 3), so = (int)((step + 1) & 3);
    const int e_n = sc->exps[sn], e_p = sc->exps[sp];
    const int e_o = scale_exponent(fmaxf(__uint_as_float(sc->amax[sn]), src_hint));
    typename K::Factors fc;
    fc.rp = pow2f(e_n - e_p);
    fc.ro = pow2f(e_o - e_n - Fmt::kRawExp);
    fc.out2true = pow2f(-e_o);
    fc.src2out = pow2f(e_o);

    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) {
            sc->exps[so] = e_o;
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
        K::consumer(rg, ringA, ringB, up, a, fc, zb, tiles_x, ntiles, nitems, rec_ptr, rec,
                    &sc->amax[so]);
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

template <class Fmt, int TX, int TY, int NA, int NB, int MINB>
cudaError_t launch16(const Maps16 &maps, uint16_t *up, const StepArgs &a, Scale16 *sc,
                     long long step, float src_hint, int zb, const int *rec_ptr,
                     const RecEntry *rec, cudaStream_t s) {
    using Cfg = Cfg16<TX, TY, NA, NB>;
    auto kern = step_stream16_kernel<Fmt, TX, TY, NA, NB, MINB>;
    static int ctas_per_sm = 0, sms = 0;
    if (ctas_per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::kSmem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm, kern, Cfg::kThreads,
                                                              Cfg::kSmem);
        if (e != cudaSuccess) return e;
        if (ctas_per_sm < 1) return cudaErrorInvalidConfiguration;
    }
    const int tiles_x = (a.g.nx + TX - 1) / TX;
    const int ntiles = tiles_x * ((a.g.ny + TY - 1) / TY);
    const int nitems = ntiles * ((a.g.nz + zb - 1) / zb);
    const int grid = min(nitems, sms * ctas_per_sm);
    kern<<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(maps, up, a, sc, step, src_hint, zb, tiles_x,
                                                 ntiles, nitems, rec_ptr, rec);
    return cudaGetLastError();
}

// Only 64-wide tiles: a half-warp then reads one 128-byte ring row with
// 64-bit loads, which is conflict-free; in a 32-wide tile a half-warp would
// read two rows whose banks overlap.
template <class Fmt>
cudaError_t dispatch16(const Maps16 &maps, uint16_t *up, const StepArgs &a, Scale16 *sc,
                       long long step, float src_hint, const StreamTiling &t, const int *rec_ptr,
                       const RecEntry *rec, cudaStream_t s) {
    if (t.tx == 64 && t.ty == 8)
        return launch16<Fmt, 64, 8, 8, 4, 3>(maps, up, a, sc, step, src_hint, t.zb, rec_ptr, rec, s);
    return cudaErrorInvalidValue;
}

}  // namespace

bool stream16_tiling_supported(int tx, int ty) { return tx == 64 && ty == 8; }

cudaError_t launch_step_stream16(int storage, const CUtensorMap *tmap_u, const CUtensorMap *tmap_up,
                                 const CUtensorMap *tmap_w, uint16_t *up, const StepArgs &a,
                                 Scale16 *sc, long long step, float src_hint,
                                 const StreamTiling &t, const int *rec_ptr, const RecEntry *rec,
                                 cudaStream_t s) {
    Maps16 maps;
    maps.u = *tmap_u;
    maps.up = *tmap_up;
    maps.w = *tmap_w;
    if (storage == WS_STORAGE_BF16)
        return dispatch16<Bf16Fmt>(maps, up, a, sc, step, src_hint, t, rec_ptr, rec, s);
    if (storage == WS_STORAGE_FP16)
        return dispatch16<Fp16Fmt>(maps, up, a, sc, step, src_hint, t, rec_ptr, rec, s);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ conversions

namespace {

// max |v| over the interior of a padded FP32 field into *amax (float bits).
__global__ void amax_kernel(const float *__restrict__ f, Geom g, unsigned *__restrict__ amax) {
    const int j = blockIdx.y, k = blockIdx.z;
    float m = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nx; i += gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(f[pidx(g, i, j, k)]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

// FP32 padded -> 16-bit padded (interior), exponent from sc->amax[slot];
// block (0,0,0) records the exponent in sc->exps[slot].
template <class Fmt>
__global__ void encode_kernel(const float *__restrict__ f, uint16_t *__restrict__ out, Geom g,
                              Scale16 *__restrict__ sc, int slot) {
    const int e = scale_exponent(__uint_as_float(sc->amax[slot]));
    const float s = pow2f(e);
    const int j = blockIdx.y, k = blockIdx.z;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (blockIdx.x == 0 && j == 0 && k == 0 && threadIdx.x == 0) sc->exps[slot] = e;
    if (i >= g.nx) return;
    const long long p = pidx(g, i, j, k);
    float4 v = make_float4(f[p] * s, 0.f, 0.f, 0.f);
    if (i + 1 < g.nx) v.y = f[p + 1] * s;
    if (i + 2 < g.nx) v.z = f[p + 2] * s;
    if (i + 3 < g.nx) v.w = f[p + 3] * s;
    const uint2 st = Fmt::encode(v);
    out[p] = (uint16_t)(st.x & 0xffffu);
    if (i + 1 < g.nx) out[p + 1] = (uint16_t)(st.x >> 16);
    if (i + 2 < g.nx) out[p + 2] = (uint16_t)(st.y & 0xffffu);
    if (i + 3 < g.nx) out[p + 3] = (uint16_t)(st.y >> 16);
}

// 16-bit padded -> FP32 padded (interior), with the exponent of sc->exps[slot].
template <class Fmt>
__global__ void decode_kernel(const uint16_t *__restrict__ in, float *__restrict__ f, Geom g,
                              const Scale16 *__restrict__ sc, int slot) {
    const float s = pow2f(-sc->exps[slot] - Fmt::kRawExp);
    const int j = blockIdx.y, k = blockIdx.z;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const long long p = pidx(g, i, j, k);
    const unsigned h = in[p];
    const float4 d = Fmt::decode(make_uint2(h, 0u));
    f[p] = d.x * s;
}

}  // namespace

cudaError_t launch_encode16(int storage, const float *f, uint16_t *out, const Geom &g, Scale16 *sc,
                            int slot, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&sc->amax[slot], 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    amax_kernel<<<dim3((g.nx + 255) / 256, g.ny, g.nz), 256, 0, s>>>(f, g, &sc->amax[slot]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + 4 * 128 - 1) / (4 * 128), g.ny, g.nz);
    if (storage == WS_STORAGE_BF16)
        encode_kernel<Bf16Fmt><<<grid, 128, 0, s>>>(f, out, g, sc, slot);
    else
        encode_kernel<Fp16Fmt><<<grid, 128, 0, s>>>(f, out, g, sc, slot);
    return cudaGetLastError();
}

cudaError_t launch_decode16(int storage, const uint16_t *in, float *f, const Geom &g,
                            const Scale16 *sc, int slot, cudaStream_t s) {
    dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
    if (storage == WS_STORAGE_BF16)
        decode_kernel<Bf16Fmt><<<grid, 128, 0, s>>>(in, f, g, sc, slot);
    else
        decode_kernel<Fp16Fmt><<<grid, 128, 0, s>>>(in, f, g, sc, slot);
    return cudaGetLastError();
}

}  // namespace ws
