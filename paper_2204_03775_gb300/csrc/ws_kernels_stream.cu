// Streaming step kernel for sm_103a: the hot path of the library.
//
// Each CTA owns a TX x TY tile of (x, y) columns and a block of zb planes.
// It walks its planes in increasing z. The paper keeps a whole z column in a
// processing element's memory and receives x/y neighbours from 4 PEs per
// direction over the fabric (Section III-B, III-C); here the column lives in
// a per-thread register queue of 9 planes (k-4 .. k+4), and the x/y
// neighbours come from a shared-memory copy of plane k with its 4-cell halo,
// brought in by TMA (cp.async.bulk.tensor) into a ring of NS slots that runs
// several planes ahead. u^{n-1} and (V dt/h)^2 are streamed with 128-bit
// loads one plane ahead; u^{n+1} is written in place of u^{n-1} with 128-bit
// stores. Taper, source injection and receiver sampling are fused into the
// same pass. Each thread owns 4 consecutive x cells of one row.
//
// Arithmetic per cell is the same expression, in the same order, as the
// direct kernel, so the two CUDA paths agree bit for bit.
#include "ws_internal.h"

namespace ws {
namespace {

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

// Wait for the phase of the given parity; false after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    unsigned n = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++n & 63u) == 0 && global_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
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

// One cell of the fused step; same expression as the direct kernel.
__device__ __forceinline__ float cell_update(const Coeffs &c, float uc, float s1, float s2,
                                             float s3, float s4, float wc, float gd, float upc) {
    float lap = c.c4 * s4;
    lap = fmaf(c.c3, s3, lap);
    lap = fmaf(c.c2, s2, lap);
    lap = fmaf(c.c1, s1, lap);
    lap = fmaf(c.c0x3, uc, lap);
    return gd * fmaf(wc, lap, fmaf(2.0f, uc, -gd * upc));
}

template <int TX, int TY, int NS>
struct StreamCfg {
    static constexpr int kThreads = (TX / 4) * TY;
    static constexpr int kRowW = TX + 2 * kHalo;   // floats per smem row
    static constexpr int kRows = TY + 2 * kHalo;
    static constexpr int kSlot = kRowW * kRows;    // floats per ring slot
    static constexpr unsigned kSlotBytes = kSlot * 4u;
    static_assert(kSlotBytes % 128 == 0, "ring slots must stay 128-byte aligned");
    static_assert(NS >= 8, "the prologue reads 8 planes before any slot is reused");
    static constexpr size_t kSmem = size_t(NS) * kSlotBytes;
};

template <int TX, int TY, int NS>
__global__ void __launch_bounds__((TX / 4) * TY, 2)
    step_stream_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ up,
                       const float *__restrict__ w, const __grid_constant__ StepArgs a, const int zb,
                       const int *__restrict__ rec_ptr, const RecEntry *__restrict__ rec) {
    using Cfg = StreamCfg<TX, TY, NS>;
    extern __shared__ __align__(128) float ring[];
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ int s_abort;

    const Geom &g = a.g;
    const int tiles_x = (g.nx + TX - 1) / TX;
    const int tile = blockIdx.x;
    const int i0 = (tile % tiles_x) * TX;
    const int j0 = (tile / tiles_x) * TY;
    const int z0 = blockIdx.y * zb;
    const int z1 = min(z0 + zb, g.nz);
    const int nplanes = (z1 - z0) + 2 * kHalo;  // relative planes 0..nplanes-1 = k in [z0-4, z1+4)

    const int tid = threadIdx.x;
    const int tx = tid % (TX / 4);
    const int ty = tid / (TX / 4);
    const int i = i0 + 4 * tx;
    const int j = j0 + ty;
    const bool col_ok = (j < g.ny) && (i < g.nx);
    const int nvalid = col_ok ? min(4, g.nx - i) : 0;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    // Relative plane pr holds interior plane z0 - 4 + pr, padded z index z0 + pr.
    // The box starts at padded (i0, j0): interior (i0 - 4, j0 - 4), i.e. the halo.
    int issued = 0;
    if (tid == 0) {
        const int first = min(NS, nplanes);
        for (int pr = 0; pr < first; ++pr) {
            mbar_arrive_expect_tx(&full[pr], Cfg::kSlotBytes);
            tma_load_3d(ring + pr * Cfg::kSlot, &tmap, &full[pr], i0, j0, z0 + pr);
        }
        issued = first;
    }

    bool ok = true;
    auto wait_plane = [&](int pr) {
        if (!mbar_wait_bounded(&full[pr % NS], (unsigned)((pr / NS) & 1))) {
            ok = false;
            atomicOr(a.status, kStatusTimeout);
            s_abort = 1;
        }
    };

    // Taper of this thread's columns (gx * gy), applied with gz per plane.
    float4 gxy = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col_ok) {
        const float gyj = a.gy[j];
        gxy.x = a.gx[i] * gyj;
        if (nvalid > 1) gxy.y = a.gx[i + 1] * gyj;
        if (nvalid > 2) gxy.z = a.gx[i + 2] * gyj;
        if (nvalid > 3) gxy.w = a.gx[i + 3] * gyj;
    }

    // Receivers of this tile with k in [z0, z1), sorted by k.
    int rcur = 0, rend = 0;
    if (rec_ptr != nullptr) {
        rcur = rec_ptr[tile];
        rend = rec_ptr[tile + 1];
        while (rcur < rend && rec[rcur].k < z0) ++rcur;
    }

    const int smem_col = kHalo + 4 * tx;        // this thread's first cell in a ring row
    const int smem_row = (kHalo + ty) * Cfg::kRowW;

    // Register queue: q[m] = u at plane k - 4 + m for this thread's 4 cells.
    float4 q[9];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        wait_plane(m);
        q[m] = lds4(ring + (m % NS) * Cfg::kSlot + smem_row + smem_col);
    }

    // u^{n-1} and (V dt/h)^2 of plane z0 (then one plane ahead).
    const long long col0 = pidx(g, i, j, 0);  // padded offset of (i, j, k = 0)
    float4 up_cur = make_float4(0.f, 0.f, 0.f, 0.f), w_cur = up_cur;
    if (col_ok) {
        up_cur = __ldcs(reinterpret_cast<const float4 *>(up + col0 + z0 * g.plane));
        w_cur = __ldcs(reinterpret_cast<const float4 *>(w + col0 + z0 * g.plane));
    }

    __syncthreads();
    // Planes z0-4 .. z0-1 were only needed for the queue: their slots are free.
    if (tid == 0) {
        fence_proxy_async_smem();
        for (int pr = 0; pr < kHalo; ++pr) {
            const int nxt = pr + NS;
            if (nxt < nplanes) {
                mbar_arrive_expect_tx(&full[nxt % NS], Cfg::kSlotBytes);
                tma_load_3d(ring + (nxt % NS) * Cfg::kSlot, &tmap, &full[nxt % NS], i0, j0,
                            z0 + nxt);
                issued = nxt + 1;
            }
        }
    }

#pragma unroll 1
    for (int k = z0; k < z1; ++k) {
        const int pc = k - z0 + kHalo;  // relative index of plane k
        wait_plane(pc + kHalo);
        q[8] = lds4(ring + ((pc + kHalo) % NS) * Cfg::kSlot + smem_row + smem_col);

        float4 up_nxt = make_float4(0.f, 0.f, 0.f, 0.f), w_nxt = up_nxt;
        if (col_ok && k + 1 < z1) {
            up_nxt = __ldcs(reinterpret_cast<const float4 *>(up + col0 + (k + 1) * g.plane));
            w_nxt = __ldcs(reinterpret_cast<const float4 *>(w + col0 + (k + 1) * g.plane));
        }

        const float *row = ring + (pc % NS) * Cfg::kSlot + smem_row + smem_col;
        const float4 xl = lds4(row - 4);   // cells x-4 .. x-1 of lane 0
        const float4 xc = q[4];
        const float4 xr = lds4(row + 4);   // cells x+4 .. x+7 of lane 0
        const float e[12] = {xl.x, xl.y, xl.z, xl.w, xc.x, xc.y, xc.z, xc.w,
                             xr.x, xr.y, xr.z, xr.w};
        float4 yp[4], ym[4];
#pragma unroll
        for (int m = 1; m <= 4; ++m) {
            yp[m - 1] = lds4(row + m * Cfg::kRowW);
            ym[m - 1] = lds4(row - m * Cfg::kRowW);
        }
        const float gzk = a.gz[k];

        float out[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            float s[5];
#pragma unroll
            for (int m = 1; m <= 4; ++m) {
                s[m] = ((e[4 + l + m] + e[4 + l - m]) + (comp(yp[m - 1], l) + comp(ym[m - 1], l))) +
                       (comp(q[4 + m], l) + comp(q[4 - m], l));
            }
            out[l] = cell_update(a.c, comp(xc, l), s[1], s[2], s[3], s[4], comp(w_cur, l),
                                 comp(gxy, l) * gzk, comp(up_cur, l));
        }
        for (int qs = 0; qs < a.src.n; ++qs) {
            const SourceSample &ss = a.src.s[qs];
            if (ss.k == k && ss.j == j && col_ok) {
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    if (ss.i == i + l) out[l] = fmaf(comp(w_cur, l), ss.amp, out[l]);
            }
        }

        if (col_ok) {
            float *dst = up + col0 + (long long)k * g.plane;
            if (nvalid == 4) {
                __stcs(reinterpret_cast<float4 *>(dst), make_float4(out[0], out[1], out[2], out[3]));
            } else {
#pragma unroll
                for (int l = 0; l < 3; ++l)
                    if (l < nvalid) dst[l] = out[l];
            }
        }
        while (rcur < rend && rec[rcur].k == k) {
            const RecEntry e_r = rec[rcur];
            if (e_r.owner == tid) {
                const float v = e_r.lane == 0 ? out[0]
                                : e_r.lane == 1 ? out[1]
                                : e_r.lane == 2 ? out[2]
                                                : out[3];
                a.traces[(long long)e_r.r * a.nt_max + a.trace_step] = v;
            }
            ++rcur;
        }

        up_cur = up_nxt;
        w_cur = w_nxt;
#pragma unroll
        for (int m = 0; m < 8; ++m) q[m] = q[m + 1];

        __syncthreads();  // every thread is done with slot(pc)
        if (s_abort) break;
        if (tid == 0) {
            const int nxt = pc + NS;
            if (nxt < nplanes) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[nxt % NS], Cfg::kSlotBytes);
                tma_load_3d(ring + (nxt % NS) * Cfg::kSlot, &tmap, &full[nxt % NS], i0, j0,
                            z0 + nxt);
                issued = nxt + 1;
            }
        }
    }

    // After a timeout, let the copies still in flight land before the CTA
    // exits (each wait bounded again).
    if (s_abort && tid == 0) {
        for (int pr = max(0, issued - NS); pr < issued; ++pr)
            mbar_wait_bounded(&full[pr % NS], (unsigned)((pr / NS) & 1));
    }
    (void)ok;
}

template <int TX, int TY, int NS>
cudaError_t launch_tile(const CUtensorMap *tmap, float *up, const float *w, const StepArgs &a,
                        int zb, const int *rec_ptr, const RecEntry *rec, cudaStream_t s) {
    using Cfg = StreamCfg<TX, TY, NS>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_stream_kernel<TX, TY, NS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::kSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((a.g.nx + TX - 1) / TX) * ((a.g.ny + TY - 1) / TY);
    const int chunks = (a.g.nz + zb - 1) / zb;
    dim3 grid(tiles, chunks, 1);
    step_stream_kernel<TX, TY, NS>
        <<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(*tmap, up, w, a, zb, rec_ptr, rec);
    return cudaGetLastError();
}

constexpr int kRing = 10;

}  // namespace

bool stream_tiling_supported(int tx, int ty) {
    return (tx == 32 || tx == 64) && (ty == 8 || ty == 16);
}

size_t stream_smem_bytes(const StreamTiling &t) {
    return size_t(kRing) * size_t(t.tx + 2 * kHalo) * size_t(t.ty + 2 * kHalo) * 4u;
}

cudaError_t launch_step_stream(const CUtensorMap *tmap_u, const float * /*u*/, float *up,
                               const float *w, const StepArgs &a, const StreamTiling &t,
                               const int *rec_ptr, const RecEntry *rec, cudaStream_t s) {
    if (t.tx == 64 && t.ty == 16)
        return launch_tile<64, 16, kRing>(tmap_u, up, w, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 64 && t.ty == 8)
        return launch_tile<64, 8, kRing>(tmap_u, up, w, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 32 && t.ty == 16)
        return launch_tile<32, 16, kRing>(tmap_u, up, w, a, t.zb, rec_ptr, rec, s);
    if (t.tx == 32 && t.ty == 8)
        return launch_tile<32, 8, kRing>(tmap_u, up, w, a, t.zb, rec_ptr, rec, s);
    return cudaErrorInvalidValue;
}

}  // namespace ws
