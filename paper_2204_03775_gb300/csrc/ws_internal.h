// Internal declarations shared by the translation units of libwavestep.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "wavestep.h"

namespace ws {

constexpr int kHalo = 4;                 // four neighbours per side (Section II)
constexpr int kMaxSources = WS_MAX_SOURCES;

// Bits of the device status word.
constexpr unsigned kStatusTimeout = 1u;

// Bounded device waits give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

// Stencil weights c_1..c_4 of the 8th-order second difference. The kernels
// evaluate sum_m c_m (s_m - 6 u), s_m the sum of the six neighbours at
// distance m: the centre weight is implied as -6 sum_m c_m, so the operator
// is exactly zero on a constant field whatever the rounding of the weights
// to float (with a separately rounded centre weight the stencil sum is off
// zero by ~2e-7, a mass term whose phase drift reached 1e-4 relative error
// after 1000 steps).
struct Coeffs {
    float c1, c2, c3, c4;
};

// The same weights in double precision, centre weight for one axis.
struct Coeffs64 {
    double c0, c1, c2, c3, c4;
};

// Per-launch source samples: cell and (h^2 * s(t_n)); the kernel multiplies
// by the stored (V dt / h)^2 of the cell, which gives (V dt)^2 s(t_n).
struct SourceSample {
    int i, j, k;
    float amp;
};
struct Sources {
    int n;
    SourceSample s[kMaxSources];
};

// Interior x offset of a padded row, in elements: 128 bytes, so that every
// interior row segment a CTA reads or writes starts on a 128-byte line and
// no 32-byte sector is written by two CTAs (a misaligned layout measured
// ~25% lower DRAM throughput for the same traffic on GB300).
#ifndef WS_XOFF
#define WS_XOFF 32
#endif
#ifndef WS_ROW_ALIGN
#define WS_ROW_ALIGN 32
#endif
constexpr int kXOff = WS_XOFF;
constexpr int kRowAlign = WS_ROW_ALIGN;  // row pitch granularity, elements
static_assert(kXOff >= 4 && kXOff % 4 == 0, "x halo of 4 cells and 16-byte TMA coordinates");

// Geometry of the padded fields: [pnz][pny][pnx], interior (i,j,k) at padded
// (i + kXOff, j + 4, k + 4). Cells outside the interior are zero. pnx is a
// multiple of kRowAlign elements (128 bytes), so every row starts on a line.
struct Geom {
    int nx, ny, nz;
    int pnx, pny, pnz;
    long long plane;  // pnx * pny
};

__host__ __device__ inline long long pidx(const Geom &g, int i, int j, int k) {
    return ((long long)(k + kHalo) * g.pny + (j + kHalo)) * g.pnx + (i + kXOff);
}

// Receivers grouped for the streaming kernels: per (xy tile, consumer warp)
// a contiguous range of entries sorted by k, ranges indexed
// tile * warps + warp. owner = thread index inside the tile's CTA (in that
// warp), lane = which of the thread's 4 x-cells, r = receiver number.
struct RecEntry {
    int k;
    int owner;
    int lane;
    int r;
};

struct StepArgs {
    Geom g;
    Coeffs c;
    Sources src;
    const float *gx, *gy, *gz;   // taper profiles (1.0 without damping)
    float *traces;               // [nrec][nt_max] or null
    int nt_max;
    long long trace_step;        // column of this step in traces
    unsigned *status;            // device status word
    float *lap;                  // if not null: receives the stencil sum L u^n (padded field)
    int stall_item;              // test hook: withhold the first copy of this work item (-1: none)
};

// Launchers (stream-ordered, no synchronization).
// out = u^{n+1} from u = u^n and up = u^{n-1}; out may be up (in place).
cudaError_t launch_step_direct(const float *u, const float *up, float *out, const float *w,
                               const StepArgs &a, cudaStream_t s);
cudaError_t launch_gather_receivers(const float *u_next, const long long *rec_pidx, int nrec,
                                    float *traces, int nt_max, long long trace_step,
                                    cudaStream_t s);
cudaError_t launch_velocity_to_w(float *w, const Geom &g, double dt_over_h,
                                 unsigned *extrema /* [2]: max bits, min bits */,
                                 cudaStream_t s);
cudaError_t launch_slowness2_to_w(float *w, const Geom &g, double dt_over_h2,
                                  unsigned *extrema /* [2]: max m bits, min m bits */,
                                  cudaStream_t s);

struct StreamTiling {
    int tx, ty, zb;
};
bool stream_tiling_supported(int tx, int ty);
// tmap_u: u^n with box (tx+8, ty+8, 1); tmap_up: u^{n-1} (written in place
// with u^{n+1} through up) and tmap_w: (V dt/h)^2, both with box (tx, ty, 1).
cudaError_t launch_step_stream(const CUtensorMap *tmap_u, const CUtensorMap *tmap_up,
                               const CUtensorMap *tmap_w, float *up, const StepArgs &a,
                               const StreamTiling &t, const int *rec_ptr, const RecEntry *rec,
                               cudaStream_t s);

// One shot of a batched step (global memory, written by the host before the
// launch). Step t of a run reads u^n from buf[cur0 ^ (t & 1)] with
// halo[cur0 ^ (t & 1)], u^{n-1} with tile[the other], writes u^{n+1} over
// u^{n-1}; src holds nsrc samples per step of the run ([t][nsrc]); trace
// column of step t = trace_col0 + t (traces null: no receivers).
// stall_item (test hook): the first step of the run withholds the first
// copy of this shot's work item stall_item (-1: none).
struct alignas(128) BatchShot {
    CUtensorMap halo[2], tile[2], w;
    float *buf[2];
    const float *gx, *gy, *gz;
    const SourceSample *src;
    float *traces;
    const int *rec_ptr;
    const RecEntry *rec;
    Geom g;
    long long trace_col0;
    int nsrc, nt_max, cur0, zb, tiles_x, ntiles, stall_item;
};

// SMs x resident CTAs of the streaming kernel (batch: the batched one) with
// tile tx x ty. Also sets the kernel's shared-memory limit, so call it once
// before capturing launches into a graph.
cudaError_t stream_slots(int tx, int ty, bool batch, int *slots);

// One launch over items[0..nitems) = (shot, item of the shot), one CTA each,
// every shot with the tile tx x ty (stream_tiling_supported).
cudaError_t launch_step_batch(const BatchShot *shots, const int2 *items, int nitems, int t,
                              const Coeffs &c, unsigned *status, int tx, int ty, cudaStream_t s);

// ---- 16-bit field storage (WS_STORAGE_BF16 / WS_STORAGE_FP16) ----
// The state is U = u^n and D = u^n - u^{n-1}, 16 bits each; the model is
// FP16 of (V dt/h)^2 * 2^kW16Exp. Ring of power-of-two exponents and maxima,
// indexed by step & 3: U and D of step n are stored as u^n * 2^e[n&3] and
// d^n * 2^e[n&3]; amax = max |u^n| (float bits, true units), accumulated by
// the step that writes u^n.
constexpr int kW16Exp = 12;
struct Scale16 {
    int e[4];
    unsigned amax[4];
};
// Stencil weights of the 16-bit kernel (centre weight c0 applied once; see
// zero_sum_weights16) and the cells whose taper is exactly 1 on each axis,
// [x0, x1) x [y0, y1) x [z0, z1) (empty ranges allowed): tiles inside them take
// the update without taper multiplies, which gives the same bits.
struct Weights16 {
    float c0, c1, c2, c3, c4;
};
struct Free16 {
    int x0, x1, y0, y1, z0, z1;
};
Weights16 zero_sum_weights16();
bool stream16_tiling_supported(int tx, int ty);
// SMs x resident CTAs of the 16-bit kernel with 64 x ty tiles.
cudaError_t stream16_slots(int ty, int *slots);
// The tensor maps of a 16-bit step: u: U (16-bit) with box (tx+16, ty+8, 1);
// d: D and w: the 16-bit model, both with box (tx, ty, 1); u_out receives U'
// (the other U buffer), D is updated in place at d_io. src_hint: bound on
// |(V dt)^2 s(t_n)| of this step's sources (picks the output exponents while
// the field is still zero).
struct Maps16In {
    const CUtensorMap *u, *d, *w;
    uint16_t *u_out, *d_io;
};
cudaError_t launch_step_stream16(int storage, const Maps16In &m, const StepArgs &a, Scale16 *sc,
                                 long long step, float src_hint, const Free16 &fr,
                                 const StreamTiling &t, const int *rec_ptr, const RecEntry *rec,
                                 cudaStream_t s);
// FP32 padded (u^n, u^{n-1}) <-> 16-bit padded (U, D) (interior), exponent slot `slot`.
cudaError_t launch_encode16(int storage, const float *u, const float *up, uint16_t *U, uint16_t *D,
                            const Geom &g, Scale16 *sc, int slot, cudaStream_t s);
cudaError_t launch_decode16(int storage, const uint16_t *U, const uint16_t *D, float *u, float *up,
                            const Geom &g, const Scale16 *sc, int slot, cudaStream_t s);
// (V dt/h)^2 (FP32 padded) -> the 16-bit model.
cudaError_t launch_model16(const float *w, uint16_t *w16, const Geom &g, cudaStream_t s);

// ---- adjoint gradient ----
int residual_partial_count();
// r = traces - d_obs (n values; r = traces when d_obs is null),
// *misfit = sum r^2 / 2 (FP64, fixed order);
// partials holds residual_partial_count() doubles.
cudaError_t launch_residual(const float *traces, const float *d_obs, long long n, float *r,
                            double *partials, double *misfit, cudaStream_t s);
// rho[rec] += W G r[:, col] at every receiver (rec_ijk: [nrec][3] device).
cudaError_t launch_inject(float *rho, const float *w, const float *gx, const float *gy,
                          const float *gz, const Geom &g, const int *rec_ijk, int nrec,
                          const float *r, int nt, int col, cudaStream_t s);
// acc (compensated FP32 {sum, correction} per cell, padded layout) +=
// rho * lapu (the stencil sum L u^n a step stored), plus rho * amp / G at
// source cells.
cudaError_t launch_imaging(const float *rho, const float *lapu, const Geom &g, const Sources &src,
                           const float *gx, const float *gy, const float *gz, float2 *acc,
                           cudaStream_t s);
// out[t] = sum over q < n of src.p[q][t], t < count (FP64 sum in the order of
// q, rounded once); out may be src.p[0]. n <= kMaxFieldList.
constexpr int kMaxFieldList = WS_MAX_SHOTS;
struct FieldList {
    const float *p[kMaxFieldList];
};
cudaError_t launch_sum_fields(const FieldList &src, int n, long long count, float *out,
                              cudaStream_t s);
// *out = sqrt(sum x^2) in FP64 over n floats: per-block partial sums into
// partials[residual_partial_count()], then their fixed-order sum.
cudaError_t launch_norm2(const float *x, long long n, double *partials, double *out,
                         cudaStream_t s);
// grad (unpadded float) = -V^2 (sum - correction) of acc, V^2 = W (h / dt)^2.
cudaError_t launch_finalize_gradient(const float2 *acc, const float *w, const Geom &g,
                                     double h_over_dt2, float *grad, cudaStream_t s);

// Discrete energy (FP64): partial sums per (row block, plane) into
// partials[energy_partial_count(ny, nz)], then their fixed-order sum into *out.
int energy_rows_per_block();
long long energy_partial_count(int ny, int nz);
cudaError_t launch_energy_padded(const float *u, const float *p, const float *w, const Geom &g,
                                 double h, const Coeffs64 &c, double *partials, double *out,
                                 cudaStream_t s);

// The same reduction over unpadded caller arrays, with the partial sums in a
// static device array instead of allocated memory (at most
// kNoAllocMaxPartials of them). out is a device pointer.
constexpr int kNoAllocMaxPartials = WS_NOALLOC_MAX_PARTIALS;
cudaError_t launch_energy_noalloc(const float *u, const float *p, const float *v, int nx, int ny,
                                  int nz, double h, double dt, const Coeffs64 &c, double *out,
                                  cudaStream_t s);

}  // namespace ws
