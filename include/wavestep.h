/*
 * wavestep.h -- C ABI of the GB300 (sm_103a) stepper for the 3D
 * constant-density acoustic wave equation of arXiv 2204.03775.
 *
 * The library advances Eq. 2 of the paper (Section II),
 *
 *     u^{n+1} - Q u^n + u^{n-1} = dt^2 V^2 f^n,   Q = 2 + dt^2 V^2 Lap,
 *
 * with Lap the 25-point, 8th-order star Laplacian of Section II (four
 * neighbours per side on each axis; weights c_0..c_4 = -205/72, 8/5, -1/5,
 * 8/315, -1/560 divided by h^2, the centre weight applied once per axis as in
 * Section III-C-2; evaluated as sum_m c_m (s_m - 6u), s_m the sum of the six
 * neighbours at distance m, which equals it in exact arithmetic and keeps the
 * float operator exactly zero on constant fields), in the time loop of
 * Algorithm 1 starting from
 * u^{-1} = u^0 = 0. Each step is one fused pass on the GPU that also applies
 * an absorbing taper, injects Ricker sources and records receivers; the paper
 * leaves boundary conditions and I/O unevaluated (Section II), so those three
 * are this library's additions, defined below.
 *
 * Conventions for every entry point:
 *  - Return value: WS_OK (0) on success, a negative WS_ERR_* code otherwise;
 *    ws_last_error() then returns a message (per calling thread).
 *  - Grid: interior cells (i, j, k), 0 <= i < nx, 0 <= j < ny, 0 <= k < nz,
 *    spacing h (metres) on all axes, k = 0 the top plane. Outside the interior
 *    the field is zero at all times (a 4-cell zero-Dirichlet halo).
 *  - User arrays of the grid are unpadded, [nz][ny][nx] row-major, x fastest,
 *    float32. The library keeps its own padded copies in device memory; it
 *    never keeps a pointer it was given.
 *  - on_device: 0 = the pointer is host memory (any, pinned is faster),
 *    1 = device memory of the current CUDA device.
 *  - Work is issued on the handle's stream (ws_set_stream; default: the
 *    legacy default stream). Calls that read into host memory synchronize
 *    that stream before returning; the others are asynchronous.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - Device memory: the handle allocates (cudaMalloc) three padded fields of
 *    P * (ny+8) * (nz+8) floats, P = 32 + nx + 4 rounded up to a multiple of
 *    32 (interior rows start on 128-byte lines), plus O(nx+ny+nz) and the
 *    trace buffer; ws_destroy frees them.
 */
#ifndef WAVESTEP_H
#define WAVESTEP_H

#ifdef __cplusplus
extern "C" {
#endif

#define WS_OK            0
#define WS_ERR_BADARG   -1  /* invalid argument or size */
#define WS_ERR_CFL      -2  /* velocity model violates the stability limit */
#define WS_ERR_OOM      -3  /* device allocation failed */
#define WS_ERR_CUDA     -4  /* CUDA runtime or driver error */
#define WS_ERR_TIMEOUT  -5  /* a bounded device-side wait ran out */
#define WS_ERR_STATE    -6  /* call not valid in the handle's current state */

/* Step kernels selectable with ws_set_kernel. */
#define WS_KERNEL_AUTO    0  /* the streaming kernel when the grid fits its tile, else DIRECT */
#define WS_KERNEL_DIRECT  1  /* one thread per cell, neighbours loaded from global memory */
#define WS_KERNEL_STREAM  2  /* z-streaming: TMA rings + 9-plane register queue, one CTA per item */

/* Storage of the two wavefield levels (ws_set_storage). */
#define WS_STORAGE_FP32   0  /* float32 fields and model: 16 bytes per cell update */
#define WS_STORAGE_BF16   1  /* bfloat16 u, u - u_prev; FP16 model: 10 bytes per cell update */
#define WS_STORAGE_FP16   2  /* float16 u, u - u_prev; FP16 model: 10 bytes per cell update */

#define WS_MAX_SOURCES   16
#define WS_MAX_SHOTS     64  /* handles in one ws_adjoint_gradient_shots call */

/* What ws_adjoint_gradient's data array holds. */
#define WS_ADJ_DATA       0  /* observed traces d: residual = traces - d */
#define WS_ADJ_RESIDUAL   1  /* the residual itself, dJ/dtraces of any J */

typedef struct ws_handle *ws_t;

/* Create a stepper for an nx x ny x nz grid with spacing h (m) and time step
 * dt (s). Fields start at zero, the step counter at 0, damping off, no
 * sources or receivers, and no velocity (ws_step fails until
 * ws_set_velocity succeeds). Sizes must be >= 1 and each <= 65535.
 * Errors: BADARG, OOM, CUDA. On error *out is NULL. */
int ws_create(ws_t *out, int nx, int ny, int nz, double h, double dt);

/* Free every device and host resource of the handle (synchronizes its
 * stream first). NULL is accepted. */
int ws_destroy(ws_t ws);

/* Issue all further work on cuda_stream (a cudaStream_t of the current
 * device; NULL = legacy default stream). The caller keeps the stream alive
 * for as long as the handle uses it. */
int ws_set_stream(ws_t ws, void *cuda_stream);

/* Set the velocity model V of Eq. 1 (m/s), [nz][ny][nx]. The library stores
 * (V dt / h)^2 in its padded layout (computed in double, rounded to float).
 * Every value must be finite and > 0, and max(V) dt / h must not exceed the
 * leapfrog stability limit of this Laplacian, 2 / sqrt(3 * sum_m |w_m|) with
 * w the 1D weights (about 0.4529); else CFL (the previous model, if any, is
 * then no longer valid and ws_step fails until a valid one is set).
 * Synchronizes the stream (it reads back the model's extrema). */
int ws_set_velocity(ws_t ws, const float *v, int on_device);

/* Set the model as squared slowness m = 1 / V^2 (s^2/m^2), [nz][ny][nx]:
 * the library stores (V dt / h)^2 = (dt / h)^2 / m. Same checks and
 * errors as ws_set_velocity, with max(V) = 1 / sqrt(min(m)). The paper has
 * no inversion; m is the parameter ws_adjoint_gradient differentiates by. */
int ws_set_slowness2(ws_t ws, const float *m, int on_device);

/* Absorbing taper (Cerjan et al. 1985): for a cell at distance d < nb cells
 * from the nearer outer face of an axis, that axis contributes
 * exp(-(a (nb - d))^2); g = gx(i) gy(j) gz(k) and each step computes
 *     u^{n+1} = g (2 u^n - g u^{n-1} + (V dt)^2 Lap u^n),
 * i.e. both time levels are multiplied by g after each plain step of Eq. 2.
 * nb = 0 turns damping off. Requires 0 <= nb and 0 <= a. */
int ws_set_sponge(ws_t ws, int nb, double a);

/* Add a point source at cell (ix, iy, iz) with Ricker time function
 *     s(t) = amp (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2).
 * Step n (producing u^{n+1}, t_n = n dt) adds (V_s dt)^2 s(t_n) at the cell
 * after damping: the right-hand side dt^2 V^2 f^n of Eq. 2. Up to
 * WS_MAX_SOURCES sources. Errors: BADARG (cell outside the grid, f0 <= 0,
 * too many sources). */
int ws_add_source(ws_t ws, int ix, int iy, int iz, double f0, double t0, double amp);

/* Remove every source. */
int ws_clear_sources(ws_t ws);

/* Record u^{n+1} at nrec cells after each step n, for steps 0..nt_max-1
 * counted from the step at which this call is made (the trace clock
 * restarts here; traces are zeroed). ijk is host memory, [nrec][3] =
 * (i, j, k) per receiver, copied. nrec = 0 removes all receivers. Stepping
 * past nt_max recorded steps fails with STATE. */
int ws_set_receivers(ws_t ws, int nrec, const int *ijk, int nt_max);

/* Advance nsteps steps (asynchronous on the stream). Requires a velocity
 * model. Errors: STATE (no velocity; receiver buffer full), CUDA. */
int ws_step(ws_t ws, int nsteps);

/* Copy the traces, [nrec][nt_max] float32, to out. Samples of steps not yet
 * taken are zero. */
int ws_read_traces(ws_t ws, float *out, int on_device);

/* Copy u^n (into u) and u^{n-1} (into u_prev) as [nz][ny][nx] float32.
 * Either pointer may be NULL. */
int ws_read_field(ws_t ws, float *u, float *u_prev, int on_device);

/* Replace u^n and u^{n-1} (NULL = zero) and set the step counter to step
 * (t_n = step * dt for the next source sample). Used to restart from a
 * saved state. */
int ws_write_field(ws_t ws, const float *u, const float *u_prev, long long step,
                   int on_device);

/* Number of steps taken since creation (or the last ws_write_field). */
int ws_get_step(ws_t ws, long long *step);

/* Discrete energy of the current state, in double precision:
 *     E = sum (u^n - u^{n-1})^2 / (V dt)^2 - sum u^n (Lap u^{n-1})
 * over the interior, Lap the 25-point Laplacian with the zero halo. Without
 * sources and damping the leapfrog recurrence of Eq. 2 conserves E exactly
 * (in exact arithmetic), since Lap is symmetric. Deterministic (fixed-order
 * reduction over per-block partial sums in memory the handle owns).
 * Synchronizes the stream. Errors: STATE (no velocity model), CUDA. */
int ws_energy(ws_t ws, double *e);

/* The energy of ws_energy for device arrays the caller
 * owns, without allocating any device memory. The paper has no counterpart;
 * this entry point exists for callers that cannot call cudaMalloc: code that
 * runs under an allocator which forbids it or has no memory to spare, and
 * code that must not risk the implicit device-wide synchronization that
 * cudaMalloc may perform.
 *
 * u, u_prev, v: device pointers to unpadded [nz][ny][nx] float32 arrays of
 * u^n, u^{n-1} and the velocity (m/s, finite and > 0; not checked); h, dt as
 * in ws_create. e: device pointer to one double, which receives E. Work is
 * issued on cuda_stream (NULL = legacy default stream) and the call returns
 * without waiting for it. E equals what ws_energy returns for a handle in
 * that state (same per-cell terms and summation order).
 *
 * Scratch: the per-block partial sums live in a static device array of
 * WS_NOALLOC_MAX_PARTIALS doubles (256 KiB) that every GPU which loads the
 * library holds until the process exits. A grid needs ceil(ny / 32) * nz
 * partial sums (1024 x 1024 x 1024 fits exactly); larger grids are rejected
 * with BADARG. Every call shares that array and leaves its partial sums
 * there; each call writes every partial it later reads, so nothing needs to
 * start at zero, but calls whose work overlaps on the GPU (other streams,
 * other host threads) race and give wrong results: serialize them.
 * Every call looks up the array's address on the current device (the
 * arrays and the stream must belong to that device), so an address is
 * never kept across a device reset; the first call on a device may also
 * load the library's kernels there, so make that first call before any
 * stream capture.
 * Errors: BADARG, CUDA. */
#define WS_NOALLOC_MAX_PARTIALS 32768
int ws_energy_noalloc(const float *u, const float *u_prev, const float *v, int nx, int ny, int nz,
                      double h, double dt, double *e, void *cuda_stream);

/* Gradient of a trace misfit with respect to the squared slowness m = 1/V^2
 * of every cell, by the discrete adjoint of the stepper (exact up to float
 * rounding: the derivative of the very recurrence ws_step computes,
 * taper and sources included). The paper solves only the forward problem
 * (Section II); this is the inversion use of its stepper.
 *
 * The call runs the forward problem from rest: fields zeroed, step 0, the
 * handle's sources, nt_max steps, traces recorded as by ws_step. With
 * mode = WS_ADJ_DATA, data is the observed traces d and the residual is
 * r = traces - d, J = |r|^2 / 2; with WS_ADJ_RESIDUAL, data is r itself
 * (any upstream dJ/dtraces) and J is reported as |r|^2 / 2. data is
 * [nrec][nt_max] float32 like ws_read_traces. grad_m receives dJ/dm,
 * [nz][ny][nx] float32; *misfit (host, may be NULL) receives J in double.
 *
 * Method: with lambda the multipliers of the step equations, rho = W G
 * lambda (W = (V dt/h)^2, G the taper) obeys the forward recurrence run
 * backwards, rho^k = G (2 rho^{k+1} - G rho^{k+2} + W Lap' rho^{k+1}) +
 * W G r^k (Lap' = h^2 Lap, r^k injected at the receivers), so the step
 * kernels advance rho; dJ/dm = -V^2 sum_n rho^{n+1} (Lap' u^n), plus
 * -V^2 sum_n rho^{n+1} h^2 s_n / G at each source cell. The states u^n are
 * recomputed, segment by segment, from ceil(N / C) - 1 checkpoint pairs,
 * C = ceil(sqrt(N)), N = nt_max; the recomputing steps store the stencil
 * sums Lap' u^n of their segment (the float values the step used) for the
 * imaging: two forward passes and one backward pass in all.
 *
 * A residual for the run that the last ws_forward left (WS_ADJ_RESIDUAL,
 * with no change to the model, taper, sources, receivers or storage since)
 * reuses that run's checkpoints instead of running the forward problem
 * again; the handle's state is then left as it is.
 *
 * Needs a velocity model, receivers and FP32 storage, else STATE. Device
 * scratch: about 3 sqrt(N) + 6 padded fields and two
 * trace arrays, allocated by the first call and kept by the handle for the
 * next ones while N, the receiver count and the tiling stay the same (freed
 * by ws_destroy).
 * Afterwards the handle holds the forward run's final state (step N) and
 * its traces. Synchronizes the stream. Errors: BADARG, STATE, OOM, CUDA,
 * TIMEOUT. */
int ws_adjoint_gradient(ws_t ws, const float *data, int mode, float *grad_m, double *misfit,
                        int on_device);

/* The gradient of the summed misfit of several shots: nshots handles (1 to
 * WS_MAX_SHOTS) on grids of one size, with the same nt_max, each with its own
 * sources, receivers and model (normally one model: the gradient is then
 * the gradient of the total misfit). data[s] is shot s's data, as for
 * ws_adjoint_gradient with the same mode. grad_m receives the sum over the
 * shots of their dJ_s/dm (FP64 sum in shot order, rounded once), *misfit
 * (may be NULL) the summed misfit, *grad_norm (may be NULL) the FP64 L2
 * norm of grad_m computed on the device (fixed summation order). Host
 * (on_device = 0) or device (1) arrays, as in ws_adjoint_gradient.
 *
 * Each shot is the computation of ws_adjoint_gradient (the same kernels and
 * values: one shot's gradient equals that call's bit for bit), issued on its
 * handle's stream, the shots interleaved step by step: shots on distinct
 * streams (ws_set_stream) run concurrently and fill the GPU that one small
 * grid leaves partly idle. The paper has no counterpart (forward problem
 * only). Synchronizes every shot's stream. Errors: BADARG (sizes or steps
 * differ, a NULL handle or array, a handle given twice), STATE, OOM, CUDA,
 * TIMEOUT; with an error the shots' states are unspecified. */
int ws_adjoint_gradient_shots(ws_t *shots, int nshots, const float *const *data, int mode,
                              float *grad_m, double *misfit, double *grad_norm, int on_device);

/* The forward run of ws_adjoint_gradient on its own: fields zeroed, step 0,
 * nt_max steps with the handle's sources, traces recorded (ws_read_traces),
 * and the sqrt(N) checkpoint pairs kept in the handle's adjoint scratch, so
 * that a following ws_adjoint_gradient(WS_ADJ_RESIDUAL) for these traces
 * skips its own forward run (the torch bridge's forward and backward). The
 * paper has no counterpart (forward problem only). Same requirements and
 * scratch as ws_adjoint_gradient; synchronizes nothing. */
int ws_forward(ws_t ws);

/* Store the state in 16 bits (WS_STORAGE_BF16 or WS_STORAGE_FP16) or back
 * in FP32. The 16-bit modes keep U = u^n and D = u^n - u^{n-1} (the
 * "velocity form": rounding then perturbs the displacement, not the discrete
 * velocity, which keeps the error from growing like N^1.5) and the model
 * (V dt/h)^2 as FP16: 10 bytes per cell update instead of 16. Arithmetic
 * stays FP32. U and D share one power-of-two scale per step, picked on the
 * device from max|u^n| and the source amplitude so that the field's maximum
 * sits near 2^12 (16x under the FP16 limit); FP16 then holds values down to
 * ~2^-36 of that maximum and smaller ones as zero. The current state is converted
 * (rounded once). 16-bit storage runs its own streaming kernel with a 64 x ty
 * tile (ty = 24 by default, 16 on grids with ny < 24; 16, 24 or 48 through
 * ws_set_kernel), single grids only (batches and the adjoint gradient need
 * FP32 storage), and needs nx >= 64, ny >= 16, else BADARG. ws_read_field,
 * ws_write_field and ws_energy convert to and from FP32 (ws_energy then uses
 * the FP32 model). Relative L2 error against the FP64 oracle, measured on the
 * layered survey at 512^3 after 100, 500, 1000 steps: FP16 8.5e-4, 2.8e-3,
 * 4.1e-3; BF16 6.1e-3, 2.3e-2, 3.5e-2 (FP32 storage 5.3e-7 ... 1.9e-6): FP16
 * stays within 1e-2, BF16 only for about the first 100 steps (its 8-bit
 * significand's rounding errors add up like a random walk); at 1024^3 after
 * 100 steps FP16 7.6e-4, BF16 5.9e-3. Speed on the 1024^3 survey: 1.28x (FP16
 * and BF16) of FP32 storage. This realizes the reduced-precision
 * storage that the paper contrasts with its FP32-only arithmetic (Section I). */
int ws_set_storage(ws_t ws, int storage);

/* Choose the step kernel (WS_KERNEL_*) and, for WS_KERNEL_STREAM, its tile:
 * tile_x x tile_y in {32x8, 32x16, 64x8, 64x16, 64x32} for the FP32 kernel
 * (0, 0 = keep the current tile; the default is 64x8) or in {64x16, 64x24,
 * 64x48} for the 16-bit kernel (64x16 selects both; a 16-bit tile leaves the
 * FP32 tile unchanged and needs nx >= 64 and ny >= tile_y), zblock >= 1 planes
 * per work item (0 = default: blocks of about 200 planes with a last block
 * about a quarter as long, so that the last items of a launch are short;
 * fewer planes on small grids).
 * WS_KERNEL_STREAM needs nx >= tile_x and ny >= tile_y; else BADARG. */
int ws_set_kernel(ws_t ws, int kernel, int tile_x, int tile_y, int zblock);

/* Pick the streaming kernel's tile and z-block for this handle's grid by
 * timing the candidates (every tile of 64x8, 32x8, 32x16 that fits: 64x16
 * and 64x32 hold too few registers per thread and are never faster; z-blocks giving the default
 * length and item counts just below and just above 1 .. 8 waves of the
 * resident CTAs) on
 * steps written to a scratch field, so the state is unchanged; then select
 * WS_KERNEL_STREAM with the fastest (WS_KERNEL_DIRECT if no tile fits).
 * Results are cached by (GPU name, storage, nx, ny, nz) in the process and
 * in a text file, so later processes on the same GPU model skip the timing:
 * the file is $WS_TUNE_CACHE if set, else $XDG_CACHE_HOME/wavestep/tune.txt,
 * else $HOME/.cache/wavestep/tune.txt (one "gpu|storage|nx|ny|nz|tx|ty|zb"
 * line per entry; unreadable lines are ignored, an unwritable file leaves
 * the in-process cache only). Outputs may be NULL.
 * Needs a velocity model and FP32 storage, else STATE. Synchronizes. */
int ws_autotune(ws_t ws, int *tile_x, int *tile_y, int *zblock);

/* ---- batched shots -------------------------------------------------------
 * A batch advances several independent handles ("shots": each its own grid
 * size, model, taper, sources and receivers) together: every step is ONE
 * launch of the streaming kernel over the work items (one CTA each) of all
 * shots, and each ws_batch_step(n) replays a CUDA graph of n such launches.
 * The results are bit for bit those of ws_step on each handle (the same
 * arithmetic per cell, whatever the tiling). The paper's many-problem use is
 * one large grid per wafer (Section IV); batching many smaller grids per
 * GPU is this library's addition.
 *
 * The batch references the handles (it does not own them; destroy the batch
 * first) and sets each shot's streaming tile to its own; the handles stay
 * usable on their own between batch steps. Every shot must have nx >= 32
 * and ny >= 8. Work runs on a stream
 * the batch creates, ordered after each shot's pending work on its own
 * stream, and each shot's later work on its own stream is ordered after it.
 *
 * Tiling: unless fixed with ws_batch_set_tiling, ws_batch_step tunes online:
 * while candidates remain untried, steps are taken two at a time with the
 * next candidate (tile x z-block rule), the second step timed; then the
 * fastest is kept. Tuning changes timing only, never results. */
typedef struct ws_batch *ws_batch_t;

/* Create a batch of nshots distinct handles. Errors: BADARG (NULL or
 * repeated handle, a shot smaller than every tile), OOM, CUDA. */
int ws_batch_create(ws_batch_t *out, int nshots, const ws_t *shots);

/* Free the batch (its stream, graphs and tables; not the handles). */
int ws_batch_destroy(ws_batch_t b);

/* Fix the tile (tile_x x tile_y, as in ws_set_kernel) and the z-block rule:
 * zmul = 0 gives each shot its default z-block, zmul >= 1 z-blocks that
 * make about zmul x (resident CTAs) items over the batch, shared among the
 * shots by their sizes. (0, 0, any) returns to online tuning. */
int ws_batch_set_tiling(ws_batch_t b, int tile_x, int tile_y, int zmul);

/* The tiling in use (all zero before the first step). */
int ws_batch_get_tiling(ws_batch_t b, int *tile_x, int *tile_y, int *zmul);

/* Advance every shot nsteps steps (asynchronous). Each shot needs a velocity
 * model, FP32 storage and room in its receiver buffer, else STATE. */
int ws_batch_step(ws_batch_t b, int nsteps);

/* Wait for the batch's stream; report (and clear) a bounded-wait timeout
 * recorded by a batched step (TIMEOUT). */
int ws_batch_synchronize(ws_batch_t b);

/* Kernel launches issued by the batch (one per step). */
long long ws_batch_launch_count(ws_batch_t b);

/* Wait for the stream, then report a device-side failure recorded since the
 * last call (TIMEOUT when a bounded wait in a kernel ran out). Clears it. */
int ws_synchronize(ws_t ws);

/* Test hook for the failure path (the paper has no counterpart): the next
 * ws_step that uses a streaming kernel (FP32, or the 16-bit kernel of
 * 16-bit storage), or the first step of the next ws_batch_step run that
 * includes this shot, withholds the first copy of the shot's work item
 * `item` (items are numbered z block by z block, then by tile),
 * so the bounded waits of the CTA that owns it give up after about one
 * second. That step's result is then invalid: ws_synchronize (for a batch,
 * ws_batch_synchronize) returns TIMEOUT, and the caller must write a new
 * state (ws_write_field) before
 * stepping on; the handle and the CUDA context stay usable. item = -1
 * clears a pending stall. No GPU fault is involved: the kernel only stops
 * waiting, records the status and drains its own copies. */
int ws_test_stall(ws_t ws, int item);

/* Test hooks for memory-safety checks (the paper has no counterpart; they
 * stand in for a sanitizer). A padded field is the interior, the 4-cell
 * zero halo and, in x, row padding beyond the halo. ws_test_fill_padding
 * writes a quiet NaN (FP32 0x7fc00000; 16-bit buffers: the format's NaN)
 * into the row padding of every field buffer of the handle (state and
 * model; with 16-bit storage the 16-bit ones too) and synchronizes. A later
 * ws_test_check_padding stores in *bad the number of cells that no longer
 * hold what they must: 0 in the halo, the NaN in the padding (bit
 * patterns); it synchronizes the handle's stream. With the padding filled,
 * the interior results must not change: nothing beyond the halo may reach
 * a result. Calls that zero whole state buffers clear their canaries, so
 * fill after them: ws_write_field, ws_forward and ws_adjoint_gradient
 * (which restart from rest) and ws_set_storage (which allocates the 16-bit
 * buffers); the model setters write the interior only. Errors: BADARG
 * (NULL), CUDA, OOM. */
int ws_test_fill_padding(ws_t ws);
int ws_test_check_padding(ws_t ws, long long *bad);

/* Number of kernel launches issued by this handle since creation. */
long long ws_launch_count(ws_t ws);

/* Message of the last failed call on this thread ("" if none). */
const char *ws_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WAVESTEP_H */
