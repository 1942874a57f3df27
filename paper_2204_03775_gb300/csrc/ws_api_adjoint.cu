// Host side of the adjoint entry points (ws_forward, ws_adjoint_gradient):
// the forward run with sqrt(N) checkpoints, the residual, and the backward
// sweep that recomputes each segment and steps rho with the forward kernel.
#include "ws_host.h"

using namespace wsh;

namespace {

// Checks shared by ws_forward and ws_adjoint_gradient; selects the kernel and
// makes sure the handle's adjoint scratch matches the run (N = nt_max steps).
int adjoint_prepare(ws_t ws, const char *who, int *kern_out, ws::StreamTiling *tiling_out,
                    AdjointCache **acp) {
    if (!ws->vel_ok) return fail(WS_ERR_STATE, "%s: no valid velocity model", who);
    if (ws->nrec == 0) return fail(WS_ERR_STATE, "%s: no receivers", who);
    if (ws->storage != WS_STORAGE_FP32) return fail(WS_ERR_STATE, "%s: needs FP32 field storage", who);
    const ws::Geom &g = ws->g;
    const int N = ws->nt_max;
    const int C = (int)std::ceil(std::sqrt((double)N));    // states per segment
    const int nck = (N + C - 1) / C;                        // segments
    int kern = WS_KERNEL_STREAM;
    ws::StreamTiling tiling{};
    int rc = prepare_fp32(ws, &kern, &tiling);
    if (rc != WS_OK) return rc;
    const bool maps = kern == WS_KERNEL_STREAM;
    const size_t fb = field_bytes(g);
    const size_t ncell = size_t(g.nx) * g.ny * g.nz;
    const size_t ntr = size_t(ws->nrec) * N;
    const cudaStream_t st = ws->stream;
    AdjointCache *ac = ws->adj;
    if (!ac || ac->N != N || ac->nrec != ws->nrec || ac->kern != kern ||
        (maps && (ac->tx != ws->tiling.tx || ac->ty != ws->tiling.ty))) {
        WS_CUDA(cudaStreamSynchronize(st), "ws_adjoint_gradient");
        delete ws->adj;
        ws->adj = nullptr;
        ac = new (std::nothrow) AdjointCache();
        if (!ac) return fail(WS_ERR_OOM, "ws_adjoint_gradient: host allocation failed");
        ws->adj = ac;
        auto grab = [&](auto **p, size_t bytes) -> cudaError_t {
            void *q = nullptr;
            cudaError_t e = cudaMalloc(&q, bytes);
            if (e == cudaSuccess) {
                ac->mem.push_back(q);
                *p = static_cast<std::remove_reference_t<decltype(**p)> *>(q);
            }
            return e;
        };
        auto field = [&](MappedField *f) -> int {
            WS_CUDA(grab(&f->p, fb), "cudaMalloc adjoint field");
            WS_CUDA(cudaMemsetAsync(f->p, 0, fb, st), "zero adjoint field");
            if (!maps) return WS_OK;
            const int tx = ws->tiling.tx, ty = ws->tiling.ty;
            int r2 = encode_map(&f->halo, f->p, g, tx + 2 * ws::kHalo, ty + 2 * ws::kHalo);
            if (r2 == WS_OK) r2 = encode_map(&f->tile, f->p, g, tx, ty);
            return r2;
        };
        // checkpoints (u^{jC}, u^{jC-1}), j = 1 .. nck-1; segment states; rho
        ac->ck.assign(2 * size_t(nck - 1), nullptr);
        for (auto &c : ac->ck) {
            cudaError_t e = grab(&c, fb);
            if (e != cudaSuccess) {
                delete ws->adj;
                ws->adj = nullptr;
                return cuda_fail(e, "cudaMalloc checkpoint");
            }
        }
        ac->lap.assign(C, nullptr);
        cudaError_t e = cudaSuccess;
        for (auto &f : ac->lap) {   // zeroed: the steps write the interior only
            if (e == cudaSuccess) e = grab(&f, fb);
            if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, fb, st);
        }
        int r3 = e == cudaSuccess ? WS_OK : cuda_fail(e, "cudaMalloc adjoint field");
        for (auto &f : ac->ring)
            if (r3 == WS_OK) r3 = field(&f);
        for (auto &f : ac->rho)
            if (r3 == WS_OK) r3 = field(&f);
        if (r3 == WS_OK) e = grab(&ac->acc, 2 * fb);   // float2 per cell, padded layout
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->partials, sizeof(double) * (ws::residual_partial_count() + 1));
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->norm, sizeof(double) * (ws::residual_partial_count() + 1));
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->r, sizeof(float) * ntr);
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->dd, sizeof(float) * ntr);
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->grad, sizeof(float) * ncell);
        if (r3 == WS_OK && e == cudaSuccess) e = grab(&ac->rec, sizeof(int) * 3 * ws->nrec);
        if (r3 != WS_OK || e != cudaSuccess) {
            delete ws->adj;
            ws->adj = nullptr;
            return r3 != WS_OK ? r3 : cuda_fail(e, "cudaMalloc adjoint scratch");
        }
        ac->N = N;
        ac->nrec = ws->nrec;
        ac->kern = kern;
        ac->tx = ws->tiling.tx;
        ac->ty = ws->tiling.ty;
    }
    *kern_out = kern;
    *tiling_out = tiling;
    *acp = ac;
    return WS_OK;
}

// The forward run from rest over N steps: traces recorded, checkpoint pairs
// (u^{jC}, u^{jC-1}) saved; the cache then holds this model version's run.
// forward_begin resets the state, forward_step issues step n.
int forward_begin(ws_t ws, AdjointCache *ac) {
    const size_t fb = field_bytes(ws->g);
    const size_t ntr = size_t(ws->nrec) * ws->nt_max;
    const cudaStream_t st = ws->stream;
    ac->fwd_valid = false;
    for (int b = 0; b < 2; ++b) WS_CUDA(cudaMemsetAsync(ws->buf[b], 0, fb, st), "zero fields");
    WS_CUDA(cudaMemsetAsync(ws->traces, 0, sizeof(float) * ntr, st), "zero traces");
    ws->step = 0;
    ws->trace_start = 0;
    return WS_OK;
}

int forward_step(ws_t ws, AdjointCache *ac, int kern, const ws::StreamTiling &tiling,
                 ws::StepArgs &a, int n) {
    const int C = (int)std::ceil(std::sqrt((double)ws->nt_max));
    const size_t fb = field_bytes(ws->g);
    const cudaStream_t st = ws->stream;
    std::vector<float *> &ck = ac->ck;
    if (n > 0 && n % C == 0) {
        const int j = n / C;
        WS_CUDA(cudaMemcpyAsync(ck[2 * (j - 1)], ws->buf[ws->cur], fb, cudaMemcpyDeviceToDevice, st),
                "save checkpoint");
        WS_CUDA(cudaMemcpyAsync(ck[2 * (j - 1) + 1], ws->buf[1 - ws->cur], fb,
                                cudaMemcpyDeviceToDevice, st),
                "save checkpoint");
    }
    const int c = ws->cur;
    int rc = step_fp32(ws, a, kern, tiling, ws->buf[c], &ws->tmap_halo[c], ws->buf[1 - c],
                       &ws->tmap_tile[1 - c], ws->buf[1 - c], n, true, true);
    if (rc != WS_OK) return rc;
    ws->cur = 1 - c;
    ws->step++;
    if (n == ws->nt_max - 1) {
        ac->fwd_valid = true;
        ac->fwd_version = ws->model_version;
    }
    return WS_OK;
}

int adjoint_forward(ws_t ws, AdjointCache *ac, int kern, const ws::StreamTiling &tiling) {
    int rc = forward_begin(ws, ac);
    ws::StepArgs a = base_args(ws);
    for (int n = 0; n < ws->nt_max && rc == WS_OK; ++n) rc = forward_step(ws, ac, kern, tiling, a, n);
    return rc;
}

// One shot of a gradient run: its handle, scratch and kernel choice, its data
// on the device, and where its gradient goes.
struct GradShot {
    ws_t ws = nullptr;
    AdjointCache *ac = nullptr;
    int kern = WS_KERNEL_STREAM;
    ws::StreamTiling tiling{};
    const float *d = nullptr;
    float *grad = nullptr;
    bool forward = true;     // run the forward problem (not reused from ws_forward)
    ws::StepArgs a{};
    int rho_cur = 0;         // rho[rho_cur] = rho^{k+1}
};

// The gradients of n shots with one grid and one step count, each shot's
// work on its handle's stream, the shots interleaved step by step.
int gradient_run(GradShot *sh, int n, int mode) {
    const ws::Geom &g = sh[0].ws->g;
    const int N = sh[0].ws->nt_max;
    const int C = (int)std::ceil(std::sqrt((double)N));    // states per segment
    const int nck = (N + C - 1) / C;                        // segments
    const size_t fb = field_bytes(g);
    const int np = ws::residual_partial_count();
    for (int q = 0; q < n; ++q) {
        GradShot &x = sh[q];
        const cudaStream_t st = x.ws->stream;
        for (auto &f : x.ac->rho) WS_CUDA(cudaMemsetAsync(f.p, 0, fb, st), "zero adjoint field");
        WS_CUDA(cudaMemsetAsync(x.ac->acc, 0, 2 * fb, st), "zero gradient accumulator");
        WS_CUDA(cudaMemcpyAsync(x.ac->rec, x.ws->rec_ijk.data(), sizeof(int) * 3 * x.ws->nrec,
                                cudaMemcpyHostToDevice, st),
                "upload receivers");
        // a residual given for the run that ws_forward left in the cache (same
        // model version) needs no new forward run
        x.forward = !(mode == WS_ADJ_RESIDUAL && x.ac->fwd_valid &&
                      x.ac->fwd_version == x.ws->model_version);
        if (x.forward) {
            int rc = forward_begin(x.ws, x.ac);
            if (rc != WS_OK) return rc;
        }
        x.a = base_args(x.ws);
        x.rho_cur = 0;
    }

    // 1. forward from rest, recording the traces and the checkpoints
    for (int t = 0; t < N; ++t)
        for (int q = 0; q < n; ++q)
            if (sh[q].forward) {
                int rc = forward_step(sh[q].ws, sh[q].ac, sh[q].kern, sh[q].tiling, sh[q].a, t);
                if (rc != WS_OK) return rc;
            }

    // 2. residual and misfit
    for (int q = 0; q < n; ++q) {
        GradShot &x = sh[q];
        const long long ntr = (long long)x.ws->nrec * N;
        WS_CUDA(ws::launch_residual(mode == WS_ADJ_DATA ? x.ws->traces : x.d,
                                    mode == WS_ADJ_DATA ? x.d : nullptr, ntr, x.ac->r,
                                    x.ac->partials, x.ac->partials + np, x.ws->stream),
                "residual kernels");
        x.ws->launches += 2;
    }

    // 3. backward: rho^k, k = N .. 1, segment by segment, the segment's
    // states recomputed from its checkpoint
    for (int j = nck - 1; j >= 0; --j) {
        const int n0 = j * C, n1 = std::min(n0 + C, N);
        // u^{n0}, u^{n0-1} into the ring, then steps n0 .. n1-1, each storing
        // L u^n into lap[n - n0] (u^{n1} itself is not needed)
        for (int q = 0; q < n; ++q) {
            AdjointCache *ac = sh[q].ac;
            const cudaStream_t st = sh[q].ws->stream;
            if (j == 0) {
                WS_CUDA(cudaMemsetAsync(ac->ring[0].p, 0, fb, st), "zero initial state");
                WS_CUDA(cudaMemsetAsync(ac->ring[1].p, 0, fb, st), "zero initial state");
            } else {
                WS_CUDA(cudaMemcpyAsync(ac->ring[0].p, ac->ck[2 * (j - 1)], fb,
                                        cudaMemcpyDeviceToDevice, st),
                        "restore checkpoint");
                WS_CUDA(cudaMemcpyAsync(ac->ring[1].p, ac->ck[2 * (j - 1) + 1], fb,
                                        cudaMemcpyDeviceToDevice, st),
                        "restore checkpoint");
            }
        }
        for (int t = 0; t < n1 - n0; ++t)
            for (int q = 0; q < n; ++q) {
                GradShot &x = sh[q];
                const int uc = t & 1;   // ring[uc] = u^{n0+t}
                MappedField &un = x.ac->ring[uc], &um = x.ac->ring[1 - uc];
                x.a.lap = x.ac->lap[t];
                int rc = step_fp32(x.ws, x.a, x.kern, x.tiling, un.p, &un.halo, um.p, &um.tile,
                                   um.p, n0 + t, true, false);
                x.a.lap = nullptr;
                if (rc != WS_OK) return rc;
            }
        for (int k = n1; k > n0; --k)
            for (int q = 0; q < n; ++q) {
                GradShot &x = sh[q];
                ws_t ws = x.ws;
                MappedField *rho = x.ac->rho;
                MappedField &r1 = rho[x.rho_cur], &r2 = rho[1 - x.rho_cur];
                int rc = step_fp32(ws, x.a, x.kern, x.tiling, r1.p, &r1.halo, r2.p, &r2.tile, r2.p,
                                   k, false, false);
                if (rc != WS_OK) return rc;
                x.rho_cur = 1 - x.rho_cur;   // rho[rho_cur] = rho^k
                WS_CUDA(ws::launch_inject(rho[x.rho_cur].p, ws->w, ws->gx, ws->gy, ws->gz, g,
                                          x.ac->rec, ws->nrec, x.ac->r, N, k - 1, ws->stream),
                        "adjoint injection kernel");
                ws::Sources src{};
                sources_of_step(ws, k - 1, &src);
                WS_CUDA(ws::launch_imaging(rho[x.rho_cur].p, x.ac->lap[k - 1 - n0], g, src, ws->gx,
                                           ws->gy, ws->gz, x.ac->acc, ws->stream),
                        "gradient imaging kernel");
                ws->launches += 2;
            }
    }
    for (int q = 0; q < n; ++q) {
        ws_t ws = sh[q].ws;
        const double hdt = ws->h / ws->dt;
        WS_CUDA(ws::launch_finalize_gradient(sh[q].ac->acc, ws->w, g, hdt * hdt, sh[q].grad,
                                             ws->stream),
                "gradient finalize kernel");
        ws->launches++;
    }
    return WS_OK;
}

// After a run: every shot's stream drained; *misfit = the summed misfits
// (host, fixed order); TIMEOUT if a bounded device wait ran out in any shot.
int gradient_finish(GradShot *sh, int n, double *misfit) {
    const int np = ws::residual_partial_count();
    double J = 0.0;
    bool timeout = false;
    for (int q = 0; q < n; ++q) {
        ws_t ws = sh[q].ws;
        double j = 0.0;
        WS_CUDA(cudaMemcpyAsync(&j, sh[q].ac->partials + np, sizeof(double), cudaMemcpyDeviceToHost,
                                ws->stream),
                "copy misfit");
        WS_CUDA(cudaStreamSynchronize(ws->stream), "ws_adjoint_gradient");
        J += j;
        unsigned status = 0;
        WS_CUDA(cudaMemcpy(&status, ws->status, sizeof status, cudaMemcpyDeviceToHost),
                "ws_adjoint_gradient");
        if (status & ws::kStatusTimeout) {
            WS_CUDA(cudaMemset(ws->status, 0, sizeof(unsigned)), "ws_adjoint_gradient");
            timeout = true;
        }
    }
    if (misfit) *misfit = J;
    if (timeout) return fail(WS_ERR_TIMEOUT, "a bounded device wait ran out in a step kernel");
    return WS_OK;
}

}  // namespace

extern "C" {

int ws_forward(ws_t ws) {
    if (!ws) return fail(WS_ERR_BADARG, "ws_forward: NULL handle");
    int kern = WS_KERNEL_STREAM;
    ws::StreamTiling tiling{};
    AdjointCache *ac = nullptr;
    int rc = adjoint_prepare(ws, "ws_forward", &kern, &tiling, &ac);
    if (rc != WS_OK) return rc;
    return adjoint_forward(ws, ac, kern, tiling);
}

int ws_adjoint_gradient(ws_t ws, const float *data, int mode, float *grad_m, double *misfit,
                        int on_device) {
    if (!ws || !data || !grad_m) return fail(WS_ERR_BADARG, "ws_adjoint_gradient: NULL argument");
    if (mode != WS_ADJ_DATA && mode != WS_ADJ_RESIDUAL)
        return fail(WS_ERR_BADARG, "ws_adjoint_gradient: unknown mode %d", mode);
    GradShot x;
    x.ws = ws;
    int rc = adjoint_prepare(ws, "ws_adjoint_gradient", &x.kern, &x.tiling, &x.ac);
    if (rc != WS_OK) return rc;
    const size_t ncell = size_t(ws->g.nx) * ws->g.ny * ws->g.nz;
    const size_t ntr = size_t(ws->nrec) * ws->nt_max;
    x.d = data;
    if (!on_device) {
        WS_CUDA(cudaMemcpyAsync(x.ac->dd, data, sizeof(float) * ntr, cudaMemcpyHostToDevice,
                                ws->stream),
                "upload observed data");
        x.d = x.ac->dd;
    }
    x.grad = on_device ? grad_m : x.ac->grad;
    rc = gradient_run(&x, 1, mode);
    if (rc != WS_OK) return rc;
    if (!on_device)
        WS_CUDA(cudaMemcpyAsync(grad_m, x.grad, sizeof(float) * ncell, cudaMemcpyDeviceToHost,
                                ws->stream),
                "copy gradient");
    return gradient_finish(&x, 1, misfit);
}

int ws_adjoint_gradient_shots(ws_t *shots, int nshots, const float *const *data, int mode,
                              float *grad_m, double *misfit, double *grad_norm, int on_device) {
    if (!shots || !data || !grad_m)
        return fail(WS_ERR_BADARG, "ws_adjoint_gradient_shots: NULL argument");
    if (nshots < 1 || nshots > WS_MAX_SHOTS)
        return fail(WS_ERR_BADARG, "ws_adjoint_gradient_shots: nshots must be in [1, %d], got %d",
                    WS_MAX_SHOTS, nshots);
    if (mode != WS_ADJ_DATA && mode != WS_ADJ_RESIDUAL)
        return fail(WS_ERR_BADARG, "ws_adjoint_gradient_shots: unknown mode %d", mode);
    for (int q = 0; q < nshots; ++q) {
        if (!shots[q] || !data[q])
            return fail(WS_ERR_BADARG, "ws_adjoint_gradient_shots: NULL handle or data of shot %d", q);
        const ws::Geom &g = shots[q]->g, &g0 = shots[0]->g;
        if (g.nx != g0.nx || g.ny != g0.ny || g.nz != g0.nz || shots[q]->nt_max != shots[0]->nt_max)
            return fail(WS_ERR_BADARG,
                        "ws_adjoint_gradient_shots: shot %d differs from shot 0 in grid size or "
                        "step count",
                        q);
        for (int p = 0; p < q; ++p)
            if (shots[p] == shots[q])
                return fail(WS_ERR_BADARG, "ws_adjoint_gradient_shots: handle given twice (%d, %d)",
                            p, q);
    }
    std::vector<GradShot> sh(nshots);
    for (int q = 0; q < nshots; ++q) {
        GradShot &x = sh[q];
        x.ws = shots[q];
        int rc = adjoint_prepare(x.ws, "ws_adjoint_gradient_shots", &x.kern, &x.tiling, &x.ac);
        if (rc != WS_OK) return rc;
        x.d = data[q];
        if (!on_device) {
            WS_CUDA(cudaMemcpyAsync(x.ac->dd, data[q],
                                    sizeof(float) * size_t(x.ws->nrec) * x.ws->nt_max,
                                    cudaMemcpyHostToDevice, x.ws->stream),
                    "upload observed data");
            x.d = x.ac->dd;
        }
        x.grad = x.ac->grad;   // each shot's own gradient, summed below
    }
    int rc = gradient_run(sh.data(), nshots, mode);
    if (rc != WS_OK) return rc;
    // the sum on shot 0's stream, after every shot's gradient
    ws_t w0 = shots[0];
    const cudaStream_t s0 = w0->stream;
    const long long ncell = (long long)w0->g.nx * w0->g.ny * w0->g.nz;
    for (int q = 1; q < nshots; ++q) {
        cudaEvent_t ev;
        WS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "ws_adjoint_gradient_shots");
        cudaError_t e = cudaEventRecord(ev, shots[q]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, ev, 0);
        cudaEventDestroy(ev);
        WS_CUDA(e, "ws_adjoint_gradient_shots");
    }
    ws::FieldList list{};
    for (int q = 0; q < nshots; ++q) list.p[q] = sh[q].grad;
    float *out = on_device ? grad_m : sh[0].ac->grad;
    WS_CUDA(ws::launch_sum_fields(list, nshots, ncell, out, s0), "gradient sum kernel");
    w0->launches++;
    double *norm = sh[0].ac->norm;
    const int np = ws::residual_partial_count();
    WS_CUDA(ws::launch_norm2(out, ncell, norm, norm + np, s0), "gradient norm kernels");
    w0->launches += 3;
    if (!on_device)
        WS_CUDA(cudaMemcpyAsync(grad_m, out, sizeof(float) * size_t(ncell), cudaMemcpyDeviceToHost,
                                s0),
                "copy gradient");
    double gn = 0.0;
    WS_CUDA(cudaMemcpyAsync(&gn, norm + np, sizeof(double), cudaMemcpyDeviceToHost, s0),
            "copy gradient norm");
    rc = gradient_finish(sh.data(), nshots, misfit);
    if (rc != WS_OK) return rc;
    if (grad_norm) *grad_norm = gn;
    return WS_OK;
}

}  // extern "C"
