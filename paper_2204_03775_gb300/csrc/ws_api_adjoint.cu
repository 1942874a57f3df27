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
    } else {
    }
    *kern_out = kern;
    *tiling_out = tiling;
    *acp = ac;
    return WS_OK;
}

// The forward run from rest over N steps: traces recorded, checkpoint pairs
// (u^{jC}, u^{jC-1}) saved; the cache then holds this model version's run.
int adjoint_forward(ws_t ws, AdjointCache *ac, int kern, const ws::StreamTiling &tiling) {
    const ws::Geom &g = ws->g;
    const int N = ws->nt_max;
    const int C = (int)std::ceil(std::sqrt((double)N));
    const size_t fb = field_bytes(g);
    const size_t ntr = size_t(ws->nrec) * N;
    const cudaStream_t st = ws->stream;
    std::vector<float *> &ck = ac->ck;
    int rc = WS_OK;
    ac->fwd_valid = false;
    for (int b = 0; b < 2; ++b) WS_CUDA(cudaMemsetAsync(ws->buf[b], 0, fb, st), "zero fields");
    WS_CUDA(cudaMemsetAsync(ws->traces, 0, sizeof(float) * ntr, st), "zero traces");
    ws->step = 0;
    ws->trace_start = 0;
    ws::StepArgs a = base_args(ws);
    for (int n = 0; n < N; ++n) {
        if (n > 0 && n % C == 0) {
            const int j = n / C;
            WS_CUDA(cudaMemcpyAsync(ck[2 * (j - 1)], ws->buf[ws->cur], fb, cudaMemcpyDeviceToDevice, st),
                    "save checkpoint");
            WS_CUDA(cudaMemcpyAsync(ck[2 * (j - 1) + 1], ws->buf[1 - ws->cur], fb,
                                    cudaMemcpyDeviceToDevice, st),
                    "save checkpoint");
        }
        const int c = ws->cur;
        rc = step_fp32(ws, a, kern, tiling, ws->buf[c], &ws->tmap_halo[c], ws->buf[1 - c],
                       &ws->tmap_tile[1 - c], ws->buf[1 - c], n, true, true);
        if (rc != WS_OK) return rc;
        ws->cur = 1 - c;
        ws->step++;
    }

    ac->fwd_valid = true;
    ac->fwd_version = ws->model_version;
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
    int kern = WS_KERNEL_STREAM;
    ws::StreamTiling tiling{};
    AdjointCache *ac = nullptr;
    int rc = adjoint_prepare(ws, "ws_adjoint_gradient", &kern, &tiling, &ac);
    if (rc != WS_OK) return rc;
    const ws::Geom &g = ws->g;
    const int N = ws->nt_max;
    const int C = (int)std::ceil(std::sqrt((double)N));    // states per segment
    const int nck = (N + C - 1) / C;                        // segments
    const size_t fb = field_bytes(g);
    const size_t ncell = size_t(g.nx) * g.ny * g.nz;
    const size_t ntr = size_t(ws->nrec) * N;
    const cudaStream_t st = ws->stream;
    for (auto &f : ac->rho) WS_CUDA(cudaMemsetAsync(f.p, 0, fb, st), "zero adjoint field");
    std::vector<float *> &ck = ac->ck;
    std::vector<float *> &lap = ac->lap;
    MappedField *ring = ac->ring;
    MappedField *rho = ac->rho;
    float2 *acc = ac->acc;
    double *partials = ac->partials;
    float *r = ac->r, *grad = on_device ? grad_m : ac->grad;
    const float *d = data;
    int *rec = ac->rec;
    const int np = ws::residual_partial_count();
    WS_CUDA(cudaMemsetAsync(acc, 0, 2 * fb, st), "zero gradient accumulator");
    WS_CUDA(cudaMemcpyAsync(rec, ws->rec_ijk.data(), sizeof(int) * 3 * ws->nrec,
                            cudaMemcpyHostToDevice, st),
            "upload receivers");
    if (!on_device) {
        WS_CUDA(cudaMemcpyAsync(ac->dd, data, sizeof(float) * ntr, cudaMemcpyHostToDevice, st),
                "upload observed data");
        d = ac->dd;
    }

    // 1. forward from rest, recording the traces and the checkpoints; a
    // residual given for the run that ws_forward left in the cache (same
    // model version) needs no new forward run
    if (!(mode == WS_ADJ_RESIDUAL && ac->fwd_valid && ac->fwd_version == ws->model_version)) {
        rc = adjoint_forward(ws, ac, kern, tiling);
        if (rc != WS_OK) return rc;
    }
    ws::StepArgs a = base_args(ws);

    // 2. residual and misfit
    WS_CUDA(ws::launch_residual(mode == WS_ADJ_DATA ? ws->traces : d,
                                mode == WS_ADJ_DATA ? d : nullptr, (long long)ntr, r, partials,
                                partials + np, st),
            "residual kernels");
    ws->launches += 2;

    // 3. backward: rho^k, k = N .. 1, segment by segment, the segment's
    // states recomputed from its checkpoint
    int rc_cur = 0;   // rho[rc_cur] = rho^{k+1}, rho[1 - rc_cur] = rho^{k+2}
    for (int j = nck - 1; j >= 0; --j) {
        const int n0 = j * C, n1 = std::min(n0 + C, N);
        // u^{n0}, u^{n0-1} into the ring, then steps n0 .. n1-1, each storing
        // L u^n into lap[n - n0] (u^{n1} itself is not needed)
        if (j == 0) {
            WS_CUDA(cudaMemsetAsync(ring[0].p, 0, fb, st), "zero initial state");
            WS_CUDA(cudaMemsetAsync(ring[1].p, 0, fb, st), "zero initial state");
        } else {
            WS_CUDA(cudaMemcpyAsync(ring[0].p, ck[2 * (j - 1)], fb, cudaMemcpyDeviceToDevice, st),
                    "restore checkpoint");
            WS_CUDA(cudaMemcpyAsync(ring[1].p, ck[2 * (j - 1) + 1], fb, cudaMemcpyDeviceToDevice, st),
                    "restore checkpoint");
        }
        int uc = 0;   // ring[uc] = u^n
        for (int t = 0; t < n1 - n0; ++t) {
            MappedField &un = ring[uc], &um = ring[1 - uc];
            a.lap = lap[t];
            rc = step_fp32(ws, a, kern, tiling, un.p, &un.halo, um.p, &um.tile, um.p, n0 + t, true,
                           false);
            a.lap = nullptr;
            if (rc != WS_OK) return rc;
            uc = 1 - uc;
        }
        for (int k = n1; k > n0; --k) {
            MappedField &r1 = rho[rc_cur], &r2 = rho[1 - rc_cur];
            rc = step_fp32(ws, a, kern, tiling, r1.p, &r1.halo, r2.p, &r2.tile, r2.p, k, false,
                           false);
            if (rc != WS_OK) return rc;
            rc_cur = 1 - rc_cur;   // rho[rc_cur] = rho^k
            WS_CUDA(ws::launch_inject(rho[rc_cur].p, ws->w, ws->gx, ws->gy, ws->gz, g, rec,
                                      ws->nrec, r, N, k - 1, st),
                    "adjoint injection kernel");
            ws::Sources src{};
            sources_of_step(ws, k - 1, &src);
            WS_CUDA(ws::launch_imaging(rho[rc_cur].p, lap[k - 1 - n0], g, src, ws->gx, ws->gy,
                                       ws->gz, acc, st),
                    "gradient imaging kernel");
            ws->launches += 2;
        }
    }
    const double hdt = ws->h / ws->dt;
    WS_CUDA(ws::launch_finalize_gradient(acc, ws->w, g, hdt * hdt, grad, st),
            "gradient finalize kernel");
    ws->launches++;
    if (!on_device)
        WS_CUDA(cudaMemcpyAsync(grad_m, grad, sizeof(float) * ncell, cudaMemcpyDeviceToHost, st),
                "copy gradient");
    double J = 0.0;
    WS_CUDA(cudaMemcpyAsync(&J, partials + np, sizeof(double), cudaMemcpyDeviceToHost, st),
            "copy misfit");
    WS_CUDA(cudaStreamSynchronize(st), "ws_adjoint_gradient");
    if (misfit) *misfit = J;
    unsigned status = 0;
    WS_CUDA(cudaMemcpy(&status, ws->status, sizeof status, cudaMemcpyDeviceToHost),
            "ws_adjoint_gradient");
    if (status & ws::kStatusTimeout) {
        WS_CUDA(cudaMemset(ws->status, 0, sizeof(unsigned)), "ws_adjoint_gradient");
        return fail(WS_ERR_TIMEOUT, "a bounded device wait ran out in a step kernel");
    }
    return WS_OK;
}

}  // extern "C"
