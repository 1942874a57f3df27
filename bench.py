#!/usr/bin/env python
"""Throughput of the fused 25-point acoustic wave step (grid-point updates/s).

A "step" is one leapfrog time step of the whole hot path (Laplacian, update,
taper, source, receivers) over the 1024^3 layered survey: FP32 fields,
h = 10 m, dt at CFL 0.4, 20-cell absorbing layer on every face, one 10 Hz
Ricker at (512, 512, 20), 32 x 32 receivers on k = 20. Inputs (three 4.4 GB
fields per step) are far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0. Under torchrun each rank advances its own
replica of the survey (the problem does not need an exchange between GPUs
to be benchmarked; replicas only), and the time is the maximum over ranks.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpoint-updates/s & % of HBM roofline, 25-pt wave step, FP32 vs BF16 at stated err"
UNIT = "Gpoint-updates/s"
BYTES_PER_POINT = 16  # read u^n, u^{n-1}, (V dt/h)^2; write u^{n+1} (FP32)
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_stream_layered512_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2204_03775_gb300", "csrc", f)
                  for f in ("ws_kernels_stream.cu", "ws_ptx.cuh", "ws_internal.h")]


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=1024, help="cells per axis (default 1024)")
    ap.add_argument("--kernel", choices=["auto", "stream", "direct"], default="auto")
    ap.add_argument("--tile", default="0x0", help="streaming tile, e.g. 64x16 (0x0 = default)")
    ap.add_argument("--zblock", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--case", choices=["survey", "fp16", "bf16", "adjoint", "batched"],
                    default="survey",
                    help="survey (default): the JSON line. The others run one workload alone "
                         "(for profilers) and print its timing: fp16/bf16 = the layered survey "
                         "of --size with 16-bit storage for --warmup + --steps steps; adjoint = "
                         "one shot of the adjoint survey (--size, --steps) gradient, three "
                         "times; batched = the 64-shot batch for --steps steps")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-shot batched-launch report")
    ap.add_argument("--shots", type=int, default=64,
                    help="--case batched: the first N shots of the 64-shot workload")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the 256^3 16-shot adjoint-gradient report")
    ap.add_argument("--no-storage16", action="store_true",
                    help="skip the BF16/FP16 storage timings and errors")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the 256^3 accuracy report against the FP64 oracle")
    return ap.parse_args()


def kernel_sources_digest() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(cells):
    """DRAM bytes per launch of the streaming kernel over `cells` cells: the
    committed ncu summary's bytes per cell (a small-case capture) times the
    cells, if the summary matches the current kernel sources; else None."""
    try:
        fields = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if line.startswith("#") or ":" not in line:
                    continue
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("kernel_sources_sha256") != kernel_sources_digest():
            return None
        return float(fields["bytes_per_cell"]) * cells
    except (OSError, KeyError, ValueError):
        return None


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """SM clocks and throttle reasons sampled while it runs (reads only).

    Primary: NVML through ctypes, polled every few milliseconds from a thread,
    so that even a timed region well under a second gets many samples.
    Fallback: nvidia-smi at its 200 ms loop."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    # NVML clock event reason bits
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap"}

    def __init__(self, gpu_id, period_s=0.005):
        self.proc = None
        self.gpu_id = gpu_id
        self.period_s = period_s
        self.rows = []
        self.source = None
        self._stop = None
        self._thread = None

    def _nvml_open(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        handle = ctypes.c_void_p()
        if self.gpu_id:
            rc = lib.nvmlDeviceGetHandleByUUID(self.gpu_id.encode(), ctypes.byref(handle))
        else:
            rc = lib.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(handle))
        if rc != 0:
            raise OSError(f"nvmlDeviceGetHandle: {rc}")
        return lib, handle

    def _poll(self, lib, handle):
        import ctypes
        mhz, mx, why = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        lib.nvmlDeviceGetMaxClockInfo(handle, 1, ctypes.byref(mx))
        while not self._stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(handle, 1, ctypes.byref(mhz)) == 0
                    and get_reasons(handle, ctypes.byref(why)) == 0):
                names = [n for bit, n in self.REASONS.items() if why.value & bit]
                self.rows.append((float(mhz.value), float(mx.value), names))
            self._stop.wait(self.period_s)

    def __enter__(self):
        import threading
        try:
            lib, handle = self._nvml_open()
            self._stop = threading.Event()
            self._thread = threading.Thread(target=self._poll, args=(lib, handle), daemon=True)
            self._thread.start()
            self.source = "nvml"
            return self
        except (OSError, AttributeError):
            pass
        cmd = ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}",
               "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.source = "nvidia-smi"
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in (self.out or "").splitlines():
                parts = [p.strip() for p in line.split(",")]
                if len(parts) != len(self.FIELDS):
                    continue
                try:
                    flags = [names[i] for i, f in enumerate(parts[3:]) if f.lower() == "active"]
                    self.rows.append((float(parts[0]), float(parts[1]), flags))
                except ValueError:
                    continue

    def summary(self):
        if not self.rows:
            return None
        reasons = sorted({n for _, _, flags in self.rows for n in flags})
        return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                "sm_max_mhz": max(r[1] for r in self.rows), "reasons": reasons,
                "samples": len(self.rows), "source": self.source}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n_gpus and world > 1:
        raise SystemExit(f"--gpus {n_gpus} but WORLD_SIZE={world}")
    return world, rank, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, points: int, steps: int, seconds: float) -> float:
    """Point updates per second of all replicas together (each rank did points x steps)."""
    return world * points * steps / seconds / 1e9


def cpu_baseline(w, target_s=15.0):
    """The FP64 oracle on a bounded slab of the same survey (host cores)."""
    import numpy as np
    import oracle

    oracle.build()
    depth = int(min(w.nz, max(w.sources[0][2] + 5, 32)))
    slab = np.ascontiguousarray(w.vel[:depth])
    win = (0, 0, 0, w.nx, w.ny, w.nz)
    cells = depth * w.nx * w.ny
    # calibrate on the slab itself (the first call also starts the thread pool),
    # then size the timed sample to about target_s seconds
    oracle.run(slab, w.h, w.dt, 1, sources=w.sources, sponge=w.sponge, window=win)
    n = 3
    while True:
        t0 = time.perf_counter()
        oracle.run(slab, w.h, w.dt, n, sources=w.sources, sponge=w.sponge, window=win)
        el = time.perf_counter() - t0
        if el > 1.0 or n >= 400:
            break
        n *= 4
    steps = int(max(3, min(4000, target_s * n / el)))
    t0 = time.perf_counter()
    oracle.run(slab, w.h, w.dt, steps, sources=w.sources, receivers=None, sponge=w.sponge,
               window=win)
    el = time.perf_counter() - t0
    pts = cells * steps
    return {"value": pts / el / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, top slab k in [0,{depth}) of the {w.nx}x{w.ny}x{w.nz} "
                      f"survey (same model, taper, source), {steps} steps from rest, "
                      f"{el:.1f} s wall"}


def storage16_report(w, K, W, stream, peak):
    """Throughput of the 16-bit storage modes on the same survey, and their
    error against the FP32 path (itself 2.5e-6 from the FP64 oracle after
    1000 steps on 256^3) at steps 100, 500 and 1000, evaluated on the device."""
    import torch
    import paper_2204_03775_gb300 as wsb

    def make(storage, nt_max):
        h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
        wsb.ws_set_stream(h, stream)
        wsb.ws_set_storage(h, storage)
        wsb.ws_set_velocity(h, w.vel)
        wsb.ws_set_sponge(h, *w.sponge)
        for s in w.sources:
            wsb.ws_add_source(h, *s)
        wsb.ws_set_receivers(h, w.receivers, nt_max)
        return h

    out = {}
    modes = [("bf16", wsb.WS_STORAGE_BF16), ("fp16", wsb.WS_STORAGE_FP16)]
    for name, st in modes:
        h = make(st, K + W)
        wsb.ws_step(h, W)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wsb.ws_step(h, K)
        e1.record(stream)
        torch.cuda.synchronize()
        wsb.ws_synchronize(h)
        sec = e0.elapsed_time(e1) / 1e3 / K
        out[name] = {"value": w.points / sec / 1e9, "unit": UNIT, "ms_per_step": 1e3 * sec,
                     "bytes_per_point": 10, "roofline_frac": 10 * w.points / sec / 1e9 / peak}
        wsb.ws_destroy(h)

    checkpoints = [100, 500, 1000]
    hs = {name: make(st, checkpoints[-1]) for name, st in [("fp32", wsb.WS_STORAGE_FP32)] + modes}
    bufs = {name: torch.empty((w.nz, w.ny, w.nx), dtype=torch.float32, device="cuda") for name in hs}
    errs = {name: [] for name, _ in modes}
    done = 0
    for c in checkpoints:
        for name, h in hs.items():
            wsb.ws_step(h, c - done)
            wsb.ws_read_field(h, bufs[name], None)
        torch.cuda.synchronize()
        ref = bufs["fp32"].double()
        nref = torch.linalg.vector_norm(ref).item()
        for name, _ in modes:
            d = torch.linalg.vector_norm(bufs[name].double() - ref).item()
            errs[name].append(d / nref)
        done = c
    for name, _ in modes:
        out[name]["rel_l2_vs_fp32_at_steps"] = dict(zip(map(str, checkpoints), errs[name]))
        out[name]["limits"] = ("single grids with nx >= 64 and ny >= 16; batches and the "
                               "adjoint gradient run FP32 storage")
    for h in hs.values():
        wsb.ws_destroy(h)
    return out


def accuracy_report(n=256, checkpoints=(100, 500, 1000)):
    """Every storage mode against the FP64 oracle on the layered survey at
    n^3 (the oracle runs on the host cores: ~30 s at 256^3 on 16 cores; the
    1024^3 field would need ~26 GB and half an hour), relative L2 of the
    field and of the traces recorded so far, at each checkpoint."""
    import numpy as np
    import oracle
    import paper_2204_03775_gb300 as wsb
    from paper_2204_03775_gb300 import synthetic

    oracle.build()
    w = synthetic.layered_survey(n, n, n, nt=checkpoints[-1])
    modes = [("fp32", wsb.WS_STORAGE_FP32), ("fp16", wsb.WS_STORAGE_FP16),
             ("bf16", wsb.WS_STORAGE_BF16)]
    hs = {}
    for name, st in modes:
        h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
        wsb.ws_set_storage(h, st)
        wsb.ws_set_velocity(h, w.vel)
        wsb.ws_set_sponge(h, *w.sponge)
        for s in w.sources:
            wsb.ws_add_source(h, *s)
        wsb.ws_set_receivers(h, w.receivers, w.nt)
        hs[name] = h
    out = {name: {"field": {}, "traces": {}} for name, _ in modes}
    v64 = w.vel.astype(np.float64)
    ref, done, ref_tr = None, 0, []
    t0 = time.perf_counter()
    for c in checkpoints:
        kw = {} if ref is None else {"n0": done, "u_init": ref["u"], "uprev_init": ref["u_prev"]}
        ref = oracle.run(v64, w.h, w.dt, c - done, sources=w.sources, receivers=w.receivers,
                         sponge=w.sponge, **kw)
        ref_tr.append(ref["traces"])
        rtr = np.concatenate(ref_tr, axis=1)
        nref, ntr = np.linalg.norm(ref["u"]), np.linalg.norm(rtr)
        for name, h in hs.items():
            wsb.ws_step(h, c - done)
            u, _ = wsb.ws_read_field(h)
            tr = wsb.ws_read_traces(h)[:, :c]
            out[name]["field"][str(c)] = float(np.linalg.norm(u - ref["u"]) / nref)
            out[name]["traces"][str(c)] = float(np.linalg.norm(tr - rtr) / ntr)
        done = c
    for h in hs.values():
        wsb.ws_destroy(h)
    bound = {"fp32": 1e-4, "fp16": 1e-2, "bf16": 1e-2}
    for name, _ in modes:
        errs = list(out[name]["field"].values()) + list(out[name]["traces"].values())
        out[name]["bound"] = bound[name]
        out[name]["within_bound_at_every_checkpoint"] = bool(max(errs) <= bound[name])
    return {"workload": f"layered_survey {n}x{n}x{n} (the benchmark's model recipe), "
                        f"{checkpoints[-1]} steps, FP64 oracle on {oracle.num_threads()} host "
                        f"cores ({time.perf_counter() - t0:.0f} s)",
            "metric": "relative L2 vs the FP64 oracle", **out}


def _shot_handle(wsb, w, nt_max):
    h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_velocity(h, w.vel)
    wsb.ws_set_sponge(h, *w.sponge)
    for s in w.sources:
        wsb.ws_add_source(h, *s)
    wsb.ws_set_receivers(h, w.receivers, nt_max)
    return h


def batched_report(peak):
    """64 shots on uneven grids (96^3 .. 320x320x256), 500 steps each: one
    persistent launch per step over all shots, replayed as a CUDA graph, with
    the tiling the batch's online tuner chose; against the same shots stepped
    one after another with ws_step (per-shot launches, default tiling)."""
    import torch
    import paper_2204_03775_gb300 as wsb
    from paper_2204_03775_gb300 import synthetic

    shots = synthetic.batched_shots()
    nt = shots[0].nt
    cells = sum(w.points for w in shots)
    hs = [_shot_handle(wsb, w, nt) for w in shots]
    b = wsb.ws_batch_create(hs)

    def restart():
        for h, w in zip(hs, shots):
            wsb.ws_write_field(h, None, None, 0)
            wsb.ws_set_receivers(h, w.receivers, nt)

    t0 = time.perf_counter()
    wsb.ws_batch_step(b, 60)            # online tuning: 18 candidates x 2 steps, then the best
    wsb.ws_batch_synchronize(b)
    tune_s = time.perf_counter() - t0
    tiling = wsb.ws_batch_get_tiling(b)
    wsb.ws_batch_set_tiling(b, *tiling)
    restart()
    wsb.ws_batch_step(b, nt)            # captures the graph of nt launches
    wsb.ws_batch_synchronize(b)
    restart()
    torch.cuda.synchronize()
    l0 = wsb.ws_batch_launch_count(b)
    t0 = time.perf_counter()
    wsb.ws_batch_step(b, nt)
    wsb.ws_batch_synchronize(b)
    batch_s = time.perf_counter() - t0
    launches = wsb.ws_batch_launch_count(b) - l0
    restart()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h in hs:
        wsb.ws_step(h, nt)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    for h in hs:
        wsb.ws_synchronize(h)
    wsb.ws_batch_destroy(b)
    for h in hs:
        wsb.ws_destroy(h)
    rate = cells * nt / batch_s / 1e9
    return {"workload": f"{len(shots)} shots on grids from the seed, sizes in [96,320]x[96,320]x"
                        f"[96,256] ({cells / 1e6:.0f} M cells), {nt} steps each, FP32",
            "value": rate, "unit": UNIT, "ms_per_step": 1e3 * batch_s / nt,
            "launches": launches, "graph": True,
            "tiling": {"tile": f"{tiling[0]}x{tiling[1]}", "zmul": tiling[2],
                       "tuning_s": tune_s},
            "roofline_frac": BYTES_PER_POINT * rate / peak,
            "sequential": {"value": cells * nt / seq_s / 1e9, "unit": UNIT,
                           "what": "the same shots one after another, ws_step each"},
            "timing": "host clock around ws_batch_step + ws_batch_synchronize"}


def adjoint_report():
    """Gradient of the L2 trace misfit w.r.t. squared slowness on the 256^3
    survey: 16 shots, 128 x 128 receivers, 800 steps, sqrt(N) checkpoints;
    time per 16-shot gradient against one 16-shot forward modelling."""
    import numpy as np
    import torch
    import paper_2204_03775_gb300 as wsb
    from paper_2204_03775_gb300 import synthetic

    w = synthetic.adjoint_survey()
    dev = torch.device("cuda")
    m_true = torch.from_numpy((1.0 / w.vel_true.astype(np.float64) ** 2).astype(np.float32)).to(dev)
    m0 = torch.from_numpy((1.0 / w.vel_start.astype(np.float64) ** 2).astype(np.float32)).to(dev)
    hs, streams = [], []
    for shot in w.shots:
        h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
        st = torch.cuda.Stream()       # one stream per shot: the shots' kernels overlap
        wsb.ws_set_stream(h, st)
        wsb.ws_set_sponge(h, *w.sponge)
        for s in shot:
            wsb.ws_add_source(h, *s)
        wsb.ws_set_receivers(h, w.receivers, w.nt)
        hs.append(h)
        streams.append(st)
    for h in hs:
        wsb.ws_set_slowness2(h, m0)
        tiling = wsb.ws_autotune(h)     # timed once, then cached for the grid size
    nrec = len(w.receivers)

    def forward(m):
        out = []
        for h in hs:
            wsb.ws_set_slowness2(h, m)
            wsb.ws_write_field(h, None, None, 0)
            wsb.ws_set_receivers(h, w.receivers, w.nt)
            wsb.ws_step(h, w.nt)
            t = torch.empty((nrec, w.nt), dtype=torch.float32, device=dev)
            wsb.ws_read_traces(h, t)
            out.append(t)
        torch.cuda.synchronize()
        return out

    d_obs = forward(m_true)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    forward(m0)
    fwd_s = time.perf_counter() - t0
    g = torch.zeros_like(m0)
    gs = torch.empty_like(m0)
    for h in hs:
        wsb.ws_set_slowness2(h, m0)
    # the 16 shots in one call (each on its own stream, interleaved step by step)
    times = []
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g, J, gnorm = wsb.ws_adjoint_gradient_shots(hs, d_obs, wsb.WS_ADJ_DATA, g)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    # the same shots one call at a time, for contrast
    g_seq = torch.zeros_like(m0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h, d in zip(hs, d_obs):
        _, j = wsb.ws_adjoint_gradient(h, d, wsb.WS_ADJ_DATA, gs)
        g_seq += gs
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    seq_rel = float((g_seq - g).abs().max() / g.abs().max())
    for h in hs:
        wsb.ws_destroy(h)
    del hs

    # the same 16-shot misfit and gradient through the torch bridge (the call a
    # user makes): traces(m) per shot, loss, backward; the backward reuses
    # each shot's forward run
    from paper_2204_03775_gb300 import autograd as wsa
    shots = [wsa.Shot((w.nz, w.ny, w.nx), w.h, w.dt, w.nt, shot, w.receivers, w.sponge)
             for shot in w.shots]
    auto_times = []
    for rep in range(2):
        m = m0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = sum(0.5 * ((wsa.traces(m, sh) - d) ** 2).sum() for sh, d in zip(shots, d_obs))
        loss.backward()
        torch.cuda.synchronize()
        auto_times.append(time.perf_counter() - t0)
    auto_rel = float((m.grad - g).abs().max() / g.abs().max())
    del shots
    cells = w.nx * w.ny * w.nz
    return {"workload": f"adjoint_survey {w.nx}^3, 16 shots, {nrec} receivers, {w.nt} steps, "
                        "true = layered + 10% Gaussian blob, start = layered",
            "gradient_s": min(times), "forward_s": fwd_s,
            "gradient_over_forward": min(times) / fwd_s,
            "forward_rate": {"value": len(w.shots) * cells * w.nt / fwd_s / 1e9, "unit": UNIT},
            "misfit": J, "grad_max_abs": float(g.abs().max()), "grad_norm_fp64": gnorm,
            "how": "ws_adjoint_gradient_shots: the 16 shots in one call, each on its own "
                   "stream, interleaved step by step",
            "sequential": {"gradient_s": seq_s, "max_rel_diff": seq_rel,
                           "what": "the same 16 shots, one ws_adjoint_gradient call each"},
            "tiling": {"tile": f"{tiling[0]}x{tiling[1]}", "zblock": tiling[2]},
            "passes": "forward (traces + sqrt(N) checkpoints), residual, then per segment a "
                      "recomputation and the adjoint steps with injection and imaging",
            "torch_autograd": {"forward_backward_s": min(auto_times),
                               "grad_vs_ws_adjoint_gradient": auto_rel,
                               "what": "loss = sum over shots of 0.5 |traces(m) - d|^2; "
                                       "loss.backward() (ws_forward + residual-mode adjoint)"},
            "timing": "host clock"}


def run_case(args):
    """One workload alone, for profiler runs (see --case)."""
    import numpy as np
    import torch
    import paper_2204_03775_gb300 as wsb
    from paper_2204_03775_gb300 import synthetic

    wsb.load_library(build_if_missing=True)
    n, K, W = args.size, args.steps, args.warmup
    t0 = time.perf_counter()
    if args.case in ("fp16", "bf16"):
        w = synthetic.layered_survey(n, n, n, nt=K + W)
        h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
        tx, ty = (int(x) for x in args.tile.split("x"))
        wsb.ws_set_kernel(h, wsb.WS_KERNEL_AUTO, tx, ty, args.zblock)
        wsb.ws_set_storage(h, wsb.WS_STORAGE_FP16 if args.case == "fp16" else wsb.WS_STORAGE_BF16)
        wsb.ws_set_velocity(h, w.vel)
        wsb.ws_set_sponge(h, *w.sponge)
        for s in w.sources:
            wsb.ws_add_source(h, *s)
        wsb.ws_set_receivers(h, w.receivers, K + W)
        wsb.ws_step(h, W)
        wsb.ws_synchronize(h)
        t0 = time.perf_counter()
        wsb.ws_step(h, K)
        wsb.ws_synchronize(h)
        cells = w.points * K
    elif args.case == "adjoint":
        w = synthetic.adjoint_survey(n, K)
        m0 = torch.from_numpy((1.0 / w.vel_start.astype(np.float64) ** 2).astype(np.float32)).cuda()
        h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
        wsb.ws_set_sponge(h, *w.sponge)
        for s in w.shots[0]:
            wsb.ws_add_source(h, *s)
        wsb.ws_set_receivers(h, w.receivers, w.nt)
        wsb.ws_set_slowness2(h, m0)
        wsb.ws_autotune(h)
        d = torch.zeros((len(w.receivers), w.nt), dtype=torch.float32, device="cuda")
        g = torch.empty_like(m0)
        for rep in range(3):
            if rep == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            wsb.ws_adjoint_gradient(h, d, wsb.WS_ADJ_DATA, g)
        torch.cuda.synchronize()
        cells = 2 * w.nx * w.ny * w.nz * w.nt   # two gradients timed, one forward-run of cells each
    else:
        shots = synthetic.batched_shots(nt=K)[:args.shots]
        hs = [_shot_handle(wsb, x, K + 60) for x in shots]
        b = wsb.ws_batch_create(hs)
        tx, ty = (int(x) for x in args.tile.split("x"))
        if tx:   # a fixed tiling (--zblock is then the z-block rule, see ws_batch_set_tiling)
            wsb.ws_batch_set_tiling(b, tx, ty, args.zblock)
        wsb.ws_batch_step(b, 60)
        wsb.ws_batch_synchronize(b)
        t0 = time.perf_counter()
        wsb.ws_batch_step(b, K)
        wsb.ws_batch_synchronize(b)
        cells = sum(x.points for x in shots) * K
    el = time.perf_counter() - t0
    print(json.dumps({"case": args.case, "size": n, "steps": K, "seconds": el,
                      "Gpoint_updates_per_s": cells / el / 1e9}), flush=True)


def run_reference(args):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    world, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2204_03775_gb300 import synthetic

    oracle.build()
    n = args.size
    w = synthetic.layered_survey(n, n, n, nt=args.steps + args.warmup)
    # per-step sample: a top slab sized so that warm-up + timed steps take ~2 minutes
    t0 = time.perf_counter()
    oracle.run(w.vel[:4], w.h, w.dt, 2, sponge=w.sponge, window=(0, 0, 0, n, n, n))
    rate = 2 * 4 * n * n / (time.perf_counter() - t0)
    depth = int(max(1, min(64, 120.0 * rate / ((args.steps + args.warmup) * n * n))))
    src = [s for s in w.sources if s[2] < depth]
    slab = np.ascontiguousarray(w.vel[:depth])
    win = (0, 0, 0, n, n, n)
    warm = oracle.run(slab, w.h, w.dt, args.warmup, sources=src, sponge=w.sponge, window=win)
    t0 = time.perf_counter()
    oracle.run(slab, w.h, w.dt, args.steps, sources=src, sponge=w.sponge, window=win,
               u_init=warm["u"], uprev_init=warm["u_prev"], n0=args.warmup)
    el = time.perf_counter() - t0
    pts = depth * n * n * args.steps
    value = pts / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"layered_survey {n}x{n}x{n}", "sample_depth": depth,
                   "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"top slab k in [0,{depth}) of the survey per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.case != "survey":
        return run_case(args)

    import numpy as np
    import torch
    import paper_2204_03775_gb300 as wsb
    from paper_2204_03775_gb300 import synthetic

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wsb.load_library(build_if_missing=True)

    n = args.size
    K, W = args.steps, args.warmup
    w = synthetic.layered_survey(n, n, n, nt=K + W)
    npts = w.points
    stream = torch.cuda.current_stream()

    h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_stream(h, stream)
    kern = {"auto": wsb.WS_KERNEL_AUTO, "stream": wsb.WS_KERNEL_STREAM,
            "direct": wsb.WS_KERNEL_DIRECT}[args.kernel]
    tx, ty = (int(x) for x in args.tile.split("x"))
    wsb.ws_set_kernel(h, kern, tx, ty, args.zblock)
    wsb.ws_set_velocity(h, w.vel)
    wsb.ws_set_sponge(h, *w.sponge)
    for s in w.sources:
        wsb.ws_add_source(h, *s)
    wsb.ws_set_receivers(h, w.receivers, K + W)

    wsb.ws_step(h, W)
    wsb.ws_synchronize(h)

    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else None
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    launches0 = wsb.ws_launch_count(h)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id) as clk:
        evs[0].record(stream)
        for s in range(K):
            wsb.ws_step(h, 1)
            evs[s + 1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wsb.ws_synchronize(h)
    launches = wsb.ws_launch_count(h) - launches0
    elapsed = evs[0].elapsed_time(evs[K]) / 1e3
    per_launch = [evs[s].elapsed_time(evs[s + 1]) / 1e3 for s in range(K)]
    if dist is not None:
        elapsed = max_over_ranks(elapsed, dist, "cuda")

    # end to end through the public API from pinned host memory: upload the
    # model, run the K steps, read the traces back
    e2e = None
    if not args.no_e2e:
        vel_pinned = torch.from_numpy(w.vel).pin_memory()
        wsb.ws_write_field(h, None, None, 0)
        wsb.ws_set_receivers(h, w.receivers, K)
        traces = torch.empty((len(w.receivers), K), dtype=torch.float32).pin_memory()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        wsb.ws_set_velocity(h, vel_pinned)
        wsb.ws_step(h, K)
        wsb.ws_read_traces(h, traces)
        e2e_s = time.perf_counter() - t0
        if dist is not None:
            e2e_s = max_over_ranks(e2e_s, dist, "cuda")
        e2e = {"value": whole_job_rate(world, npts, K, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": vel_pinned.numel() * 4 / K,
               "d2h_bytes_per_step": traces.numel() * 4 / K,
               "what": "ws_set_velocity (pinned host model) + ws_step(K) + ws_read_traces (pinned host)"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    avg_launch = statistics.mean(per_launch)
    peak, peak_kind = measured_peak()
    achieved = BYTES_PER_POINT * npts / avg_launch / 1e9
    value = whole_job_rate(world, npts, K, elapsed)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * elapsed / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"layered_survey {n}x{n}x{n}, h=10 m, CFL 0.4, 20-cell Cerjan "
                               f"layer, 10 Hz Ricker at ({n // 2},{n // 2},20), 32x32 receivers "
                               f"at k=20", "kernel": args.kernel, "tile": args.tile,
                   "zblock": args.zblock, "l2": "inputs larger than L2 (3 x 4.4 GB per step)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(npts),
                     "traffic_source": "profiles/step_stream_layered512_traffic.txt: DRAM bytes "
                                       "per cell of a 512^3 capture x the launch's cells",
                     "peak_source": peak_kind,
                     "bytes_per_point": BYTES_PER_POINT,
                     "kernel_ms": 1e3 * avg_launch},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    wsb.ws_destroy(h)
    if world == 1 and not args.no_storage16 and n >= 64:
        line["storage16"] = storage16_report(w, K, W, stream, peak)
        for mode in line["storage16"].values():     # speed relative to FP32 storage
            mode["vs_fp32_storage"] = mode["value"] / line["value"]
    if world == 1 and not args.no_accuracy:
        line["accuracy_vs_oracle"] = accuracy_report()
        if "storage16" in line:
            for name, mode in line["storage16"].items():
                mode["rel_l2_vs_oracle_at_steps"] = line["accuracy_vs_oracle"][name]["field"]
                mode["within_1e-2_vs_oracle"] = \
                    line["accuracy_vs_oracle"][name]["within_bound_at_every_checkpoint"]
    if world == 1 and not args.no_batched:
        line["batched"] = batched_report(peak)
    if world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_report()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
