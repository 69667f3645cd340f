"""Served form: a request loop with continuous batching over device-resident scans.

Requests (scans) arrive over time. The loop admits a request when it has arrived, a slot
is free and its device memory (inputs, state, workspace) fits the budget; the scan's
frames, reference image and pixel map then stay on the device until it finishes. Every
pass over the active scans launches one iteration (make_object_map, update_pixel_map,
through pxst_iterate) of each scan whose previous iteration has completed, on a pool of
streams, so the iterations of scans admitted at different times run side by side on the
GPU and a new scan joins at the next pass instead of waiting for the others to finish.
A scan's completion time is a CUDA event after its last iteration; its latency is that
time minus its arrival. A request whose scan is returned on the host (pinned CPU tensors) is
copied to the device at admission, on the admission stream, so the copy counts in its
latency. A request larger than the whole memory budget is rejected at once (it could never
be admitted); a request can be cancelled at any time: it is dropped if still waiting, or its
slot is freed after its iteration in flight, and the other scans are not affected.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from . import FORM_FP32, Reconstruction


@dataclass
class Request:
    rid: int
    arrival: float                      # seconds after the loop starts
    make: Callable                      # () -> object with frames, W, M, delta, u_init, ref_shape, window (device)
    est_bytes: int                      # device memory the request will hold (for admission)
    n_iter: int = 10
    form: int = FORM_FP32
    tile: int = 0
    quadratic: bool = True              # the 3x3 fit (False: integer argmin)
    keep_result: bool = False
    # filled by the server
    admitted: float | None = None
    done: float | None = None
    evals: int = 0
    result: dict | None = None
    iterations_done: int = 0
    cancelled: bool = False
    rejected: str | None = None         # why the request was not admitted
    charged_bytes: int = 0              # device bytes charged against the budget

    def cancel(self):
        """Drop the request: no further iteration is launched for it (safe from any thread)."""
        self.cancelled = True


@dataclass
class _Slot:
    req: Request
    rec: Reconstruction
    stream: object
    event: object
    iters: int = 0
    inflight: bool = False
    nbytes: int = 0


def estimate_bytes(dims, window, form):
    """Device bytes of one scan: inputs, state and workspace (pxst_workspace_size)."""
    from . import Dims, Options, workspace_size
    n, ny, nx, Ry, Rx = dims
    P, R = ny * nx, Ry * Rx
    inputs = 4 * n * P + 4 * P + P + 16 * n + 16 * P
    state = 8 * R + 4 * P
    return inputs + state + workspace_size(Dims(n, ny, nx, Ry, Rx), Options(window[0], window[1], True, form))


class Server:
    def __init__(self, mem_budget, n_streams=8, max_active=64, device="cuda"):
        import torch
        self.budget = int(mem_budget)
        self.max_active = int(max_active)
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]
        self.admit_stream = torch.cuda.Stream(device=self.device)

    def run(self, requests, realtime=True, idle_sleep=2e-4):
        """Serve every request; returns a summary (throughput, latency percentiles). With
        realtime=False every request counts as arrived at time 0."""
        import torch
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        active: list[_Slot] = []
        used = 0
        nxt = 0
        torch.cuda.synchronize(self.device)
        t_start = torch.cuda.Event(enable_timing=True)
        t_start.record(torch.cuda.current_stream(self.device))
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        peak_active = 0
        peak_used = 0
        while pending or active:
            now = time.perf_counter() - t0
            # admission: arrived, a slot free, memory available
            while pending and (not realtime or pending[0].arrival <= now) and len(active) < self.max_active:
                r = pending[0]
                if r.cancelled:
                    pending.pop(0)
                    continue
                if r.est_bytes > self.budget:
                    # it could never fit: rejected, and it does not hold up the requests behind it
                    pending.pop(0)
                    r.rejected = f"needs {r.est_bytes} B of device memory, the budget is {self.budget} B"
                    continue
                if used + r.est_bytes > self.budget:
                    break
                pending.pop(0)
                with torch.cuda.stream(self.admit_stream):
                    sc = r.make()
                    dev = lambda t: t.to(self.device, non_blocking=True) if not t.is_cuda else t
                    rec = Reconstruction.from_device(dev(sc.frames), dev(sc.W), dev(sc.M), dev(sc.delta),
                                                     dev(sc.u_init), sc.ref_shape, sc.window, quadratic=r.quadratic,
                                                     form=r.form, tile=r.tile)
                ready = torch.cuda.Event()
                ready.record(self.admit_stream)
                st = self.streams[nxt % len(self.streams)]
                nxt += 1
                st.wait_event(ready)
                r.admitted = time.perf_counter() - t0
                r.evals = int(sc.M.sum().item()) * (2 * sc.window[0] + 1) * (2 * sc.window[1] + 1) * \
                    int(sc.frames.shape[0]) * r.n_iter
                # charged: the larger of the estimate and what the scan holds
                slot = _Slot(r, rec, st, torch.cuda.Event(enable_timing=True),
                             nbytes=max(int(r.est_bytes), rec.device_bytes()))
                r.charged_bytes = slot.nbytes
                used += slot.nbytes
                peak_used = max(peak_used, used)
                active.append(slot)
            peak_active = max(peak_active, len(active))
            # one iteration of every scan whose previous one has finished
            launched = False
            for slot in list(active):
                if slot.inflight and not slot.event.query():
                    continue
                slot.inflight = False
                slot.req.iterations_done = slot.iters
                if slot.req.cancelled:
                    active.remove(slot)
                    used -= slot.nbytes
                    del slot
                    continue
                if slot.iters == slot.req.n_iter:
                    r = slot.req
                    r.done = t_start.elapsed_time(slot.event) / 1e3
                    if r.keep_result:
                        r.result = dict(u=slot.rec.u.clone(), I_ref=slot.rec.I_ref.clone(), w=slot.rec.w.clone(),
                                        err=slot.rec.err.clone())
                    active.remove(slot)
                    used -= slot.nbytes
                    del slot
                    continue
                with torch.cuda.stream(slot.stream):
                    slot.rec.run(1, slot.stream)
                    slot.event.record(slot.stream)
                slot.iters += 1
                slot.inflight = True
                launched = True
            if not launched:
                if pending and realtime and not active:
                    time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.01)))
                else:
                    time.sleep(idle_sleep)
        torch.cuda.synchronize(self.device)
        wall = time.perf_counter() - t0
        done = [r for r in requests if r.done is not None]
        if not done:
            return dict(scans=0, rejected=sum(r.rejected is not None for r in requests),
                        cancelled=sum(r.cancelled for r in requests), wall_s=wall, peak_active=peak_active,
                        peak_bytes=peak_used)
        lat = np.array([r.done - r.arrival for r in done])
        span = max(r.done for r in done) - min(r.arrival for r in done)
        return dict(scans=len(done), rejected=sum(r.rejected is not None for r in requests),
                    cancelled=sum(r.cancelled for r in requests), wall_s=wall, span_s=span,
                    scans_per_s=len(done) / span, evals_per_s=sum(r.evals for r in done) / span,
                    p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                    mean_s=float(lat.mean()), peak_active=peak_active, peak_bytes=peak_used)


def poisson_arrivals(n, rate, seed):
    """Arrival times of a Poisson process of the given rate (per second)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n)) - 0.0
