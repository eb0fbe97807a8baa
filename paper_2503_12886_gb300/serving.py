"""Continuous-batching server for forward-only animation renders of resident avatars.

Every avatar's base Gaussians and blendshapes stay on the device. Requests (avatar, weights psi,
camera, resolution) arrive over time; the loop
  - admits a request when its memory (output image, per-pixel state, its share of the splat
    records and tile pairs) fits the HBM budget, rejecting requests that can never fit or that
    name an unknown avatar;
  - whenever one of its launch slots (a CUDA stream with its own workspace and output buffers)
    is free, packs every admitted request (up to max_frames) into one uneven batch and launches
    preprocess -> bin/sort -> compositing on that slot, so requests that arrive while earlier
    batches run are batched together and their work overlaps on the device;
  - polls completion events, records arrival-to-completion latency and frees the memory.
The per-frame path (one request per launch, a host sync per request) is the comparison.
"""
from __future__ import annotations

import collections
import contextlib
import ctypes as C
import gc
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api, synth
from .rasterizer import DeviceModel, Renderer


@dataclass
class Request:
    rid: int
    avatar: int
    width: int
    height: int
    psi: np.ndarray          # float32 [k]
    fparams: np.ndarray      # float32 [20]
    t_arrival: float = 0.0
    t_done: float = -1.0
    status: str = "pending"  # pending, admitted, running, done, rejected
    error: str = ""
    image: np.ndarray | None = None


@contextlib.contextmanager
def _no_gc_pauses():
    """The request loops run with Python's cyclic garbage collector off (one collection and a
    freeze of what exists before the loop): a full collection stops the host thread, and with it
    every queued request, for tens of milliseconds (measured: single 31-36 ms stalls of both
    loops at 2,000 requests/s). Reference counting still frees the loop's own objects."""
    was = gc.isenabled()
    gc.collect()
    gc.freeze()
    gc.disable()
    try:
        yield
    finally:
        gc.unfreeze()
        if was:
            gc.enable()


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    ws: torch.Tensor
    img: torch.Tensor
    T: torch.Tensor
    n: torch.Tensor
    psi_h: torch.Tensor
    fp_h: torch.Tensor
    psi_d: torch.Tensor
    fp_d: torch.Tensor
    cnt_h: torch.Tensor
    event: torch.cuda.Event
    reqs: list = field(default_factory=list)
    busy: bool = False
    keep: tuple = ()


class Server:
    def __init__(self, avatars: list[synth.Model], device: int = 0, hbm_budget: float = 40e9,
                 max_frames: int = 32, slots: int = 2, max_res: int = 1024, tile=(16, 16),
                 smem_batch: int = 64, pairs_per_gaussian: float | None = None,
                 headroom: float = 1.3):
        if any(m.binding is not None for m in avatars):
            raise ValueError("the server renders world-space avatars; a tangent-space avatar "
                             "needs a deformed mesh per request")
        self.device = device
        dev = f"cuda:{device}"
        self.r = Renderer(device)
        self.models = [DeviceModel(m.n, m.k, m.mask, torch.from_numpy(m.g0).to(dev),
                                   torch.from_numpy(m.dg).to(dev)) for m in avatars]
        self.k_stride = max(m.k for m in avatars)
        self.budget = hbm_budget
        self.used = 0.0
        self.max_frames = max_frames
        self.tile, self.smem_batch = tile, smem_batch
        max_n = max(m.n_pad for m in self.models)
        max_pix = max_frames * max_res * max_res
        self.max_res = max_res
        self.regrowths = 0
        # (Gaussian, tile) pairs per Gaussian at the largest resolution, measured once at start-up
        # (every avatar from the corners of the request camera range), times the headroom: the
        # slot workspaces then hold a batch of max_frames such frames of the largest avatar, so
        # that no batch overflows and nothing is allocated inside the request loop
        self.ppg = (pairs_per_gaussian if pairs_per_gaussian is not None
                    else headroom * self._measure_pairs_per_gaussian(max_res))
        frames = [(0, max_res, max_res)] * max_frames
        probe = self._struct([0] * 0, frames, None, None, models=[self.models[int(np.argmax(
            [m.n_pad for m in self.models]))]])
        pairs = int(max_frames * max_n * self.ppg) + 4096
        ws_bytes = api.rgba_workspace_size(probe, pairs)
        self.pair_capacity = pairs
        # the slots' device memory (workspaces, outputs, weights and cameras) is held for the
        # server's life and counts against the HBM budget; requests are admitted in what is left
        self.fixed_bytes = float(slots * (ws_bytes + 4 * (5 * max_pix + max_frames * (self.k_stride
                                                                                     + api.RGBA_FP_STRIDE))))
        if self.fixed_bytes >= self.budget:
            self.r.close()
            raise ValueError(f"the slots alone need {self.fixed_bytes / 1e9:.2f} GB, more than the "
                             f"{self.budget / 1e9:.2f} GB budget")
        self.slots = []
        for _ in range(slots):
            self.slots.append(_Slot(
                stream=torch.cuda.Stream(device=dev),
                ws=torch.empty(ws_bytes, dtype=torch.uint8, device=dev),
                img=torch.empty(3 * max_pix, dtype=torch.float32, device=dev),
                T=torch.empty(max_pix, dtype=torch.float32, device=dev),
                n=torch.empty(max_pix, dtype=torch.int32, device=dev),
                psi_h=torch.zeros(max_frames, self.k_stride).pin_memory(),
                fp_h=torch.zeros(max_frames, api.RGBA_FP_STRIDE).pin_memory(),
                psi_d=torch.zeros(max_frames, self.k_stride, device=dev),
                fp_d=torch.zeros(max_frames, api.RGBA_FP_STRIDE, device=dev),
                cnt_h=torch.zeros(24, dtype=torch.uint8).pin_memory(),
                event=torch.cuda.Event()))
        self.lat: list[float] = []
        self.frames_done = 0

    def _measure_pairs_per_gaussian(self, res: int) -> float:
        """The largest (Gaussian, tile) pair count per Gaussian over every avatar rendered at
        res x res from five cameras (straight on and the four corners of the +-20 deg yaw /
        pitch range), zero weights."""
        from .rasterizer import DeviceBatch
        worst = 0.0
        for a, m in enumerate(self.models):
            cams = [(0.0, 0.0)] + [(sy * np.radians(20.0), sp * np.radians(20.0))
                                   for sy in (-1, 1) for sp in (-1, 1)]
            fp = np.stack([synth.camera_params(res, res, y, p) for y, p in cams]).astype(np.float32)
            b = synth.Batch([], [synth.Frame(0, res, res)] * len(cams),
                            np.zeros((len(cams), self.k_stride), np.float32), fp, self.k_stride)
            db = DeviceBatch(b, self.models[0].g0.device, tile=self.tile,
                             smem_batch=self.smem_batch, grads=False, models=[m])
            self.r.forward(db)
            worst = max(worst, self.r.counters(db)["pairs"] / (len(cams) * m.n))
        self.r.ws = None  # the probe's workspace goes back to the caching allocator
        return worst

    # -- helpers ---------------------------------------------------------------------------
    def _struct(self, order, frames, psi_ptr, fp_ptr, models=None):
        models = models if models is not None else self.models
        ms = (api.RgbaModel * len(models))()
        for i, m in enumerate(models):
            ms[i] = api.RgbaModel(m.n, m.n_pad, m.k, m.mask, m.g0.data_ptr(), m.dg.data_ptr(),
                                  None, None)
        fs = (api.RgbaFrame * max(1, len(frames)))()
        for i, (mi, w, h) in enumerate(frames):
            fs[i] = api.RgbaFrame(mi, w, h)
        b = api.RgbaBatch()
        b.n_models, b.models = len(models), C.cast(ms, C.POINTER(api.RgbaModel))
        b.n_frames, b.frames = len(frames), C.cast(fs, C.POINTER(api.RgbaFrame))
        b.k_stride = self.k_stride
        b.psi = psi_ptr if psi_ptr is not None else 16
        b.fparams = fp_ptr if fp_ptr is not None else 16
        b.grad_psi = None
        b.tile_w, b.tile_h = self.tile
        b.smem_batch = self.smem_batch
        b._keep = (ms, fs)
        return b

    def request_bytes(self, q: Request) -> float:
        m = self.models[q.avatar]
        hw = q.width * q.height
        return 3 * hw * 4 + 8 * hw + 104 * m.n_pad + 12 * self.ppg * m.n

    def _launch(self, slot: _Slot, reqs: list[Request]):
        avatars = sorted({q.avatar for q in reqs})
        remap = {a: i for i, a in enumerate(avatars)}
        frames = [(remap[q.avatar], q.width, q.height) for q in reqs]
        for j, q in enumerate(reqs):
            slot.psi_h[j, :len(q.psi)] = torch.from_numpy(q.psi)
            slot.fp_h[j] = torch.from_numpy(q.fparams)
            q.status = "running"
        b = self._struct(None, frames, slot.psi_d.data_ptr(), slot.fp_d.data_ptr(),
                         models=[self.models[a] for a in avatars])
        with torch.cuda.stream(slot.stream):
            slot.psi_d.copy_(slot.psi_h, non_blocking=True)
            slot.fp_d.copy_(slot.fp_h, non_blocking=True)
            s = slot.stream.cuda_stream
            ws = slot.ws
            api.rgba_preprocess(self.r.ctx, b, ws.data_ptr(), ws.numel(), s)
            api.rgba_bin_sort(self.r.ctx, b, ws.data_ptr(), ws.numel(), s)
            api.rgba_render_fwd(self.r.ctx, b, ws.data_ptr(), ws.numel(), slot.img.data_ptr(),
                                slot.T.data_ptr(), slot.n.data_ptr(), s)
            lay = api.rgba_workspace_layout(b, ws.numel())
            slot.cnt_h.copy_(ws[lay.counters: lay.counters + 24], non_blocking=True)
            slot.event.record(slot.stream)
        slot.reqs, slot.busy, slot.keep = reqs, True, (b, frames)

    def _finish(self, slot: _Slot, now: float, keep_images: bool):
        u = slot.cnt_h.numpy()[:16].view(np.uint32)
        if u[1]:  # overflow (not expected: the capacity is sized at start-up): grow, render again
            b, _ = slot.keep
            need = api.rgba_workspace_size(b, int(u[0] * 1.25) + 4096)
            self.fixed_bytes += need - slot.ws.numel()
            slot.ws = torch.empty(need, dtype=torch.uint8, device=slot.ws.device)
            self.regrowths += 1
            self._launch(slot, slot.reqs)
            return
        off = 0
        for q in slot.reqs:
            hw = q.width * q.height
            if keep_images:
                q.image = slot.img[3 * off: 3 * (off + hw)].view(3, q.height, q.width).cpu().numpy()
            off += hw
            q.t_done = now
            q.status = "done"
            self.lat.append(q.t_done - q.t_arrival)
            self.used -= self.request_bytes(q)
            self.frames_done += 1
        slot.reqs, slot.busy = [], False

    # -- the loop ---------------------------------------------------------------------------
    def run(self, requests: list[Request], realtime: bool = True, keep_images: bool = False,
            timeout_s: float = 600.0) -> dict:
        """Serves the requests (sorted by t_arrival). With realtime, request i becomes visible
        at t0 + t_arrival; otherwise all are visible at once. Returns throughput and latency."""
        with _no_gc_pauses():
            return self._run(requests, realtime, keep_images, timeout_s)

    def _run(self, requests, realtime, keep_images, timeout_s) -> dict:
        reqs = sorted(requests, key=lambda q: q.t_arrival)
        arrivals = collections.deque(reqs)
        waiting: collections.deque = collections.deque()  # arrived, waiting for budget
        admitted: collections.deque = collections.deque()
        self.lat, self.frames_done = [], 0
        regrow0 = self.regrowths
        t0 = time.perf_counter()
        n_total = len(reqs)
        finished = 0
        batches = 0
        while finished < n_total:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise TimeoutError("serving loop exceeded its time limit")
            while arrivals and (not realtime or arrivals[0].t_arrival <= now):
                q = arrivals.popleft()
                if not realtime:
                    q.t_arrival = now
                if not (0 <= q.avatar < len(self.models)):
                    q.status, q.error = "rejected", "unknown avatar"
                    finished += 1
                    continue
                if self.request_bytes(q) > self.budget - self.fixed_bytes:
                    q.status, q.error = "rejected", "request larger than the HBM budget"
                    finished += 1
                    continue
                if not (0 < q.width <= self.max_res and 0 < q.height <= self.max_res):
                    q.status, q.error = "rejected", "resolution above the server's maximum"
                    finished += 1
                    continue
                waiting.append(q)
            while waiting and self.used + self.request_bytes(waiting[0]) <= self.budget - self.fixed_bytes:
                q = waiting.popleft()
                self.used += self.request_bytes(q)
                q.status = "admitted"
                admitted.append(q)
            for slot in self.slots:
                if slot.busy and slot.event.query():
                    before = self.frames_done
                    self._finish(slot, time.perf_counter() - t0, keep_images)
                    finished += self.frames_done - before
            for slot in self.slots:
                if not slot.busy and admitted:
                    batch = [admitted.popleft() for _ in range(min(self.max_frames, len(admitted)))]
                    self._launch(slot, batch)
                    batches += 1
            if not any(s.busy for s in self.slots) and not admitted and arrivals and realtime:
                dt = arrivals[0].t_arrival - (time.perf_counter() - t0)
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
        wall = time.perf_counter() - t0
        lat = np.sort(np.array(self.lat)) if self.lat else np.zeros(1)
        return {"requests": n_total, "served": self.frames_done, "batches": batches,
                "wall_s": wall, "frames_per_s": self.frames_done / wall,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "max_ms": 1e3 * float(lat.max()), "regrowths": self.regrowths - regrow0}

    def run_per_frame(self, requests: list[Request], realtime: bool = True) -> dict:
        """The per-frame path: each request rendered alone as soon as the previous one finished,
        with a host synchronisation per request."""
        with _no_gc_pauses():
            return self._run_per_frame(requests, realtime)

    def _run_per_frame(self, requests, realtime) -> dict:
        reqs = sorted(requests, key=lambda q: q.t_arrival)
        slot = self.slots[0]
        lat = []
        t0 = time.perf_counter()
        for q in reqs:
            now = time.perf_counter() - t0
            if realtime and q.t_arrival > now:
                time.sleep(max(0.0, q.t_arrival - now - 1e-4))
                while time.perf_counter() - t0 < q.t_arrival:
                    pass
            if not realtime:
                q.t_arrival = time.perf_counter() - t0
            self._launch(slot, [q])
            slot.event.synchronize()
            self._finish(slot, time.perf_counter() - t0, False)
            lat.append(q.t_done - q.t_arrival)
        wall = time.perf_counter() - t0
        lat = np.sort(np.array(lat))
        return {"requests": len(reqs), "wall_s": wall, "frames_per_s": len(reqs) / wall,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "max_ms": 1e3 * float(lat.max())}

    def close(self):
        self.r.close()


def requests_from_trace(trace, avatars: list[synth.Model], seed: int = 5000) -> list[Request]:
    """Turns synth.serving_requests tuples into Requests with cameras (random yaw/pitch within
    +-20 deg and a random background per request)."""
    st = synth.Stream(seed, 23)
    out = []
    for rid, (t, a, res, psi) in enumerate(trace):
        yp = (st.uniform(2) * 2 - 1) * np.radians(20.0)
        bg = tuple(st.uniform(3))
        fp = synth.camera_params(res, res, float(yp[0]), float(yp[1]), bg)
        out.append(Request(rid, a, res, res, psi[:avatars[a].k].astype(np.float32), fp,
                           t_arrival=t))
    return out
