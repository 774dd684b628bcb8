"""Continuous-batching server for freezing simulations.

Requests -- a lattice size and the paper's dimensionless parameters -- arrive
over time.  Every admitted simulation stays resident on the GPU; all of them
advance together, one batched launch per time step (``lbm_batch_step``),
in chunks of ``chunk`` steps.  After each chunk the FP64 observables of every
member are reduced on the GPU; a member whose frozen fraction has reached
the target is retired (its device memory freed) and waiting requests are
admitted as soon as the device-memory budget has room for them, so requests
that arrive while others run join the running batch at the next chunk.

Every member advances by whole chunks from its own admission, so its
observables are taken at the same step counts as when it runs alone with the
same cadence: in FP64 the results are identical alone and in the mix.

The host works one chunk behind the GPU: a tick enqueues the next chunk
(and the copy of every member's observables into page-locked host memory)
before it reads the observables of the chunk before, so the GPU is never
idle while the host decides retirements and admissions.  A member that
turns out to be finished has then run one more chunk, which is discarded;
its result is the observation that finished it, and its memory is freed
once that extra chunk has completed.

Scheduling is host logic only; all arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, List, Optional

from . import lbm

STORAGE_BYTES = {lbm.FP64: 8, lbm.FP32: 4, lbm.FP16S: 2}


def footprint_bytes(params: dict) -> int:
    """Device bytes of one instance: ONE population copy (9 f planes and 23
    h, g, l planes, streamed in place), two copies of the 7 auxiliary planes,
    sigma, the halo records (16 bytes per cell, 32 in FP64) and the
    reduction workspace, rows padded to 32 elements."""
    nx, ny, prec = int(params["nx"]), int(params["ny"]), int(params["precision"])
    pitch = (nx + 31) // 32 * 32
    plane = pitch * ny
    sb = STORAGE_BYTES[prec]
    fb = 8 if prec == lbm.FP64 else 4        # half storage keeps f in single precision
    ab = 8 if prec == lbm.FP64 else 4        # auxiliary and arithmetic type
    rec = 32 if prec == lbm.FP64 else 16
    blocks = ((nx + 31) // 32) * ((ny + 7) // 8)
    ws = blocks * 7 * 8 + (3 * ny + 8) * 8 + nx * 8 + 4096
    return (9 * fb + 23 * sb) * plane + 2 * 7 * plane * ab + plane * ab + rec * plane + ws


@dataclasses.dataclass
class Request:
    id: int
    arrival: float                  # seconds after the server starts
    params: dict
    R: float
    xc: float
    yc: float
    presolve: int = 0
    psi: Optional[object] = None    # an initial order-parameter field (ny x nx) instead of the cap


def _init(sim, req: "Request"):
    if req.psi is not None:
        sim.init_psi(req.psi, req.presolve)
    else:
        sim.init_droplet(req.R, req.xc, req.yc, req.presolve)


@dataclasses.dataclass
class Result:
    id: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    t_fre: int
    frozen: bool
    obs: dict

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """Admit, batch, observe and retire freezing simulations on one GPU."""

    def __init__(self, budget_bytes: int, stream=None, chunk: int = 200, frozen_target: float = 0.99,
                 max_steps: int = 2_000_000, tile_rows: int = 4,
                 clock: Callable[[], float] = time.perf_counter):
        self.budget = int(budget_bytes)
        self.stream = stream
        self.chunk = int(chunk)
        self.target = float(frozen_target)
        self.max_steps = int(max_steps)
        self.tile_rows = int(tile_rows)
        self.clock = clock
        self.pending: List[Request] = []
        self.active = []                # (request, simulation, admitted time, bytes)
        self.results: List[Result] = []
        self.used = 0
        self.lattice_updates = 0
        self.gpu_busy_s = 0.0           # device time of the chunks (events on the stream)
        self._batch = None
        self._members = None
        self._t0 = None
        self._inflight = None           # (members, events, host buffers) of the chunk on the GPU
        self._retiring = []             # (simulation, bytes) to free once the in-flight chunk is done
        self._old_batches = []          # batches whose launches may still be in flight

    # -- time ------------------------------------------------------------
    def now(self) -> float:
        return self.clock() - self._t0

    # -- queue -----------------------------------------------------------
    def submit(self, req: Request):
        fp = footprint_bytes(req.params)
        if fp > self.budget:
            raise ValueError(f"request {req.id} needs {fp} bytes, more than the whole budget")
        self.pending.append(req)
        self.pending.sort(key=lambda r: r.arrival)

    def _admit(self, now: float):
        admitted = False
        while self.pending and self.pending[0].arrival <= now:
            req = self.pending[0]
            fp = footprint_bytes(req.params)
            if self.used + fp > self.budget:
                break                   # first come, first served: wait for memory
            self.pending.pop(0)
            sim = lbm.Simulation(req.params, self.stream)
            _init(sim, req)
            self.active.append((req, sim, now, fp))
            self.used += fp
            admitted = True
        return admitted

    # -- one chunk of work ------------------------------------------------
    def tick(self) -> int:
        """Admit what has arrived, enqueue one chunk for every resident
        member with its observables, then read the observables of the
        chunk before and retire the finished members.  Returns members
        retired."""
        if self._t0 is None:
            self._t0 = self.clock()
        changed = self._admit(self.now())
        launched = None
        if self.active:
            sims = [s for _, s, _, _ in self.active]
            if changed or self._batch is None or self._members != [id(s) for s in sims]:
                if self._batch is not None:
                    self._old_batches.append(self._batch)
                self._batch = lbm.Batch(sims, self.stream, tile_rows=self.tile_rows)
                self._members = [id(s) for s in sims]
            launched = self._enqueue(list(self.active))
        retired = self._collect()
        self._inflight = launched
        return retired

    def _enqueue(self, members):
        """One chunk of the current batch and every member's observables,
        bracketed by two events; the observables land in page-locked host
        memory (or are fetched synchronously without torch)."""
        ev = _events(self.stream)
        bufs = _pinned(len(members)) if ev else None
        if ev:
            ev[0].record(ev[2])
        self._batch.step(self.chunk)
        for j, (_, sim, _, _) in enumerate(members):
            if bufs is not None:
                sim.observables_to_host(bufs.data_ptr() + j * _OBS_BYTES)
            else:
                sim.observables_async()
        if ev:
            ev[1].record(ev[2])
        return members, ev, bufs

    def _collect(self) -> int:
        """Wait for the chunk before, free what retired before it, read its
        observations and retire the finished members."""
        if self._inflight is None:
            return 0
        members, ev, bufs = self._inflight
        self._inflight = None
        if ev:
            ev[1].synchronize()
            self.gpu_busy_s += ev[0].elapsed_time(ev[1]) / 1e3
        for sim, fp in self._retiring:      # their last chunk is the one just finished
            sim.close()
            self.used -= fp
        self._retiring = []
        for b in self._old_batches:
            b.close()
        self._old_batches = []
        active_ids = {id(e[1]) for e in self.active}
        retired = 0
        for j, (req, sim, adm, fp) in enumerate(members):
            if id(sim) not in active_ids:
                continue                    # retired at the chunk before: this chunk is discarded
            self.lattice_updates += self.chunk * sim.nx * sim.ny    # work that counts
            if bufs is not None:
                o = lbm.Obs.from_address(bufs.data_ptr() + j * _OBS_BYTES).as_dict()
            else:
                o = sim.observables_fetch()
            done = o["t_fre"] >= 0 or o["frozen_fraction"] >= self.target
            if done or o["step"] >= self.max_steps or o["status"] != 0:
                self.results.append(Result(req.id, req.arrival, adm, self.now(), o["step"], o["t_fre"],
                                           done and o["status"] == 0, o))
                # the chunk enqueued after this one may still use its memory
                self._retiring.append((sim, fp))
                retired += 1
        if retired:
            gone = {id(sim) for sim, _ in self._retiring}
            self.active = [e for e in self.active if id(e[1]) not in gone]
        return retired

    def run(self, requests: Optional[List[Request]] = None, idle_sleep: float = 1e-3) -> List[Result]:
        """Serve until every submitted request has finished."""
        for r in requests or []:
            self.submit(r)
        self._t0 = self.clock()
        while self.pending or self.active or self._inflight is not None:
            if (not self.active and self._inflight is None and self.pending
                    and self.pending[0].arrival > self.now()):
                time.sleep(min(idle_sleep, self.pending[0].arrival - self.now()))
                continue
            self.tick()
        self.drain()
        return sorted(self.results, key=lambda r: r.id)

    def drain(self):
        """Wait for the GPU and free everything retired."""
        while self._inflight is not None:
            self._collect()
        # nothing was enqueued after the chunk just collected
        for sim, fp in self._retiring:
            sim.close()
            self.used -= fp
        self._retiring = []
        for b in self._old_batches:
            b.close()
        self._old_batches = []
        if self._batch is not None and not self.active:
            self._batch.close()
            self._batch = None


_OBS_BYTES = 0


def _pinned(n: int):
    """Page-locked host memory for n lbm_obs records (None without torch)."""
    global _OBS_BYTES
    try:
        import ctypes
        import torch
        _OBS_BYTES = ctypes.sizeof(lbm.Obs)
        return torch.empty(max(1, n) * _OBS_BYTES, dtype=torch.uint8, pin_memory=True)
    except Exception:
        return None


def _events(stream):
    """Two timing events and the torch stream to record them on (None
    without torch or CUDA)."""
    try:
        import torch
        if not torch.cuda.is_available():
            return None
        if stream is None:
            st = torch.cuda.current_stream()
        elif isinstance(stream, torch.cuda.Stream):
            st = stream
        else:
            st = torch.cuda.ExternalStream(int(getattr(stream, "cuda_stream", stream)))
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True), st
    except Exception:
        return None


def run_alone(req: Request, chunk: int, frozen_target: float = 0.99, max_steps: int = 2_000_000, stream=None):
    """The same request on its own, observed with the same cadence."""
    sim = lbm.Simulation(req.params, stream)
    _init(sim, req)
    while True:
        sim.step(chunk)
        o = sim.observables()
        if o["t_fre"] >= 0 or o["frozen_fraction"] >= frozen_target or sim.t >= max_steps or o["status"] != 0:
            sim.close()
            return o
