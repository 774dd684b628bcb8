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
        """Admit what has arrived, advance every resident member by one chunk,
        observe them and retire the frozen ones.  Returns members retired."""
        if self._t0 is None:
            self._t0 = self.clock()
        changed = self._admit(self.now())
        if not self.active:
            return 0
        sims = [s for _, s, _, _ in self.active]
        if changed or self._batch is None or self._members != [id(s) for s in sims]:
            if self._batch is not None:
                self._batch.close()
            self._batch = lbm.Batch(sims, self.stream, tile_rows=self.tile_rows)
            self._members = [id(s) for s in sims]
        ev = _events(self.stream)
        if ev:
            ev[0].record(ev[2])
        self._batch.step(self.chunk)
        self.lattice_updates += self.chunk * sum(s.nx * s.ny for s in sims)
        for s in sims:
            s.observables_async()
        if ev:
            ev[1].record(ev[2])
        keep, retired = [], 0
        for entry in self.active:
            req, sim, adm, fp = entry
            o = sim.observables_fetch()
            done = o["t_fre"] >= 0 or o["frozen_fraction"] >= self.target
            if done or sim.t >= self.max_steps or o["status"] != 0:
                self.results.append(Result(req.id, req.arrival, adm, self.now(), sim.t, o["t_fre"],
                                           done and o["status"] == 0, o))
                sim.close()
                self.used -= fp
                retired += 1
            else:
                keep.append(entry)
        if ev:
            self.gpu_busy_s += ev[0].elapsed_time(ev[1]) / 1e3    # the fetches synchronised
        if retired:
            self.active = keep
            self._batch.close()
            self._batch = None
        return retired

    def run(self, requests: Optional[List[Request]] = None, idle_sleep: float = 1e-3) -> List[Result]:
        """Serve until every submitted request has finished."""
        for r in requests or []:
            self.submit(r)
        self._t0 = self.clock()
        while self.pending or self.active:
            if not self.active and self.pending and self.pending[0].arrival > self.now():
                time.sleep(min(idle_sleep, self.pending[0].arrival - self.now()))
                continue
            self.tick()
        if self._batch is not None:
            self._batch.close()
            self._batch = None
        return sorted(self.results, key=lambda r: r.id)


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
