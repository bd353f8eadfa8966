"""Continuous-batching request loop over one eulbfs solver.

Solidification cases arrive over time (a Poisson trace).  The loop keeps
every admitted case's state resident on the GPU as a domain of one solver,
so all running cases advance together in the same stage launches:

  admit  -- between step chunks, queued cases whose arrival time has passed
            are added in arrival order while they fit the device-memory
            budget (eulbfs_add_domain returns EBUSY otherwise; the case waits);
  step   -- one eulbfs_step(chunk) advances every running case (each stops
            at its own step count, its slot leaves the work list);
  retire -- finished cases have their fields copied to the host and their
            memory released; their time to solution is completion - arrival.
            A case whose own state became NaN or Inf (its per-domain flag,
            read after every chunk) is retired with that error at once.

Results do not depend on which other cases share the launches (the per-cell
arithmetic is independent of the batch), which the tests check bit for bit.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import eulbfs


@dataclass
class Outcome:
    rid: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    cells: int
    steps: int
    fields: Optional[Dict[str, np.ndarray]] = None
    diag: Optional[dict] = None
    error: Optional[str] = None

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


@dataclass
class ServeReport:
    outcomes: List[Outcome]
    wall_s: float
    cell_steps: int
    max_resident: int
    budget_bytes: int
    rejected_busy: int = 0
    extra: dict = field(default_factory=dict)

    def latency_percentiles(self, q=(50, 99)) -> Dict[str, float]:
        lat = np.array([o.latency_s for o in self.outcomes if o.error is None])
        return {f"p{k}_s": float(np.percentile(lat, k)) for k in q} if lat.size else {}

    def summary(self) -> dict:
        done = [o for o in self.outcomes if o.error is None]
        out = {"requests": len(self.outcomes), "completed": len(done),
               "failed": len(self.outcomes) - len(done), "wall_s": self.wall_s,
               "gcups": self.cell_steps / self.wall_s / 1e9 if self.wall_s > 0 else 0.0,
               "max_resident": self.max_resident, "budget_bytes": self.budget_bytes,
               "admissions_deferred": self.rejected_busy}
        out.update(self.latency_percentiles())
        if done:
            out["mean_queue_s"] = float(np.mean([o.admitted_s - o.arrival_s for o in done]))
        out.update(self.extra)
        return out


def serve(requests, precision: int = eulbfs.FP32C, budget_bytes: int = 0, chunk: int = 16,
          keep_fields: bool = False, stream: Optional[int] = None, realtime: bool = True,
          clock=time.perf_counter, resident_cap: int = 0) -> ServeReport:
    """Serve `requests` (workloads.Request: rid, arrival_s, case, steps).

    realtime=True replays arrivals against the wall clock (arrival_s after the
    start); realtime=False admits every case as soon as it fits (a closed loop,
    for tests).  resident_cap > 0 caps the cases on the device at once (1:
    one solve after another, no batching).  A case whose state becomes non-finite is retired with that
    error after the chunk in which it diverged and does not affect the others.
    A CUDA error from a launch is sticky for the whole context, so it retires
    every running case with that error."""
    reqs = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
    solver = eulbfs.Solver([], precision=precision, stream=stream)
    if budget_bytes:
        solver.set_memory_budget(budget_bytes)
    lib = eulbfs.lib()
    pending = list(reqs)
    running: Dict[int, tuple] = {}      # slot -> (request, admitted time)
    outcomes: List[Outcome] = []
    cell_steps = 0
    max_resident = 0
    deferred = 0
    t0 = clock()
    now = lambda: clock() - t0  # noqa: E731
    try:
        while pending or running:
            # admit in arrival order while the budget allows
            while pending and (not realtime or pending[0].arrival_s <= now()) and \
                    (resident_cap <= 0 or len(running) < resident_cap):
                r = pending[0]
                need = lib.eulbfs_domain_bytes(r.case.nx, r.case.ny, precision)
                if budget_bytes and need > budget_bytes:
                    pending.pop(0)
                    outcomes.append(Outcome(r.rid, r.arrival_s, now(), now(), r.case.cells, r.steps,
                                            error="case larger than the memory budget"))
                    continue
                try:
                    slot = solver.add(r.case, max_steps=r.steps)
                except eulbfs.EulbfsError as e:
                    if e.code == eulbfs.EBUSY:
                        deferred += 1
                        break
                    pending.pop(0)
                    outcomes.append(Outcome(r.rid, r.arrival_s, now(), now(), r.case.cells, r.steps, error=str(e)))
                    continue
                pending.pop(0)
                running[slot] = (r, now() if realtime else max(now(), 0.0))
            max_resident = max(max_resident, len(running))
            if not running:
                if pending and realtime:
                    time.sleep(max(0.0, min(pending[0].arrival_s - now(), 0.05)))
                continue
            step_error = None
            diverged = set()
            try:
                solver.step(chunk)
                diverged = set(solver.nonfinite_slots())     # one flag per case; synchronises
            except eulbfs.EulbfsError as e:
                step_error = str(e)
            # retire finished and diverged cases
            for slot in list(running):
                r, t_adm = running[slot]
                done, left = solver.progress(slot)
                if left != 0 and step_error is None and slot not in diverged:
                    continue
                err = None
                fields = diag = None
                try:
                    if keep_fields:
                        fields = solver.fields(slot)
                    diag = solver.diag(slot)
                except eulbfs.EulbfsError as e:
                    err = str(e)
                if slot in diverged:
                    err = err or "ENONFINITE: the case's state became NaN or Inf"
                if step_error is not None and left != 0:
                    err = err or step_error
                cell_steps += r.case.cells * done
                outcomes.append(Outcome(r.rid, r.arrival_s, t_adm, now(), r.case.cells, done, fields, diag, err))
                solver.remove(slot)
                del running[slot]
    finally:
        wall = now()
        solver.close()
    outcomes.sort(key=lambda o: o.rid)
    return ServeReport(outcomes, wall, cell_steps, max_resident, budget_bytes, deferred)
