"""Continuous-batching request loop for pressurised-crack solves.

Host scheduling only: every numeric step runs in libpff through the batch ABI.  Each request is a
fracture instance (mesh, material, crack layout) with a pressure ramp over load steps; each load
step is solved by the active-set Newton iteration (Algorithm 1) with the pressure p_n = n/N p.

Every tick:
  1. admit waiting requests in arrival order while the device-memory budget allows
     (pff_hierarchy_bytes + the instance's state vectors) and the batch is not full;
  2. run one batched Newton step over all active instances (pff_batch_newton_step);
  3. instances whose load step converged (active set unchanged and ||R~|| <= eps_as, Algorithm 1)
     or reached the Newton cap advance to the next load step (phi_old := phi, new pressure) or
     retire, freeing their memory for waiting requests.
Requests that arrive while others are on the GPU join at the next tick, so their work overlaps
on the device with the instances already running.  Hierarchies, active sets and the Krylov
workspace stay on the device across Newton and load steps.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as W


@dataclass
class Request:
    rid: int
    workload: W.Workload
    load_steps: int = 1
    arrival: float = 0.0
    max_newton: int = 12


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float = 0.0
    finished: float = 0.0
    newton_steps: list = field(default_factory=list)     # per load step
    gmres_iterations: list = field(default_factory=list)  # per Newton step
    load_step_latency: list = field(default_factory=list)
    solve_latency: list = field(default_factory=list)     # per Newton step (linear solve)
    converged: list = field(default_factory=list)         # per load step
    U: np.ndarray | None = None
    cancelled: bool = False


class PffBackend:
    """Real backend: hierarchies on one CUDA stream, batched Newton steps."""

    def __init__(self, device="cuda:0", restart=30):
        import torch
        from . import pff
        self.torch, self.pff = torch, pff
        self.dev = torch.device(device)
        self.stream = torch.cuda.Stream(device=self.dev)
        self.restart = restart
        self._batch, self._members = None, []
        self.batches_built = 0          # ticks whose batch membership changed (device state rebuilt)

    def mesh(self, w):
        return self.pff.make_mesh(w.dim, w.deg, w.n_cells, w.n_levels, w.lo, w.hi,
                                  dirichlet_faces=w.dirichlet_faces, cell_mask=w.cell_mask(),
                                  dirichlet_mask=w.dirichlet_mask())

    def bytes_for(self, w) -> int:
        return self.pff.hierarchy_bytes(self.mesh(w), self.restart) + 3 * w.n_dofs * 8

    def params(self, w, pressure):
        return self.pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, pressure=pressure,
                                       mg_precision=32, seed=w.seed)

    def create(self, w, pressure):
        h = self.pff.create_hierarchy(self.mesh(w), self.params(w, pressure), self.stream)
        U0, po, pt = W.initial_state(w)
        with self.torch.cuda.stream(self.stream):
            U = self.torch.from_numpy(U0).to(self.dev)
            phi_old = self.torch.from_numpy(po).to(self.dev)
        self.stream.synchronize()
        return {"h": h, "U": U, "phi_old": phi_old, "w": w}

    def start_load_step(self, inst, pressure, frac=1.0):
        """Load step at the fraction 'frac' of the request's ramp: phi_old := phi, the pressure p_n and, for
        displacement-driven instances, the prescribed boundary displacements of this step."""
        w = inst["w"]
        nn = w.n_nodes
        ud = w.u_dirichlet(frac)
        with self.torch.cuda.stream(self.stream):
            inst["phi_old"].copy_(inst["U"][w.dim * nn:])
            inst["ud"] = self.torch.from_numpy(ud).to(self.dev) if ud is not None else None
        self.pff.set_params(inst["h"], self.params(w, pressure))
        self.pff.set_state(inst["h"], inst["U"], inst["phi_old"], inst["phi_old"], inst["ud"])

    def newton(self, insts):
        """One batched Newton step.  The batch (descriptor tables, device FGMRES state, captured Arnoldi
        graph, tuned kernels) lives across ticks: instances that joined are submitted to it and those
        that left are retired (pff_batch_submit / pff_batch_retire), and the library rebuilds its device
        state only when the membership changed."""
        if self._batch is None:
            self._batch = self.pff.batch_create([], self.restart)
            self._members = []
        want = {i["h"].value for i in insts}
        changed = False
        for idx in reversed(range(len(self._members))):
            if self._members[idx] not in want:
                self.pff.batch_retire(self._batch, idx)
                self._members.pop(idx)
                changed = True
        for i in insts:
            if i["h"].value not in self._members:
                self.pff.batch_submit(self._batch, i["h"])
                self._members.append(i["h"].value)
                changed = True
        self.batches_built += changed
        order = {hv: k for k, hv in enumerate(self._members)}
        Us = [None] * len(self._members)
        for i in insts:
            Us[order[i["h"].value]] = i["U"]
        infos = self.pff.batch_newton_step(self._batch, Us, allow_noconv=True)
        return [infos[order[i["h"].value]] for i in insts]

    def release(self):
        """Destroy the batch (not its instances)."""
        if self._batch is not None:
            self.pff.batch_destroy(self._batch)
        self._batch, self._members = None, []

    def fetch(self, inst):
        self.stream.synchronize()
        return inst["U"].cpu().numpy()

    def destroy(self, inst):
        hv = inst["h"].value
        if self._batch is not None and hv in self._members:   # the batch holds the hierarchy: retire it first
            idx = self._members.index(hv)
            self.pff.batch_retire(self._batch, idx)
            self._members.pop(idx)
        self.pff.destroy_hierarchy(inst["h"])


class Server:
    def __init__(self, backend, hbm_budget: int, max_active: int = 256, clock=time.perf_counter):
        self.backend = backend
        self.budget = hbm_budget
        self.max_active = max_active
        self.clock = clock
        self.waiting: list = []
        self.active: list = []
        self.used = 0
        self.results: dict = {}
        self.ticks = 0
        self.t0 = clock()

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)
        self.results[req.rid] = Result(req.rid, arrival=req.arrival)

    def cancel(self, rid: int) -> bool:
        """Withdraw a request between ticks: a waiting request leaves the queue; an admitted one has
        its instance destroyed and its device bytes returned to the budget.  False if the request
        already finished or is unknown."""
        for i, req in enumerate(self.waiting):
            if req.rid == rid:
                self.waiting.pop(i)
                self.results[rid].cancelled = True
                return True
        for i, s in enumerate(self.active):
            if s["req"].rid == rid:
                self.backend.destroy(s["inst"])
                self.used -= s["bytes"]
                self.active.pop(i)
                self.results[rid].cancelled = True
                self.results[rid].finished = self.now()
                return True
        return False

    def _pressure(self, req, step):
        return req.workload.pressure * step / req.load_steps

    def _start(self, slot):
        req, step = slot["req"], slot["step"]
        self.backend.start_load_step(slot["inst"], self._pressure(req, step), frac=step / req.load_steps)

    def _admit(self):
        admitted = []
        while self.waiting and len(self.active) < self.max_active:
            req = self.waiting[0]
            need = self.backend.bytes_for(req.workload)
            if need > self.budget:
                raise ValueError(f"request {req.rid} needs {need} bytes, more than the whole budget")
            if self.used + need > self.budget:
                break
            self.waiting.pop(0)
            inst = self.backend.create(req.workload, self._pressure(req, 1))
            slot = {"req": req, "inst": inst, "bytes": need, "step": 1, "newton": 0, "t_step": self.now()}
            self._start(slot)
            self.active.append(slot)
            self.used += need
            self.results[req.rid].admitted = self.now()
            admitted.append(req.rid)
        return admitted

    def tick(self):
        """Admit, run one batched Newton step for every active instance, advance or retire."""
        self._admit()
        if not self.active:
            return []
        self.ticks += 1
        t0 = self.now()
        infos = self.backend.newton([s["inst"] for s in self.active])
        t1 = self.now()
        retired, keep = [], []
        for s, info in zip(self.active, infos):
            res = self.results[s["req"].rid]
            res.solve_latency.append(t1 - t0)
            res.gmres_iterations.append(info.solve.iterations)
            s["newton"] += 1
            done_step = bool(info.converged) or s["newton"] >= s["req"].max_newton
            if not done_step:
                keep.append(s)
                continue
            res.newton_steps.append(s["newton"])
            res.converged.append(bool(info.converged))
            res.load_step_latency.append(t1 - s["t_step"])
            if s["step"] < s["req"].load_steps:
                s["step"] += 1
                s["newton"] = 0
                s["t_step"] = t1
                self._start(s)
                keep.append(s)
            else:
                res.U = self.backend.fetch(s["inst"])
                res.finished = t1
                self.backend.destroy(s["inst"])
                self.used -= s["bytes"]
                retired.append(s["req"].rid)
        self.active = keep
        return retired

    def run(self, requests, realtime: bool = True, idle_sleep: float = 1e-3):
        """Serve 'requests' (sorted by arrival, seconds from start).  With realtime, requests are
        submitted when the clock reaches their arrival time; otherwise all are queued at once."""
        pending = sorted(requests, key=lambda r: r.arrival)
        while pending or self.waiting or self.active:
            while pending and (not realtime or pending[0].arrival <= self.now()):
                self.submit(pending.pop(0))
            if not self.waiting and not self.active:
                if pending:
                    time.sleep(max(0.0, min(idle_sleep, pending[0].arrival - self.now())))
                continue
            self.tick()
        if hasattr(self.backend, "release"):
            self.backend.release()
        return self.results


def summarize(results: dict, wall: float) -> dict:
    """p50/p99 latency per linear solve, per load step and per request, and solves/s."""
    solves = [x for r in results.values() for x in r.solve_latency]
    steps = [x for r in results.values() for x in r.load_step_latency]
    reqs = [r.finished - r.arrival for r in results.values() if r.finished and not r.cancelled]

    def pct(v, q):
        return float(np.percentile(v, q)) * 1e3 if v else None

    n_solves = sum(len(r.solve_latency) for r in results.values())
    return {"requests": len(results), "linear_solves": n_solves, "solves_per_s": n_solves / wall if wall > 0 else None,
            "solve_ms_p50": pct(solves, 50), "solve_ms_p99": pct(solves, 99),
            "load_step_ms_p50": pct(steps, 50), "load_step_ms_p99": pct(steps, 99),
            "request_ms_p50": pct(reqs, 50), "request_ms_p99": pct(reqs, 99)}


def poisson_requests(count: int, rate_per_s: float, sizes=(16, 24, 32), load_steps=2, seed: int = W.SEED,
                     coarsest: int = 4, lshape_every: int = 0, lshape_sizes=(16, 32, 64, 128),
                     lshape_steps: int = 20) -> list:
    """Seeded Poisson arrivals of random pressurised-crack instances (the batch recipe, 'load_steps'
    pressure steps each); with lshape_every = k every k-th request is a 3D L-shaped panel (edge n cells,
    n from lshape_sizes) loaded by a prescribed displacement ramp over 'lshape_steps' load steps."""
    rng = np.random.default_rng(seed)
    inst = W.batch_instances(count, sizes=sizes, seed=seed, coarsest=coarsest)
    t = 0.0
    out = []
    for i, w in enumerate(inst):
        t += rng.exponential(1.0 / rate_per_s)
        steps = load_steps
        if lshape_every and i % lshape_every == lshape_every - 1:
            n = int(rng.choice(lshape_sizes))
            w = W.config_3d_lshape(n, n_levels=lshape_levels(n))
            steps = lshape_steps
        out.append(Request(i, w, load_steps=steps, arrival=t))
    return out


def lshape_levels(n: int) -> int:
    """Levels of an L-shaped panel with n cells per edge (n/4 through the depth): down to 2 cells through
    the depth, at most 5 levels."""
    levels, m = 1, n // 4
    while m % 2 == 0 and m // 2 >= 1 and levels < 5 and n // (1 << levels) >= 4:
        m //= 2
        levels += 1
    return levels
