"""Benchmark of the matrix-free phase-field fracture solver on one GB300 (or N replicas).

Workload (default): 3D pressurised penny crack, [-10,10]^3, 128^3 Q1 hexahedra (8.6M DoFs),
5-level geometric multigrid, E=1, nu=0.2, Gc=1, kappa=1e-10, eps=2h, p=1e-3; synthetic seeded
state (initial crack phase field, smooth displacement), active set from Algorithm 1 step 3.

One timed step = one primal-dual active-set step (Algorithm 1) on that system: residual,
active set, restriction of state and active set to all levels, diagonals and CG eigenvalue
estimates, FGMRES to 1e-8 with the FP32 V-cycle, update.  The reported metric is the
Jacobian-apply throughput in GDoF/s: fine DoFs / mean device time of the FP64 fine-level
Jacobian applies launched inside the timed steps (CUDA events on the library's stream).
Secondary keys give the V-cycle time and the time to a 1e-8 solve with FP32-MG and FP64-MG.

--impl reference times the CPU oracle (assembled CSR Jacobian, scipy SpMV, 1 thread) on a
bounded sample of the same recipe.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Jacobian-apply GDoF/s; time-to-1e-8 solve FP32-MG vs FP64-MG; solves/s, p99"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# DRAM bytes per cell of the FP64-accurate apply k_q1_apply_cell<df64, false> from one ncu capture at
# 64^3 (157.5 MB per launch over 262,144 cells): the df64 Gauss-point data plus x, mask and y
TRAFFIC_DF64_PER_CELL = 157.498368e6 / 262144
# Algorithmic work of that kernel per cell, counted from its operations: 572 double-float adds
# (8 FP32 flops each: TwoSum and two low-part adds) and 223 double-float multiplies (7 flops:
# product and three fused multiply-adds).  Displacement transforms 144 adds + 36 multiplies, phi
# values 48 + 8, Gauss-point loop 148 adds (8 x 23, less the 36 flux sums' first terms) + 128
# multiplies, flux integration 153 + 36, phi rows 79 + 15.
DF64_ADDS_PER_CELL, DF64_MULS_PER_CELL = 572, 223


def vcycle_bytes_per_node(prec: int) -> float:
    """Algorithmic bytes of one V-cycle per fine node: on every level nine operator applies (degree-4
    Chebyshev pre- and post-smoothing from and to the level's vectors, 2 x 4 + 1 applies with the
    residual) at 53 B/node in FP32 or 105 B/node FP64-accurate, five vector passes per Chebyshev step
    over eight steps and two for the transfers (4 components of 4 or 8 bytes), summed over the levels
    of a 3D hierarchy (factor 8/7)."""
    s = 4 if prec == 32 else 8
    b_apply = 53.0 if prec == 32 else 105.0
    return (9 * b_apply + 8 * 5 * 4 * s + 2 * 4 * s) * 8.0 / 7.0


def _nvtx(name: str, push: bool):
    """NVTX range around the timed region, so that a profiler can select exactly its launches."""
    try:
        import torch
        torch.cuda.nvtx.range_push(name) if push else torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(vals, ws, device=None):
    """Each entry's maximum over the ranks (the slowest replica sets the job's time)."""
    if ws <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_gdofs(ws, n_dofs, apply_ms):
    """Whole-job Jacobian-apply throughput of ws replicas, each applying n_dofs in apply_ms."""
    return ws * n_dofs / (apply_ms * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi clock/throttle sampling (every 50 ms, timestamped).  Start it before the warm-up
    so that it is sampling when the timed region opens; mark() records the region's host times and
    summary() keeps the samples inside it."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: str | None = None):
        self.index = index
        self.proc = None
        self.window = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"pff_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def mark(self, t0: float, t1: float):
        """Host wall-clock bounds (time.time()) of the timed region."""
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self, running: bool = True):
        if running and not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, p[1:]))
        inside = rows
        if self.window and rows:
            lo, hi = self.window[0] - 0.05, self.window[1] + 0.05
            sel = [r for r in rows if r[0] is not None and lo <= r[0] <= hi]
            inside = sel if sel else rows
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        vals = [r[1] for r in inside]
        sm = [float(v[1]) for v in vals if v[1].replace(".", "").isdigit()]
        mx = [float(v[2]) for v in vals if v[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for v in vals for i in range(4) if v[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(vals)}


def bench_config(n: int = 128, levels: int = 5, ws: int = 1) -> dict:
    """The workload the JSON line is quoted on (shared by both arms)."""
    nn = (n + 1) ** 3
    return {"workload": f"3d_penny_q1_{n}", "n_dofs": 4 * nn, "levels": levels,
            "step": "one active-set Newton step (FP32 V-cycle in FP64 FGMRES to 1e-8)",
            "state": "U^3 after load steps p_n = n p / 3, n = 1..3; the step is the first of load step 4",
            "l2": "inputs larger than L2 (one FP64 apply touches ~%.0f MB)" % (105.0 * nn / 1e6),
            "parallelism": f"replicas{ws}"}


def _oracle_slab(n: int = 128, layers: int = 2):
    """The oracle's assembled Jacobian of a slab of the n^3 penny workload: the n x n x 'layers' cells
    through the crack plane z = 0 (same cell size, eps and crack recipe as the full mesh), at the
    workload's synthetic state.  Assembly (element by element, full Gauss quadrature) is not timed."""
    from oracle import fem
    from paper_1902_08112_gb300 import workloads as W
    full = W.config_3d_penny(n=n)
    dz = (full.hi[2] - full.lo[2]) / n
    w = W.Workload("penny_slab", 3, 1, (n, n, layers), 1, full.lo[:2] + (-dz * layers / 2,),
                   full.hi[:2] + (dz * layers / 2,), eps=full.eps, cracks=full.cracks)
    U, po, pt = W.initial_state(w, displacement="smooth")
    m = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi)
    ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure)
    t0 = time.perf_counter()
    G = fem.assemble(m, ph, U, pt, fem.dirichlet_face_mask(m, 0x3F))
    return G, m.n_dofs, time.perf_counter() - t0


def _spmv_rate(G, threads: int, reps: int = 5, min_s: float = 0.4):
    """Median over 'reps' timings of the oracle's CSR product y = G x split into 'threads' row blocks run
    on a thread pool (scipy's product releases the GIL); each timing repeats the product for >= min_s.
    Returns DoF/s."""
    from concurrent.futures import ThreadPoolExecutor
    n = G.shape[0]
    x = np.random.default_rng(7).standard_normal(n)
    y = np.empty(n)
    b = np.linspace(0, n, threads + 1).astype(int)
    parts = [(G[b[i]:b[i + 1]], b[i], b[i + 1]) for i in range(threads)]

    def f(p):
        M, a, c = p
        y[a:c] = M @ x

    rates = []
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(f, parts))
        for _ in range(reps):
            k, t0 = 0, time.perf_counter()
            while True:
                list(ex.map(f, parts))
                k += 1
                el = time.perf_counter() - t0
                if el >= min_s:
                    break
            rates.append(n * k / el)
    return float(np.median(rates))


def cpu_baseline():
    """Oracle Jacobian apply (assembled CSR product) on the host cores, on a slab of the benchmark
    workload: 1 thread and every core, median of 5."""
    G, nd, t_asm = _oracle_slab()
    cores = os.cpu_count() or 1
    r1 = _spmv_rate(G, 1)
    rn = _spmv_rate(G, cores)
    return {"value": rn / 1e9, "unit": "GDoF/s", "cores": cores, "kind": "oracle",
            "single_thread": {"value": r1 / 1e9, "unit": "GDoF/s", "cores": 1},
            "sample": f"3d_penny_q1_128: slab of 128 x 128 x 2 cells through the crack plane ({nd} DoFs, "
                      f"{G.nnz} nonzeros) of the oracle's assembled Jacobian (assembly {t_asm:.1f} s, not timed); "
                      f"CSR product in {cores} row blocks on {cores} threads, median of 5"}


SMALL_SOLVE = (32, 3)     # 3D penny recipe on 32^3 Q1 with 3 levels: the solve both the GPU and the oracle time


def bench_small_solve(dev, pending: list):
    """The GPU side of the solve comparison with the oracle: V-cycle and 1e-8 FGMRES solve (FP32-MG and
    FP64-MG) of the system G~ x = -A(U) on the penny recipe at 32^3 Q1 (3 levels, smooth displacement
    state, the active set of Algorithm 1).  The oracle's times for the same system are added by the CPU
    leg (oracle_solve_times)."""
    import torch
    from paper_1902_08112_gb300 import pff, workloads as W
    n, levels = SMALL_SOLVE
    w = W.small(W.config_3d_penny(), n, levels)
    U, po, pt = W.initial_state(w, displacement="smooth")
    stream = torch.cuda.Stream(device=dev)
    rec = {"workload": f"3d_penny_q1_{n} ({levels} levels, {w.n_dofs} DoFs)", "rtol": 1e-8}
    for mgp in (32, 64):
        prm = pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, pressure=w.pressure,
                                 mg_precision=mgp)
        h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, levels, w.lo, w.hi), prm, stream)
        try:
            with torch.cuda.stream(stream):
                Ud, pod, ptd = (torch.from_numpy(a).to(dev) for a in (U, po, pt))
                R = torch.empty(w.n_dofs, dtype=torch.float64, device=dev)
                z = torch.empty_like(R)
                xs = torch.zeros_like(R)
            stream.synchronize()
            pff.set_state(h, Ud, pod, ptd)
            na, _ = pff.update_active_set(h)
            stream.synchronize()
            t0 = time.perf_counter()
            pff.setup(h)
            stream.synchronize()
            setup_ms = (time.perf_counter() - t0) * 1e3
            pff.residual(h, R)
            pff.vcycle(h, R, z)
            stream.synchronize()
            t0 = time.perf_counter()
            for _ in range(10):
                pff.vcycle(h, R, z)
            stream.synchronize()
            vc_ms = (time.perf_counter() - t0) * 1e3 / 10
            t0 = time.perf_counter()
            info = pff.gmres_solve(h, R, xs, rtol=1e-8, restart=30, maxit=200, allow_noconv=True)
            stream.synchronize()
            rec[f"gpu_fp{mgp}_mg"] = {"setup_ms": setup_ms, "vcycle_ms": vc_ms,
                                      "solve_ms": (time.perf_counter() - t0) * 1e3, "iterations": info.iterations,
                                      "rel_res": info.res_final / max(info.res0, 1e-300), "n_active": na}
        finally:
            pff.destroy_hierarchy(h)
    pending.append({"solve": rec, "w": w, "U": U, "po": po, "pt": pt})
    return rec


def oracle_solve_times(pending: list):
    """The oracle's side of the solve comparison (CPU leg): the same system, assembled element by element
    with the active set of Algorithm 1, its V-cycle (FP64, Chebyshev-Jacobi) and FGMRES to 1e-8, timed on
    the host; setup = assembly of every level plus the eigenvalue estimates."""
    from oracle import fem, krylov, multigrid as mg, pdas
    for p in pending:
        if "solve" not in p:
            continue
        w, U, po, pt = p["w"], p["U"], p["po"], p["pt"]
        m = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi)
        ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure)
        t0 = time.perf_counter()
        R = -fem.residual_A(m, ph, U, pt)
        dmask = fem.dirichlet_face_mask(m, w.dirichlet_faces)
        act = pdas.active_set(m, R, fem.lumped_mass(m), U, po, 100.0, 1e-10, fixed=(dmask & fem.BIT_PHI_DIR) != 0)
        mask = dmask | (act * fem.BIT_ACTIVE).astype(np.uint8)
        lv = mg.build_levels(m, w.n_levels, ph, U, pt, mask)
        mg.estimate_levels(lv, 12345, 10)
        setup_s = time.perf_counter() - t0
        prm = mg.MGParams()
        t0 = time.perf_counter()
        for _ in range(3):
            mg.precondition(lv, R, prm)
        vc_s = (time.perf_counter() - t0) / 3
        G = lv[-1].G
        t0 = time.perf_counter()
        _, its, res, res0, _ = krylov.fgmres(lambda v: G @ v, R, lambda v: mg.precondition(lv, v, prm),
                                             rtol=1e-8, restart=30, maxit=200)
        p["solve"]["oracle_fp64_mg"] = {"setup_ms": setup_s * 1e3, "vcycle_ms": vc_s * 1e3,
                                        "solve_ms": (time.perf_counter() - t0) * 1e3, "iterations": its,
                                        "rel_res": res / max(res0, 1e-300), "n_active": int(act.sum()),
                                        "threads": 1}


def oracle_rows_check(pending: list):
    """Error of the GPU's multi-crack solutions against the FP64 oracle: the oracle's own rows (element by
    element, full Gauss quadrature) of the eliminated Jacobian applied to each solution on its seeded rows,
    against the right-hand side, max |b - G x| / max |b| over the sample.  Part of the CPU leg (rank 0,
    one GPU), after the GPU sections."""
    from oracle import fem
    for p in pending:
        if "rows" not in p:
            continue
        w = p["w"]
        m = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi)
        ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure)
        Gx = fem.apply_rows(m, ph, p["U"], p["pt"], p["mask"], p["x"], p["rows"])
        p["out"]["oracle_rows_rel_residual"] = float(np.abs(p["b_rows"] - Gx).max() / p["b_max"])


def bench_batch(count: int, dev):
    """Batching pattern: 'count' instances of the batch recipe (N in {16,24,32,48,64}, 1-6 cracks), one
    active-set step each (one linear solve to 1e-8).  Solves/s of the batched solver (one persistent
    launch per level and operation, device-side FGMRES state, the Arnoldi step replayed from a captured
    graph, autotuned level kernels) with the FP32 V-cycle (instances that stall switch to the FP64
    V-cycle after 10 iterations) and with the FP64 V-cycle, against the same instances solved one after
    another by the single-instance solver."""
    import torch
    from paper_1902_08112_gb300 import pff, workloads as W
    ws = W.batch_instances(count)
    stream = torch.cuda.Stream(device=dev)

    def build(mgp, phi_max=0):
        hs, Us = [], []
        for w in ws:
            U, po, pt = W.initial_state(w, displacement="smooth")
            prm = pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, pressure=w.pressure,
                                     mg_precision=mgp, seed=w.seed, coarse_phi_max=phi_max)
            h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, w.n_levels, w.lo, w.hi), prm, stream)
            Ud = torch.from_numpy(U).to(dev)
            pff.set_state(h, Ud, torch.from_numpy(po).to(dev), torch.from_numpy(pt).to(dev))
            hs.append(h)
            Us.append(Ud)
        torch.cuda.synchronize()
        return hs, Us

    def batched(hs, Us, U0, label):
        b = pff.batch_create(hs)
        for u, u0 in zip(Us, U0):
            u.copy_(u0)
        torch.cuda.synchronize()
        pff.batch_newton_step(b, Us, allow_noconv=True)          # warm-up: tuning, graph capture
        for u, u0 in zip(Us, U0):
            u.copy_(u0)
        torch.cuda.synchronize()
        _nvtx(f"batched_step_{label}", True)
        t0 = time.perf_counter()
        infos = pff.batch_newton_step(b, Us, allow_noconv=True)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        _nvtx("", False)
        precs = pff.batch_mg_precisions(b, len(hs))
        Lmax = max(w.n_levels for w in ws)
        tune = {}
        for level in list(range(Lmax)) + [-1]:
            for prec in (32, 64):
                try:
                    st, cps, ms = pff.batch_tuning(b, level, prec)
                except pff.PffError:
                    continue
                if st:
                    tune[f"{'fine' if level < 0 else 'l%d' % level}_fp{prec}"] = {
                        "kernels": "per_cell" if st == 2 else "small_level", "ctas_per_sm": cps, "ms": ms}
        pff.batch_destroy(b)
        return el, infos, precs, tune

    def single(hs, Us, U0):
        for u, u0 in zip(Us, U0):
            u.copy_(u0)
        pff.newton_step(hs[0], Us[0].clone(), allow_noconv=True)   # warm-up
        for u, u0 in zip(Us, U0):
            u.copy_(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sinfos = [pff.newton_step(h, u, allow_noconv=True) for h, u in zip(hs, Us)]
        torch.cuda.synchronize()
        return time.perf_counter() - t0, [i.solve.iterations for i in sinfos]

    out = {"instances": count, "dofs": int(sum(w.n_dofs for w in ws)), "sizes": sorted({w.n_cells[0] for w in ws}),
           "stream": "non-default (captured Arnoldi step replayed)"}
    hs, Us = build(32)
    U0 = [u.clone() for u in Us]
    tb32, infos32, precs32, tune32 = batched(hs, Us, U0, "fp32mg")
    ts32, its_s32 = single(hs, Us, U0)
    for h in hs:
        pff.destroy_hierarchy(h)
    hs, _ = build(64)
    tb64, infos64, _, tune64 = batched(hs, Us, U0, "fp64mg")
    ts64, its_s64 = single(hs, Us, U0)
    for h in hs:
        pff.destroy_hierarchy(h)
    # the option beyond the paper: phi~ on the coarse levels as the neighbourhood maximum
    hs, _ = build(32, phi_max=1)
    tbx, infosx, precsx, _ = batched(hs, Us, U0, "fp32mg_phimax")
    for h in hs:
        pff.destroy_hierarchy(h)
    out.update({
        "batched_fp32mg_solves_per_s": count / tb32,
        "batched_fp64mg_solves_per_s": count / tb64,
        "single_fp32mg_solves_per_s": count / ts32,
        "single_fp64mg_solves_per_s": count / ts64,
        "batched_fp32mg_vs_single_fp64mg": ts64 / tb32,
        "gmres_its_batched_fp32mg": [i.solve.iterations for i in infos32],
        "switched_to_fp64mg": int(sum(p == 64 for p in precs32)),
        "gmres_its_batched_fp64mg": [i.solve.iterations for i in infos64],
        "gmres_its_single_fp32mg": its_s32, "gmres_its_single_fp64mg": its_s64,
        "all_converged": all(i.solve.converged for i in infos32 + infos64 + infosx),
        "coarse_phi_max": {"batched_fp32mg_solves_per_s": count / tbx,
                           "batched_fp32mg_vs_single_fp64mg": ts64 / tbx,
                           "gmres_its_batched_fp32mg": [i.solve.iterations for i in infosx],
                           "switched_to_fp64mg": int(sum(p == 64 for p in precsx))},
        "autotuner_fp32mg": tune32, "autotuner_fp64mg": tune64})
    return out


def bench_multi(n: int, dev, pending: list):
    """3D multi-crack configuration (n^3 Q1, 8 penny cracks, 6 levels) at eps = 2h and 4h: FP64-accurate
    fine apply, V-cycle and time to a 1e-8 FGMRES solve of the Newton right-hand side with the FP32 and the
    FP64 V-cycle, at the initial crack state with the active set of Algorithm 1.  Each solution's error
    against the FP64 oracle is taken later, in the CPU leg (oracle_rows_check): this function only keeps
    the solution, the right-hand side on 4,000 seeded rows (a third of them on cracks) and the level's
    mask in 'pending'."""
    import torch
    from paper_1902_08112_gb300 import pff, workloads as W
    stream = torch.cuda.Stream(device=dev)

    def timed(fn, reps=3):
        fn()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    for ef in (2.0, 4.0):
        w = W.config_3d_multi(n=n, n_levels=6 if n >= 128 else 4, eps_factor=ef)
        U, po, pt = W.initial_state(w, displacement="smooth")
        rng = np.random.default_rng(17)
        crack_nodes = np.flatnonzero(po == 0.0)
        rows = np.concatenate([rng.choice(w.n_dofs, 2700, replace=False),
                               rng.choice(crack_nodes, 1300, replace=False) + rng.integers(0, 4, 1300) * w.n_nodes])
        rec = {"workload": f"3d_multi_q1_{n}_eps{int(ef)}h", "n_dofs": w.n_dofs, "levels": w.n_levels, "eps": w.eps}
        for mgp in (32, 64):
            prm = pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, pressure=w.pressure,
                                     mg_precision=mgp)
            h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, w.n_levels, w.lo, w.hi), prm, stream)
            try:
                with torch.cuda.stream(stream):
                    Ud, pod, ptd = (torch.from_numpy(a).to(dev) for a in (U, po, pt))
                    x = torch.randn(w.n_dofs, dtype=torch.float64, device=dev)
                    y = torch.empty_like(x)
                    z = torch.empty_like(x)
                    R = torch.empty_like(x)
                    xs = torch.zeros_like(x)
                    mask = torch.empty(w.n_nodes, dtype=torch.uint8, device=dev)
                stream.synchronize()
                pff.set_state(h, Ud, pod, ptd)
                na, _ = pff.update_active_set(h)
                pff.setup(h)
                if mgp == 32:
                    ms = timed(lambda: pff.apply_jacobian(h, -1, x, y), reps=5)
                    rec["apply64_ms"] = ms
                    rec["apply_gdofs"] = w.n_dofs / (ms * 1e-3) / 1e9
                    rec["n_active"] = na
                vc = timed(lambda: pff.vcycle(h, x, z))
                pff.residual(h, R)
                stream.synchronize()
                t0 = time.perf_counter()
                info = pff.gmres_solve(h, R, xs, rtol=1e-8, restart=30, maxit=300, allow_noconv=True)
                stream.synchronize()
                solve_ms = (time.perf_counter() - t0) * 1e3
                pff.level_state(h, -1, None, None, mask)
                stream.synchronize()
                Rh, xh, mh = R.cpu().numpy(), xs.cpu().numpy(), mask.cpu().numpy()
                rec[f"fp{mgp}_mg"] = {"vcycle_ms": vc, "solve_ms": solve_ms, "iterations": info.iterations,
                                      "rel_res": info.res_final / max(info.res0, 1e-300),
                                      "converged": bool(info.converged), "oracle_rows_rel_residual": None}
                pending.append({"out": rec[f"fp{mgp}_mg"], "w": w, "U": U, "pt": pt, "mask": mh, "x": xh,
                                "rows": rows, "b_rows": Rh[rows].copy(), "b_max": float(np.abs(Rh).max())})
            finally:
                pff.destroy_hierarchy(h)
        out[f"eps_{int(ef)}h"] = rec
    return out


def bench_q2(dev, sizes=((64, "penny", 5), (128, "multi", 6))):
    """Q2 on the sum-factorised fast path: the 3D penny crack on 64^3 Q2 hexahedra (8.6M DoFs) and the
    multi-crack recipe on 128^3 Q2 (67.9M DoFs).  FP64-accurate and FP32 fine applies (GDoF/s, HBM
    fraction of the 105 B/node algorithmic bytes), V-cycles and a 1e-8 FGMRES solve of the Newton
    right-hand side with the FP32 and the FP64 V-cycle, at the initial crack state with the active set
    of Algorithm 1."""
    import torch
    from paper_1902_08112_gb300 import pff, workloads as W
    hbm = _peaks().get("hbm_gbs", 6800.0)
    stream = torch.cuda.Stream(device=dev)

    def timed(fn, reps=3):
        fn()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    for n, kind, levels in sizes:
        w = (W.config_3d_penny(n=n, deg=2, n_levels=levels) if kind == "penny"
             else W.config_3d_multi(n=n, deg=2, n_levels=levels))
        U, po, pt = W.initial_state(w, displacement="smooth")
        rec = {"workload": f"3d_{kind}_q2_{n}", "n_dofs": w.n_dofs, "levels": levels}
        for mgp in (32, 64):
            prm = pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, pressure=w.pressure,
                                     mg_precision=mgp)
            h = pff.create_hierarchy(pff.make_mesh(3, 2, w.n_cells, levels, w.lo, w.hi), prm, stream)
            try:
                with torch.cuda.stream(stream):
                    Ud, pod, ptd = (torch.from_numpy(a).to(dev) for a in (U, po, pt))
                    x = torch.randn(w.n_dofs, dtype=torch.float64, device=dev)
                    y = torch.empty_like(x)
                    z = torch.empty_like(x)
                    R = torch.empty_like(x)
                    xs = torch.zeros_like(x)
                    x32 = x.float()
                    y32 = torch.empty_like(x32)
                stream.synchronize()
                pff.set_state(h, Ud, pod, ptd)
                pff.update_active_set(h)
                pff.setup(h)
                if mgp == 32:
                    ms = timed(lambda: pff.apply_jacobian(h, -1, x, y), reps=5)
                    ms32 = timed(lambda: pff.apply_jacobian_f32(h, -1, x32, y32), reps=5)
                    if kind == "penny":
                        # the generic direct-evaluation kernels (native FP64) for comparison
                        pff.set_kernel_variant(h, 1)
                        rec["generic_apply64_ms"] = timed(lambda: pff.apply_jacobian(h, -1, x, y), reps=2)
                        pff.set_kernel_variant(h, 0)
                        pff.setup(h)
                    nn = w.n_nodes
                    rec["apply64_ms"] = ms
                    rec["apply64_gdofs"] = w.n_dofs / (ms * 1e-3) / 1e9
                    rec["apply64_hbm_frac"] = 105.0 * nn / (ms * 1e-3) / 1e9 / hbm
                    rec["apply32_ms"] = ms32
                    rec["apply32_gdofs"] = w.n_dofs / (ms32 * 1e-3) / 1e9
                    rec["apply32_hbm_frac"] = 53.0 * nn / (ms32 * 1e-3) / 1e9 / hbm
                vc = timed(lambda: pff.vcycle(h, x, z))
                pff.residual(h, R)
                stream.synchronize()
                t0 = time.perf_counter()
                info = pff.gmres_solve(h, R, xs, rtol=1e-8, restart=30, maxit=100, allow_noconv=True)
                stream.synchronize()
                rec[f"fp{mgp}_mg"] = {"vcycle_ms": vc, "solve_ms": (time.perf_counter() - t0) * 1e3,
                                      "iterations": info.iterations, "converged": bool(info.converged),
                                      "rel_res": info.res_final / max(info.res0, 1e-300)}
            finally:
                pff.destroy_hierarchy(h)
        out[rec["workload"]] = rec
    return out


def bench_variants(n: int, dev):
    """Next-row variants on the 3D penny crack (n^3 Q1, smooth displacement, active set of
    Algorithm 1): P_full vs P_diag (Sec. 3.3), the Miehe split (Sec. 2.1, generic kernels) and a
    spatially varying E.  Per variant: FP64-accurate fine apply time and a 1e-8 FGMRES solve of the
    Newton right-hand side with the FP32 V-cycle."""
    import torch
    from paper_1902_08112_gb300 import pff, workloads as W
    w = W.config_3d_penny(n=n, n_levels=4)
    U, po, pt = W.initial_state(w, displacement="smooth")
    stream = torch.cuda.Stream(device=dev)
    out = {"workload": f"3d_penny_q1_{n}", "n_dofs": w.n_dofs}
    cases = {"p_full": dict(), "p_diag": dict(preconditioner=1), "miehe_split": dict(split=1),
             "varying_E": dict()}
    for name, extra in cases.items():
        prm = pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, pressure=w.pressure,
                                 mg_precision=32, **extra)
        h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, w.n_levels, w.lo, w.hi), prm, stream)
        try:
            with torch.cuda.stream(stream):
                Ud, pod, ptd = (torch.from_numpy(a).to(dev) for a in (U, po, pt))
                x = torch.randn(w.n_dofs, dtype=torch.float64, device=dev)
                y = torch.empty_like(x)
                R = torch.empty_like(x)
                xs = torch.zeros_like(x)
                es = torch.from_numpy(W.modulus_field(w)).to(dev) if name == "varying_E" else None
            stream.synchronize()
            if es is not None:
                pff.set_modulus(h, es)
            pff.set_state(h, Ud, pod, ptd)
            pff.update_active_set(h)
            pff.setup(h)
            pff.apply_jacobian(h, -1, x, y)
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                pff.apply_jacobian(h, -1, x, y)
            e1.record(stream)
            e1.synchronize()
            pff.residual(h, R)
            stream.synchronize()
            t0 = time.perf_counter()
            info = pff.gmres_solve(h, R, xs, rtol=1e-8, restart=30, maxit=300, allow_noconv=True)
            stream.synchronize()
            out[name] = {"apply64_ms": e0.elapsed_time(e1) / 5, "solve_ms": (time.perf_counter() - t0) * 1e3,
                         "iterations": info.iterations, "converged": bool(info.converged)}
        finally:
            pff.destroy_hierarchy(h)
    return out


def bench_serve(count: int):
    """Serving pattern: Poisson arrivals of random pressurised-crack requests (the batch recipe with
    N in {16,24,32}, 2 pressure load steps) mixed with displacement-driven 3D L-shaped panels (every 4th
    request, 2^k cells per edge for k = 4..7, a 20-step displacement ramp), served by the
    continuous-batching loop at 50, 80 and 95 % of the measured closed-loop capacity."""
    from paper_1902_08112_gb300 import serve
    # capacity: all requests queued at once
    cal = serve.poisson_requests(max(4, count // 4), 1.0, seed=99, lshape_every=4)
    be = serve.PffBackend()
    srv = serve.Server(be, hbm_budget=64 << 30)
    t0 = srv.now()
    srv.run(cal, realtime=False)
    cap = len(cal) / (srv.now() - t0)       # requests per second
    out = {"capacity_requests_per_s": cap, "load_steps": {"crack": 2, "lshape": 20},
           "mix": "batch recipe (N 16/24/32) + displacement-driven 3D L-shape (edge 16..128) every 4th"}
    for frac in (0.5, 0.8, 0.95):
        reqs = serve.poisson_requests(count, frac * cap, seed=12345, lshape_every=4)
        be = serve.PffBackend()
        srv = serve.Server(be, hbm_budget=64 << 30)
        t0 = srv.now()
        srv.run(reqs, realtime=True)
        wall = srv.now() - t0
        res = serve.summarize(srv.results, wall)
        res.update({"arrival_rate_per_s": frac * cap, "ticks": srv.ticks, "batches_built": be.batches_built,
                    "lshape_sizes": sorted({r.workload.n_cells[0] for r in reqs if r.workload.domain == "lshape"})})
        out[f"load_{int(frac * 100)}"] = res
    return out


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    G, nd, t_asm = _oracle_slab()
    cores = os.cpu_count() or 1
    from concurrent.futures import ThreadPoolExecutor
    n = G.shape[0]
    x = np.random.default_rng(7).standard_normal(n)
    y = np.empty(n)
    b = np.linspace(0, n, cores + 1).astype(int)
    parts = [(G[b[i]:b[i + 1]], b[i], b[i + 1]) for i in range(cores)]

    def f(p):
        M, a, c = p
        y[a:c] = M @ x

    reps_per_step = 20
    with ThreadPoolExecutor(cores) as ex:
        for _ in range(args.warmup):
            list(ex.map(f, parts))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for _ in range(reps_per_step):
                list(ex.map(f, parts))
        el = time.perf_counter() - t0
    val = nd * reps_per_step * args.steps / el / 1e9
    sample = (f"3d_penny_q1_128: slab of 128 x 128 x 2 cells through the crack plane ({nd} DoFs) of the oracle's "
              f"assembled Jacobian (assembly {t_asm:.1f} s, not timed); {reps_per_step} CSR products per step on "
              f"{cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(128, 5, args.gpus),
            "cpu_baseline": {"value": val, "unit": "GDoF/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pff", choices=["pff", "reference"])
    ap.add_argument("--n", type=int, default=128, help="cells per edge of the 3D penny workload")
    ap.add_argument("--levels", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small-solve", type=int, default=1, help="GPU vs oracle solve on the 32^3 penny (0: off)")
    ap.add_argument("--batch", type=int, default=256, help="instances in the batching measurement (0: skip)")
    ap.add_argument("--serve", type=int, default=24, help="requests in the serving measurement (0: skip)")
    ap.add_argument("--multi", type=int, default=256, help="cells per edge of the multi-crack measurement (0: skip)")
    ap.add_argument("--variants", type=int, default=64, help="cells per edge of the variant measurements (0: skip)")
    ap.add_argument("--q2", type=int, default=1, help="Q2 measurements (64^3 penny, 128^3 multi-crack; 0: skip)")
    ap.add_argument("--q2-case", type=int, default=0,
                    help="run the Q2 section on an n^3 Q2 penny crack (3 levels) only (a small profiling case)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_1902_08112_gb300 import pff, workloads as W

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if ws > 1:
            dist.barrier()

    w = W.config_3d_penny(n=args.n, n_levels=args.levels)
    U0, po, pt = W.initial_state(w)
    stream = torch.cuda.Stream(device=dev)
    prm = pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, pressure=w.pressure,
                             mg_precision=32)
    h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, w.n_levels, w.lo, w.hi), prm, stream)
    nd, nn = w.n_dofs, w.n_nodes
    with torch.cuda.stream(stream):
        U = torch.from_numpy(U0).to(dev)
        po_d = torch.from_numpy(po).to(dev)
        pt_d = torch.from_numpy(pt).to(dev)
    stream.synchronize()
    pff.set_state(h, U, po_d, pt_d)
    # linearisation point: three load steps p_n = n p / 3 from u = 0 (untimed)
    prev, load_info = None, []
    for n in (1, 2, 3):
        with torch.cuda.stream(stream):
            phi_nm1 = U[3 * nn:].clone()
        li = pff.load_step(h, U, prev, w.pressure * n / 3, max_newton=12, allow_noconv=True)
        load_info.append({"newton_steps": li.newton_steps, "converged": li.converged,
                          "gmres_iterations": li.gmres_iterations})
        prev = phi_nm1
    with torch.cuda.stream(stream):
        U3 = U.clone()
        phi2 = prev
    stream.synchronize()
    p4 = w.pressure * 4 / 3

    def step():
        # first active-set Newton step of load step 4, linearised at U^3
        with torch.cuda.stream(stream):
            U.copy_(U3)
        li = pff.load_step(h, U, phi2, p4, max_newton=1, allow_noconv=True)
        return li.last

    infos = []
    # the clock sampler runs from the warm-up on, so it is sampling when the timed region opens
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        barrier()
        pff.profile(h, True)
        launches0 = pff.launch_count()
        barrier()
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        _nvtx("timed_steps", True)
        t_wall0 = time.time()
        ev0.record(stream)
        for _ in range(args.steps):
            infos.append(step())
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        clk.mark(t_wall0, time.time())
        _nvtx("timed_steps", False)
        barrier()
    launches = pff.launch_count() - launches0
    ms_total = ev0.elapsed_time(ev1)
    cnt64, ms64 = pff.profile_read(h, pff.PROF_APPLY64_FINE)
    cnt64c, ms64c = pff.profile_read(h, pff.PROF_APPLY64_COARSE)
    cnt32, ms32 = pff.profile_read(h, pff.PROF_APPLY32)
    cntv, msv = pff.profile_read(h, pff.PROF_VCYCLE)
    pff.profile(h, False)
    ms_total, apply_ms = max_over_ranks([ms_total, ms64 / max(cnt64, 1)], ws, dev)
    ms_step = ms_total / args.steps
    value = job_gdofs(ws, nd, apply_ms)

    # ---- secondary measurements (outside the timed region)
    def timed(fn, reps=3):
        fn()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    rng = np.random.default_rng(3)
    with torch.cuda.stream(stream):
        r = torch.from_numpy(rng.standard_normal(nd)).to(dev)
        z = torch.empty_like(r)
        xs = torch.zeros_like(r)
    stream.synchronize()
    # linear system of the timed step (state U^3, phi_old = phi^3, extrapolated phi~, p_4)
    pt4 = torch.empty(nn, dtype=torch.float64, device=dev)
    pff.level_state(h, -1, None, pt4, None)
    with torch.cuda.stream(stream):
        phi3 = U3[3 * nn:].clone()
    res = {}
    for mgp in (32, 64):
        pff.set_params(h, pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps,
                                             pressure=p4, mg_precision=mgp))
        pff.set_state(h, U3, phi3, pt4)
        pff.update_active_set(h)
        pff.setup(h)
        vc_ms = timed(lambda: pff.vcycle(h, r, z))
        R = torch.empty(nd, dtype=torch.float64, device=dev)
        pff.residual(h, R)
        stream.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            xs.zero_()
        info = pff.gmres_solve(h, R, xs, rtol=1e-8, restart=30, maxit=200, allow_noconv=True)
        stream.synchronize()
        solve_ms = (time.perf_counter() - t0) * 1e3
        vc_gbs = vcycle_bytes_per_node(mgp) * nn / (vc_ms * 1e-3) / 1e9
        res[f"fp{mgp}_mg"] = {"vcycle_ms": vc_ms, "solve_ms": solve_ms, "iterations": info.iterations,
                              "rel_res": info.res_final / max(info.res0, 1e-300),
                              "vcycle_gdofs": nd / (vc_ms * 1e-3) / 1e9,
                              "vcycle_hbm_frac": vc_gbs / _peaks().get("hbm_gbs", 6800.0),
                              "vcycle_bytes_per_node": vcycle_bytes_per_node(mgp)}

    # ---- end to end through the C ABI with host buffers: pff_apply_jacobian_host copies x from
    # pinned host memory, applies and copies y back (slab-pipelined on three streams) and returns
    # when y is on the host; timed by the host clock around the synchronous calls
    xh = torch.from_numpy(rng.standard_normal(nd)).pin_memory()
    yh = torch.empty(nd, dtype=torch.float64).pin_memory()
    pff.apply_jacobian_host(h, -1, xh, yh)
    reps = max(3, args.steps)
    t0 = time.perf_counter()
    for _ in range(reps):
        pff.apply_jacobian_host(h, -1, xh, yh)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / reps
    e2e_ms = max_over_ranks([e2e_ms], ws, dev)[0]

    # ---- FP32 fine-level apply (the V-cycle operator), timed alone
    x32 = torch.randn(nd, dtype=torch.float32, device=dev)
    y32 = torch.empty_like(x32)
    torch.cuda.synchronize()   # x32 is written on torch's stream, read on the library's
    ms32_fine = timed(lambda: pff.apply_jacobian_f32(h, -1, x32, y32), reps=10)

    # ---- rooflines.  Headline: the FP64-accurate fine apply against HBM with the algorithmic bytes
    # of the on-the-fly linearisation (x, U, phi~, y and the mask: 105 B per node in 3D), over the
    # measured copy bandwidth.  Secondary: its arithmetic, which is what bounds it on GB300 -- the
    # FP64-accurate apply runs as double-float on the FP32 pipes -- over the FP32 FMA rate measured
    # by pff_fp32_fma_tflops.  Algorithmic FP32 flops per cell of the double-float per-cell apply:
    # 572 adds x 8 + 223 multiplies x 7 = 6137; the FP32 per-cell apply runs the same operations in
    # FP32: 572 + 223 = 795.
    classes = {"apply64_fine": (cnt64, ms64), "apply64_coarse": (cnt64c, ms64c), "apply32": (cnt32, ms32),
               "vcycle_graph": (cntv, msv)}
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    try:
        fp32_peak = pff.fp32_fma_tflops(stream)
        fp32_note = "peak: FP32 FMA rate measured on this GPU by pff_fp32_fma_tflops"
    except pff.PffError:
        fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        fp32_note = "peak: FP32 pipe derived from unit counts (152 SMs x 128 lanes x 2 flops x 2.07 GHz)"
    cells = w.n_cells_total
    fl64 = (8.0 * DF64_ADDS_PER_CELL + 7.0 * DF64_MULS_PER_CELL) * cells
    fl32 = float(DF64_ADDS_PER_CELL + DF64_MULS_PER_CELL) * cells
    bytes64 = 105.0 * nn
    gbs64 = bytes64 / (apply_ms * 1e-3) / 1e9
    roof = {"kernel": "k_q1_apply_cell<df64, false> (FP64-accurate fine-level Jacobian apply)",
            "bound": "hbm", "achieved": gbs64, "peak": hbm, "unit": "GB/s", "frac": gbs64 / hbm,
            "peak_note": "MEASURED_PEAKS.json hbm_gbs (of measured)",
            "algorithmic_bytes_per_launch": bytes64,
            "bytes_note": "105 B per node: x, U (4 x 8 B each), phi~ and y (8 B, 32 B) and the 1-byte mask",
            "traffic": TRAFFIC_DF64_PER_CELL * cells if TRAFFIC_DF64_PER_CELL else None,
            "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at 64^3 "
                            "(%.1f MB), scaled by cells" % (TRAFFIC_DF64_PER_CELL * 262144 / 1e6),
            "alu": {"achieved": fl64 / (apply_ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": fl64 / (apply_ms * 1e-3) / 1e12 / fp32_peak, "algorithmic_flops_per_launch": fl64,
                    "note": fp32_note + "; double-float arithmetic on the FP32 pipes (the kernel's bound)"},
            "fp64_equivalent_tflops": (DF64_ADDS_PER_CELL + DF64_MULS_PER_CELL) * cells / (apply_ms * 1e-3) / 1e12}
    roof32 = {"kernel": "k_q1_apply_cell<float, false> (FP32 fine-level V-cycle operator)", "ms": ms32_fine,
              "bound": "alu", "achieved": fl32 / (ms32_fine * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
              "frac": fl32 / (ms32_fine * 1e-3) / 1e12 / fp32_peak,
              "hbm_frac": 53.0 * nn / (ms32_fine * 1e-3) / 1e9 / hbm, "gdofs": nd / (ms32_fine * 1e-3) / 1e9}
    line = {
        "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "df64", "data": "synthetic",
        "dtype_note": "double-float (pairs of FP32) arithmetic, FP64 vectors in memory; matches the FP64 "
                      "oracle's assembled product to 1e-12 relative",
        "config": bench_config(args.n, w.n_levels, ws),
        "clocks": clk.summary(),
        "e2e": {"value": job_gdofs(ws, nd, e2e_ms), "unit": "GDoF/s", "h2d_bytes_per_step": nd * 8,
                "d2h_bytes_per_step": nd * 8},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_fp32_apply": roof32,
        "kernel_ms": {k: {"launches": v[0], "total_ms": v[1]} for k, v in classes.items()},
        "newton": {"gmres_iterations": [i.solve.iterations for i in infos], "n_active": infos[-1].n_active,
                   "load_steps_to_state": load_info},
        "solve": res,
    }
    pff.destroy_hierarchy(h)
    if args.batch > 0:
        line["batch"] = bench_batch(args.batch, dev)
    if args.serve > 0:
        line["serve"] = bench_serve(args.serve)
    pending = []
    if args.small_solve:
        line["solve_small"] = bench_small_solve(dev, pending)
    if args.multi > 0:
        line["multi_crack"] = bench_multi(args.multi, dev, pending)
    if args.variants > 0:
        line["variants"] = bench_variants(args.variants, dev)
    if args.q2_case > 0:
        line["q2"] = bench_q2(dev, sizes=((args.q2_case, "penny", 3),))
    elif args.q2 > 0:
        line["q2"] = bench_q2(dev)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the CPU leg: the oracle on the host cores, timed (cpu_baseline), and its rows of the multi-crack
        # systems applied to the GPU's solutions
        oracle_rows_check(pending)
        oracle_solve_times(pending)
        line["cpu_baseline"] = cpu_baseline()
    pending.clear()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
