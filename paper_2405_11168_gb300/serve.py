"""Continuous-batching RVE solve service on one GPU with device-resident solver slots.

Requests (a microstructure, its phase table, 1-6 load cases, a precision and a
tolerance) are queued as they arrive.  Up to ``slots`` requests run at once,
each on its own worker thread.  The device memory is a pool of resident solver
contexts owned by the HBM budget: a context (workspace, launch shapes, twiddle
tables, captured iteration graphs, its own CUDA stream, and field buffers when
asked for) is created for a (grid, precision, phase capacity, fields) key the
first time a request needs one and stays resident afterwards; a later request of
the same key binds its microstructure to an idle context with hs_set_material
instead of allocating anything.  A request is admitted, in arrival order, when a
worker is free and an idle context of its key exists, or a new one fits in the
budget next to the resident ones (idle contexts of other keys are released to
make room).  Solves of different requests run on their contexts' streams and
overlap on the device (the C ABI releases the GIL while it waits).  Every
kernel reduction is deterministic, so a request's results do not depend on what
runs beside it or on which resident context serves it.

A context's launch shapes come from the autotuner's plan cache when
``autotune=True`` (tuned once per grid and precision, then reused).

The batched form of the 6 unit load cases (the columns of the effective
stiffness, Eqs. final_fields) is a request with ``loads=unit_loads()``.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import hs

# phase capacity of a resident context: materials of up to this many phases share one layout
LAYOUT_PHASES = 64


def unit_loads():
    """The 6 unit macroscopic strains (tensor components); column J of C_eff is <sigma> under load J."""
    out = []
    for J in range(6):
        e = np.zeros(6)
        e[J] = 1.0 if J < 3 else 0.5
        out.append(e)
    return out


@dataclass
class Request:
    ids: np.ndarray                 # [N3][N2][N1] phase ids (uint8 / uint16)
    table: np.ndarray               # nphase x 6 x 6 Voigt stiffness
    loads: list                     # macroscopic strains (6 tensor components each)
    precision: int = hs.HS_FP32_REFINED
    tol: float = 1e-6
    max_iter: int = 5000
    fields: bool = False            # return eps/sig of the last load case (host arrays)
    tag: object = None
    arrival: float = field(default=0.0)


@dataclass
class Result:
    tag: object
    sig_eff: np.ndarray             # len(loads) x 6
    iters: list
    errs: list
    status: list
    eps: np.ndarray = None
    sig: np.ndarray = None
    latency_s: float = 0.0
    queued_s: float = 0.0
    bytes: int = 0


def layout_phases(nphase: int) -> int:
    """Phase capacity of the context that serves a material of ``nphase`` phases."""
    n = LAYOUT_PHASES
    while n < nphase:
        n *= 2
    return min(n, hs.HS_MAX_PHASES)


def pool_key(req: Request):
    n3, n2, n1 = req.ids.shape
    return ((n1, n2, n3), int(req.precision), layout_phases(len(req.table)), bool(req.fields))


def key_bytes(key) -> int:
    """Device bytes a resident context of this key holds (workspace + field buffers)."""
    (n1, n2, n3), prec, lnp, fields = key
    opt = hs.default_options(precision=prec)
    nb = hs.workspace_size((n1, n2, n3), lnp, opt) + 256
    if fields:
        nb += 2 * 6 * n1 * n2 * n3 * 8
    return nb


def request_bytes(req: Request) -> int:
    """Device bytes the context that serves this request holds."""
    return key_bytes(pool_key(req))


@dataclass
class _Slot:
    """One resident solver context and what belongs to it."""
    key: tuple
    bytes: int
    stream: object = None
    solver: object = None
    fields: tuple = None
    uses: int = 0


class Server:
    def __init__(self, budget_bytes: int, slots: int = 4, device="cuda", autotune: bool = False):
        import torch

        self.torch = torch
        dev = torch.device(device)
        if dev.index is None:
            dev = torch.device(dev.type, torch.cuda.current_device())
        self.device = dev
        self.budget = int(budget_bytes)
        self.used = 0               # bytes of every resident context, busy or idle
        self.max_used = 0
        self.running = 0
        self.max_running = 0
        self.created = 0            # contexts created (the rest of the requests reused one)
        self.released = 0           # idle contexts released to make room for another key
        self.autotune = autotune
        self._cv = threading.Condition()
        self._pending = collections.deque()
        self._idle = collections.defaultdict(list)   # key -> idle resident slots
        self._closed = False
        self._workers = []
        for i in range(slots):
            t = threading.Thread(target=self._worker, name=f"hs-slot-{i}", daemon=True)
            t.start()
            self._workers.append(t)

    def request_bytes(self, req: Request) -> int:
        """Device bytes the context that serves the request holds (admission uses this)."""
        return request_bytes(req)

    def _start_slot(self):
        """Per-worker set-up: the worker's device."""
        self.torch.cuda.set_device(self.device)

    def submit(self, req: Request) -> Future:
        need = self.request_bytes(req)
        if need > self.budget:
            raise ValueError(f"request needs {need} bytes, above the budget of {self.budget}")
        fut = Future()
        req.arrival = req.arrival or time.perf_counter()
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            self._pending.append((req, pool_key(req), need, fut))
            self._cv.notify_all()
        return fut

    def close(self):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for t in self._workers:
            t.join()
        with self._cv:
            for slots in self._idle.values():
                for sl in slots:
                    self._free(sl)
            self._idle.clear()

    def _free(self, sl: _Slot):
        if sl.solver is not None:
            sl.solver.close()
        sl.solver = sl.fields = None
        self.used -= sl.bytes

    # admission: the head of the queue runs when an idle context of its key is resident, or a new
    # one fits next to the resident contexts once idle contexts of other keys are released
    def _take(self):
        with self._cv:
            while True:
                if self._pending:
                    req, key, need, fut = self._pending[0]
                    if self._idle[key]:
                        sl = self._idle[key].pop()
                    else:
                        others = [s for k, lst in self._idle.items() if k != key for s in lst]
                        while self.used + need > self.budget and others:
                            victim = others.pop(0)
                            self._idle[victim.key].remove(victim)
                            self._free(victim)
                            self.released += 1
                        sl = None
                        if self.used + need <= self.budget:
                            sl = _Slot(key=key, bytes=need)
                            self.used += need
                            self.created += 1
                    if sl is not None:
                        self._pending.popleft()
                        self.running += 1
                        self.max_used = max(self.max_used, self.used)
                        self.max_running = max(self.max_running, self.running)
                        return req, sl, fut
                elif self._closed:
                    return None
                self._cv.wait()

    def _release(self, sl: _Slot, ok: bool):
        with self._cv:
            self.running -= 1
            if ok and sl.solver is not None:
                self._idle[sl.key].append(sl)       # stays resident for the next request of its key
            else:
                self._free(sl)
            self._cv.notify_all()

    def _fail_pending(self, exc):
        with self._cv:
            while self._pending:
                _, _, _, fut = self._pending.popleft()
                fut.set_exception(exc)
            self._closed = True
            self._cv.notify_all()

    def _worker(self):
        try:
            self._start_slot()
        except BaseException as e:  # noqa: BLE001 - a slot that cannot start fails the queue, not silently
            self._fail_pending(e)
            return
        while True:
            item = self._take()
            if item is None:
                return
            req, sl, fut = item
            t_start = time.perf_counter()
            ok = False
            try:
                res = self._run(req, sl)
                res.queued_s = t_start - req.arrival
                res.latency_s = time.perf_counter() - req.arrival
                res.bytes = sl.bytes
                ok = True
                fut.set_result(res)
            except BaseException as e:  # noqa: BLE001 - report any failure through the future
                fut.set_exception(e)
            finally:
                self._release(sl, ok)

    def _bind(self, req: Request, sl: _Slot):
        """The slot's context bound to the request's microstructure (created on first use)."""
        torch = self.torch
        if sl.solver is not None:
            sl.solver.set_material(req.ids, req.table)
            return
        sl.stream = torch.cuda.Stream(self.device)
        kw = {}
        if self.autotune:
            opts, _ = hs.autotune(torch.from_numpy(np.ascontiguousarray(req.ids)).to(self.device), req.table,
                                  precision=req.precision, device=self.device, stream=sl.stream)
            kw = {k: opts[k] for k in ("ytile", "zchunk", "col_tile")}
        sl.solver = hs.Solver(req.ids, req.table, precision=req.precision, device=self.device, stream=sl.stream,
                              layout_nphase=sl.key[2], **kw)
        if req.fields:
            n3, n2, n1 = req.ids.shape
            sl.fields = (torch.empty((6, n3, n2, n1), dtype=torch.float64, device=self.device),
                         torch.empty((6, n3, n2, n1), dtype=torch.float64, device=self.device))

    def _run(self, req: Request, sl: _Slot) -> Result:
        self._bind(req, sl)
        sl.uses += 1
        s = sl.solver
        sig_eff, iters, errs, status = [], [], [], []
        out = None
        for k, E in enumerate(req.loads):
            last = k == len(req.loads) - 1
            out = s.solve(E, tol=req.tol, max_iter=req.max_iter, fields=req.fields and last,
                          out=sl.fields if (req.fields and last) else None)
            sig_eff.append(out["sig_eff"])
            iters.append(out["iters"])
            errs.append(out["err"])
            status.append(out["status"])
        res = Result(tag=req.tag, sig_eff=np.array(sig_eff), iters=iters, errs=errs, status=status)
        if req.fields:
            sl.stream.synchronize()
            res.eps = out["eps"].cpu().numpy()
            res.sig = out["sig"].cpu().numpy()
        return res


def run_stream(server: Server, requests, rate_hz: float, seed: int = 0):
    """Submit requests with Poisson arrivals at ``rate_hz`` (0: all at once); returns (results, wall s)."""
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    futs = []
    t_next = t0
    for req in requests:
        t_next += rng.exponential(1.0 / rate_hz) if rate_hz > 0 else 0.0
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        req.arrival = time.perf_counter()
        futs.append(server.submit(req))
    results = [f.result(timeout=3600) for f in futs]
    return results, time.perf_counter() - t0


def latency_stats(results):
    lat = np.array([r.latency_s for r in results])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}


def synthetic_requests(n, sizes, seed, precision, tol, max_iter, loads_per_request=(1, 6)):
    """Seeded request stream: random-sphere two-phase RVEs (contrast log-uniform in
    1e-3..1e3, plus voids and the rigid surrogate) or 50-grain cubic Voronoi
    polycrystals, sizes drawn from ``sizes``, 1-6 unit load cases each."""
    from synth import polycrystal_table, random_rotations, random_spheres, two_phase_table, voronoi_grains

    rng = np.random.default_rng(seed)
    loads = unit_loads()
    reqs = []
    for i in range(n):
        N = int(rng.choice(sizes))
        grid = (N, N, N)
        if rng.random() < 0.5:
            ids, _ = random_spheres(grid, max(2.0, N / 8.0), 0.2, seed=int(rng.integers(1 << 30)))
            u = rng.random()
            contrast = 0.0 if u < 0.05 else (1e6 if u < 0.1 else float(10.0 ** rng.uniform(-3, 3)))
            table = two_phase_table(1.0, 0.3, contrast, 0.3)
        else:
            ids, _ = voronoi_grains(grid, 50, seed=int(rng.integers(1 << 30)))
            ids = ids.astype(np.uint8)
            table = polycrystal_table(168.4, 121.4, 75.4, random_rotations(50, seed=int(rng.integers(1 << 30))))
        k = int(rng.integers(loads_per_request[0], loads_per_request[1] + 1))
        reqs.append(Request(ids=ids, table=table, loads=loads[:k], precision=precision, tol=tol,
                            max_iter=max_iter, tag=i))
    return reqs


def main(argv=None):
    """Serve a seeded synthetic request stream and print one JSON line of throughput and latency."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--sizes", default="32,48,64,96")
    ap.add_argument("--rate", type=float, default=0.0, help="Poisson arrivals per second (0: all at once)")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--precision", default="refined", choices=["fp64", "fp32", "refined"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--seed", type=int, default=5)
    a = ap.parse_args(argv)
    prec = {"fp64": hs.HS_FP64, "fp32": hs.HS_FP32, "refined": hs.HS_FP32_REFINED}[a.precision]
    sizes = [int(x) for x in a.sizes.split(",")]
    hs.load()
    reqs = synthetic_requests(a.requests, sizes, a.seed, prec, a.tol, a.max_iter)
    srv = Server(int(a.budget_gb * 2**30), slots=a.slots, autotune=a.autotune)
    try:
        res, wall = run_stream(srv, reqs, a.rate, seed=a.seed)
    finally:
        srv.close()
    solves = sum(len(r.iters) for r in res)
    conv = sum(int(st == hs.HS_OK) for r in res for st in r.status)
    line = {"metric": "served RVE solves/s", "value": solves / wall, "unit": "solves/s", "requests": len(res),
            "solves": solves, "converged": conv, "wall_s": wall, "precision": a.precision, "tol": a.tol,
            "max_iter": a.max_iter, "sizes": sizes, "rate_hz": a.rate, "slots": a.slots,
            "budget_gb": a.budget_gb, "max_running": srv.max_running, "max_used_gb": srv.max_used / 2**30,
            "contexts_created": srv.created, "contexts_released": srv.released,
            "evaluations": int(sum(sum(r.iters) for r in res)), **latency_stats(res)}
    # requests whose every solve met the tolerance, and the stream split by grid size
    ok = [r for r in res if all(st == hs.HS_OK for st in r.status)]
    if ok:
        line["converged_requests"] = len(ok)
        line.update({k + "_converged": v for k, v in latency_stats(ok).items()})
    size_of = {q.tag: q.ids.shape[0] for q in reqs}
    by = {}
    for r in res:
        d = by.setdefault(str(size_of[r.tag]), {"requests": 0, "solves": 0, "converged": 0, "lat": []})
        d["requests"] += 1
        d["solves"] += len(r.status)
        d["converged"] += sum(int(st == hs.HS_OK) for st in r.status)
        d["lat"].append(r.latency_s)
    for d in by.values():
        lat = d.pop("lat")
        d["p50_s"] = float(np.percentile(lat, 50))
        d["p99_s"] = float(np.percentile(lat, 99))
    line["by_size"] = by
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    import sys

    sys.exit(main())
