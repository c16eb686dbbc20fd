"""Continuous-batching request loop for shallow-water runs on one GPU.

Requests (a mesh size, a degree, a number of steps, a seed, an arrival time) are admitted
while both a slot and device memory are free -- the memory each needs is the library's own
``hdgdg_bytes_required`` -- and stay resident until done.  Every admitted simulation is
stepped by its own host thread on its own CUDA stream (the library creates one per handle;
ctypes releases the GIL during each call), so the device work of all admitted requests
overlaps, and requests that arrive while others run join as soon as a slot and memory free
up.  Each step's arithmetic is the same as when the simulation runs alone, so results do not
depend on the mix (the reductions have a fixed order).

Requests that share a mesh size, degree, step count and arithmetic can instead be grouped
(``batch_requests``) and served as one batched handle each: one launch per kernel per stage
then covers the whole group.  A batch's trace systems are solved together, so its Krylov
iteration count is that of its hardest member and its results agree with the members' lone
runs to the solver tolerance, not bit for bit.

Reported: throughput in DOF-steps/s over the whole run, and the time to solution of each
request (arrival to result copied back), summarised as p50 / p99.
"""
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import hdgdg as hd
from . import workloads as W


@dataclass
class Request:
    rid: int
    N: int
    k: int
    steps: int
    seed: int
    arrival: float                      # seconds after the loop starts
    precision: str = "mixed"
    bottom_amp: float = 0.1
    result: tuple = None
    admitted: float = None
    finished: float = None
    bytes: int = 0
    error: str = None


def poisson_requests(n, rate_per_s, seed=5000, n_range=(32, 256), degrees=(2, 3, 4),
                     steps_range=(50, 500), precision="mixed"):
    """Seeded Poisson arrivals; N log-uniform in n_range, k uniform in degrees, steps uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_per_s)
        N = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        k = int(rng.choice(degrees))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(Request(i, N, k, steps, seed + 1 + i, t, precision, bottom_amp=0.0))
    return out


def ensemble_requests(n=256, seed=4000, sides=(16, 32, 64, 128), degrees=(2, 3, 4), steps=100,
                      precision="mixed"):
    """The batched-ensemble workload: n instances, all submitted at once, mesh side uniform in
    sides, k uniform in degrees, each with its own seeded bump and bottom amplitude U[0, 0.1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [Request(i, int(rng.choice(sides)), int(rng.choice(degrees)), steps, seed + 1 + i, 0.0,
                    precision, float(rng.uniform(0.0, 0.1))) for i in range(n)]


def initial_state(req):
    """The request's seeded state on the library's own nodes: one seeded Gaussian bump on a lake
    at rest over a sinusoidal bottom of the request's amplitude (flat for the Poisson serving
    requests, like the 8 x 8 bump; U[0, 0.1] for the ensemble), and its advective time step."""
    x, y = hd.node_coords(req.N, req.k)
    h, hu, hv, b = W.bump_at_rest_state(x, y, req.seed, req.bottom_amp)
    dt = W.advective_dt(x, h, hu, hv, req.N)
    return h, hu, hv, b, dt


@dataclass
class Batch:
    """Requests of one mesh size, degree, step count and arithmetic served as ONE batched handle:
    every kernel then covers all of them in one launch per stage, each keeping its own bottom,
    state and time step."""
    rid: int
    members: list
    arrival: float
    result: tuple = None
    admitted: float = None
    finished: float = None
    bytes: int = 0
    error: str = None

    @property
    def N(self):
        return self.members[0].N

    @property
    def k(self):
        return self.members[0].k

    @property
    def steps(self):
        return self.members[0].steps

    @property
    def precision(self):
        return self.members[0].precision


def batch_requests(requests, max_batch=64):
    """Group requests by (N, k, steps, precision) in arrival order, at most max_batch per group."""
    groups = {}
    for r in sorted(requests, key=lambda r: r.arrival):
        groups.setdefault((r.N, r.k, r.steps, r.precision), []).append(r)
    out = []
    for members in groups.values():
        for i in range(0, len(members), max_batch):
            part = members[i:i + max_batch]
            out.append(Batch(len(out), part, max(m.arrival for m in part)))
    return sorted(out, key=lambda b: b.arrival)


def bytes_of(req):
    """Device bytes one request (or batch) needs, from the library's own plan."""
    B = len(req.members) if isinstance(req, Batch) else 1
    return hd.bytes_required(hd.make_config(req.N, req.k, 1.0, batch=B, **form_options(req.precision)))


def run_batch(batch, chunk=10):
    """Run every member of a batch in one handle; sets each member's result."""
    states = [initial_state(r) for r in batch.members]
    cat = lambda j: np.concatenate([s[j] for s in states])  # noqa: E731
    dts = np.array([s[4] for s in states])
    n = batch.N * batch.N
    with hd.Sim(batch.N, batch.k, float(dts.max()), bottom=cat(3), batch=len(states), dt_per_instance=dts,
                **form_options(batch.precision)) as s:
        s.set_state(cat(0), cat(1), cat(2))
        done = 0
        while done < batch.steps:
            m = min(chunk, batch.steps - done)
            s.step(m)
            done += m
        out = s.get_state()
    for i, r in enumerate(batch.members):
        r.result = tuple(a[i * n:(i + 1) * n] for a in out)
    return out


def form_options(precision):
    """Library options of a request's arithmetic: the mixed form runs its FP64-bound parts (local
    contractions, refinement residuals) as FP32 pairs."""
    if precision == "mixed":
        return {"precision": "mixed", "local_precision": "f32x2", "residual_f32x2": True}
    return {"precision": precision}


def run_one(req, chunk=10):
    """Run one request to completion on a fresh handle; returns the final (h, hu, hv)."""
    h, hu, hv, b, dt = initial_state(req)
    with hd.Sim(req.N, req.k, dt, bottom=b, **form_options(req.precision)) as s:
        s.set_state(h, hu, hv)
        done = 0
        while done < req.steps:
            n = min(chunk, req.steps - done)
            s.step(n)
            done += n
        return s.get_state()


@dataclass
class Server:
    hbm_budget: int                      # bytes the loop may hand out
    max_slots: int = 8
    chunk: int = 10
    log: list = field(default_factory=list)

    def serve(self, requests, time_scale=1.0):
        """Serve requests (or batches of them) arriving at time_scale * arrival seconds; returns a
        summary dict over the individual requests."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue, running = [], {}
        used = 0
        lock = threading.Lock()
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def worker(req):
            try:
                if isinstance(req, Batch):
                    run_batch(req, self.chunk)
                else:
                    req.result = run_one(req, self.chunk)
            except Exception as ex:           # the request fails, the server carries on
                req.error = str(ex)
            req.finished = now()
            for m in getattr(req, "members", ()):
                m.admitted, m.finished, m.error = req.admitted, req.finished, req.error

        finished = []
        while pending or queue or running:
            t = now()
            while pending and pending[0].arrival * time_scale <= t:
                r = pending.pop(0)
                r.bytes = bytes_of(r)
                queue.append(r)
            with lock:
                for rid in [rid for rid, (r, th) in running.items() if not th.is_alive()]:
                    r, th = running.pop(rid)
                    th.join()
                    used -= r.bytes
                    finished.append(r)
                # admit in arrival order while a slot and memory are free (no overtaking)
                while queue and len(running) < self.max_slots and used + queue[0].bytes <= self.hbm_budget:
                    r = queue.pop(0)
                    r.admitted = now()
                    used += r.bytes
                    th = threading.Thread(target=worker, args=(r,), daemon=True)
                    running[r.rid] = (r, th)
                    th.start()
                if queue and not running and queue[0].bytes > self.hbm_budget:
                    r = queue.pop(0)
                    r.error = "exceeds the memory budget"
                    r.finished = now()
                    finished.append(r)
            self.log.append({"t": round(now(), 4), "queued": len(queue), "running": len(running),
                             "hbm_used": used})
            time.sleep(0.002)
        wall = now()
        finished = [m for r in finished for m in (r.members if isinstance(r, Batch) else [r])]
        ok = [r for r in finished if r.error is None]
        tts = sorted((r.finished - r.arrival * time_scale) for r in ok)
        dof_steps = sum(3 * r.N * r.N * (r.k + 1) ** 2 * r.steps for r in ok)

        def pct(p):
            return tts[min(len(tts) - 1, max(0, math.ceil(p * len(tts)) - 1))] if tts else None

        return {"requests": len(finished), "completed": len(ok), "wall_s": wall,
                "throughput_dof_steps_per_s": dof_steps / wall if wall > 0 else None,
                "tts_p50_s": pct(0.5), "tts_p99_s": pct(0.99),
                "max_running": max((e["running"] for e in self.log), default=0),
                "max_queued": max((e["queued"] for e in self.log), default=0),
                "errors": [r.error for r in finished if r.error]}
