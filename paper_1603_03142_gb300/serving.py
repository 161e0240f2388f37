"""Open-loop client of the request loop (sgf_server_* in libsgf).

A stream of force requests arrives at seeded Poisson times; each is submitted
to the server when its arrival time has come, and the server admits it as soon
as a slot and device memory allow (continuous batching: requests that arrive
while others run join them on the device).  Densities come from a per-shape
pool of pinned host arrays (one concentric nest problem per shape); forces go
to pinned host buffers that are recycled when their request completes.

Latency of a request = the server-clock time its completion was seen minus its
arrival time: queueing, admission, copies in and out and the solve.  This
module only drives the server and summarises; every solve runs in libsgf.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import sgf
from . import workloads as W


def pinned(shape, dtype) -> np.ndarray:
    """A page-locked host array (through torch's pinned allocator); a plain host
    array where no CUDA device exists (a simulating server touches no buffer)."""
    import torch
    if not torch.cuda.is_available():
        return np.empty(shape, dtype=dtype)
    tdt = torch.float64 if np.dtype(dtype) == np.float64 else torch.float32
    return torch.empty(shape, dtype=tdt, pin_memory=True).numpy()


@dataclass
class Arrival:
    t: float          # seconds after the stream starts
    n: int
    levels: int
    precision: str
    seed: int


def poisson_arrivals(rate: float, duration: float, seed: int, sizes: Sequence[int],
                     levels: Tuple[int, int], precisions: Sequence[str] = ("fp32",)) -> List[Arrival]:
    """Seeded Poisson process of rate `rate` over [0, duration): shape n ~ U(sizes),
    levels ~ U{levels[0]..levels[1]}, precision ~ U(precisions)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        n = int(rng.choice(list(sizes)))
        L = int(rng.integers(levels[0], levels[1] + 1))
        prec = str(rng.choice(list(precisions)))
        out.append(Arrival(t, n, L, prec, int(rng.integers(0, 2 ** 31 - 1))))


@dataclass
class ShapePool:
    nest: object
    precision: str
    sigma: List[np.ndarray]
    free: List[Tuple[List[np.ndarray], List[np.ndarray]]] = field(default_factory=list)

    def take(self):
        if self.free:
            return self.free.pop()
        dt = np.float64 if self.precision == "fp64" else np.float32
        n, L = self.nest.n, self.nest.levels
        return [pinned((n, n), dt) for _ in range(L)], [pinned((n, n), dt) for _ in range(L)]


def make_pools(shapes, seed: int = 0) -> Dict[tuple, ShapePool]:
    """One concentric nest problem (Maclaurin disk + clumps) per (n, levels, precision)."""
    pools = {}
    for k, (n, L, prec) in enumerate(sorted(set(shapes))):
        rng = np.random.Generator(np.random.PCG64(seed + 7919 * k))
        nest, sig = W.random_nest_problem(rng, n, L)
        dt = np.float64 if prec == "fp64" else np.float32
        arrs = []
        for s in sig:
            a = pinned((n, n), dt)
            a[...] = s
            arrs.append(a)
        pools[(n, L, prec)] = ShapePool(nest, prec, arrs)
    return pools


@dataclass
class Record:
    id: int
    n: int
    levels: int
    precision: str
    t_arrival: float   # server clock
    status: int = -1
    t_admit: float = 0.0
    t_done: float = 0.0
    built_shape: bool = False

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def run_stream(server: "sgf.Server", arrivals: Sequence[Arrival], pools: Dict[tuple, ShapePool],
               poll_s: float = 2e-4, id_base: int = 0, keep_outputs: bool = False,
               max_seconds: Optional[float] = None):
    """Release the arrivals at their times, drive the server until every accepted
    request has completed.  Returns (records, outputs) where outputs maps id ->
    (fx, fy) when keep_outputs (buffers are then not recycled)."""
    recs: Dict[int, Record] = {}
    bufs: Dict[int, tuple] = {}
    outputs = {}
    t0 = server.clock()
    i, pending = 0, 0
    deadline = None if max_seconds is None else t0 + max_seconds
    while i < len(arrivals) or pending:
        now = server.clock()
        while i < len(arrivals) and t0 + arrivals[i].t <= now:
            a = arrivals[i]
            rid = id_base + i
            pool = pools[(a.n, a.levels, a.precision)]
            fx, fy = pool.take()
            r = Record(rid, a.n, a.levels, a.precision, t0 + a.t)
            st = server.submit(rid, pool.nest, a.precision, pool.sigma, fx, fy)
            if st == sgf.SGF_OK:
                pending += 1
                bufs[rid] = (pool, fx, fy)
            else:
                r.status = st
                pool.free.append((fx, fy))
            recs[rid] = r
            i += 1
        done = server.progress()
        for c in done:
            r = recs[c["id"]]
            r.status, r.t_admit, r.t_done, r.built_shape = c["status"], c["t_admit"], c["t_done"], c["built_shape"]
            pool, fx, fy = bufs.pop(c["id"])
            if keep_outputs:
                outputs[c["id"]] = (fx, fy)
            else:
                pool.free.append((fx, fy))
            pending -= 1
        if deadline is not None and now > deadline:
            raise TimeoutError(f"stream not drained after {max_seconds} s ({pending} requests pending)")
        if not done:
            time.sleep(poll_s)
    return [recs[k] for k in sorted(recs)], outputs


def percentile(xs: Sequence[float], q: float) -> float:
    """Nearest-rank percentile (q in [0, 100]) of a non-empty sample."""
    s = sorted(xs)
    k = max(0, min(len(s) - 1, int(np.ceil(q / 100.0 * len(s))) - 1))
    return float(s[k])


def summarize(records: Sequence[Record], duration: float) -> dict:
    """Latency percentiles, served cells/s and offered vs achieved load of one stream."""
    ok = [r for r in records if r.status == sgf.SGF_OK]
    rejected = [r for r in records if r.status == sgf.SGF_ENOMEM]
    failed = [r for r in records if r.status not in (sgf.SGF_OK, sgf.SGF_ENOMEM)]
    if not ok:
        return {"completed": 0, "rejected": len(rejected), "failed": len(failed)}
    start = min(r.t_arrival for r in records)
    end = max(r.t_done for r in ok)
    span = end - start
    lat = [r.latency for r in ok]
    cells = sum(r.n * r.n * r.levels for r in ok)
    return {
        "completed": len(ok), "rejected": len(rejected), "failed": len(failed),
        "p50_ms": 1e3 * percentile(lat, 50), "p90_ms": 1e3 * percentile(lat, 90),
        "p99_ms": 1e3 * percentile(lat, 99), "max_ms": 1e3 * max(lat), "mean_ms": 1e3 * float(np.mean(lat)),
        "cells": cells, "span_s": span, "cells_per_s": cells / span,
        "offered_rps": len(records) / duration, "achieved_rps": len(ok) / span,
        "offered_cells_per_s": sum(r.n * r.n * r.levels for r in records) / duration,
    }
