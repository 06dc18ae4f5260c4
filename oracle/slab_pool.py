"""Whole-grid oracle steps evaluated slab by slab on a pool of worker processes.

TEST INFRASTRUCTURE ONLY (see the package docstring): the test suite and the
benchmark's CPU-baseline legs use it to step grids too large for one core, such
as the 256^3 head-on collision, in bounded time and memory.

It adds no arithmetic to the oracle.  A step is the oracle's own ``step`` taken
apart along its stages:
  * the potential (Sec. 2.3) is ``solve_poisson`` of the whole grid and the step
    size is ``cfl_dt`` of the whole grid (reading s10), both in the parent;
  * the Eulerian stage, Lagrangian stage and energy balance (Sec. 2.1, 2.2, 2.4)
    are ``advance_window(zslab=(k0, k1))`` on z-slabs, one slab per task.  The new
    value of a cell depends only on cells within L1 distance 2, so a slab cut
    with a margin of two planes (wrapped on a periodic grid, clamped on an outflow
    grid) reproduces ``advance`` on the whole grid exactly, and the slabs together
    are the whole new state;
  * the signal speed of the new state is ``max_signal_speed`` of the whole grid.

The state lives in shared memory (one block for the input state, one for the
output, one for the potential), so a task moves only its slab indices.  The pool
is started with the ``spawn`` method: workers import numpy and the oracle only,
never a CUDA context, so the pool may be created in a process that already uses
the GPU.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import flic_oracle as O

__all__ = ["SlabPool", "host_cores"]


def host_cores() -> int:
    """Cores this process may run on (affinity mask), else the machine's count."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# worker side
# ---------------------------------------------------------------------------
_W = {}


def _attach(names, shape):
    _W.clear()
    nf = len(O.FIELDS)
    for key, name in names.items():
        shm = shared_memory.SharedMemory(name=name)
        n = nf if key in ("a", "b") else (2 if key == "kap" else 1)
        _W[key] = (shm, np.ndarray((n,) + tuple(shape), dtype=np.float64, buffer=shm.buf))


def _slab_task(args):
    src, dst, k0, k1, tau, prm = args
    a = _W[src][1]
    b = _W[dst][1]
    phi = _W["phi"][1][0]
    kap = _W["kap"][1]
    st = {f: a[i] for i, f in enumerate(O.FIELDS)}
    new, kp = O.advance_window(st, phi, tau, prm, zslab=(k0, k1))
    for i, f in enumerate(O.FIELDS):
        b[i, k0:k1] = new[f]
    kap[0, k0:k1] = kp["kappa_gas"]
    kap[1, k0:k1] = kp["kappa_bme"]
    return k1 - k0


# ---------------------------------------------------------------------------
# parent side
# ---------------------------------------------------------------------------
class SlabPool:
    """Steps one grid of ``shape`` (nz, ny, nx) with ``workers`` processes.

    ``slab``: z planes per task (default: the grid split into about two tasks
    per worker, at least 4 planes each).  Use as a context manager, or call
    ``close()``.
    """

    def __init__(self, shape, workers: int | None = None, slab: int | None = None):
        self.shape = tuple(int(s) for s in shape)
        nz = self.shape[0]
        self.workers = max(1, int(workers or host_cores()))
        if slab is None:
            slab = max(4, math.ceil(nz / (2 * self.workers)))
        self.slab = max(1, min(int(slab), nz))
        cells = int(np.prod(self.shape))
        nf = len(O.FIELDS)
        sizes = {"a": nf * cells, "b": nf * cells, "phi": cells, "kap": 2 * cells}
        self._shm = {k: shared_memory.SharedMemory(create=True, size=8 * v) for k, v in sizes.items()}
        self._arr = {}
        for k, shm in self._shm.items():
            n = sizes[k] // cells
            self._arr[k] = np.ndarray((n,) + self.shape, dtype=np.float64, buffer=shm.buf)
        self.cur = "a"
        ctx = mp.get_context("spawn")
        names = {k: s.name for k, s in self._shm.items()}
        self._pool = ctx.Pool(self.workers, initializer=_attach, initargs=(names, self.shape))

    # -- state access ----------------------------------------------------------
    def state_view(self, which: str | None = None) -> dict:
        """The current state as a dict of views into shared memory."""
        a = self._arr[which or self.cur]
        return {f: a[i] for i, f in enumerate(O.FIELDS)}

    def load(self, st: dict):
        a = self._arr[self.cur]
        for i, f in enumerate(O.FIELDS):
            a[i] = st[f]

    def state(self) -> dict:
        """A copy of the current state."""
        return {f: v.copy() for f, v in self.state_view().items()}

    # -- one step ----------------------------------------------------------------
    def step(self, prm: O.Params, dt: float | None = None, with_kappa: bool = False) -> dict:
        """Advances the current state by one step of the oracle; returns a record
        with the step size ``dt``, the signal speed ``vmax`` of the new state and,
        if asked, the kappa sums (plain float64 sums)."""
        st = self.state_view()
        phi = O.solve_poisson(st, prm)
        self._arr["phi"][0] = phi
        tau = dt if (dt is not None and dt > 0.0) else O.cfl_dt(st, prm)
        nxt = "b" if self.cur == "a" else "a"
        nz = self.shape[0]
        tasks = [(self.cur, nxt, k0, min(k0 + self.slab, nz), tau, prm) for k0 in range(0, nz, self.slab)]
        done = sum(self._pool.map(_slab_task, tasks, chunksize=1))
        if done != nz:
            raise RuntimeError(f"slab tasks covered {done} of {nz} planes")
        self.cur = nxt
        new = self.state_view()
        rec = {"dt": tau, "vmax": O.max_signal_speed(new, prm)}
        if with_kappa:
            rec["kappa_gas"] = float(np.sum(self._arr["kap"][0]))
            rec["kappa_bme"] = float(np.sum(self._arr["kap"][1]))
        return rec

    def run(self, st: dict, prm: O.Params, nsteps: int, dt: float | None = None):
        """``nsteps`` steps from ``st``; returns (copy of the final state, records)."""
        self.load(st)
        recs = [self.step(prm, dt) for _ in range(nsteps)]
        return self.state(), recs

    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None
        self._arr = {}
        for shm in self._shm.values():
            shm.close()
            shm.unlink()
        self._shm = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
