"""Continuous-batching search server on one GPU.

Systems (determinants, coefficients, E0, integrals) are registered once and
stay resident on the device.  Requests name a system and (C, N) and are
admitted in arrival order as soon as a slot is free and their device-memory
footprint fits the budget; admitted searches run concurrently, each on its
own CUDA stream from its own worker thread, so requests that arrive while
others are on the GPU join them as slots and memory free up.  Each search
caps its constraint batches to its memory share, so a result does not depend
on what else is running (the batch size does not change any output).
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import search as _search, FP64

__all__ = ["Server", "footprint"]


def footprint(norb: int, ndets: int, C: int, N: int, batch_pairs: int) -> int:
    """Upper estimate of one search's device bytes beyond its resident inputs:
    the staging of one constraint batch (16-byte pairs, 1.5 slots each, and the
    alpha word), item lists, the candidate pool (two buffers of N + 2^29 entries
    at most, 16 bytes each), the psi hash and routing, and the integral tables."""
    staging = 28 * batch_pairs
    pool = 32 * (N + min(batch_pairs, 1 << 29))
    psi = 48 * ndets
    tables = 40 * norb ** 4
    items = 64 * C * (1 + norb * norb)
    return int(staging + pool + psi + tables + items + (64 << 20))


class Server:
    """Search requests against resident systems, continuously batched.

    ``slots``: searches in flight at most; ``budget``: device bytes the running
    searches may hold together (default: half the free memory at start);
    ``search_fn``: the search call (the library's by default; tests may pass a
    stand-in with the same signature).
    """

    def __init__(self, slots: int = 8, budget: int | None = None, search_fn=None):
        import torch
        self._torch = torch
        self._fn = search_fn or _search
        if budget is None:
            free, _ = torch.cuda.mem_get_info()
            budget = free // 2
        self.budget = int(budget)
        self.slots = int(slots)
        self._systems = {}
        self._pending = collections.deque()
        self._cv = threading.Condition()
        self._in_use = 0
        self._running = 0
        self._closed = False
        self.peak_bytes = 0
        self.peak_running = 0
        self.cancelled = 0  # requests withdrawn before admission
        self._workers = [threading.Thread(target=self._work, daemon=True) for _ in range(slots)]
        for t in self._workers:
            t.start()

    # -------------------------------------------------------------- systems ---
    def register(self, name, dets, coeffs, E0, h1, eri, ecore):
        """Keep a system resident (inputs are copied to the device once)."""
        torch = self._torch
        dev = torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu")

        def dv(x, dt):
            return x.to(dev) if hasattr(x, "to") else torch.tensor(np.asarray(x), dtype=dt, device=dev)

        d = dets if hasattr(dets, "to") else torch.tensor(np.asarray(dets).astype(np.int64))
        h = dv(h1, torch.float64)
        self._systems[name] = dict(dets=d.to(dev), coeffs=dv(coeffs, torch.float64), E0=float(E0),
                                   h1=h, eri=dv(eri, torch.float64), ecore=float(ecore),
                                   norb=int(round(h.numel() ** 0.5)), ndets=int(d.shape[0]))

    # ------------------------------------------------------------- requests ---
    def submit(self, name, C: int, N: int, precision: int = FP64, batch_pairs: int = 1 << 26):
        """Queue a search of system ``name``; returns a Future of
        (dets, scores, stats, latency_s) with latency from submission.  A
        request still in the queue is withdrawn by the future's cancel()
        (which then returns True); one already admitted runs to its end."""
        sy = self._systems[name]
        fp = footprint(sy["norb"], sy["ndets"], C, N, batch_pairs)
        if fp > self.budget:
            raise ValueError(f"request needs {fp} bytes, more than the budget {self.budget}")
        fut = Future()
        fut.add_done_callback(self._on_done)
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            self._pending.append((name, C, N, precision, batch_pairs, fp, fut, time.perf_counter()))
            self._cv.notify_all()
        return fut

    def _on_done(self, fut):
        # a withdrawn request may have been the one holding up the queue
        if fut.cancelled():
            with self._cv:
                self._cv.notify_all()

    def close(self):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for t in self._workers:
            t.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- workers ---
    def _next(self):
        """The oldest pending request, once it fits the budget (arrival order:
        a large request is not overtaken indefinitely)."""
        with self._cv:
            while True:
                # withdrawn requests leave the queue without taking a slot
                while self._pending and self._pending[0][6].cancelled():
                    self._pending.popleft()
                    self.cancelled += 1
                if self._pending:
                    fp = self._pending[0][5]
                    if self._in_use + fp <= self.budget:
                        req = self._pending.popleft()
                        if not req[6].set_running_or_notify_cancel():  # withdrawn just now
                            self.cancelled += 1
                            continue
                        self._in_use += fp
                        self._running += 1
                        self.peak_bytes = max(self.peak_bytes, self._in_use)
                        self.peak_running = max(self.peak_running, self._running)
                        return req
                elif self._closed:
                    return None
                self._cv.wait()

    def _work(self):
        torch = self._torch
        stream = torch.cuda.Stream() if torch.cuda.is_available() else None
        while True:
            req = self._next()
            if req is None:
                return
            name, C, N, prec, bp, fp, fut, t0 = req
            sy = self._systems[name]
            try:
                if stream is not None:
                    with torch.cuda.stream(stream):
                        od, osc, st = self._fn(sy["dets"], sy["coeffs"], sy["E0"], sy["h1"],
                                               sy["eri"], sy["ecore"], C, N, precision=prec,
                                               max_batch_pairs=bp, stream=stream)
                        stream.synchronize()
                else:
                    od, osc, st = self._fn(sy["dets"], sy["coeffs"], sy["E0"], sy["h1"], sy["eri"],
                                           sy["ecore"], C, N, precision=prec, max_batch_pairs=bp,
                                           stream=None)
                fut.set_result((od, osc, st, time.perf_counter() - t0))
            except Exception as e:  # reported through the future
                fut.set_exception(e)
            finally:
                with self._cv:
                    self._in_use -= fp
                    self._running -= 1
                    self._cv.notify_all()
