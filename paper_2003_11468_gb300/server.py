"""Continuous-batching Friends-of-Friends server over the C ABI.

The paper runs FoF on-the-fly at fixed intervals of a simulation (Sec. 1)
and its users analyse many snapshots; a GPU serving such jobs sees requests
of very different sizes arriving at random times.  This server

* queues requests as they arrive (`submit` returns a Future);
* admits waiting requests, oldest first, while device memory (workspace from
  `fof_batch_workspace_bytes` plus input/output buffers) fits the budget and
  a slot (CUDA stream) is free; requests admitted together form one batch
  plan (`fof_batch_create` with a caller-owned workspace), so small jobs share
  one set of launches; each slot keeps its device and pinned host buffers
  and only grows them, so steady-state serving allocates nothing;
* runs each batch on its slot's stream (H2D copy, `fof_link`,
  `fof_groups_async`, D2H copy of ids, sizes and the catalogue), so batches
  on different slots overlap on the device;
* polls completion events and hands finished batches to a completion
  thread, which reads the status (`fof_result`), copies each request's
  results out of the slot's pinned buffers with a pool of host threads,
  resolves the futures and only then returns the slot and the batch's share
  of the budget; the scheduler meanwhile keeps admitting and launching.

Results are exactly those of a solo run (the partition is unique).  Memory
comes from PyTorch's caching allocator, the only allocator used.
"""
from __future__ import annotations

import collections
import os
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor, wait
from dataclasses import dataclass, field

import numpy as np

from . import fof


@dataclass
class Request:
    pos: object                   # float32 [n, 3], host (pinned torch tensor or numpy)
    box: float
    l_x: float
    min_size: int = 1
    t_arrive: float = field(default_factory=time.perf_counter)
    future: Future = field(default_factory=Future)


@dataclass
class Result:
    ids: np.ndarray
    sizes: np.ndarray
    catalogue: np.ndarray         # [k, 2] (label, size), ascending label
    n_groups: int
    latency_s: float


class _SlotBuffers:
    """Device and pinned host buffers of one slot, grown on demand and kept,
    so that steady-state serving allocates nothing."""

    def __init__(self, device):
        self.device = device
        self.cap_ws = 0
        self.cap_n = 0
        self.ws = self.pos = self.ids = self.sizes = self.cat = None
        self.ids_h = self.sizes_h = None

    def ensure(self, ws_bytes, total):
        import torch
        if ws_bytes > self.cap_ws:
            self.ws = None
            self.cap_ws = int(ws_bytes * 1.25) + 4096
            self.ws = torch.empty(self.cap_ws + 256, dtype=torch.uint8, device=self.device)
        n = max(total, 1)
        if n > self.cap_n:
            self.pos = self.ids = self.sizes = self.cat = self.ids_h = self.sizes_h = None
            self.cap_n = int(n * 1.25) + 1024
            c = self.cap_n
            self.pos = torch.empty((c, 3), dtype=torch.float32, device=self.device)
            self.ids = torch.empty(c, dtype=torch.int32, device=self.device)
            self.sizes = torch.empty(c, dtype=torch.int32, device=self.device)
            self.cat = torch.empty((c, 2), dtype=torch.int32, device=self.device)
            self.ids_h = torch.empty(c, dtype=torch.int32).pin_memory()
            self.sizes_h = torch.empty(c, dtype=torch.int32).pin_memory()

    def ws_ptr(self):
        return (self.ws.data_ptr() + 255) // 256 * 256


class _Batch:
    def __init__(self, reqs, slot, stream, bufs: _SlotBuffers):
        self.reqs = reqs
        self.slot = slot
        self.stream = stream
        ns = [r.pos.shape[0] for r in reqs]
        self.ns = ns
        self.total = int(sum(ns))
        self.offsets = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        boxes = [r.box for r in reqs]
        lxs = [r.l_x for r in reqs]
        self.ws_bytes = fof.fof_batch_workspace_bytes(boxes, lxs, ns)
        if self.ws_bytes == 0:
            raise ValueError("invalid request geometry")
        bufs.ensure(self.ws_bytes, self.total)
        self.b = bufs
        self.h = fof.fof_batch_create(boxes, lxs, ns, None, bufs.ws_ptr(), self.ws_bytes)
        self.min_size = min(r.min_size for r in reqs)
        import torch
        self.event = torch.cuda.Event()

    @staticmethod
    def io_bytes(n):
        return 12 * n + 8 * n + 8 * n

    def launch(self):
        import torch
        b, t = self.b, self.total
        with torch.cuda.stream(self.stream):
            for r, o in zip(self.reqs, self.offsets[:-1]):
                n = r.pos.shape[0]
                if n:
                    src = r.pos if hasattr(r.pos, "is_pinned") else torch.from_numpy(np.ascontiguousarray(r.pos))
                    b.pos[o:o + n].copy_(src, non_blocking=True)
            fof.fof_link(self.h, b.pos, self.stream)
            fof.fof_groups_async(self.h, b.ids, b.sizes, b.cat, t, self.min_size, self.stream)
            b.ids_h[:t].copy_(b.ids[:t], non_blocking=True)
            b.sizes_h[:t].copy_(b.sizes[:t], non_blocking=True)
            self.event.record(self.stream)

    # elements per host copy task: large enough to amortise the task, small
    # enough to spread one big request over the copy threads
    COPY_CHUNK = 1 << 22

    def finish(self, copy_pool):
        code, ng, nk = fof.fof_result(self.h, len(self.reqs), self.stream)
        b = self.b
        ids = b.ids_h.numpy()
        sizes = b.sizes_h.numpy()
        cat = b.cat[: int(sum(nk))].cpu().numpy()     # only the rows that exist
        outs = [(np.empty(n, np.int32), np.empty(n, np.int32)) for n in self.ns]

        def copy(i, a, e):
            o = int(self.offsets[i])
            outs[i][0][a:e] = ids[o + a:o + e]
            outs[i][1][a:e] = sizes[o + a:o + e]

        tasks = [copy_pool.submit(copy, i, a, min(a + self.COPY_CHUNK, n))
                 for i, n in enumerate(self.ns) for a in range(0, n, self.COPY_CHUNK)]
        wait(tasks)
        for t in tasks:
            t.result()
        now = time.perf_counter()
        k0 = 0
        for i, r in enumerate(self.reqs):
            rows = cat[k0:k0 + nk[i]]
            k0 += nk[i]
            rows = rows[rows[:, 1] >= max(r.min_size, 1)].copy()
            r.future.set_result(Result(outs[i][0], outs[i][1], rows, ng[i], now - r.t_arrive))
        fof.fof_destroy(self.h)
        self.h = None


class Server:
    """Continuous-batching FoF server on one GPU.

    memory_budget: device bytes the server may hold for admitted work.
    slots: concurrent batches (one CUDA stream each).
    max_batch_boxes / max_batch_particles: limits of one batch plan.
    prealloc: optional (box, l_x, n) of the largest batch expected; every
    slot's buffers are sized for it up front.
    copy_threads: host threads that copy results out of the slot buffers.
    """

    def __init__(self, memory_budget: int = 120 << 30, slots: int = 3, max_batch_boxes: int = 64,
                 max_batch_particles: int = 1 << 27, device: int = 0, prealloc=None,
                 copy_threads: int | None = None):
        import torch
        fof.load()
        self.device = torch.device("cuda", device)
        self.budget = int(memory_budget)
        self.in_use = 0
        self.max_boxes = max_batch_boxes
        self.max_particles = max_batch_particles
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.buffers = [_SlotBuffers(self.device) for _ in range(slots)]
        if prealloc is not None:
            # (box, l_x, n) of the largest expected batch: size every slot now
            box, l_x, n = prealloc
            ws = fof.fof_batch_workspace_bytes([box], [l_x], [n])
            for b in self.buffers:
                b.ensure(ws, n)
        self.free_slots = list(range(slots))
        self.waiting = collections.deque()
        self.running = []
        self.finishing = 0
        nthr = copy_threads or max(1, min(8, (os.cpu_count() or 2) // 2))
        self.copy_pool = ThreadPoolExecutor(max_workers=nthr)
        self.completer = ThreadPoolExecutor(max_workers=1, initializer=torch.cuda.set_device,
                                            initargs=(self.device,))
        self.lock = threading.Condition()
        self.stop_flag = False
        self.latencies = []
        self.completed_particles = 0
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # -- public ----------------------------------------------------------
    def submit(self, pos, box: float, l_x: float, min_size: int = 1) -> Future:
        req = Request(pos, float(box), float(l_x), int(min_size))
        with self.lock:
            self.waiting.append(req)
            self.lock.notify()
        return req.future

    def close(self):
        with self.lock:
            self.stop_flag = True
            self.lock.notify()
        self.thread.join()
        self.completer.shutdown(wait=True)
        self.copy_pool.shutdown(wait=True)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- scheduler -------------------------------------------------------
    def _need_bytes(self, req):
        n = req.pos.shape[0]
        ws = fof.fof_batch_workspace_bytes([req.box], [req.l_x], [n])
        return ws + _Batch.io_bytes(n) + 4096

    def _admit(self):
        """Form one batch from the head of the queue if memory and a slot allow."""
        if not self.free_slots or not self.waiting:
            return None
        take, need, total = [], 0, 0
        for req in self.waiting:
            b = self._need_bytes(req)
            n = req.pos.shape[0]
            if take and (len(take) >= self.max_boxes or total + n > self.max_particles):
                break
            if self.in_use + need + b > self.budget:
                break
            take.append(req)
            need += b
            total += n
        if not take:
            if not self.running and not self.finishing and self.waiting:
                # a single request larger than the budget can never run
                req = self.waiting.popleft()
                req.future.set_exception(MemoryError("request exceeds the memory budget"))
            return None
        for _ in take:
            self.waiting.popleft()
        slot = self.free_slots.pop()
        try:
            batch = _Batch(take, slot, self.streams[slot], self.buffers[slot])
        except Exception as e:                      # geometry errors: fail those requests
            self.free_slots.append(slot)
            for r in take:
                r.future.set_exception(e)
            return None
        batch.reserved = need
        self.in_use += need
        batch.launch()
        return batch

    def _complete(self, b):
        """Completion thread: results out, futures resolved, slot returned."""
        try:
            b.finish(self.copy_pool)
        except Exception as e:                      # a failed batch fails its requests
            for r in b.reqs:
                if not r.future.done():
                    r.future.set_exception(e)
        with self.lock:
            self.in_use -= b.reserved
            self.free_slots.append(b.slot)
            self.finishing -= 1
            for r in b.reqs:
                if r.future.exception() is None:
                    self.latencies.append(r.future.result().latency_s)
            self.completed_particles += b.total
            self.lock.notify()

    def _loop(self):
        import torch
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                if self.stop_flag and not self.waiting and not self.running and not self.finishing:
                    return
                while True:
                    b = self._admit()
                    if b is None:
                        break
                    self.running.append(b)
                if not self.running and (not self.waiting or self.finishing):
                    self.lock.wait(timeout=0.05)
                    continue
            done = [b for b in self.running if b.event.query()]
            for b in done:
                with self.lock:
                    self.running.remove(b)
                    self.finishing += 1
                self.completer.submit(self._complete, b)
            if not done:
                time.sleep(0.0002)
