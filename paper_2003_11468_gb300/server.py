"""Continuous-batching Friends-of-Friends server over the C ABI.

The paper runs FoF on-the-fly at fixed intervals of a simulation (Sec. 1)
and its users analyse many snapshots; a GPU serving such jobs sees requests
of very different sizes arriving at random times.  This server

* queues requests as they arrive (`submit` returns a Future);
* admits waiting requests, oldest first, while a slot (CUDA stream) is free
  and the device memory all slots hold stays within the budget; requests
  admitted together form one batch plan (`fof_batch_create` with a
  caller-owned workspace), so small jobs share one set of launches; each slot
  keeps its device and pinned host buffers and only grows them, so
  steady-state serving allocates nothing.  The budget covers what the slots
  keep (workspace from `fof_batch_workspace_bytes` plus input/output buffers,
  with the growth margin), idle or busy: a batch goes to the free slot that
  needs the least growth, and idle slots give their buffers back when a
  batch would otherwise not fit;
* runs each batch on its slot's stream (H2D copy, `fof_link`,
  `fof_groups_async`, D2H copy of each request's ids and sizes straight
  into that request's own pinned host arrays), so batches on different
  slots overlap on the device and the host copies nothing;
* polls completion events and hands finished batches to a completion
  thread, which reads the status and the catalogue (`fof_result`),
  resolves the futures and only then returns the slot; the scheduler
  meanwhile keeps admitting and launching.

Results are exactly those of a solo run (the partition is unique).  Memory
comes from PyTorch's caching allocators (device and pinned host), the only
allocators used; result arrays return to the host cache once dropped.
"""
from __future__ import annotations

import collections
import os
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
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


# device bytes per particle of a slot's input/output buffers: positions
# (12), ids (4), sizes (4), catalogue rows (8)
_IO_BYTES = 28


class _SlotBuffers:
    """Device and pinned host buffers of one slot, grown on demand and kept,
    so that steady-state serving allocates nothing.  held() is the device
    memory the slot keeps whether or not a batch runs on it; the server's
    budget covers the sum over all slots."""

    GROW = 1.25

    def __init__(self, device):
        self.device = device
        self.cap_ws = 0
        self.cap_n = 0
        self.ws = self.pos = self.ids = self.sizes = self.cat = None

    @staticmethod
    def _ws_cap(ws_bytes):
        return int(ws_bytes * _SlotBuffers.GROW) + 4096

    @staticmethod
    def _n_cap(n):
        return int(n * _SlotBuffers.GROW) + 1024

    def held(self) -> int:
        ws = self.cap_ws + 256 if self.cap_ws else 0
        return ws + _IO_BYTES * self.cap_n

    def held_after(self, ws_bytes, total) -> int:
        """Device bytes the slot holds after ensure(ws_bytes, total)."""
        cw = self.cap_ws if ws_bytes <= self.cap_ws else self._ws_cap(ws_bytes)
        cn = self.cap_n if max(total, 1) <= self.cap_n else self._n_cap(max(total, 1))
        return (cw + 256 if cw else 0) + _IO_BYTES * cn

    def release(self):
        self.ws = self.pos = self.ids = self.sizes = self.cat = None
        self.cap_ws = self.cap_n = 0

    def ensure(self, ws_bytes, total):
        import torch
        if ws_bytes > self.cap_ws:
            self.ws = None
            self.cap_ws = self._ws_cap(ws_bytes)
            self.ws = torch.empty(self.cap_ws + 256, dtype=torch.uint8, device=self.device)
        n = max(total, 1)
        if n > self.cap_n:
            self.pos = self.ids = self.sizes = self.cat = None
            self.cap_n = self._n_cap(n)
            c = self.cap_n
            self.pos = torch.empty((c, 3), dtype=torch.float32, device=self.device)
            self.ids = torch.empty(c, dtype=torch.int32, device=self.device)
            self.sizes = torch.empty(c, dtype=torch.int32, device=self.device)
            self.cat = torch.empty((c, 2), dtype=torch.int32, device=self.device)

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
            # each request's ids and sizes go straight into its own pinned
            # host arrays (PyTorch's caching host allocator recycles them
            # once the caller drops the result): no host-side copy
            self.outs = []
            for r, o in zip(self.reqs, self.offsets[:-1]):
                n = r.pos.shape[0]
                ids_r = torch.empty(n, dtype=torch.int32, pin_memory=True)
                sizes_r = torch.empty(n, dtype=torch.int32, pin_memory=True)
                if n:
                    ids_r.copy_(b.ids[o:o + n], non_blocking=True)
                    sizes_r.copy_(b.sizes[o:o + n], non_blocking=True)
                self.outs.append((ids_r, sizes_r))
            self.event.record(self.stream)

    def finish(self):
        code, ng, nk = fof.fof_result(self.h, len(self.reqs), self.stream)
        cat = self.b.cat[: int(sum(nk))].cpu().numpy()     # only the rows that exist
        now = time.perf_counter()
        k0 = 0
        for i, r in enumerate(self.reqs):
            rows = cat[k0:k0 + nk[i]]
            k0 += nk[i]
            rows = rows[rows[:, 1] >= max(r.min_size, 1)].copy()
            ids_r, sizes_r = self.outs[i]
            r.future.set_result(Result(ids_r.numpy(), sizes_r.numpy(), rows, ng[i], now - r.t_arrive))
        self.outs = None
        fof.fof_destroy(self.h)
        self.h = None


class Server:
    """Continuous-batching FoF server on one GPU.

    memory_budget: device bytes the server may hold for admitted work.
    slots: concurrent batches (one CUDA stream each).
    max_batch_boxes / max_batch_particles: limits of one batch plan.
    prealloc: optional (box, l_x, n) of the largest batch expected; every
    slot's buffers are sized for it up front.
    """

    def __init__(self, memory_budget: int = 120 << 30, slots: int = 3, max_batch_boxes: int = 64,
                 max_batch_particles: int = 1 << 27, device: int = 0, prealloc=None):
        import torch
        fof.load()
        self.device = torch.device("cuda", device)
        self.budget = int(memory_budget)
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

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- scheduler -------------------------------------------------------
    def held_bytes(self) -> int:
        """Device memory all slots keep (the quantity the budget bounds)."""
        return sum(b.held() for b in self.buffers)

    def _fit(self, ws, total):
        """A free slot that can take a batch of (ws, total) within the budget,
        releasing idle slots' buffers if needed; None if it cannot fit now."""
        busy = [s for s in range(len(self.buffers)) if s not in self.free_slots]
        busy_bytes = sum(self.buffers[s].held() for s in busy)
        idle = list(self.free_slots)
        # the free slot that grows least
        slot = min(idle, key=lambda s: self.buffers[s].held_after(ws, total) - self.buffers[s].held())
        after = self.buffers[slot].held_after(ws, total)
        others = sum(self.buffers[s].held() for s in idle if s != slot)
        if busy_bytes + others + after <= self.budget:
            return slot, []
        # idle slots (and the chosen one's old buffers) can be given back
        fresh = _SlotBuffers._ws_cap(ws) + 256 + _IO_BYTES * _SlotBuffers._n_cap(max(total, 1))
        if busy_bytes + min(after, fresh) <= self.budget:
            drop = [s for s in idle if s != slot]
            if after > fresh:
                drop.append(slot)
            return slot, drop
        return None

    def _admit(self):
        """Form one batch from the head of the queue if memory and a slot allow."""
        if not self.free_slots or not self.waiting:
            return None
        take, ws, total, choice = [], 0, 0, None
        for req in self.waiting:
            n = req.pos.shape[0]
            if take and (len(take) >= self.max_boxes or total + n > self.max_particles):
                break
            w1 = fof.fof_batch_workspace_bytes([req.box], [req.l_x], [n])
            if w1 == 0:
                w1 = 0                              # invalid geometry: fails in _Batch
            # a batch's workspace is at most the sum of its boxes' plus alignment
            c = self._fit(ws + w1 + 4096, total + n)
            if c is None:
                break
            take.append(req)
            ws += w1 + 4096
            total += n
            choice = c
        if not take:
            if not self.running and not self.finishing and self.waiting:
                # a single request larger than the budget can never run
                req = self.waiting.popleft()
                req.future.set_exception(MemoryError("request exceeds the memory budget"))
            return None
        for _ in take:
            self.waiting.popleft()
        slot, drop = choice
        if drop:
            import torch
            for s in drop:
                self.buffers[s].release()
            torch.cuda.empty_cache()               # hand the memory back to the device
        self.free_slots.remove(slot)
        try:
            batch = _Batch(take, slot, self.streams[slot], self.buffers[slot])
        except Exception as e:                      # geometry errors: fail those requests
            self.free_slots.append(slot)
            for r in take:
                r.future.set_exception(e)
            return None
        batch.launch()
        return batch

    def _complete(self, b):
        """Completion thread: results out, futures resolved, slot returned."""
        try:
            b.finish()
        except Exception as e:                      # a failed batch fails its requests
            for r in b.reqs:
                if not r.future.done():
                    r.future.set_exception(e)
        with self.lock:
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
