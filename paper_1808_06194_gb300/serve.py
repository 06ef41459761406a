"""Serving loop: continuous batching of registration jobs over one GPU.

A job is one image pair.  The server keeps every admitted job's CFOG volumes
resident, admits waiting jobs in arrival order while the HBM budget allows,
and drains the control points of all resident jobs through batched matching
launches (`cfog_match_batched`, one persistent launch over a device job
table).  Admission work (host-to-device copy from pinned memory, CFOG of both
images, Harris CPs) runs on its own stream and overlaps the matching launch
in flight; a job's CPs join the next matching launch once its features are
ready.  Per-CP results depend only on the CP's own inputs and (N, r), so a
job's result is the same alone and in any mix.

Host-side bookkeeping (`Admission`, `CpRing`) is plain Python and is tested
without a GPU; `Server` drives the library through the C ABI.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import _lib as L


# ------------------------------------------------------------ host logic --

class Admission:
    """HBM budget ledger: admit in arrival order while the resident bytes fit."""

    def __init__(self, budget_bytes):
        self.budget = int(budget_bytes)
        self.resident = {}
        self.used = 0
        self.peak = 0

    def fits(self, nbytes):
        return self.used + nbytes <= self.budget

    def admit(self, key, nbytes):
        if nbytes > self.budget:
            raise ValueError(f"job needs {nbytes} bytes, more than the whole budget {self.budget}")
        if not self.fits(nbytes):
            raise RuntimeError("admission over budget")
        self.resident[key] = nbytes
        self.used += nbytes
        self.peak = max(self.peak, self.used)

    def release(self, key):
        self.used -= self.resident.pop(key)


class CpRing:
    """First-fit allocator of contiguous CP ranges in a fixed-size ring of slots."""

    def __init__(self, capacity):
        self.capacity = int(capacity)
        self.free = [(0, self.capacity)]   # sorted, non-overlapping (start, length)

    def alloc(self, n):
        for i, (s, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (s + n, ln - n)
                return s
        return None

    def release(self, start, n):
        self.free.append((start, n))
        self.free.sort()
        merged = []
        for s, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == s:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((s, ln))
        self.free = merged

    @property
    def free_slots(self):
        return sum(ln for _, ln in self.free)


@dataclasses.dataclass
class Job:
    """One registration request: a reference and a sensed image on the host."""
    ref: np.ndarray
    sen: np.ndarray
    tmpl: int = 64
    radius: int = 16
    cp_block: int = 64          # one CP per cp_block x cp_block block of the interior
    arrival: float = None       # seconds on the server clock (None: at submit)
    key: int = -1
    # filled by the server
    n_cp: int = 0
    cps: np.ndarray = None
    results: np.ndarray = None
    done_time: float = None

    @property
    def margin(self):
        return self.tmpl // 2 + self.radius + 8

    def grid(self):
        h, w = self.ref.shape
        gy = max(1, (h - 2 * self.margin) // self.cp_block)
        gx = max(1, (w - 2 * self.margin) // self.cp_block)
        return gx, gy


def job_bytes(job, m=9):
    """Device bytes a resident job holds: both images and both CFOG volumes."""
    h, w = job.ref.shape
    rp = (w + 31) // 32 * 32
    itemsize = job.ref.element_size() if hasattr(job.ref, "element_size") else job.ref.itemsize
    img = 2 * h * w * itemsize
    feats = 2 * (m + 1) * h * rp * 4
    gx, gy = job.grid()
    return img + feats + gx * gy * (8 + 24)


# ------------------------------------------------------------ GPU server --

def _pinned(torch, a):
    """A pinned host tensor for a numpy array or an (already pinned) CPU tensor."""
    if isinstance(a, torch.Tensor):
        return a if a.is_pinned() else a.pin_memory()
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


class Server:
    """Continuous-batching matcher over one device.

    submit(job) queues a job; step() admits, launches and retires work without
    blocking; results of finished jobs are collected by `finished`.
    tune_classes: the (N, r) classes the jobs will use; with the AUTO variant
    the server applies (or first measures) the autotuner's choices for them.
    """

    def __init__(self, device="cuda", hbm_budget=150 * 2**30, ring=1 << 20, max_batch=32768,
                 max_jobs=512, tmpl_max=96, radius_max=20, variant=L.CFOG_MATCH_VARIANT_AUTO,
                 precision=L.CFOG_PREC_FP32_FFT, clock=time.perf_counter, tune_classes=None):
        import torch
        from . import api
        self.torch, self.api = torch, api
        self.dev = torch.device(device)
        self.adm = Admission(hbm_budget)
        self.ring = CpRing(ring)
        self.max_batch = max_batch
        self.max_jobs = max_jobs
        self.tmpl_max, self.radius_max = tmpl_max, radius_max
        self.variant, self.precision = variant, precision
        self.clock = clock
        self.t0 = clock()
        self.s_admit = torch.cuda.Stream(self.dev)
        self.s_match = torch.cuda.Stream(self.dev)
        ti = dict(dtype=torch.int32, device=self.dev)
        self.cps = torch.zeros((ring, 2), **ti)
        self.tmpl = torch.zeros(ring, **ti)
        self.radius = torch.zeros(ring, **ti)
        self.job_of = torch.full((ring,), -1, **ti)
        self.res = torch.zeros((ring, 6), **ti)
        self.res_host = torch.zeros((ring, 6), dtype=torch.int32).pin_memory()
        self.cps_host = torch.zeros((ring, 2), dtype=torch.int32).pin_memory()
        # pinned staging for the per-CP (N, r, job slot) rows and the job table
        # entries: a job writes only its own ring range and slot, which are
        # not reused before the job retires, so no staging copy is overwritten
        # while in flight and nothing is pinned per job
        self.side_host = torch.zeros((3, ring), dtype=torch.int32).pin_memory()
        self.jobs_host = torch.zeros(max_jobs * L.ctypes.sizeof(L.cfog_job),
                                     dtype=torch.uint8).pin_memory()
        self.jobs_dev = torch.zeros(max_jobs * L.ctypes.sizeof(L.cfog_job), dtype=torch.uint8,
                                    device=self.dev)
        # two match launches may be queued at once, each with its own workspace
        self.max_inflight = 2
        self.ws = [api.match_workspace(max_batch, self.dev) for _ in range(self.max_inflight)]
        self.free_job_slots = list(range(max_jobs))[::-1]
        self.waiting = collections.deque()
        self.resident = {}          # key -> dict(job, slot, off, ready_event, tensors)
        self.pending = collections.deque()   # (key, start, n) CP ranges not yet matched
        self.inflight = collections.deque()  # (event, [(key, start, n)]), oldest first
        self.finished = []
        self.next_key = 0
        self.launches = 0
        # AUTO runs the autotuner's variant and plans for the expected classes
        # (cached per GPU and library build; tuned once when absent)
        self.tuning = None
        if tune_classes and variant == L.CFOG_MATCH_VARIANT_AUTO:
            from . import autotune
            self.tuning = autotune.ensure(tune_classes, 9, tmpl_max, radius_max, precision,
                                          device=self.dev)
        self.variant_used = api.resolve_variant(tmpl_max, radius_max, 9, precision, variant)

    # -- requests ------------------------------------------------------------
    def now(self):
        return self.clock() - self.t0

    def submit(self, job):
        job.key = self.next_key
        self.next_key += 1
        if job.arrival is None:
            job.arrival = self.now()
        self.waiting.append(job)
        return job.key

    def idle(self):
        return not (self.waiting or self.resident or self.inflight)

    # -- admission -----------------------------------------------------------
    def _admit_one(self, job):
        torch, api = self.torch, self.api
        gx, gy = job.grid()
        n = gx * gy
        nbytes = job_bytes(job)
        if not self.adm.fits(nbytes) or not self.free_job_slots:
            return False
        off = self.ring.alloc(n)
        if off is None:
            return False
        self.adm.admit(job.key, nbytes)
        slot = self.free_job_slots.pop()
        job.n_cp = n
        st = self.s_admit
        with torch.cuda.stream(st):
            ref_h, sen_h = _pinned(torch, job.ref), _pinned(torch, job.sen)
            ref = torch.empty(ref_h.shape, dtype=ref_h.dtype, device=self.dev)
            sen = torch.empty(sen_h.shape, dtype=sen_h.dtype, device=self.dev)
            ref.copy_(ref_h, non_blocking=True)
            sen.copy_(sen_h, non_blocking=True)
            fr = api.cfog_extract(ref, stream=st)
            fs = api.cfog_extract(sen, stream=st)
            api.cfog_detect_cps(ref, gx, gy, 1, 0, job.margin, out=self.cps[off:off + n], stream=st)
            side = self.side_host[:, off:off + n].numpy()
            side[0] = job.tmpl
            side[1] = job.radius
            side[2] = slot
            self.tmpl[off:off + n].copy_(self.side_host[0, off:off + n], non_blocking=True)
            self.radius[off:off + n].copy_(self.side_host[1, off:off + n], non_blocking=True)
            self.job_of[off:off + n].copy_(self.side_host[2, off:off + n], non_blocking=True)
            entry = (L.cfog_job * 1)()
            entry[0].ref = fr.struct()
            entry[0].sen = fs.struct()
            sz = L.ctypes.sizeof(L.cfog_job)
            self.jobs_host[slot * sz:(slot + 1) * sz].numpy()[:] = np.frombuffer(bytes(entry),
                                                                                 dtype=np.uint8)
            self.jobs_dev[slot * sz:(slot + 1) * sz].copy_(self.jobs_host[slot * sz:(slot + 1) * sz],
                                                           non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        self.resident[job.key] = {"job": job, "slot": slot, "off": off, "ready": ev,
                                  "keep": (ref_h, sen_h, ref, sen, fr, fs),
                                  "left": n}
        self.pending.append((job.key, off, n))
        return True

    def _admit(self):
        while self.waiting:
            if not self._admit_one(self.waiting[0]):
                break
            self.waiting.popleft()

    # -- matching ------------------------------------------------------------
    def _launch(self):
        torch, api = self.torch, self.api
        if len(self.inflight) >= self.max_inflight or not self.pending:
            return
        batch, total = [], 0
        # one launch covers one contiguous ring range (CP ranges adjacent in the ring)
        while self.pending and total < self.max_batch:
            key, start, n = self.pending[0]
            if batch and batch[-1][1] + batch[-1][2] != start:
                break
            take = min(n, self.max_batch - total)
            batch.append((key, start, take))
            total += take
            if take == n:
                self.pending.popleft()
            else:
                self.pending[0] = (key, start + take, n - take)
        st = self.s_match
        for key, _, _ in batch:
            st.wait_event(self.resident[key]["ready"])
        s0 = batch[0][1]
        wi = self.launches % self.max_inflight
        self.launches += 1
        with torch.cuda.stream(st):
            api.cfog_match_batched(self.jobs_dev, self.max_jobs, self.cps[s0:s0 + total],
                                   self.tmpl[s0:s0 + total], self.radius[s0:s0 + total],
                                   self.tmpl_max, self.radius_max,
                                   job_of_cp=self.job_of[s0:s0 + total],
                                   precision=self.precision, variant=self.variant,
                                   out=self.res[s0:s0 + total], workspace=self.ws[wi], stream=st)
            self.res_host[s0:s0 + total].copy_(self.res[s0:s0 + total], non_blocking=True)
            self.cps_host[s0:s0 + total].copy_(self.cps[s0:s0 + total], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        self.inflight.append((ev, batch))

    def _retire(self):
        # launches complete in order on the one match stream
        while self.inflight and self.inflight[0][0].query():
            _, batch = self.inflight.popleft()
            t = self.now()
            for key, start, n in batch:
                ent = self.resident[key]
                ent["left"] -= n
                if ent["left"] == 0:
                    job = ent["job"]
                    off = ent["off"]
                    job.results = self.res_host[off:off + job.n_cp].numpy().copy()
                    job.cps = self.cps_host[off:off + job.n_cp].numpy().copy()
                    job.done_time = t
                    self.ring.release(off, job.n_cp)
                    self.adm.release(key)
                    self.free_job_slots.append(ent["slot"])
                    del self.resident[key]
                    self.finished.append(job)

    def step(self):
        """Admit, launch and retire without blocking; returns True if work remains."""
        self._retire()
        self._admit()
        self._launch()
        return not self.idle()

    def drain(self, poll=0.0002):
        while self.step():
            time.sleep(poll)


def latency_summary(jobs):
    lat = np.array([j.done_time - j.arrival for j in jobs])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "p999_ms": float(np.percentile(lat, 99.9) * 1e3), "jobs": int(len(jobs))}
