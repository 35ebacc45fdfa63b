"""Continuous-batching request loop for race checks.

Requests arrive over time and are of two kinds:

* trace checks: a prefix of a device-resident trace (from a pool built with
  the generators in ``tracegen``), checked chunk by chunk; the job's shadow
  stays resident in its region between chunks;
* instrumented kernels: a hand-instrumented synthetic kernel (stencil,
  histogram or reduction) run with ``hr_access()`` inline on the job's region.

The server owns one checker context with ``n_slots`` pre-allocated regions.
A queued request is admitted (first come, first served) when a slot is free
and its shadow footprint (n_words x 8 B + its report ring) fits the memory
budget; its slot is reconfigured to the job's geometry without allocating.
Each loop iteration gathers the next chunk of every active trace job into one
batched check (``hr_check_batch``: one persistent launch, stages interleaved
across jobs), so requests that arrive while others run join the next
iteration; up to ``max_inflight`` iterations are queued on the GPU at once.
An iteration shares a record budget among the active jobs (each gets at least
one chunk), so a lone job is checked whole and iterations stay short under
load.
Latency is measured from the request's arrival to the moment the host sees
its last chunk complete.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import hirace
from . import tracegen as tg

RING = 1 << 17  # race records kept per request
CANCELLED = -1  # Result.status of a request cancelled before it finished


@dataclass
class Request:
    rid: int
    arrival: float                      # seconds after the run starts
    kind: str                           # "trace" or "kernel"
    source: str = ""                    # trace pool entry, or kernel name
    length: int = 0                     # records (trace) or threads (kernel)
    seed: int = 0
    timeout: float = 0.0                # cancel if not done this long after arrival (0: never)


@dataclass
class Result:
    rid: int
    kind: str
    status: int
    races: np.ndarray          # the request's race records (hirace.RACE_DTYPE)
    n_races: int
    accesses: int
    arrival: float
    admitted: float = 0.0
    done: float = 0.0

    @property
    def latency(self):
        return self.done - self.arrival

    def keys(self) -> set:
        """{(kernel, word, epoch)} of the request's races."""
        return hirace.race_keys(self.races)


class TracePool:
    """Device-resident traces requests take prefixes of (a prefix of a
    wave-sorted trace is itself a valid trace)."""

    def __init__(self, device, scale: str = "full"):
        import torch
        self.entries = {}
        small = scale != "full"
        tr, info = tg.gen_tree_reduction(tg.seed_for(5, 1), inject=True)
        self._add("tree", tr, info, device)
        tr, info = tg.gen_global_mix(tg.seed_for(5, 2), inject=True, n_blocks=16 if small else 1024)
        self._add("global", tr, info, device)
        tr, info = tg.gen_powerlaw_push(tg.seed_for(5, 3), log2_vertices=16 if small else 22,
                                        sweeps=2 if small else 2)
        self._add("graph", tr, info, device)
        torch.cuda.synchronize(device)

    def _add(self, name, trace, info, device):
        import torch
        self.entries[name] = dict(host=trace, dev=torch.from_numpy(trace.view(np.uint8)).to(device),
                                  n=len(trace), n_words=info["n_words"], block_dim=info["block_dim"],
                                  acc_prefix=np.cumsum(trace["op"] <= tg.OP_A))

    def prefix(self, name, length):
        e = self.entries[name]
        length = max(1, min(length, e["n"]))
        return e["dev"][: length * 16], length

    def accesses(self, name, length):
        e = self.entries[name]
        return int(e["acc_prefix"][min(length, e["n"]) - 1])


KERNELS = ("stencil", "histogram", "reduction")


def kernel_words(name, threads):
    return {"stencil": 2 * threads, "histogram": 4096, "reduction": threads}[name]


def kernel_accesses(name, threads):
    if name == "stencil":
        return 4 * threads - 2
    if name == "histogram":
        return threads
    return 3 * threads - 3 * (threads // 512)  # tree levels of a 256-thread block over 512 elements


class Server:
    def __init__(self, pool: TracePool, device, n_slots=64, slot_words=1 << 26, budget_bytes=64 << 30,
                 chunk_records=1 << 22, max_inflight=2, iteration_records=1 << 26, n_kernel_streams=4):
        import torch
        self.pool = pool
        self.device = device
        self.n_slots = n_slots
        self.slot_words = slot_words
        self.budget = budget_bytes
        self.chunk = chunk_records          # smallest chunk a job gets per iteration
        self.iteration_records = iteration_records  # records shared by the active jobs per iteration
        self.max_inflight = max_inflight
        self.ck = hirace.Checker([dict(n_words=slot_words, block_dim=256, report_capacity=RING)] * n_slots,
                                 report_capacity=RING)
        self.ck.batch_reserve(n_slots, 1 << 18)
        hirace.load_workloads()
        self.stream = torch.cuda.Stream(device)           # trace batches
        # instrumented-kernel jobs run on streams of their own, so they overlap
        # the trace batches (and each other) on the device
        self.kernel_streams = [torch.cuda.Stream(device) for _ in range(n_kernel_streams)]
        self.next_kernel_stream = 0
        self.free = list(range(n_slots))
        self.used = 0
        self.queue = collections.deque()
        self.active = {}        # slot -> job dict (trace jobs with chunks left)
        self.inflight = collections.deque()   # (event, [finishing slots], is a trace iteration)
        self.results = {}
        self.t0 = None
        self.iterations = 0
        self.overlapped = 0     # launches queued while work of the other kind was in flight

    # ------------------------------------------------------------- helpers
    def _now(self):
        return time.perf_counter() - self.t0

    def _footprint(self, req):
        if req.kind == "trace":
            words = self.pool.entries[req.source]["n_words"]
        else:
            words = kernel_words(req.source, req.length)
        return words * 8 + RING * 16

    def _words(self, req):
        if req.kind == "trace":
            return self.pool.entries[req.source]["n_words"]
        return kernel_words(req.source, req.length)

    def _finish_unserved(self, req, status):
        t = self._now() if self.t0 is not None else 0.0
        self.results[req.rid] = Result(req.rid, req.kind, status, np.zeros(0, hirace.RACE_DTYPE), 0, 0,
                                       req.arrival, t, t)

    def submit(self, req: Request):
        """Queue a request.  One that can never be admitted (its shadow does not
        fit a slot or the whole budget) is answered at once with HR_ERR_OOM
        instead of blocking the queue behind it."""
        if self._words(req) > self.slot_words or self._footprint(req) > self.budget:
            self._finish_unserved(req, hirace.STATUS_CODE["HR_ERR_OOM"])
            return
        self.queue.append(req)

    def _expire(self, now):
        """Cancel queued or running requests whose timeout has passed."""
        late = [r.rid for r in self.queue if r.timeout and now > r.arrival + r.timeout]
        late += [j["req"].rid for j in self.active.values()
                 if j["req"].timeout and now > j["req"].arrival + j["req"].timeout]
        for rid in late:
            self.cancel(rid)

    def cancel(self, rid: int) -> bool:
        """Cancel a request: dropped if still queued; a trace job being checked
        gets no further chunks and its slot is freed once its launched chunks
        finish.  Its result has status CANCELLED.  False if it already finished."""
        for req in self.queue:
            if req.rid == rid:
                self.queue.remove(req)
                self._finish_unserved(req, CANCELLED)
                return True
        for slot, job in list(self.active.items()):
            if job["req"].rid == rid:
                del self.active[slot]
                job["cancelled"] = True
                # the slot comes back once the chunks already queued on the GPU are done
                import torch
                ev = torch.cuda.Event()
                ev.record(self.stream)
                self.inflight.append((ev, [(slot, job)], False))
                return True
        return False

    def _admit(self):
        import torch
        while self.queue and self.free:
            req = self.queue[0]
            need = self._footprint(req)
            if self.used + need > self.budget:
                break
            self.queue.popleft()
            slot = self.free.pop()
            self.used += need
            admitted = self._now()
            if req.kind == "trace":
                e = self.pool.entries[req.source]
                self.ck.reconfigure(slot, e["n_words"], e["block_dim"], stream=self.stream)
                dev, length = self.pool.prefix(req.source, req.length)
                self.active[slot] = dict(req=req, dev=dev, length=length, next=0, need=need, admitted=admitted,
                                         accesses=self.pool.accesses(req.source, length))
            else:
                n = req.length
                # the slot's reset is queued on the trace stream; the job's stream waits for it
                self.ck.reconfigure(slot, kernel_words(req.source, n), 256, stream=self.stream)
                ready = torch.cuda.Event()
                ready.record(self.stream)
                if any(e[2] for e in self.inflight):
                    self.overlapped += 1
                ks = self.kernel_streams[self.next_kernel_stream]
                self.next_kernel_stream = (self.next_kernel_stream + 1) % len(self.kernel_streams)
                ks.wait_event(ready)
                view = self.ck.device_view(slot)
                g = torch.Generator(device=self.device).manual_seed(req.seed)
                with torch.cuda.stream(ks):
                    if req.source == "stencil":
                        a = torch.rand(n, device=self.device, generator=g)
                        bufs = (a, torch.empty_like(a))
                        hirace.run_stencil(view, bufs[0], bufs[1], racy_stride=(req.seed % 3) * 97, stream=ks)
                    elif req.source == "histogram":
                        k = torch.randint(0, 4096, (n,), device=self.device, dtype=torch.int32, generator=g)
                        bufs = (k, torch.zeros(4096, dtype=torch.int32, device=self.device))
                        hirace.run_histogram(view, bufs[0], bufs[1], racy_stride=(req.seed % 3) * 101, stream=ks)
                    else:
                        bufs = (torch.rand(n, device=self.device, generator=g),)
                        hirace.run_reduce(view, bufs[0], drop_level=(req.seed % 4) - 1, stream=ks)
                ev = torch.cuda.Event()
                ev.record(ks)
                job = dict(req=req, need=need, admitted=admitted, bufs=bufs,
                           accesses=kernel_accesses(req.source, n))
                self.inflight.append((ev, [(slot, job)], False))

    def _launch_iteration(self):
        import torch
        if not self.active or sum(1 for e in self.inflight if e[2]) >= self.max_inflight:
            return False
        batch, finishing = [], []
        # share the iteration's record budget: a lone job takes its whole remainder,
        # many jobs take at least one chunk each
        share = max(self.chunk, self.iteration_records // len(self.active))
        for slot, job in list(self.active.items()):
            a = job["next"]
            b = min(job["length"], a + share)
            batch.append((slot, job["dev"][a * 16: b * 16]))
            job["next"] = b
            if b >= job["length"]:
                finishing.append((slot, job))
                del self.active[slot]
        if any(not e[2] for e in self.inflight):
            self.overlapped += 1
        self.ck.check_batch(batch, stream=self.stream)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        self.inflight.append((ev, finishing, True))
        self.iterations += 1
        return True

    def _poll(self):
        # entries finish out of order (kernel jobs run on their own streams)
        done = [e for e in self.inflight if e[0].query()]
        for e in done:
            self.inflight.remove(e)
            finished = e[1]
            t = self._now()
            for slot, job in finished:
                races, status, n_total, _ = self.ck.report(slot)
                req = job["req"]
                acc = job["accesses"]
                if job.get("cancelled"):
                    status, races, n_total, acc = CANCELLED, races[:0], 0, 0
                self.results[req.rid] = Result(req.rid, req.kind, status, races.copy(), n_total,
                                               acc, req.arrival, job["admitted"], t)
                self.free.append(slot)
                self.used -= job["need"]

    # ------------------------------------------------------------- driving
    def warmup(self):
        """One untimed request of every trace kind and every kernel: first launches
        load kernel modules and set up generators, which should not count as
        request latency."""
        reqs = [Request(-1 - i, 0.0, "trace", name, 200_000, i) for i, name in enumerate(self.pool.entries)]
        reqs += [Request(-10 - i, 0.0, "kernel", name, 1 << 16, i) for i, name in enumerate(KERNELS)]
        saved = self.results
        self.results = {}
        self._drive(reqs, None)
        self._drive(reqs, None, serial=True)
        self.results = saved

    def run(self, requests, time_limit=None, warm=True):
        """Serve ``requests`` (sorted by arrival) in real time; returns results by rid."""
        if warm:
            self.warmup()
        return self._drive(requests, time_limit)

    def _drive(self, requests, time_limit, serial=False):
        import torch
        if serial:
            return self._serial(requests, time_limit)
        torch.cuda.synchronize(self.device)
        self.t0 = time.perf_counter()
        pending = collections.deque(requests)
        while pending or self.queue or self.active or self.inflight:
            now = self._now()
            if time_limit is not None and now > time_limit:
                break
            while pending and pending[0].arrival <= now:
                self.submit(pending.popleft())
            self._expire(now)
            self._admit()
            launched = self._launch_iteration()
            self._poll()
            if not launched and self.inflight:
                time.sleep(20e-6)
        torch.cuda.synchronize(self.device)
        self._poll()
        return self.results

    def run_serial(self, requests, time_limit=None, warm=True):
        """One request at a time, in arrival order, whole trace in one check."""
        if warm:
            self.warmup()
        return self._serial(requests, time_limit)

    def _serial(self, requests, time_limit):
        import torch
        torch.cuda.synchronize(self.device)
        self.t0 = time.perf_counter()
        for req in requests:
            now = self._now()
            if time_limit is not None and now > time_limit:
                break
            if req.arrival > now:
                time.sleep(req.arrival - now)
            old = self.chunk, self.iteration_records
            self.chunk = self.iteration_records = 1 << 40
            self.submit(req)
            self._admit()
            self._launch_iteration()
            self.chunk, self.iteration_records = old
            while self.inflight:
                self.inflight[0][0].synchronize()
                self._poll()
        return self.results


def make_requests(seed: int, rate: float, duration: float, min_len=10_000, max_len=50_000_000,
                  kernel_frac=0.25, min_grid=64, max_grid=4096):
    """Poisson arrivals at ``rate`` per second for ``duration`` seconds."""
    rng = np.random.default_rng(seed)
    t, rid, out = 0.0, 0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            break
        if rng.random() < kernel_frac:
            grid = int(np.exp(rng.uniform(np.log(min_grid), np.log(max_grid))))
            out.append(Request(rid, t, "kernel", KERNELS[int(rng.integers(0, 3))], grid * 256,
                               int(rng.integers(0, 1 << 30))))
        else:
            length = int(np.exp(rng.uniform(np.log(min_len), np.log(max_len))))
            out.append(Request(rid, t, "trace", ("tree", "global", "graph")[int(rng.integers(0, 3))], length,
                               int(rng.integers(0, 1 << 30))))
        rid += 1
    return out


def summarize(results, wall=None):
    lat = np.array([r.latency for r in results.values()]) if results else np.zeros(1)
    acc = sum(r.accesses for r in results.values())
    span = wall if wall else (max(r.done for r in results.values()) if results else 1.0)
    return {"completed": len(results), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "accesses_per_s": acc / max(span, 1e-9),
            "errors": sum(1 for r in results.values() if r.status != hirace.HR_OK)}
