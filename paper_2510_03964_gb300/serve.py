"""Serving many viewers' foveated frame streams on one GPU.

Viewers join and leave over time; each sends frames as a Poisson process,
and every frame returns the viewer's resolved frame (the update and the
resolve in one pass, into the viewer's output buffer). Every admitted
viewer's reservoirs and output stay resident in HBM, and viewers are admitted
while their device bytes (reservoir state and output) fit under an HBM budget (the rest wait in a
FIFO queue and are admitted as others leave; frames a viewer sends before
admission are rejected).

Parking (``park_idle_ms``): when a joining viewer does not fit the budget,
admitted viewers with nothing pending or in flight for at least that long are
moved to host memory, least recently active first: their reservoirs through
wrs_export_state and their last resolved frame, freeing their device bytes.
A parked viewer stays admitted; when its next frame is due it is restored
through wrs_import_state (parking other idle viewers if it must) and carries
on bit for bit as if it had stayed resident.

Overload policy: a frame still waiting on the host ``deadline_ms`` after it
arrived is dropped (shed) instead of launched: it could no longer be shown in
time, and launching it would delay every later frame. Both modes keep a
bounded number of launches in flight, so waiting frames stay on the host where
the deadline applies.

Two dispatch modes run the same arrival trace:

* ``batched`` (continuous batching): launches go out in arrival order on
  one CUDA stream (by default; viewers can be spread over ``n_streams``
  streams, each keeping its viewers' frames in order). Whenever fewer than
  ``depth`` launches are queued, every viewer with a pending frame
  contributes its oldest one to one persistent batched launch
  (wrs_push_batch, a CUDA-graph kernel node); frames that arrive while
  launches run join the next one. A launch that would hold a single frame
  goes out as that viewer's own update (wrs_push_frame, or wrs_push_foveated
  for rendered frames) instead: a batch of one gains nothing and costs the
  graph update. At light load this is the plain path; when frames queue up,
  they share launches.
* ``plain``: every frame is launched on its own (wrs_push_frame), in arrival
  order, on one stream, with at most ``plain_depth`` launches in flight.

Both modes keep at most ``plain_depth`` frames on the GPU at a time.

A frame's latency is the time from its arrival to the host observing its
launch's completion event. Results per frame are identical in both modes and
to a viewer served alone (each viewer's frames are applied in arrival order).

Frames come from one of two sources: a ``FramePool`` of foveated frames made
beforehand, or a ``RenderPool`` holding each resolution class's rendered
image and its mip levels on the device, from which every request's frame is
foveated on the device for that request's gaze (Sec. 4.3's post-process)
inside the update kernel: wrs_push_foveated in plain mode (and for batches of
one), wrs_push_batch_foveated for batches. Either way a request carries only
a gaze and no frame is written to memory.
"""
from __future__ import annotations

import collections
import dataclasses
import statistics
import time

import numpy as np
import torch

from .wrs import Batch, Foveation, Stream, make_config, state_bytes

# resolution classes of the mixed-viewer workload: (width, height, ring radii)
CLASSES = ((3840, 2160, (200.0, 500.0, 1000.0)), (2064, 2208, (200.0, 500.0, 1000.0)),
           (1440, 1600, (150.0, 375.0, 750.0)), (1920, 1080, (120.0, 300.0)))


@dataclasses.dataclass
class ViewerSpec:
    vid: int
    width: int
    height: int
    K: int
    radii: tuple
    seed: int
    rate_hz: float
    join_s: float
    leave_s: float
    cls: int
    color_fp16: bool = True

    @property
    def pixels(self) -> int:
        return self.width * self.height

    def state_bytes(self) -> int:
        return state_bytes(make_config(self.width, self.height, self.K, self.radii[0],
                                       color_fp16=self.color_fp16))

    def frame_bytes(self) -> int:
        return self.pixels * 12  # one RGB float frame (the output, or a staged frame)


def viewer_mix(n: int = 64, duration_s: float = 60.0, seed: int = 0,
               rate_hz=(72.0, 120.0), classes=CLASSES) -> list[ViewerSpec]:
    """n viewers cycling through the resolution classes, K = 8 for even and 4
    for odd viewer index, frame rates uniform in rate_hz, joining within the
    first half of the run and staying 30-90% of it."""
    g = np.random.Generator(np.random.Philox(key=[seed, 11]))
    out = []
    for i in range(n):
        w, h, radii = classes[i % len(classes)]
        join = float(g.random() * 0.5 * duration_s)
        stay = float((0.3 + 0.6 * g.random()) * duration_s)
        out.append(ViewerSpec(vid=i, width=w, height=h, K=8 if i % 2 == 0 else 4, radii=radii,
                              seed=i + 1, rate_hz=float(rate_hz[0] + g.random() * (rate_hz[1] - rate_hz[0])),
                              join_s=join, leave_s=min(duration_s, join + stay), cls=i % len(classes)))
    return out


def arrivals(specs, seed: int = 0):
    """Sorted (time_s, vid) of every frame each viewer sends between join and leave."""
    g = np.random.Generator(np.random.Philox(key=[seed, 12]))
    ev = []
    for v in specs:
        t = v.join_s
        while True:
            t += float(g.exponential(1.0 / v.rate_hz))
            if t >= v.leave_s:
                break
            ev.append((t, v.vid))
    ev.sort()
    return ev


class FramePool:
    """A few pre-generated foveated frames per resolution class, resident on the
    device; viewer frame t uses frame t mod F of its class with its gaze."""

    def __init__(self, classes, frames_per_class: int, device, seed: int = 0):
        from synth import Foveator, gaze_path  # input generator, not part of the method
        self.frames, self.gaze = [], []
        for ci, (w, h, radii) in enumerate(classes):
            fv = Foveator(w, h, radii, seed=seed + ci, device=device)
            gz = gaze_path(w, h, frames_per_class, seed=seed + ci)
            fr = torch.empty((frames_per_class, h, w, 3), dtype=torch.float32, device=device)
            for t in range(frames_per_class):
                fv.frame(float(gz[t, 0]), float(gz[t, 1]), out=fr[t])
            self.frames.append(fr)
            self.gaze.append(gz)
        self.F = frames_per_class

    def get(self, cls: int, t: int):
        i = t % self.F
        return self.frames[cls][i], self.gaze[cls][i]


class RenderPool:
    """Each resolution class's rendered image and mip levels, resident on the
    device, and a gaze path per class; viewer frame t is foveated on the device
    from its class's image for gaze t mod F."""

    def __init__(self, classes, frames_per_class: int, device, seed: int = 0, filter: str = "bilinear"):
        from synth import gaze_path, ground_truth  # input generator, not part of the method
        self.fov, self.gaze = [], []
        for ci, (w, h, radii) in enumerate(classes):
            img = torch.from_numpy(ground_truth(w, h, seed + ci)).to(device)
            self.fov.append(Foveation(img, radii, filter=filter))
            self.gaze.append(gaze_path(w, h, frames_per_class, seed=seed + ci))
        self.F = frames_per_class

    def get(self, cls: int, t: int):
        i = t % self.F
        return self.fov[cls], self.gaze[cls][i]


@dataclasses.dataclass
class ServeStats:
    mode: str
    duration_s: float
    frames_served: int
    frames_rejected: int
    pixel_updates: int
    latencies_ms: list
    launches: int
    viewers_admitted: int
    viewers_queued_max: int
    peak_state_bytes: int
    single_launches: int = 0  # batched mode: launches that held one frame (the viewer's own kernel)
    frames_shed: int = 0      # dropped on the host after waiting past the deadline
    peak_device_bytes: int = 0  # states + outputs (+ frame buffers) of the admitted viewers
    deadline_ms: float | None = None
    parks: int = 0              # viewers moved to host memory (wrs_export_state)
    restores: int = 0           # parked viewers brought back (wrs_import_state)

    def summary(self) -> dict:
        lat = sorted(self.latencies_ms)

        def pct(q):
            if not lat:
                return None
            return round(lat[min(len(lat) - 1, int(q * len(lat)))], 3)

        return {"mode": self.mode, "duration_s": round(self.duration_s, 2),
                "frames_served": self.frames_served, "frames_rejected": self.frames_rejected,
                "frames_shed": self.frames_shed, "deadline_ms": self.deadline_ms,
                "p50_ms": pct(0.50), "p99_ms": pct(0.99),
                "mean_ms": round(statistics.mean(lat), 3) if lat else None,
                "mpx_updates_per_s": round(self.pixel_updates / self.duration_s / 1e6, 1),
                "launches": self.launches, "frames_per_launch": round(self.frames_served / max(1, self.launches), 2),
                "single_frame_launches": self.single_launches,
                "viewers_admitted": self.viewers_admitted, "viewers_queued_max": self.viewers_queued_max,
                "viewers_parked": self.parks, "viewers_restored": self.restores,
                "peak_state_gb": round(self.peak_state_bytes / 1e9, 2),
                "peak_device_gb": round(self.peak_device_bytes / 1e9, 2)}


class Server:
    """Runs one arrival trace in real time in one of the two dispatch modes."""

    def __init__(self, specs, pool: FramePool, budget_bytes: int, mode: str = "batched",
                 n_streams: int = 1, depth: int = 12, device=None, keep_states: bool = False,
                 batch_launch=None, single_direct: bool = True, deadline_ms: float | None = None,
                 plain_depth: int = 12, park_idle_ms: float | None = None):
        assert mode in ("batched", "plain")
        self.specs = {v.vid: v for v in specs}
        self.pool = pool
        self.budget = int(budget_bytes)
        self.mode = mode
        self.depth = depth
        self.plain_depth = plain_depth
        self.deadline_s = None if deadline_ms is None else deadline_ms * 1e-3
        self.park_idle_s = None if park_idle_ms is None else park_idle_ms * 1e-3
        self.parked = {}          # vid -> (state bytes, frame index, last resolved frame), on the host
        self.parks = 0
        self.restores = 0
        self.single_direct = single_direct
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.keep_states = keep_states
        n_streams = n_streams if mode == "batched" else 1
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]
        # one launcher per stream: a launcher's graph is updated in place, so
        # two launches queued on different streams must not share one
        self.batches = []
        if mode == "batched":
            for _ in range(n_streams):
                b = Batch(min(64, max(1, len(specs))))
                if batch_launch:
                    b.set_launch(*batch_launch)
                self.batches.append(b)
        self.init_stream = torch.cuda.Stream(device=self.device)
        self.init_ev = {}         # vid -> event after its state initialisation
        self.used = 0             # device bytes of the admitted viewers
        self.used_state = 0       # of which reservoir states
        self.outs = {}            # vid -> resolved frame of the viewer's latest served frame
        self.live = {}            # vid -> Stream
        self.pushed = collections.defaultdict(list)  # vid -> frame counters pushed, in order
        self.kept = {}            # vid -> Stream kept after leaving (keep_states)
        self.kept_out = {}        # vid -> its last resolved frame
        self.render = isinstance(pool, RenderPool)

    # -- admission ---------------------------------------------------------
    def viewer_bytes(self, v: ViewerSpec) -> int:
        return v.state_bytes() + v.frame_bytes()  # reservoirs + resolved output

    def _admit(self, vid) -> bool:
        v = self.specs[vid]
        need = self.viewer_bytes(v)
        if self.used + need > self.budget:
            return False
        st = Stream(v.width, v.height, v.K, v.radii[0], seed=v.seed, stream_id=vid,
                    color_fp16=v.color_fp16, device=self.device, stream=self.init_stream)
        ev = torch.cuda.Event()
        ev.record(self.init_stream)
        self.init_ev[vid] = ev
        self.live[vid] = st
        self.used += need
        self.used_state += v.state_bytes()
        self.outs[vid] = torch.empty((v.height, v.width, 3), dtype=torch.float32, device=self.device)
        return True

    def _stream_of(self, vid):
        return self.streams[vid % len(self.streams)]

    def _park(self, vid):
        # an idle viewer's reservoirs and last resolved frame to host memory
        stream = self._stream_of(vid)
        ev = self.init_ev.pop(vid, None)
        if ev is not None:
            stream.wait_event(ev)
        st = self.live.pop(vid)
        buf = st.export_raw(stream=stream)  # waits for its copies
        out = self.outs.pop(vid)
        with torch.cuda.stream(stream):
            host_out = out.to("cpu")
        self.parked[vid] = (buf, st.frame_index, host_out)
        st.close()
        v = self.specs[vid]
        self.used -= self.viewer_bytes(v)
        self.used_state -= v.state_bytes()
        self.parks += 1

    def _restore(self, vid):
        v = self.specs[vid]
        stream = self._stream_of(vid)
        buf, t, host_out = self.parked.pop(vid)
        st = Stream(v.width, v.height, v.K, v.radii[0], seed=v.seed, stream_id=vid,
                    color_fp16=v.color_fp16, device=self.device, stream=stream)
        st.import_raw(buf, t, stream=stream)
        with torch.cuda.stream(stream):
            self.outs[vid] = host_out.to(self.device)
        self.live[vid] = st
        self.used += self.viewer_bytes(v)
        self.used_state += v.state_bytes()
        self.restores += 1

    def _make_room(self, need, exclude, idle_since):
        # parks admitted viewers that are idle (nothing pending or in flight,
        # last active at or before idle_since), least recently active first,
        # until `need` more bytes fit the budget; True if they do
        cands = sorted((self._last[vid], vid) for vid in self.live
                       if vid not in exclude and self._busy[vid] == 0 and not self._pending[vid]
                       and vid not in self._leaving and self._last[vid] <= idle_since)
        for _, vid in cands:
            if self.used + need <= self.budget:
                break
            self._park(vid)
        return self.used + need <= self.budget

    def _keep_parked(self, vid):
        # a parked viewer that leaves: its state back on the device for the
        # caller (keep_states), outside the budget
        buf, t, host_out = self.parked.pop(vid)
        if self.keep_states:
            v = self.specs[vid]
            st = Stream(v.width, v.height, v.K, v.radii[0], seed=v.seed, stream_id=vid,
                        color_fp16=v.color_fp16, device=self.device)
            st.import_raw(buf, t)
            self.kept[vid] = st
            self.kept_out[vid] = host_out.to(self.device)

    def _ready(self, vid, stream):
        # a launch that touches a newly admitted viewer waits for its initialisation
        ev = self.init_ev.pop(vid, None)
        if ev is not None:
            stream.wait_event(ev)

    def _release(self, vid):
        self.init_ev.pop(vid, None)
        st = self.live.pop(vid)
        self.used -= self.viewer_bytes(self.specs[vid])
        self.used_state -= self.specs[vid].state_bytes()
        out = self.outs.pop(vid)
        if self.keep_states:
            self.kept[vid] = st
            self.kept_out[vid] = out
        else:
            st.close()
            del st

    def run(self, trace, duration_s: float) -> ServeStats:
        dev = self.device
        torch.cuda.synchronize(dev)
        joins = sorted((v.join_s, vid) for vid, v in self.specs.items())
        leaves = sorted((v.leave_s, vid) for vid, v in self.specs.items())
        ji = li = ai = 0
        waitq = collections.deque()
        pending = collections.defaultdict(collections.deque)  # vid -> deque of arrival times
        next_t = collections.defaultdict(int)                 # vid -> next frame counter
        busy = collections.Counter()  # vid -> frames in flight
        leaving = set()
        last = collections.defaultdict(float)  # vid -> last arrival or completion (s)
        self._busy, self._pending, self._leaving, self._last = busy, pending, leaving, last
        inflight = []         # (event, stream index, [(vid, arrival_s)])
        queued = collections.Counter()  # stream index -> launches in flight
        lat, served, rejected, pix, launches, singles, shed = [], 0, 0, 0, 0, 0, 0
        admitted_total, queued_max, peak, peak_state = 0, 0, 0, 0
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            # joins
            while ji < len(joins) and joins[ji][0] <= now:
                vid = joins[ji][1]
                ji += 1
                last[vid] = now
                if not waitq and self.park_idle_s is not None:
                    self._make_room(self.viewer_bytes(self.specs[vid]), {vid}, now - self.park_idle_s)
                if not waitq and self._admit(vid):
                    admitted_total += 1
                else:
                    waitq.append(vid)
                queued_max = max(queued_max, len(waitq))
            # leaves: release once nothing of the viewer is pending or in flight
            while li < len(leaves) and leaves[li][0] <= now:
                leaving.add(leaves[li][1])
                li += 1
            for vid in list(leaving):
                if vid in waitq:
                    waitq.remove(vid)
                    leaving.discard(vid)
                elif vid in self.live and busy[vid] == 0 and not pending[vid]:
                    self._release(vid)
                    leaving.discard(vid)
                elif vid in self.parked and not pending[vid]:
                    self._keep_parked(vid)
                    leaving.discard(vid)
                elif vid not in self.live and vid not in self.parked and vid not in waitq:
                    leaving.discard(vid)
            if waitq and self.park_idle_s is not None:
                self._make_room(self.viewer_bytes(self.specs[waitq[0]]), {waitq[0]}, now - self.park_idle_s)
            while waitq and self._admit(waitq[0]):
                waitq.popleft()
                admitted_total += 1
            peak = max(peak, self.used)
            peak_state = max(peak_state, self.used_state)
            # arrivals
            while ai < len(trace) and trace[ai][0] <= min(now, duration_s):
                ta, vid = trace[ai]
                ai += 1
                if (vid in self.live or vid in self.parked) and vid not in leaving:
                    pending[vid].append(ta)
                    last[vid] = max(last[vid], ta)
                else:
                    rejected += 1
            # completions
            still = []
            done_now = time.perf_counter() - t0
            for ev, si, frames in inflight:
                if ev.query():
                    queued[si] -= 1
                    for vid, ta in frames:
                        lat.append((done_now - ta) * 1e3)
                        last[vid] = done_now
                        busy[vid] -= 1
                        served += 1
                        pix += self.specs[vid].pixels
                else:
                    still.append((ev, si, frames))
            inflight = still
            # overload: frames that waited past the deadline are dropped
            if self.deadline_s is not None:
                late = time.perf_counter() - t0 - self.deadline_s
                for vid in list(self.live) + list(self.parked):
                    q = pending[vid]
                    while q and q[0] < late:
                        q.popleft()
                        shed += 1
            # parked viewers with a frame due come back, oldest frame first
            if self.parked:
                due = sorted((pending[vid][0], vid) for vid in self.parked if pending[vid])
                for _, vid in due:
                    need = self.viewer_bytes(self.specs[vid])
                    if self.used + need <= self.budget or self._make_room(need, {vid}, now):
                        self._restore(vid)
            # dispatch
            if self.mode == "batched":
                for si, stream in enumerate(self.streams):
                    if queued[si] >= self.depth:
                        continue
                    # at most plain_depth frames on the GPU in either mode: waiting
                    # frames stay on the host, where the deadline applies
                    room = self.plain_depth - sum(len(fr) for _, _, fr in inflight)
                    if room <= 0:
                        break
                    ready = [vid for vid in self.live
                             if vid % len(self.streams) == si and pending[vid]]
                    ready.sort(key=lambda v: pending[v][0])  # oldest frames first
                    ready = ready[:min(self.batches[si].max_streams, room)]
                    if not ready:
                        continue
                    if self.single_direct and len(ready) == 1:
                        # a batch of one: the viewer's own update on its stream
                        vid = ready[0]
                        ta = pending[vid].popleft()
                        t = next_t[vid]
                        next_t[vid] += 1
                        fr, gz = self.pool.get(self.specs[vid].cls, t)
                        self._ready(vid, stream)
                        if self.render:
                            self.live[vid].push_foveated(fr, gz, out=self.outs[vid], stream=stream)
                        else:
                            self.live[vid].push_frame(fr, gz, out=self.outs[vid], stream=stream)
                        busy[vid] += 1
                        self.pushed[vid].append(t)
                        ev = torch.cuda.Event()
                        ev.record(stream)
                        inflight.append((ev, si, [(vid, ta)]))
                        queued[si] += 1
                        launches += 1
                        singles += 1
                        continue
                    sts, frs, gzs, frames, outs = [], [], [], [], []
                    for vid in ready:
                        ta = pending[vid].popleft()
                        t = next_t[vid]
                        next_t[vid] += 1
                        fr, gz = self.pool.get(self.specs[vid].cls, t)
                        self._ready(vid, stream)
                        sts.append(self.live[vid])
                        frs.append(fr)
                        gzs.append(gz)
                        outs.append(self.outs[vid])
                        frames.append((vid, ta))
                        busy[vid] += 1
                        self.pushed[vid].append(t)
                    if self.render:
                        # each frame foveated on read inside the batched update
                        self.batches[si].push_foveated(sts, frs, gzs, outs=outs, stream=stream)
                    else:
                        self.batches[si].push(sts, frs, gzs, outs=outs, stream=stream)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                    inflight.append((ev, si, frames))
                    queued[si] += 1
                    launches += 1
            else:
                stream = self.streams[0]
                # oldest frame first, one launch each, at most plain_depth in flight
                heads = [(pending[vid][0], vid) for vid in self.live if pending[vid]]
                heads.sort()
                while heads and queued[0] < self.plain_depth:
                    _, vid = heads.pop(0)
                    ta = pending[vid].popleft()
                    if pending[vid]:
                        heads.append((pending[vid][0], vid))
                        heads.sort()
                    t = next_t[vid]
                    next_t[vid] += 1
                    fr, gz = self.pool.get(self.specs[vid].cls, t)
                    self._ready(vid, stream)
                    if self.render:
                        self.live[vid].push_foveated(fr, gz, out=self.outs[vid], stream=stream)
                    else:
                        self.live[vid].push_frame(fr, gz, out=self.outs[vid], stream=stream)
                    busy[vid] += 1
                    ev = torch.cuda.Event()
                    ev.record(stream)
                    inflight.append((ev, 0, [(vid, ta)]))
                    queued[0] += 1
                    self.pushed[vid].append(t)
                    launches += 1
            if now >= duration_s and not inflight and all(not q for q in pending.values()):
                break
            if not inflight and ai < len(trace) and trace[ai][0] > now + 0.0005:
                time.sleep(min(0.0005, trace[ai][0] - now))
        torch.cuda.synchronize(dev)
        elapsed = time.perf_counter() - t0
        for vid in list(self.live):
            self._release(vid)
        for vid in list(self.parked):
            self._keep_parked(vid)
        return ServeStats(self.mode, max(elapsed, duration_s), served, rejected, pix, lat, launches,
                          admitted_total, queued_max, peak_state, singles, shed, peak,
                          None if self.deadline_s is None else round(self.deadline_s * 1e3, 3),
                          self.parks, self.restores)

    def close(self):
        for b in self.batches:
            b.close()
        for st in list(self.live.values()) + list(self.kept.values()):
            st.close()
        self.live.clear()
        self.kept.clear()
        self.outs.clear()
        self.kept_out.clear()


def replay_alone(spec: ViewerSpec, pushed, pool: FramePool, device=None):
    """The viewer's frames pushed alone, in the same order, one launch each;
    returns the stream and the resolved frame of the last one."""
    st = Stream(spec.width, spec.height, spec.K, spec.radii[0], seed=spec.seed, stream_id=spec.vid,
                color_fp16=spec.color_fp16, device=device)
    out = torch.empty((spec.height, spec.width, 3), dtype=torch.float32, device=st.device)
    for t in pushed:
        fr, gz = pool.get(spec.cls, t)
        if isinstance(pool, RenderPool):
            st.push_foveated(fr, gz, out=out)
        else:
            st.push_frame(fr, gz, out=out)
    return st, out


def serve_compare(n_viewers=64, duration_s=10.0, budget_gb=60.0, seed=0, frames_per_class=8,
                  device=None, rate_hz=(72.0, 120.0), batch_launch=None, classes=CLASSES,
                  n_streams=1, depth=12, source="frames", deadline_ms=20.0,
                  park_idle_ms=None) -> dict:
    """Both modes on the same trace; returns their summaries. source: "frames"
    (foveated beforehand) or "render" (foveated on the device per request);
    deadline_ms: frames waiting longer on the host are shed (None: never);
    park_idle_ms: park idle viewers to admit joining ones (None: never)."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    specs = viewer_mix(n_viewers, duration_s, seed, rate_hz, classes)
    trace = arrivals(specs, seed)
    if source == "render":
        pool = RenderPool(classes, frames_per_class, dev, seed)
    else:
        pool = FramePool(classes, frames_per_class, dev, seed)
    out = {"viewers": n_viewers, "duration_s": duration_s, "budget_gb": budget_gb,
           "rate_hz": list(rate_hz), "frames_offered": len(trace), "source": source,
           "batched_streams": n_streams, "batched_depth": depth, "deadline_ms": deadline_ms,
           "outputs": "every frame resolved into its viewer's output buffer (fused update + resolve)"}
    for mode in ("batched", "plain"):
        srv = Server(specs, pool, int(budget_gb * 1e9), mode=mode, n_streams=n_streams, depth=depth,
                     device=dev, batch_launch=batch_launch, deadline_ms=deadline_ms,
                     park_idle_ms=park_idle_ms)
        out[mode] = srv.run(trace, duration_s).summary()
        srv.close()
        torch.cuda.synchronize(dev)
    return out
