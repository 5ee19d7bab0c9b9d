"""Multi-step rollouts captured in one CUDA graph.

A rollout evaluates the same population on T consecutive input batches (one
per environment step).  The transformation stage runs once; the T forward
launches, each reading its step's inputs and writing its step's outputs, are
captured together with it into a single CUDA graph, so a whole rollout costs
one graph launch.  With `events=k` an event pair brackets every k-th forward
launch inside the graph (an interval then also holds the event records and
the launch gap).  `capture_split` captures the transform and the T forward
steps as two graphs instead, replayed back to back by `run_split`: an event
recorded between them times the forward launches alone, with no event node
among them.

From host buffers (`run_host`) the rollout is a pipeline of chunks of
consecutive steps, one graph each: the input copies of later chunks (a copy
stream) and the output copies of earlier ones (a second copy stream) run
while a chunk computes, so the host link and the kernels overlap.  The step
inputs are all known when the call is made (open loop).
"""
from __future__ import annotations

import torch

from .api import Plan, Transformed


class Rollout:
    def __init__(self, plan: Plan, T: int, S: int = 1, ring: int | None = None,
                 events: int = 0, plain: bool = False, chunk: int | None = None):
        """T steps of S input vectors per genome.  `ring` (<= T) input buffers
        are cycled through (step t reads buffer t % ring); default ring = T.
        `chunk`: steps per pipeline chunk of `run_host` (default T / 16,
        at least 1)."""
        self.plan, self.T, self.S = plan, int(T), int(S)
        self.ring = int(ring or T)
        self.chunk = max(1, int(chunk) if chunk else -(-self.T // 16))
        P, N, C, I, O = plan.P, plan.N, plan.C, plan.I, plan.O
        dev = plan.device
        self.nodes = torch.empty((P, N, 5), dtype=torch.float32, device=dev)
        self.conns = torch.empty((P, C, 4), dtype=torch.float32, device=dev)
        self.inputs = torch.empty((self.ring, P, S, I), dtype=torch.float32, device=dev)
        self.outputs = torch.empty((self.T, P, S, O), dtype=torch.float32, device=dev)
        self.tr = Transformed(torch.empty((P, N), dtype=torch.int32, device=dev),
                              torch.empty((P, N), dtype=torch.int32, device=dev),
                              torch.empty((P,), dtype=torch.int32, device=dev),
                              torch.empty((P,), dtype=torch.int32, device=dev))
        self.plain = plain
        self.every = int(events)
        self.ev = None
        if self.every > 0:
            mk = lambda: torch.cuda.Event(enable_timing=True, external=True)  # noqa: E731
            self.ev = {t: (mk(), mk()) for t in range(0, self.T, self.every)}
        self.graph = None
        self.split = None       # (transform graph, graph of the T forward steps)
        self.parts = None       # [transform graph, graph of each chunk]
        self.copy_streams = None

    def _steps(self, t0, t1, events=True):
        for t in range(t0, t1):
            ev = self.ev.get(t) if (events and self.ev is not None) else None
            if ev is not None:
                ev[0].record()
            self.plan.forward(self.inputs[t % self.ring], out=self.outputs[t], plain=self.plain)
            if ev is not None:
                ev[1].record()

    def _body(self):
        self.plan.transform(self.nodes, self.conns, out=self.tr)
        self._steps(0, self.T)

    def _warm(self):
        """One transform and one forward on a side stream before a capture."""
        s = torch.cuda.Stream(device=self.plan.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.plan.transform(self.nodes, self.conns, out=self.tr)
            self.plan.forward(self.inputs[0], out=self.outputs[0], plain=self.plain)
        torch.cuda.current_stream().wait_stream(s)

    def capture(self):
        """Capture transform + T forward steps into one graph (run once eagerly
        first on the capture stream)."""
        self._warm()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()
        return self

    def capture_split(self):
        """Capture the transform and the T forward steps as two graphs."""
        self._warm()
        g_tr, g_fwd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_tr):
            self.plan.transform(self.nodes, self.conns, out=self.tr)
        with torch.cuda.graph(g_fwd):
            self._steps(0, self.T, events=False)
        self.split = (g_tr, g_fwd)
        return self

    def run_split(self, ev_mid=None, ev_end=None):
        """One rollout as two graph launches (transform, then the T steps);
        ev_mid / ev_end (optional CUDA events) are recorded after each, so
        ev_mid.elapsed_time(ev_end) is the device time of the T forward
        launches."""
        if self.split is None:
            self.capture_split()
        self.split[0].replay()
        if ev_mid is not None:
            ev_mid.record()
        self.split[1].replay()
        if ev_end is not None:
            ev_end.record()
        return self.outputs

    def load(self, nodes, conns, inputs=None, non_blocking=True):
        """Copy a population (and optionally the input ring) into the graph's
        buffers; host tensors should be pinned for an asynchronous copy."""
        self.nodes.copy_(nodes, non_blocking=non_blocking)
        self.conns.copy_(conns, non_blocking=non_blocking)
        if inputs is not None:
            self.inputs.copy_(inputs, non_blocking=non_blocking)

    def run(self):
        """One rollout on the device-resident buffers (one graph launch)."""
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.outputs

    def _capture_parts(self):
        """The transform and each chunk of steps as graphs of their own."""
        if self.graph is None:
            self._warm()
        parts = []
        for k, t0 in enumerate([None] + list(range(0, self.T, self.chunk))):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                if t0 is None:
                    self.plan.transform(self.nodes, self.conns, out=self.tr)
                else:
                    self._steps(t0, min(t0 + self.chunk, self.T), events=False)
            parts.append(g)
        self.parts = parts
        dev = self.plan.device
        self.copy_streams = (torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))

    def run_host(self, nodes, conns, inputs, out_host):
        """End-to-end rollout from host buffers: the population and the step
        inputs in (host to device), every step's outputs out (device to host),
        pipelined by chunks of steps on the current stream and two copy
        streams.  `inputs` holds the `ring` input buffers [ring, P, S, I];
        host tensors should be pinned for the copies to overlap.  Returns
        out_host [T, P, S, O], complete once the current stream reaches this
        point (e.g. after torch.cuda.synchronize())."""
        if self.parts is None:
            self._capture_parts()
        main = torch.cuda.current_stream()
        h2d, d2h = self.copy_streams
        c, T, ring = self.chunk, self.T, self.ring
        starts = list(range(0, T, c))
        # the previous call's kernels and output copies are done with the buffers
        h2d.wait_stream(main)
        h2d.wait_stream(d2h)
        ev_in = []
        with torch.cuda.stream(h2d):
            self.nodes.copy_(nodes, non_blocking=True)
            self.conns.copy_(conns, non_blocking=True)
            ev_pop = torch.cuda.Event()
            ev_pop.record(h2d)
            for t0 in starts:
                # the input buffers first read by this chunk (steps t0..t1-1
                # read buffers t % ring)
                a, b = min(t0, ring), min(t0 + c, ring)
                if b > a:
                    self.inputs[a:b].copy_(inputs[a:b], non_blocking=True)
                e = torch.cuda.Event()
                e.record(h2d)
                ev_in.append(e)
        main.wait_event(ev_pop)
        self.parts[0].replay()                       # transform
        ev_out = []
        for k, t0 in enumerate(starts):
            main.wait_event(ev_in[k])
            self.parts[1 + k].replay()
            e = torch.cuda.Event()
            e.record(main)
            ev_out.append(e)
        with torch.cuda.stream(d2h):
            for k, t0 in enumerate(starts):
                d2h.wait_event(ev_out[k])
                t1 = min(t0 + c, T)
                out_host[t0:t1].copy_(self.outputs[t0:t1], non_blocking=True)
        main.wait_stream(d2h)
        return out_host

    def launch_durations_ms(self):
        """Device duration of the timed forward launches of the last replay."""
        if self.ev is None:
            return None
        return [a.elapsed_time(b) for a, b in self.ev.values()]
