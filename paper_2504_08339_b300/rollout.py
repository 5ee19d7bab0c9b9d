"""Multi-step rollouts captured in one CUDA graph.

A rollout evaluates the same population on T consecutive input batches (one
per environment step).  The transformation stage runs once; the T forward
launches, each reading its step's inputs and writing its step's outputs, are
captured together with it into a single CUDA graph, so a whole rollout costs
one graph launch.  With `events=k` an event pair brackets every k-th forward
launch inside the graph, which gives per-launch device durations.
"""
from __future__ import annotations

import torch

from .api import Plan, Transformed


class Rollout:
    def __init__(self, plan: Plan, T: int, S: int = 1, ring: int | None = None,
                 events: int = 0, plain: bool = False):
        """T steps of S input vectors per genome.  `ring` (<= T) input buffers
        are cycled through (step t reads buffer t % ring); default ring = T."""
        self.plan, self.T, self.S = plan, int(T), int(S)
        self.ring = int(ring or T)
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

    def _body(self):
        self.plan.transform(self.nodes, self.conns, out=self.tr)
        for t in range(self.T):
            ev = self.ev.get(t) if self.ev is not None else None
            if ev is not None:
                ev[0].record()
            self.plan.forward(self.inputs[t % self.ring], out=self.outputs[t], plain=self.plain)
            if ev is not None:
                ev[1].record()

    def capture(self):
        """Capture transform + T forward steps into one graph (run once eagerly
        first on the capture stream)."""
        s = torch.cuda.Stream(device=self.plan.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.plan.transform(self.nodes, self.conns, out=self.tr)
            self.plan.forward(self.inputs[0], out=self.outputs[0], plain=self.plain)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()
        return self

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

    def run_host(self, nodes, conns, inputs, out_host):
        """End-to-end rollout from host buffers: H2D copy of the population and
        all step inputs, the graph, and a D2H copy of all step outputs."""
        self.load(nodes, conns, inputs)
        self.run()
        out_host.copy_(self.outputs, non_blocking=True)
        return out_host

    def launch_durations_ms(self):
        """Device duration of the timed forward launches of the last replay."""
        if self.ev is None:
            return None
        return [a.elapsed_time(b) for a, b in self.ev.values()]
