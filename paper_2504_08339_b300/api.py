"""Torch-facing wrapper of the C ABI: device memory and streams come from
PyTorch, every computation happens in libneat.so's kernels."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, name, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise _lib.NeatError(f"{name} must be a CUDA tensor (no CPU path exists)")
    if t.dtype != dtype:
        raise _lib.NeatError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise _lib.NeatError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise _lib.NeatError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


@dataclass
class Transformed:
    order: torch.Tensor      # [P, N] int32, node rows in topological order, -1 padded
    layer: torch.Tensor      # [P, N] int32
    n_layers: torch.Tensor   # [P] int32
    status: torch.Tensor     # [P] int32 (uint32 bits)


class Plan:
    """A population plan: P genomes of N node rows and C connection rows with
    I inputs and O outputs, bound to the current CUDA device.  The workspace
    (device memory for the transformed programs) is a torch allocation."""

    def __init__(self, P, N, C, I, O, device=None):
        lib = _lib.load()
        self.P, self.N, self.C, self.I, self.O = int(P), int(N), int(C), int(I), int(O)
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        nbytes = lib.neat_workspace_bytes(self.P, self.N, self.C, self.I, self.O)
        if nbytes == 0:
            raise _lib.NeatError(f"unsupported sizes P={P} N={N} C={C} I={I} O={O}")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self._h = ctypes.c_void_p()
        self.generation = 0  # bumped by every transform (the programs it built)
        with torch.cuda.device(self.device):
            _lib.check(lib.neat_plan_create(ctypes.byref(self._h), self.P, self.N, self.C, self.I,
                                            self.O, ctypes.c_void_p(self._ws_ptr), nbytes),
                       "neat_plan_create")
        self._lib = lib

    # -- lifecycle -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.neat_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- tuning ------------------------------------------------------------------
    def get_tuning(self) -> dict:
        t = _lib.neat_tuning()
        _lib.check(self._lib.neat_plan_get_tuning(self._h, ctypes.byref(t)), "get_tuning")
        return {k: getattr(t, k) for k, _ in t._fields_}

    def set_tuning(self, **kw):
        """Set the tuning knobs (neat_tuning); knobs not named are 0, the
        library's default.  An unknown knob name is an error."""
        t = _lib.neat_tuning()
        names = {k for k, _ in t._fields_}
        for k, v in kw.items():
            if k not in names:
                raise _lib.NeatError(f"set_tuning: unknown knob {k!r} (knobs: {sorted(names)})")
            setattr(t, k, int(v))
        _lib.check(self._lib.neat_plan_set_tuning(self._h, ctypes.byref(t)), "set_tuning")

    # -- device failures -----------------------------------------------------------
    def device_errors(self, clear=True, stream=None) -> int:
        """The plan's device failure bits (_lib.DEV_*) OR-ed by its kernels since
        the last clear (synchronises with the stream)."""
        word = torch.zeros((1,), dtype=torch.int32, device=self.device)
        _lib.check(self._lib.neat_plan_device_errors(self._h, _ptr(word), int(bool(clear)),
                                                     _stream(stream)), "neat_plan_device_errors")
        return int(word.item()) & 0xffffffff

    def check(self, stream=None) -> None:
        """Raise NeatError if a kernel of this plan gave up on some genomes
        (their outputs are NaN) since the last check or transform."""
        _lib.check(self._lib.neat_plan_check(self._h, _stream(stream)), "neat_plan_check")

    def validate(self, stream=None) -> int:
        """neat_plan_validate: the NEAT_BAD_* bits (_lib.BAD_*) of the
        structures the last transform wrote, 0 when every index they hold is
        in range (synchronises with the stream)."""
        bits = torch.zeros((1,), dtype=torch.int32, device=self.device)
        _lib.check(self._lib.neat_plan_validate(self._h, _ptr(bits), _stream(stream)),
                   "neat_plan_validate")
        return int(bits.item()) & 0xffffffff

    # -- transformation stage -----------------------------------------------------
    def transform(self, nodes, conns, out: Transformed | None = None, stream=None) -> Transformed:
        P, N, C = self.P, self.N, self.C
        _need(nodes, "nodes", torch.float32, (P, N, 5))
        _need(conns, "conns", torch.float32, (P, C, 4))
        if out is None:
            dev = nodes.device
            out = Transformed(torch.empty((P, N), dtype=torch.int32, device=dev),
                              torch.empty((P, N), dtype=torch.int32, device=dev),
                              torch.empty((P,), dtype=torch.int32, device=dev),
                              torch.empty((P,), dtype=torch.int32, device=dev))
        _lib.check(self._lib.neat_transform(self._h, _ptr(nodes), _ptr(conns), _ptr(out.order),
                                            _ptr(out.layer), _ptr(out.n_layers),
                                            _ptr(out.status), _stream(stream)),
                   "neat_transform")
        self.generation += 1
        return out

    def hyperneat_substrate(self, inputs, grid=32, thresh=0.2, act=2, weights=None, out=None,
                            stream=None):
        """Query every CPPN on the grid, then evaluate its two-sheet substrate
        on inputs [P or 1, S, grid^2]: (outputs [P, S, grid^2], weights)."""
        K = grid * grid
        _need(inputs, "inputs", torch.float32)
        if inputs.dim() != 3 or inputs.shape[2] != K:
            raise _lib.NeatError(f"inputs must be [P or 1, S, {K}]")
        S = inputs.shape[1]
        stride = 0 if inputs.shape[0] == 1 and self.P != 1 else S * K
        dev = inputs.device
        if weights is None:
            weights = torch.empty((self.P, K, K), dtype=torch.float32, device=dev)
        if out is None:
            out = torch.empty((self.P, S, K), dtype=torch.float32, device=dev)
        _need(weights, "weights", torch.float32, (self.P, K, K))
        _need(out, "out", torch.float32, (self.P, S, K))
        _lib.check(self._lib.neat_hyperneat_substrate(
            self._h, int(grid), float(thresh), _ptr(inputs), stride, S, int(act),
            _ptr(weights), _ptr(out), _stream(stream)), "neat_hyperneat_substrate")
        return out, weights

    def mutate_transform(self, nodes, conns, ops, op_status=None, out: Transformed | None = None,
                         stream=None):
        """Apply the Sec. 3.2 operation list ops [P, K, 8] to nodes / conns in
        place, then transform; returns (Transformed, op_status [P])."""
        P, N, C = self.P, self.N, self.C
        _need(nodes, "nodes", torch.float32, (P, N, 5))
        _need(conns, "conns", torch.float32, (P, C, 4))
        _need(ops, "ops", torch.float32)
        if ops.dim() != 3 or ops.shape[0] != P or ops.shape[2] != 8:
            raise _lib.NeatError("ops must be [P, K, 8]")
        dev = nodes.device
        if op_status is None:
            op_status = torch.empty((P,), dtype=torch.int32, device=dev)
        if out is None:
            out = Transformed(torch.empty((P, N), dtype=torch.int32, device=dev),
                              torch.empty((P, N), dtype=torch.int32, device=dev),
                              torch.empty((P,), dtype=torch.int32, device=dev),
                              torch.empty((P,), dtype=torch.int32, device=dev))
        _lib.check(self._lib.neat_mutate_transform(
            self._h, _ptr(nodes), _ptr(conns), _ptr(ops), ops.shape[1], _ptr(op_status),
            _ptr(out.order), _ptr(out.layer), _ptr(out.n_layers), _ptr(out.status),
            _stream(stream)), "neat_mutate_transform")
        self.generation += 1
        return out, op_status

    def transform_recurrent(self, nodes, conns, status=None, stream=None):
        """Transformation for recurrent networks (cycles legal); returns the
        per-genome status words [P] (int32 view of the u32 bits)."""
        P, N, C = self.P, self.N, self.C
        _need(nodes, "nodes", torch.float32, (P, N, 5))
        _need(conns, "conns", torch.float32, (P, C, 4))
        if status is None:
            status = torch.empty((P,), dtype=torch.int32, device=nodes.device)
        _lib.check(self._lib.neat_transform_recurrent(self._h, _ptr(nodes), _ptr(conns),
                                                      _ptr(status), _stream(stream)),
                   "neat_transform_recurrent")
        self.generation += 1
        return status

    def forward_recurrent(self, inputs, T, out=None, stream=None):
        """outputs [P, S, O] after T synchronous iterations."""
        S, stride = self._inputs(inputs)
        if out is None:
            out = torch.empty((self.P, S, self.O), dtype=torch.float32, device=inputs.device)
        _need(out, "out", torch.float32, (self.P, S, self.O))
        _lib.check(self._lib.neat_forward_recurrent(self._h, _ptr(inputs), stride, S, int(T),
                                                    _ptr(out), _stream(stream)),
                   "neat_forward_recurrent")
        return out

    # -- calculation stage ---------------------------------------------------------
    def _inputs(self, inputs):
        _need(inputs, "inputs", torch.float32)
        if inputs.dim() != 3 or inputs.shape[2] != self.I:
            raise _lib.NeatError(f"inputs must be [P or 1, S, {self.I}]")
        S = inputs.shape[1]
        if inputs.shape[0] == self.P:
            stride = S * self.I
        elif inputs.shape[0] == 1:
            stride = 0
        else:
            raise _lib.NeatError("inputs must have P or 1 rows")
        return S, stride

    def forward(self, inputs, out=None, saved=None, plain=False, stream=None):
        """outputs [P, S, O]; inputs [P, S, I] or [1, S, I] (shared)."""
        S, stride = self._inputs(inputs)
        if out is None:
            out = torch.empty((self.P, S, self.O), dtype=torch.float32, device=inputs.device)
        _need(out, "out", torch.float32, (self.P, S, self.O))
        if plain:
            code = self._lib.neat_forward_plain(self._h, _ptr(inputs), stride, S, _ptr(out),
                                                _stream(stream))
            _lib.check(code, "neat_forward_plain")
        else:
            if saved is not None:
                _need(saved, "saved", torch.float32, (self.P, self.N, S))
            code = self._lib.neat_forward(self._h, _ptr(inputs), stride, S, _ptr(out),
                                          _ptr(saved), _stream(stream))
            _lib.check(code, "neat_forward")
        return out

    def backward(self, inputs, grad_out, saved=None, want_inputs=True, stream=None):
        """(grad_weight [P,C], grad_bias [P,N], grad_response [P,N], grad_inputs [P,S,I] or None)."""
        S, stride = self._inputs(inputs)
        _need(grad_out, "grad_out", torch.float32, (self.P, S, self.O))
        if saved is not None:
            _need(saved, "saved", torch.float32, (self.P, self.N, S))
        dev = inputs.device
        gw = torch.empty((self.P, self.C), dtype=torch.float32, device=dev)
        gb = torch.empty((self.P, self.N), dtype=torch.float32, device=dev)
        gr = torch.empty((self.P, self.N), dtype=torch.float32, device=dev)
        gi = torch.empty((self.P, S, self.I), dtype=torch.float32, device=dev) if want_inputs else None
        code = self._lib.neat_backward(self._h, _ptr(inputs), stride, S, _ptr(grad_out),
                                       _ptr(saved), _ptr(gw), _ptr(gb), _ptr(gr), _ptr(gi),
                                       _stream(stream))
        _lib.check(code, "neat_backward")
        return gw, gb, gr, gi

    def sum_genomes(self, x, out=None, stream=None):
        """[P, ...] -> [...]: the sum over genomes (neat_sum_genomes), e.g. the
        gradient of an input set all genomes share from backward()'s
        per-genome grad_inputs."""
        _need(x, "x", torch.float32)
        if x.shape[0] != self.P:
            raise ValueError(f"x: expected {self.P} genomes, got {x.shape[0]}")
        n = 1
        for d in x.shape[1:]:
            n *= int(d)
        if out is None:
            out = torch.empty(x.shape[1:], dtype=torch.float32, device=x.device)
        _need(out, "out", torch.float32, tuple(x.shape[1:]))
        _lib.check(self._lib.neat_sum_genomes(_ptr(x), self.P, n, _ptr(out), _stream(stream)),
                   "neat_sum_genomes")
        return out

    def hyperneat(self, grid=32, thresh=0.2, out=None, stream=None):
        """Substrate weights [P, grid^2, grid^2] of every CPPN (I=5, O=1)."""
        G2 = grid * grid
        if out is None:
            out = torch.empty((self.P, G2, G2), dtype=torch.float32, device=self.device)
        _need(out, "out", torch.float32, (self.P, G2, G2))
        _lib.check(self._lib.neat_hyperneat_query(self._h, int(grid), float(thresh), _ptr(out),
                                                  _stream(stream)), "neat_hyperneat_query")
        return out


def substrate_forward(weights, inputs, act=2, out=None, stream=None):
    """Two-sheet substrate outputs [P, S, K] = act(inputs @ weights) per genome
    (weights [P, K, K], inputs [P or 1, S, K])."""
    lib = _lib.load()
    _need(weights, "weights", torch.float32)
    _need(inputs, "inputs", torch.float32)
    P, K = weights.shape[0], weights.shape[1]
    S = inputs.shape[1]
    stride = 0 if inputs.shape[0] == 1 and P != 1 else S * K
    if out is None:
        out = torch.empty((P, S, K), dtype=torch.float32, device=weights.device)
    _lib.check(lib.neat_substrate_forward(_ptr(weights), P, K, _ptr(inputs), stride, S, int(act),
                                          _ptr(out), _stream(stream)), "neat_substrate_forward")
    return out


def apply_ops(nodes, conns, ops, op_status=None, stream=None):
    """Sec. 3.2 operations ops [P, K, 8] on nodes [P, N, 5] / conns [P, C, 4]
    in place; returns op_status [P] (int32 view of the failed-op bits)."""
    lib = _lib.load()
    _need(nodes, "nodes", torch.float32)
    _need(conns, "conns", torch.float32)
    _need(ops, "ops", torch.float32)
    P, N, C = nodes.shape[0], nodes.shape[1], conns.shape[1]
    if ops.dim() != 3 or ops.shape[0] != P or ops.shape[2] != 8:
        raise _lib.NeatError("ops must be [P, K, 8]")
    if op_status is None:
        op_status = torch.empty((P,), dtype=torch.int32, device=nodes.device)
    _lib.check(lib.neat_apply_ops(_ptr(nodes), _ptr(conns), P, N, C, _ptr(ops), ops.shape[1],
                                  _ptr(op_status), _stream(stream)), "neat_apply_ops")
    return op_status


def distance(nodes, conns, I, O, status=None, c_disjoint=1.0, c_homologous=0.5, out=None,
             stream=None):
    """Compatibility distance of every pair of genomes: [P, P] f32 on the
    device of `nodes` (status: optional [P] status words of a transform)."""
    lib = _lib.load()
    _need(nodes, "nodes", torch.float32)
    _need(conns, "conns", torch.float32)
    P, N, C = nodes.shape[0], nodes.shape[1], conns.shape[1]
    if out is None:
        out = torch.empty((P, P), dtype=torch.float32, device=nodes.device)
    _need(out, "out", torch.float32, (P, P))
    nbytes = lib.neat_distance_scratch_bytes(P, N, C)
    if nbytes == 0:
        raise _lib.NeatError("distance: unsupported sizes")
    scratch = torch.empty((nbytes + 255,), dtype=torch.uint8, device=nodes.device)
    base = (scratch.data_ptr() + 255) // 256 * 256
    code = lib.neat_distance(_ptr(nodes), _ptr(conns), _ptr(status), P, N, C, I, O,
                             float(c_disjoint), float(c_homologous), _ptr(out),
                             ctypes.c_void_p(base), nbytes, _stream(stream))
    _lib.check(code, "neat_distance")
    return out


# Default cap on the per-node aggregates an autograd forward keeps for its
# backward ([P, N, S] f32): above it the backward recomputes the forward
# values inside its kernel instead of reading them.
SAVED_BUDGET_BYTES = 8 << 30


def saved_bytes(plan: Plan, S: int) -> int:
    """Bytes of the aggregates a forward over S samples per genome saves."""
    return 4 * plan.P * plan.N * int(S)


def choose_store(plan: Plan, S: int, budget: int | None = None) -> bool:
    """True when the saved aggregates fit the budget (default
    SAVED_BUDGET_BYTES), False to recompute them in the backward."""
    return saved_bytes(plan, S) <= (SAVED_BUDGET_BYTES if budget is None else int(budget))


class NeatFunction(torch.autograd.Function):
    """outputs = network(nodes, conns)(inputs), differentiable with respect to
    the bias/response columns of nodes, the weight column of conns and the
    inputs.  Stores the per-node aggregates when `store` is True; recomputes
    the forward values in the backward kernel when it is False; with `store`
    None it stores them if they fit `budget` bytes (choose_store)."""

    @staticmethod
    def forward(ctx, plan: Plan, nodes, conns, inputs, store=None, budget=None):
        plan.transform(nodes, conns)
        S = inputs.shape[1]
        if store is None:
            store = choose_store(plan, S, budget)
        saved = None
        if store:
            saved = torch.empty((plan.P, plan.N, S), dtype=torch.float32, device=inputs.device)
        out = plan.forward(inputs, saved=saved)
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.saved_agg = saved
        ctx.save_for_backward(nodes, conns, inputs)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        nodes, conns, inputs = ctx.saved_tensors
        plan = ctx.plan
        if plan.generation != ctx.generation:
            # the plan was transformed again since this forward (e.g. another
            # evaluate on the same plan): rebuild this population's programs,
            # which the saved aggregates were taken on
            plan.transform(nodes, conns)
        gw, gb, gr, gi = plan.backward(inputs, grad_out.contiguous(), saved=ctx.saved_agg,
                                       want_inputs=ctx.needs_input_grad[3])
        g_nodes = g_conns = g_inputs = None
        if ctx.needs_input_grad[1]:
            g_nodes = torch.zeros_like(nodes)
            g_nodes[..., 1] = gb
            g_nodes[..., 2] = gr
        if ctx.needs_input_grad[2]:
            g_conns = torch.zeros_like(conns)
            g_conns[..., 2] = gw
        if ctx.needs_input_grad[3]:
            g_inputs = gi if inputs.shape[0] == plan.P else plan.sum_genomes(gi).unsqueeze(0)
        return None, g_nodes, g_conns, g_inputs, None, None


def evaluate(plan: Plan, nodes, conns, inputs, store=None, budget=None):
    """Differentiable population evaluation (see NeatFunction): `store` True
    keeps the aggregates, False recomputes them in the backward, None (the
    default) keeps them if 4 P N S bytes fit `budget` (SAVED_BUDGET_BYTES)."""
    return NeatFunction.apply(plan, nodes, conns, inputs, store, budget)
