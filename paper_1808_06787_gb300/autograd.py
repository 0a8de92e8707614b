"""Gradients of a loss of the final mole fractions with respect to the binary
diffusivities and the initial field, through the hand-written adjoint kernels.

``MaxwellStefanLB.apply(x0, d_pairs, spec)`` runs ``spec.steps`` steps of the
model from the initial mole fractions ``x0`` ([n, nz, ny, nx], on the device,
the solver's dtype) with the pair diffusivities ``d_pairs`` (1-D float64 CPU
tensor, pairs (0,1), (0,2), .., (0,n-1), (1,2), ..) and returns the mole
fractions at the final step.  Its backward pass applies the adjoint step
kernels from the last step to the first with sqrt(T) checkpointing: the
forward keeps the populations every K = ceil(sqrt(T)) steps, and the backward
pass recomputes each segment of K states from its checkpoint (bit for bit:
the step count keys the stochastic rounding) before stepping the adjoint
through it, so the extra cost is one forward pass (run on a second stream,
overlapping the adjoint steps) and the memory is about 3 sqrt(T) population
buffers.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from .lbms import Solver


@dataclass
class RunSpec:
    lattice: str
    grid: tuple
    steps: int
    bc: object = "periodic"
    relax: str = "magic"
    dtype: torch.dtype = torch.float32
    stats: dict = field(default_factory=dict)
    boundary: dict = None  # {face: composition} of the Dirichlet faces


def pairs_to_matrix(d_pairs, n: int) -> np.ndarray:
    D = np.ones((n, n))
    k = 0
    for p in range(n):
        for q in range(p + 1, n):
            D[p, q] = D[q, p] = float(d_pairs[k])
            k += 1
    return D


def n_from_pairs(npairs: int) -> int:
    n = int(round((1 + math.sqrt(1 + 8 * npairs)) / 2))
    if n * (n - 1) // 2 != npairs:
        raise ValueError("d_pairs must hold n (n - 1) / 2 entries")
    return n


class MaxwellStefanLB(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0: torch.Tensor, d_pairs: torch.Tensor, spec: RunSpec):
        n = n_from_pairs(d_pairs.numel())
        D = pairs_to_matrix(d_pairs.detach().cpu().double().numpy(), n)
        solver = Solver(spec.lattice, D, spec.grid, bc=spec.bc, relax=spec.relax, dtype=spec.dtype,
                        device=x0.device, boundary=spec.boundary)
        solver.set_state(x0.detach().to(spec.dtype).contiguous())
        T = int(spec.steps)
        K = max(1, int(math.ceil(math.sqrt(T))))
        ckpts = []
        t = 0
        launches = 1  # set_state
        while t < T:
            ckpts.append((t, solver.get_state()))
            m = min(K, T - t)
            solver.step(m)
            launches += m  # m step kernels (the mass partials are reduced on demand only)
            t += m
        xT = solver.moments()
        spec.stats["launches"] = launches + 1
        ctx.solver = solver
        ctx.D = D
        ctx.x0_dtype = x0.dtype
        ctx.ckpts = ckpts
        ctx.K = K
        ctx.T = T
        ctx.spec = spec
        spec.stats["checkpoints"] = len(ckpts)
        spec.stats["segment"] = K
        return xT

    @staticmethod
    def backward(ctx, grad_xT: torch.Tensor):
        s = ctx.solver
        spec = ctx.spec
        lam = s.adjoint_state()
        lam2 = torch.empty_like(lam)
        s.adjoint_seed(grad_xT.to(s.dtype), lam)
        gacc = s.adjoint_scratch()
        # Segment recomputation runs on a second stream through a second handle
        # (its own step counters), one segment ahead of the adjoint steps, which
        # are latency-bound and leave most of the GPU to it; two segment buffers
        # alternate.  The results are those of the serial order, bit for bit.
        side = torch.cuda.Stream(device=s.device)
        side.wait_stream(s.stream)  # the checkpoints come from the forward
        helper = Solver(spec.lattice, ctx.D, spec.grid, bc=spec.bc, relax=spec.relax,
                        dtype=spec.dtype, device=s.device, stream=side, boundary=spec.boundary)
        shape = (max(ctx.K - 1, 1),) + tuple(s.state_shape)
        segs = [torch.empty(shape, dtype=s.dtype, device=s.device) for _ in range(2)]
        order = list(reversed(ctx.ckpts))
        rec_done, adj_done = [None] * len(order), [None] * len(order)
        launches = 1  # seed

        def recompute(i):
            nonlocal launches
            t0, ck = order[i]
            count = min(t0 + ctx.K, ctx.T) - t0 - 1
            if i >= 2:
                side.wait_event(adj_done[i - 2])  # the buffer's previous segment is done
            # f+(t0 + 1) .. f+(t1 - 1) from the checkpoint f+(t0)
            helper.recompute(ck, t0, count, segs[i % 2])
            launches += count + 2 if count > 0 else 0
            ev = torch.cuda.Event()
            ev.record(side)
            rec_done[i] = ev

        # optional timing of the adjoint-step loops (CUDA events on the solver's stream)
        events = spec.stats.get("adjoint_events")
        recompute(0)
        for i, (t0, ck) in enumerate(order):
            t1 = min(t0 + ctx.K, ctx.T)
            if i + 1 < len(order):
                recompute(i + 1)
            s.stream.wait_event(rec_done[i])
            seg = segs[i % 2]
            if events is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(s.stream)
            # adjoint steps t1 .. t0 + 1 (step t reads f+(t - 1)), one native call
            count = t1 - t0
            s.adjoint_steps(ck, seg if count > 1 else None, count, lam, lam2, gacc)
            if count % 2:
                lam, lam2 = lam2, lam
            launches += count
            if events is not None:
                e1 = torch.cuda.Event(enable_timing=True)
                e1.record(s.stream)
                events.append((e0, e1, t1 - t0))
            ev = torch.cuda.Event()
            ev.record(s.stream)
            adj_done[i] = ev
        grad_x0 = s.adjoint_initial(lam).to(ctx.x0_dtype)
        gD = torch.from_numpy(s.adjoint_reduce(gacc))
        spec.stats["launches"] = spec.stats.get("launches", 0) + launches + 2
        return grad_x0, gD, None


def simulate(x0: torch.Tensor, d_pairs: torch.Tensor, spec: RunSpec) -> torch.Tensor:
    """Differentiable final mole fractions (see the module docstring)."""
    return MaxwellStefanLB.apply(x0, d_pairs, spec)
