"""Differentiable runs: receivers, discrete adjoint and checkpointing.

``run(plan, x0, nhalf, checkpoint_every, c)`` (``HermiteRun``) returns the
state after `nhalf` half steps as a differentiable function of x0 and c.
``receiver_traces(plan, u0, nhalf, receivers, checkpoint_every, c)`` runs
`nhalf` half steps from the state u0, records the value of u at the receiver
nodes after every half step (whatever grid the state is on), and returns the
traces (nhalf x nrec, FP64).  It is a torch.autograd.Function: the backward
pass is the hand-written discrete adjoint of the half step (hermite_adjoint_
step), swept backwards over segments of `checkpoint_every` half steps.  Each
segment's forward states are recomputed from the checkpoint stored at its start
during the forward pass; they are needed for the gradient with respect to the
wave speed c,

    dL/dc = sum_t < lambda_{t+1}, (dS_t/dc) x_t >,

x_t the forward state before half step t and lambda_{t+1} the adjoint state
after it.  The gradient with respect to u0 is lambda_0.  All arithmetic runs
in libhermite's kernels; torch provides memory, streams and autograd glue.
"""
import torch


def _forward(plan, x0, nhalf, every, after_step=None):
    """nhalf half steps from x0 (parity t % 2 for step t); keeps the state at
    the start of every segment of `every` half steps.  after_step(y, t) sees
    the output of step t.  Returns (final state, checkpoints)."""
    x = x0.detach().clone()
    y = torch.empty_like(x)
    ckpt = {0: x.clone()}
    for t in range(nhalf):
        plan.step(x, y, t % 2)
        if after_step is not None:
            after_step(y, t)
        x, y = y, x
        if (t + 1) % every == 0 and t + 1 < nhalf:
            ckpt[t + 1] = x.clone()
    return x, ckpt


def _sweep(plan, nhalf, every, ckpt, need_c, seed):
    """The discrete adjoint swept backwards over the segments: seed(adj, t)
    adds the cotangent of the output of half step t, then adj <- S_t^T adj.
    With need_c the segment's forward states are recomputed from its
    checkpoint and sum_t < adj_{t+1}, (dS_t/dc) x_t > is accumulated.
    Returns (the gradient with respect to the initial state, dL/dc)."""
    start0 = ckpt[0]
    adj = torch.zeros_like(start0)
    tmp = torch.empty_like(start0)
    grad_c = 0.0
    for s0 in sorted(ckpt, reverse=True):
        s1 = min(s0 + every, nhalf)
        states = None
        if need_c:   # recompute the segment's forward states from its checkpoint
            states = [ckpt[s0]]
            for t in range(s0, s1 - 1):
                nxt = torch.empty_like(start0)
                plan.step(states[-1], nxt, t % 2)
                states.append(nxt)
        for t in range(s1 - 1, s0 - 1, -1):
            seed(adj, t)
            if need_c:
                plan.step_dc(states[t - s0], tmp, t % 2)
                grad_c += plan.dot(adj, tmp)
            plan.adjoint(adj, tmp, t % 2)
            adj, tmp = tmp, adj
    return adj, grad_c


class _ReceiverRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, c, plan, nhalf, idx, every):
        traces = torch.empty((nhalf, idx.numel()), dtype=torch.float64, device=u0.device)
        _, ckpt = _forward(plan, u0, nhalf, every, lambda y, t: plan.record(y, idx, traces[t]))
        ctx.plan, ctx.nhalf, ctx.every, ctx.ckpt = plan, nhalf, every, ckpt
        ctx.save_for_backward(idx)
        return traces

    @staticmethod
    def backward(ctx, g):
        (idx,) = ctx.saved_tensors
        g = g.contiguous().to(torch.float64)
        need_c = ctx.needs_input_grad[1]
        plan = ctx.plan
        adj, grad_c = _sweep(plan, ctx.nhalf, ctx.every, ctx.ckpt, need_c,
                             lambda adj, t: plan.inject(adj, idx, g[t]))   # transpose of recording after step t
        gc = torch.tensor(grad_c, dtype=torch.float64) if need_c else None
        return adj, gc, None, None, None, None


class HermiteRun(torch.autograd.Function):
    """x_n = S_{n-1} ... S_1 S_0 x0: `nhalf` half steps from the state x0
    (step t has parity t % 2), differentiable in x0 and in the wave speed c.
    The backward pass is the discrete adjoint swept from the output's
    cotangent (the gradient for x0 needs no forward state: the half step is
    linear in the state); the forward states that dS/dc needs are recomputed
    per segment of `checkpoint_every` half steps from checkpoints kept by the
    forward pass.  Call as HermiteRun.apply(x0, c, plan, nhalf,
    checkpoint_every), c a 0-d FP64 tensor equal to the plan's wave speed;
    ``run`` fills in c."""

    @staticmethod
    def forward(ctx, x0, c, plan, nhalf, every):
        out, ckpt = _forward(plan, x0, nhalf, every)
        ctx.plan, ctx.nhalf, ctx.every, ctx.ckpt = plan, nhalf, every, ckpt
        return out

    @staticmethod
    def backward(ctx, g):
        need_c = ctx.needs_input_grad[1]
        last = ctx.nhalf - 1
        g = g.contiguous()

        def seed(adj, t):
            if t == last:
                adj.add_(g)
        adj, grad_c = _sweep(ctx.plan, ctx.nhalf, ctx.every, ctx.ckpt, need_c, seed)
        gc = torch.tensor(grad_c, dtype=torch.float64) if need_c else None
        return adj, gc, None, None, None


def _wave_speed(plan, c):
    if c is None:
        return torch.tensor(plan.c, dtype=torch.float64)
    if abs(float(c.detach()) - plan.c) > 1e-15 * plan.c:
        raise ValueError("c must equal the plan's wave speed")
    return c


def run(plan, x0, nhalf, checkpoint_every=20, c=None):
    """The state after `nhalf` half steps from x0 (on the primal grid), as a
    differentiable function of x0 (and of c: pass a 0-d FP64 tensor equal to
    the plan's wave speed with requires_grad)."""
    if nhalf < 1 or checkpoint_every < 1:
        raise ValueError("nhalf and checkpoint_every must be >= 1")
    return HermiteRun.apply(x0, _wave_speed(plan, c), plan, int(nhalf), int(checkpoint_every))


def receiver_traces(plan, u0, nhalf, receivers, checkpoint_every=20, c=None):
    """Traces of u at `receivers` (int64 device tensor of flat node indices)
    after each of `nhalf` half steps starting on the primal grid.  Pass a
    0-d tensor `c` (equal to the plan's wave speed, requires_grad) to also get
    dL/dc."""
    c = _wave_speed(plan, c)
    if checkpoint_every < 1:
        raise ValueError("checkpoint_every must be >= 1")
    return _ReceiverRun.apply(u0, c, plan, int(nhalf), receivers, int(checkpoint_every))
