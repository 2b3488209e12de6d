"""Differentiable runs: receivers, discrete adjoint and checkpointing.

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


class _ReceiverRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, c, plan, nhalf, idx, every):
        x = u0.detach().clone()
        y = torch.empty_like(x)
        traces = torch.empty((nhalf, idx.numel()), dtype=torch.float64, device=u0.device)
        ckpt = {0: x.clone()}
        for t in range(nhalf):
            plan.step(x, y, t % 2)
            plan.record(y, idx, traces[t])
            x, y = y, x
            if (t + 1) % every == 0 and t + 1 < nhalf:
                ckpt[t + 1] = x.clone()
        ctx.plan, ctx.nhalf, ctx.every, ctx.ckpt = plan, nhalf, every, ckpt
        ctx.save_for_backward(idx)
        return traces

    @staticmethod
    def backward(ctx, g):
        (idx,) = ctx.saved_tensors
        plan, nhalf, every, ckpt = ctx.plan, ctx.nhalf, ctx.every, ctx.ckpt
        g = g.contiguous().to(torch.float64)
        need_c = ctx.needs_input_grad[1]
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
                plan.inject(adj, idx, g[t])              # transpose of recording after step t
                if need_c:
                    plan.step_dc(states[t - s0], tmp, t % 2)
                    grad_c += plan.dot(adj, tmp)
                plan.adjoint(adj, tmp, t % 2)
                adj, tmp = tmp, adj
        gc = torch.tensor(grad_c, dtype=torch.float64) if need_c else None
        return adj, gc, None, None, None, None


def receiver_traces(plan, u0, nhalf, receivers, checkpoint_every=20, c=None):
    """Traces of u at `receivers` (int64 device tensor of flat node indices)
    after each of `nhalf` half steps starting on the primal grid.  Pass a
    0-d tensor `c` (equal to the plan's wave speed, requires_grad) to also get
    dL/dc."""
    if c is None:
        c = torch.tensor(plan.c, dtype=torch.float64)
    elif abs(float(c.detach()) - plan.c) > 1e-15 * plan.c:
        raise ValueError("c must equal the plan's wave speed")
    if checkpoint_every < 1:
        raise ValueError("checkpoint_every must be >= 1")
    return _ReceiverRun.apply(u0, c, plan, int(nhalf), receivers, int(checkpoint_every))
