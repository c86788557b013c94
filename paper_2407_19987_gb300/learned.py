"""Training and evaluation of the learned flip proposal.

The proposal network (MLP: 3 -> H -> H -> 1, bf16 weights) scores each bit
of a state from (clamp(beta*g_i, +-vmax)/8, 2x_i - 1, -ln(beta)/4).  It is
trained on trajectories of the plain annealer: every recorded attempt of
bit i is labelled 1 if the bit then differs from the state's final best
state, 0 otherwise, and the network minimises the mean binary
cross-entropy with Adam.  Recording, the forward and backward passes and
the optimiser all run in the library's kernels (hobo_anneal_learned with
recording, hobo_mlp_train_step); this module only schedules the calls and
draws minibatch indices.

The paper has no learned component; this is the tuned proposal of the
annealer (simulated annealing, Sec. II.D.1), measured against the plain
sweep by time to a target energy.
"""
from __future__ import annotations

import math
import time

import numpy as np

from .binding import MLP, Instance, anneal_learned


def record(instances, *, seed: int, B: int, betas: np.ndarray, rec_every: int, rec_states: int):
    """Run plain sweeps (no network) on each instance and collect the
    recorded (features, label) rows of every attempted bit.  Returns CUDA
    tensors F [rows, 3] and y [rows]."""
    import torch
    Fs, ys = [], []
    for t, inst in enumerate(instances):
        r = anneal_learned(inst, None, seed + t, B, betas, rec_every=rec_every, rec_states=rec_states)
        keep = r["rec_y"] >= 0
        Fs.append(r["rec_F"][keep])
        ys.append(r["rec_y"][keep])
    return torch.cat(Fs), torch.cat(ys)


def train(mlp: MLP, F, y, *, steps: int, batch: int, lr: float, seed: int = 0, log_every: int = 0):
    """Adam on minibatches drawn uniformly (with replacement) from (F, y).
    Returns the mean loss of every log_every-th step (device-side losses
    read back at the end)."""
    import torch
    gen = torch.Generator(device=F.device)
    gen.manual_seed(seed)
    loss = torch.zeros(max(steps, 1), dtype=torch.float32, device=F.device)
    n = F.shape[0]
    for s in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device=F.device, generator=gen)
        mlp.train_step(F[idx].contiguous(), y[idx].contiguous(), lr, loss[s:s + 1])
    out = loss.cpu().numpy()
    return out[::log_every] if log_every else out


def full_loss(mlp: MLP, F, y, chunk: int = 1 << 18) -> float:
    """Mean cross-entropy of the network over all rows."""
    tot = 0.0
    for r0 in range(0, F.shape[0], chunk):
        l, _ = mlp.loss_grad(F[r0:r0 + chunk].contiguous(), y[r0:r0 + chunk].contiguous())
        tot += float(l.item()) * min(chunk, F.shape[0] - r0)
    return tot / max(F.shape[0], 1)


def _timed(fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def run_schedule(inst: Instance, mlp, *, seed: int, B: int, betas: np.ndarray, **kw):
    """One anneal with the learned proposal (mlp=None: the tuned plain
    sweep).  Returns (best energies as numpy float64, milliseconds of the
    whole call including initial energies and the float64 re-score)."""
    if mlp is None:
        r, ms = _timed(lambda: inst.anneal(seed, B, betas, mode=0))
    else:
        r, ms = _timed(lambda: anneal_learned(inst, mlp, seed, B, betas, **kw))
    return r["bestE"].cpu().numpy(), ms


def time_to_target(inst: Instance, target: float, mlp, *, seed: int, B: int, T0: float, T1: float,
                   sweeps_list=(5, 10, 15, 20, 25, 35, 50, 70, 100, 140, 200, 280, 400, 560, 800, 1120, 1600,
                                2240, 3200), **kw) -> dict:
    """Time to target: for schedules of growing length (geometric, T0 ->
    T1), the wall time of the first whole anneal whose best state reaches
    ``target`` (energy <= target).  Each length is a fresh anneal of B
    states; the time of the shorter ones that missed is reported apart."""
    from workloads import geometric_betas  # seeded schedule helper, no solver arithmetic
    spent = 0.0
    for S in sweeps_list:
        E, ms = run_schedule(inst, mlp, seed=seed, B=B, betas=geometric_betas(T0, T1, S), **kw)
        if float(E.min()) <= target:
            return dict(sweeps=S, ms=ms, ms_including_misses=spent + ms, best=float(E.min()))
        spent += ms
    return dict(sweeps=None, ms=None, ms_including_misses=spent, best=float(E.min()))
