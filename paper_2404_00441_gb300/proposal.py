"""Learned proposal: training pairs, training loop and gap calibration.

The paper has no learned component; this is the library's addition on top of
the best-match search of Algorithm 1. Every numeric step (simulation, encoder
inputs, forward/backward passes, AdamW, embedding tables, nearest-neighbour
selection) runs in libccw's kernels; this module only draws indices and moves
tensors between those calls.

Pairs: the plain method (K = 1, full search) runs on the TI and records, for
every searched patch, the facies counts of its level-J data event and the
candidate it picked (the exact best match). The encoder learns to map a data
event and the TI window of its best match, masked like the data event, to
nearby unit vectors (InfoNCE, temperature tau, in-batch plus random TI
negatives).
"""
from __future__ import annotations

import math

import torch

from . import ccw


def generate_pairs(ti: "ccw.TI", grid, n_real: int, seed: int, real_base: int = 0,
                   path_random: int = 0, chunk: int = 256):
    """Runs the plain method and returns (counts uint8 [n, F, tj*tj],
    best int32 [n]) for every patch it searched (not the uniform ones)."""
    counts_all, best_all = [], []
    done = 0
    while done < n_real:
        n = min(chunk, n_real - done)
        res = ccw.simulate_groups(ti, [dict(grid=grid, n_real=n, real_base=real_base + done)],
                                  topk=1, seed=seed, path_random=path_random, want_log=True,
                                  want_counts=True)
        _, log, counts = res[0]
        flags = log[..., 3]
        searched = ((flags & ccw.LOG_FLAG_DONE) != 0) & ((flags & ccw.LOG_FLAG_UNIFORM) == 0)
        counts_all.append(counts[searched].reshape(-1, counts.shape[2], counts.shape[3]))
        best_all.append(log[..., 0][searched].contiguous())
        done += n
    return torch.cat(counts_all).contiguous(), torch.cat(best_all).contiguous()


def train(ti: "ccw.TI", net: "ccw.Net", counts: torch.Tensor, best: torch.Tensor, steps: int,
          batch: int = 256, n_neg: int = 255, tau: float = 0.1, lr: float = 2e-3,
          wd: float = 1e-4, seed: int = 0, bf16: int = 1, log_every: int = 0):
    """InfoNCE training of ``net`` on (counts, best) pairs. Candidates of a
    step: the batch's positives, then ``n_neg`` random TI windows masked like
    random anchors of the batch. Returns the list of logged losses."""
    x_all, types = ti.proposal_inputs(0, counts=counts)
    n = x_all.shape[0]
    g = torch.Generator(device=counts.device)
    g.manual_seed(seed)
    losses = []
    for step in range(steps):
        # cosine learning-rate decay
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(steps, 1)))
        idx = torch.randint(0, n, (batch,), device=counts.device, generator=g)
        neg = torch.randint(0, ti.n_cand, (n_neg,), device=counts.device, generator=g,
                            dtype=torch.int64).to(torch.int32)
        neg_t = types[idx[torch.randint(0, batch, (n_neg,), device=counts.device, generator=g)]]
        cand = torch.cat([best[idx], neg]).contiguous()
        ctyp = torch.cat([types[idx], neg_t]).contiguous()
        cands = ti.proposal_inputs(1, cand=cand, types=ctyp)
        anchors = x_all[idx].contiguous()
        loss = net.train_step(anchors, cands, tau=tau, lr=lr_t, wd=wd, bf16=bf16)
        if log_every and (step % log_every == 0 or step == steps - 1):
            losses.append(float(loss.item()))
    return losses


def proposal_hits(ti: "ccw.TI", counts: torch.Tensor, best: torch.Tensor):
    """(hit bool [n], gap float [n], types int32 [n]): whether the exact best
    match is among the proposals of each data event (the attached tables)."""
    prop, gap, typ = ti.proposal_query(counts)
    hit = (prop == best[:, None]).any(dim=1) & (gap >= 0)
    return hit, gap, typ


def calibrate_gap(hit: torch.Tensor, gap: torch.Tensor, target_miss: float) -> float:
    """Smallest relative gap theta such that, among the data events with
    proposals and gap >= theta, the fraction whose best match is missed is
    at most ``target_miss``. Returns +inf when no theta meets the target."""
    ok = gap >= 0
    g = gap[ok]
    h = hit[ok]
    if g.numel() == 0:
        return float("inf")
    order = torch.argsort(g, descending=True)
    gs, miss = g[order], (~h[order]).to(torch.float64)
    rate = torch.cumsum(miss, 0) / torch.arange(1, gs.numel() + 1, device=gs.device)
    good = torch.nonzero(rate <= target_miss).flatten()
    if good.numel() == 0:
        return float("inf")
    return float(gs[good[-1]].item())
