"""Row sharding of one fit (Algorithm 4 across devices).

Algorithm 4 accumulates F = sum_s U_s^T X_s over row slices X_s, so a fit
shards by rows: every rank holds a contiguous block of rows, regenerates Omega
from the seed (counter-based, nothing is broadcast), computes its own partial
F_g = U_g^T X_g (and G_g = U_g^T U_g) with the library, and one exchange sums
the partials.  The k x k step then runs replicated on every rank; projection
is row-parallel with V replicated.

The exchange gathers every rank's FP64 partial and adds them in rank order, so
all ranks hold bit-identical sums whatever the collective's own reduction
order.  ``virtual_shards`` runs the same split on one device: S row ranges
whose partials are added in the same fixed order.
"""
from __future__ import annotations

import torch


def row_range(m: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block of rows of rank ``rank`` out of ``world`` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    q, r = divmod(m, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def ordered_sum(parts: list[torch.Tensor]) -> torch.Tensor:
    """sum_g parts[g] in index order, in FP64."""
    acc = parts[0].to(torch.float64).clone()
    for p in parts[1:]:
        acc += p.to(torch.float64)
    return acc


def reduce_partials(F: torch.Tensor, G: torch.Tensor | None = None, group=None, ctx=None) -> tuple:
    """Sum the per-rank partials F (k x n) and G (k x k) over the process group.

    All-gathers the FP64 partials and adds them in rank order -- on CUDA
    tensors in the library (lspca_sum_partials, with ``ctx``), on host tensors
    with ``ordered_sum`` -- so every rank ends with the same bits.  Without an
    initialised process group this is the identity.
    """
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return F, G
    ws = dist.get_world_size(group)
    if ws == 1:
        return F, G
    outs = []
    for t in (F, G):
        if t is None:
            outs.append(None)
            continue
        t64 = t.to(torch.float64).contiguous()
        parts = [torch.empty_like(t64) for _ in range(ws)]
        dist.all_gather(parts, t64, group=group)
        if t64.is_cuda:
            gathered = torch.stack(parts)
            if ctx is None:
                raise ValueError("a CUDA exchange needs the library context")
            from . import lspca as L
            out = torch.empty_like(t64)
            rc = L.lspca_sum_partials(ctx.handle, gathered, out)
            if rc != L.OK:
                raise L.LspcaError(rc, "lspca_sum_partials")
            outs.append(out)
        else:
            outs.append(ordered_sum(parts))
    return outs[0], outs[1]


def max_over_ranks(x: float, device=None, group=None) -> float:
    """Largest value of ``x`` over the ranks (a timing reduction)."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_fit(ctx, X_local: torch.Tensor, m_total: int, k: int, om, want_gram: bool = False,
                group=None, virtual_shards: int = 1, vt=torch.float32):
    """Lazy SPCA fit of the row-sharded matrix whose rows ``X_local`` this rank holds.

    Per rank (and per virtual shard): U_g = X_g Omega (library sketch), then
    F_g = U_g^T X_g (library chain, FP64 partial).  The partials are summed in
    a fixed order (virtual shards first, then ranks), and the library's k x k
    step gives V and sigma from the summed F, with the rank rule evaluated for
    the global row count ``m_total``.
    Returns (V, sigma, rank, F, G).
    """
    rows = X_local.shape[0]
    Fs, Gs = [], []
    for s in range(max(1, virtual_shards)):
        lo, hi = row_range(rows, max(1, virtual_shards), s)
        Xs = X_local[lo:hi]
        U = ctx.sketch(Xs, k, om)
        F, G = ctx.chain(Xs, U, want_gram=want_gram)
        Fs.append(F)
        Gs.append(G)
    F = ordered_sum(Fs)
    G = ordered_sum(Gs) if want_gram else None
    F, G = reduce_partials(F, G, group, ctx)
    V, sigma, rank = ctx.decompose(F, m_total, vt=vt)
    return V, sigma, rank, F, G
