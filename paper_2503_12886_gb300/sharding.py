"""Frame-sharded data-parallel training step: one process per GPU, one all-reduce per step.

The frames of a batch are independent through every step of the rasterizer (blend, projection,
binning, compositing, the compositing and projection backward; Sec. 3.2, Fig. 4c); they meet
only in the adjoint of Eq. 1, whose sums over the batch's frames give dL/dG0 and dL/ddG. So
each rank renders its own share of the batch's frames against a replica of the avatar, with
the loss averaged over the whole batch (rgba_batch.loss_frames = the global batch size), which
makes its dG0 and ddG its share of the batch's; one sum all-reduce of one flat buffer holding
every model's dG0 and ddG then gives each rank the batch gradient, and the identical Adam update
on every rank keeps the replicas equal. dL/dpsi belongs to each frame (it feeds the MLP that
produced that frame's weights, outside this path): it stays on the rank that rendered the frame
and is gathered only for reporting.

The helpers work on any torch.distributed backend: NCCL with CUDA tensors on GPUs, gloo with
CPU tensors in the tests.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(n_frames: int, world: int, rank: int) -> range:
    """The contiguous frames [start, stop) of rank `rank` when n_frames are split over `world`
    ranks as evenly as possible (the first n_frames % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_frames, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def grad_layout(models) -> list[tuple[int, int, int]]:
    """Offsets in the flat gradient buffer: per model (offset of dG0 [14][n_pad], offset of
    ddG [k][A][n_pad], end), for models with n_pad and a dg array of that shape. Every offset
    is a multiple of 4 floats (n_pad is), so every view is 16-byte aligned as the library
    requires."""
    out, at = [], 0
    for m in models:
        g0 = 14 * m.n_pad
        dg = 1
        for d in m.dg.shape:  # [k][A][n_pad]
            dg *= int(d)
        out.append((at, at + g0, at + g0 + dg))
        at += g0 + dg
    return out


def attach_flat_grads(models, device=None, dtype=torch.float32) -> torch.Tensor:
    """One zeroed buffer for every model's dG0 and ddG, with each DeviceModel's grad_g0 and
    grad_dg set to views of it (so the backward writes straight into what the all-reduce
    sends). Returns the buffer."""
    lay = grad_layout(models)
    total = lay[-1][2] if lay else 0
    dev = device if device is not None else (models[0].g0.device if models else "cpu")
    flat = torch.zeros(total, dtype=dtype, device=dev)
    for m, (a, b, c) in zip(models, lay):
        m.grad_g0 = flat[a:b].view(14, m.n_pad)
        m.grad_dg = flat[b:c].view(*m.dg.shape)
    return flat


def all_reduce_grads(flat: torch.Tensor, group=None) -> None:
    """The step's one exchange: the sum over ranks of every model's dG0 and ddG, in place.
    Each rank's share is already scaled by its loss normalisation (loss_frames), so the sum is
    the batch gradient; ranks end with identical buffers."""
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)


def all_reduce_loss(loss: float, device, group=None) -> float:
    """The batch loss: the sum of the ranks' shares (each already divided by the global frame
    count)."""
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return float(loss)
    t = torch.tensor([loss], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def gather_psi_grads(local: torch.Tensor, n_frames: int, group=None) -> torch.Tensor:
    """dL/dpsi of the whole batch ([n_frames][k_stride]) from each rank's rows of its own
    frames (the shard() split), for reporting; every rank receives it."""
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return local.clone()
    world = dist.get_world_size(group)
    k = local.shape[1]
    rows = max(len(shard(n_frames, world, r)) for r in range(world))
    pad = torch.zeros(rows, k, dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][:len(shard(n_frames, world, r))] for r in range(world)], 0)
