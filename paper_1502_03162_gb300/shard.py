"""Source sharding over processes, one GPU each (Sec. II: the render is linear in the sources
and the resonance f of Eq. 2 is shared by all of them).

Rank r of a world of W renders the reflection mix z_r of its contiguous slice of the sources
(``shard_range``) with the sparse taps alone; the W mixes are gathered in rank order (the
one exchange of the path: 2 x z_len FP32 per rank), and every rank applies the resonance once
to their sum, added in rank order, so that every rank holds the same stereo output

    out_e = f_e * sum_r z_{r,e},

which equals the single-GPU render of the whole batch up to the order of the FP32 sums.  The
arithmetic runs in the library (hrir_render_reflections, hrir_apply_resonance); this module
only partitions the sources and moves the mixes between ranks (torch.distributed).
"""
from __future__ import annotations


def shard_range(n_src: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous source slice [s0, s1) of `rank`: sizes differ by at most one, earlier
    ranks take the larger ones."""
    if world < 1 or not 0 <= rank < world or n_src < 0:
        raise ValueError(f"bad shard (n_src={n_src}, rank={rank}, world={world})")
    base, extra = divmod(n_src, world)
    s0 = rank * base + min(rank, extra)
    return s0, s0 + base + (1 if rank < extra else 0)


def gather_parts(z, group=None):
    """[2][z_len] on every rank -> [world][2][z_len], rank r's mix at index r (all ranks get
    the same tensor).  A single process (no process group) returns z as one part."""
    import torch
    import torch.distributed as dist
    z = z.contiguous()
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return z.unsqueeze(0)
    world = dist.get_world_size(group)
    parts = torch.empty((world,) + tuple(z.shape), dtype=z.dtype, device=z.device)
    dist.all_gather(list(parts.unbind(0)), z, group=group)
    return parts


def render_sharded(rend, src, dirs, full=True, length=None, group=None, stream=None):
    """Render this rank's sources (src [S_r][ld], dirs [S_r] on its GPU) and return the stereo
    output of every rank's sources together ([2][out_len], the same on every rank).
    `rend` needs render_reflections(src, dirs, full, length, stream) and
    apply_resonance(parts, full, stream) (hrir.Renderer has both)."""
    z = rend.render_reflections(src, dirs, full=full, length=length, stream=stream)
    parts = gather_parts(z, group)
    return rend.apply_resonance(parts, full=full, stream=stream)
