"""Slab decomposition of one domain along y, and the halo exchange between
ranks that hold different slabs.

On one device the library splits a domain itself (eulbfs_add_split_domain)
and copies the halo rows between its slabs after every Runge-Kutta stage.
This module holds the same schedule on the host -- which rows each slab
owns, which slabs are neighbours, which rows go where -- for slabs spread
over several processes, and runs the exchange with torch.distributed
point-to-point messages (gloo on the CPU, NCCL on GPUs).  The arrays hold a
slab's planes with its halo rows, in the library's layout: (planes,
halo_lo + rows + halo_hi, nx), row-major, x fastest.

HALO is the stencil's ghost width: two rows for the gradients of Eq. 54 and
a third for the Laplacian of C in mu_c (Sec. 2.3.1).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

HALO = 3


def split_rows(ny: int, k: int) -> List[Tuple[int, int]]:
    """Rows [y0, y1) of each of the k slabs (the library's rule)."""
    return [(i * ny // k, (i + 1) * ny // k) for i in range(k)]


def halo_sides(k: int, periodic: bool) -> List[Tuple[int, int]]:
    """(halo rows below, halo rows above) of each slab."""
    return [(HALO if (i > 0 or periodic) and k > 1 else 0, HALO if (i < k - 1 or periodic) and k > 1 else 0)
            for i in range(k)]


def halo_links(k: int, periodic: bool) -> List[Tuple[int, int]]:
    """(lower slab, upper slab) pairs whose halo rows are exchanged; on a
    periodic axis the top slab is also the bottom slab's lower neighbour."""
    if k < 2:
        return []
    links = [(i, i + 1) for i in range(k - 1)]
    if periodic:
        links.append((k - 1, 0))
    return links


def owners(k: int, world: int) -> List[int]:
    """Rank of each slab: contiguous blocks of slabs per rank."""
    return [i * world // k for i in range(k)]


def _rows(a, lo: int, hi: int) -> int:
    """Interior rows of a slab's array with lo and hi halo rows."""
    return a.shape[1] - lo - hi


def exchange(planes: Dict[int, "object"], k: int, periodic: bool, rank: int = 0, world: int = 1) -> int:
    """Fill the halo rows of this rank's slabs (`planes`: slab index -> array
    of shape (planes, lo + rows + hi, nx), torch tensors or numpy arrays) from
    their neighbours' outermost interior rows: copies between this rank's own
    slabs, point-to-point messages to and from the other ranks' slabs.
    Returns the number of messages sent.  Every rank calls it with the same
    k and periodic; the messages of all links are posted before any is
    waited for, so the order of links cannot deadlock."""
    sides = halo_sides(k, periodic)
    own = owners(k, world)
    sends, recvs, local = [], [], []
    for lo_s, hi_s in halo_links(k, periodic):
        for src, dst, up in ((lo_s, hi_s, True), (hi_s, lo_s, False)):
            if own[src] != rank and own[dst] != rank:
                continue
            if own[src] == rank:
                a = planes[src]
                slo, shi = sides[src]
                n = _rows(a, slo, shi)
                rows = a[:, slo + n - HALO: slo + n] if up else a[:, slo: slo + HALO]
            if own[dst] == rank:
                b = planes[dst]
                dlo, dhi = sides[dst]
                m = _rows(b, dlo, dhi)
                halo = b[:, 0: HALO] if up else b[:, dlo + m: dlo + m + HALO]
            if own[src] == rank and own[dst] == rank:
                local.append((halo, rows))
            elif own[src] == rank:
                sends.append((rows, own[dst], src, up))
            else:
                recvs.append((halo, own[src], src, up))
    for halo, rows in local:
        halo[...] = rows
    if not sends and not recvs:
        return 0
    import torch
    import torch.distributed as dist

    def tag(src_slab: int, up: bool) -> int:
        return 2 * src_slab + (1 if up else 0)

    reqs, bufs = [], []
    for rows, peer, src, up in sends:
        t = torch.as_tensor(rows).contiguous()
        bufs.append(t)
        reqs.append(dist.isend(t, peer, tag=tag(src, up)))
    pending = []
    for halo, peer, src, up in recvs:
        t = torch.empty(tuple(halo.shape), dtype=torch.as_tensor(halo).dtype)
        reqs.append(dist.irecv(t, peer, tag=tag(src, up)))
        pending.append((halo, t))
    for r in reqs:
        r.wait()
    for halo, t in pending:
        halo[...] = t.numpy() if not hasattr(halo, "copy_") else t
    return len(sends)


def assemble(parts: Sequence, k: int, periodic: bool):
    """The interior rows of the k slabs (in slab order) stacked back into the
    domain's planes."""
    import numpy as np
    sides = halo_sides(k, periodic)
    return np.concatenate([p[:, lo: p.shape[1] - hi] for p, (lo, hi) in zip(parts, sides)], axis=1)
