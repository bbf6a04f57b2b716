"""One large O-grid split over ranks along its periodic angular index.

The method's step is local: a node's new populations come from the Q2
element around its departure point (Eq. SemiLagrProp), which lies in a cell
next to the node, and its correction field Y (Sec. II C) is a second
derivative of the moment field; the only global coupling is the load on the
body (Sec. III), which drives the rigid-body update (Sec. III B).  So one
mesh splits into contiguous ranges of angular columns, one per rank, with

  - one exchange per step of halo columns: a rank needs, beside its own
    columns, a few columns of each neighbour's state, as many as the step's
    stencils reach (the step kernel keeps pre-collision populations and the
    moment field between launches and reads them on +-2 and +-4 columns; a
    stepper that keeps post-collision populations reads both on +-4: its own
    columns collide with Y, which reaches the moments two columns out, and
    those moments come from populations streamed from a Q2 window two
    columns further, or, on the wall and far-field rows, from the previous
    moment field at the target point B, whose window reaches as far);
  - the load as a fixed-order sum: every rank contributes the terms of the
    wall edges it owns, all ranks gather every rank's terms and sum them in
    the global edge order, so the load (and the body update that every rank
    then computes for itself) is bit-identical to the one-rank sum and the
    same on every rank.

Ranges are whole tiles of the step kernel (32 columns), so that a rank's
launch covers whole tiles.  Exchanges are point-to-point sends and receives
of column strips between angular neighbours (torch.distributed: gloo on CPU
ranks, NCCL between GPUs), no collective on the field data.
"""
from __future__ import annotations

from dataclasses import dataclass

TILE = 32

# columns of state read beyond a rank's own range, per representation of the
# state kept between steps
HALO_PRE_COLLISION = {"populations": 2, "moments": 4}    # the step kernel
HALO_POST_COLLISION = {"populations": 4, "moments": 4}   # stream-then-collide steppers


@dataclass(frozen=True)
class AngularPartition:
    """Contiguous angular ranges [j0, j1) of an O-grid with nt columns over
    nranks ranks, each a whole number of tiles (the last may be ragged)."""
    nt: int
    nranks: int
    tile: int = TILE

    def __post_init__(self):
        ntiles = -(-self.nt // self.tile)
        if self.nranks < 1 or self.nranks > ntiles:
            raise ValueError(f"{self.nranks} ranks for {ntiles} tiles of {self.tile} columns")

    @property
    def ntiles(self) -> int:
        return -(-self.nt // self.tile)

    def tiles(self, rank: int) -> tuple[int, int]:
        """Tile range [t0, t1) of a rank: as even as the tile count allows."""
        t0 = (rank * self.ntiles) // self.nranks
        t1 = ((rank + 1) * self.ntiles) // self.nranks
        return t0, t1

    def owned(self, rank: int) -> tuple[int, int]:
        t0, t1 = self.tiles(rank)
        return t0 * self.tile, min(t1 * self.tile, self.nt)

    def neighbours(self, rank: int) -> tuple[int, int]:
        """Ranks owning the columns just before and just after this rank's
        range (the angular index is periodic)."""
        return (rank - 1) % self.nranks, (rank + 1) % self.nranks

    def check_halo(self, width: int):
        """A halo must come from the adjacent rank alone: no range narrower
        than the widest halo."""
        narrow = min(self.owned(r)[1] - self.owned(r)[0] for r in range(self.nranks))
        if width > narrow:
            raise ValueError(f"halo of {width} columns wider than the narrowest range ({narrow})")

    def halo_columns(self, rank: int, width: int):
        """Global column indices of the left and right halo of a rank, in
        increasing angular order (wrapped)."""
        j0, j1 = self.owned(rank)
        left = [(j0 - width + k) % self.nt for k in range(width)]
        right = [(j1 + k) % self.nt for k in range(width)]
        return left, right

    def local_columns(self, rank: int, width: int):
        """Global columns a rank holds: left halo, own range, right halo."""
        left, right = self.halo_columns(rank, width)
        j0, j1 = self.owned(rank)
        return left + list(range(j0, j1)) + right


def exchange_halos(part: AngularPartition, rank: int, arrays, width: int, dist=None):
    """Fill the halo columns of full-width arrays [..., nt] (angular index
    last) from the angular neighbours: this rank's first `width` own columns
    go to the left neighbour (its right halo) and its last `width` to the
    right neighbour (its left halo).  Arrays are torch tensors (CPU for gloo,
    CUDA for NCCL); the strips travel as contiguous copies.  With one rank
    the periodic wrap is a local copy."""
    if width == 0:
        return
    part.check_halo(width)
    j0, j1 = part.owned(rank)
    lo, hi = part.neighbours(rank)
    left, right = part.halo_columns(rank, width)
    for a in arrays:
        first = a[..., j0:j0 + width].contiguous()
        last = a[..., j1 - width:j1].contiguous()
        if part.nranks == 1:
            a[..., left] = last
            a[..., right] = first
            continue
        recv_left = last.new_empty(last.shape)
        recv_right = first.new_empty(first.shape)
        # tags tell the strips apart where both neighbours are one rank (two
        # ranks on a ring): 0 fills a left halo, 1 a right halo
        ops = [dist.P2POp(dist.isend, first, lo, tag=1), dist.P2POp(dist.isend, last, hi, tag=0),
               dist.P2POp(dist.irecv, recv_left, lo, tag=0), dist.P2POp(dist.irecv, recv_right, hi, tag=1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        a[..., left] = recv_left
        a[..., right] = recv_right


def gather_in_order(part: AngularPartition, local, dist=None):
    """Concatenate every rank's 1-D float64 tensor of terms in rank order
    (the global order of the terms, since ranks own increasing ranges).
    Ranks may hold different counts."""
    if part.nranks == 1:
        return local
    import torch
    n = torch.tensor([local.numel()], dtype=torch.int64)
    counts = [torch.zeros_like(n) for _ in range(part.nranks)]
    dist.all_gather(counts, n)
    width = int(max(c.item() for c in counts))
    pad = torch.zeros(width, dtype=local.dtype)
    pad[:local.numel()] = local
    bufs = [torch.zeros_like(pad) for _ in range(part.nranks)]
    dist.all_gather(bufs, pad)
    return torch.cat([b[:int(c.item())] for b, c in zip(bufs, counts)])


def ordered_sum(terms):
    """Left-to-right sum of a sequence of floats (the one-rank order)."""
    s = 0.0
    for t in terms:
        s += float(t)
    return s
