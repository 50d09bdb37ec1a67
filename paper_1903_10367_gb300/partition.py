"""Slab partition of a regular tree for several GPUs (the vertical-integration
split of Sec. 4.3 and Sec. 5.5, "Parallel adAFAC").

Host-side planning only: which fine planes a rank owns, which planes it needs
from its neighbours, and which coarse planes receive partial sums from more
than one rank.  The arithmetic of the cycle is unchanged; every run of this
repository has one GPU, so no multi-GPU cycle is built on it (the plan is
exercised by a two-rank CPU test).

The finest level (n cells per axis, interior planes 1 .. n-1 along z) is cut
into contiguous slabs of planes, one per rank.  Every rank keeps all coarser
levels in full (the paper's replicated ancestors).  One cycle then needs:

* one halo exchange of the iterate: the fine residual of plane z reads planes
  z - 1 .. z + 1, so a rank needs the plane just below and just above its
  slab;
* one sum over the ranks of the partial level-(L-1) vectors: a rank restricts
  the residual of its own planes (R r_L and the damping right-hand side
  R~ r_L, both sums over the 5^d window of fine vertices 3J + o), and coarse
  planes whose window reaches into two slabs receive a part from each;
* nothing else: the levels below L - 1 and the prolongation to the rank's own
  planes are computed redundantly from the summed vectors.
"""
from __future__ import annotations

import dataclasses


@dataclasses.dataclass(frozen=True)
class Slab:
    rank: int
    world: int
    n: int                      # fine cells per axis
    z0: int                     # owned interior fine planes [z0, z1)
    z1: int
    halo: tuple                 # fine planes read from the neighbours' slabs
    coarse_shared: tuple        # coarse planes whose windows reach another slab

    @property
    def planes(self) -> range:
        return range(self.z0, self.z1)


def plan(n: int, world: int) -> list:
    """Balanced contiguous slabs of the interior fine planes 1 .. n-1 (n = 3^L)
    for `world` ranks, with the halo planes and the shared coarse planes."""
    if n < 3 or n % 3 != 0:
        raise ValueError("n must be a power of 3, at least 3")
    interior = n - 1
    if not 1 <= world <= interior:
        raise ValueError("between 1 and n - 1 ranks")
    cuts = [1 + (interior * r) // world for r in range(world + 1)]
    nc = n // 3

    def owner(z):
        for r in range(world):
            if cuts[r] <= z < cuts[r + 1]:
                return r
        return None            # boundary plane (Dirichlet data, no owner)

    slabs = []
    for r in range(world):
        z0, z1 = cuts[r], cuts[r + 1]
        halo = tuple(z for z in (z0 - 1, z1) if owner(z) not in (None, r))
        shared = []
        for m in range(1, nc):
            owners = {owner(z) for z in range(3 * m - 2, 3 * m + 3)} - {None}
            if r in owners and len(owners) > 1:
                shared.append(m)
        slabs.append(Slab(r, world, n, z0, z1, halo, tuple(shared)))
    return slabs
