"""Row decomposition of one large instance into y-slabs, one per rank.

Host-side index logic only; no kernels and no collectives live here. With PLM
(two cells on each side of a face) the update of row j reads rows j-2 .. j+2,
so a rank that owns rows [y0, y1) and also holds HALO rows on each side that
has a neighbour computes its own rows exactly as the whole-domain step does.
Before every RK stage the neighbours refresh those halo rows: each rank sends
its lowest HALO rows down and its highest HALO rows up. The time step is the
minimum over ranks of each slab's crossing-time minimum, and sums over cells
(objective, constraint) are sums over ranks of each slab's own rows. At the
physical walls (y = y0 and y = y1 of the domain) the slab holds no halo and
the boundary condition applies as in the whole-domain step.

The reverse sweep works on whole steps: the transposed step maps the
cotangent of row k back to rows k-4 .. k+4 (two stages of two rows each), and
the forward map behind row k reads the state four rows further out. A rank
therefore applies the reverse of one step to its own rows exactly when it
holds the step's input state and the incoming cotangent with STEP_REVERSE_HALO
rows on each side; after the step it refreshes the cotangent halos.
"""
from __future__ import annotations

from dataclasses import dataclass

HALO = 2               # rows on each side that one PLM + flux + update stage reads
STEP_REVERSE_HALO = 8  # rows on each side that the reverse of one RK2 step reads


@dataclass(frozen=True)
class Slab:
    rank: int
    world: int
    y0: int          # first owned row
    y1: int          # one past the last owned row
    e0: int          # first held row (owned rows plus halos)
    e1: int          # one past the last held row
    down: int | None  # rank owning the rows below, or None at the bottom wall
    up: int | None    # rank owning the rows above, or None at the top wall
    halo: int = HALO  # halo rows held on each side with a neighbour

    @property
    def own(self) -> slice:
        """Owned rows as a slice of the held rows."""
        return slice(self.y0 - self.e0, self.y1 - self.e0)

    def send_down(self) -> slice:
        """Held-row slice sent to the rank below (its upper halo)."""
        return slice(self.y0 - self.e0, self.y0 - self.e0 + self.halo)

    def send_up(self) -> slice:
        """Held-row slice sent to the rank above (its lower halo)."""
        return slice(self.y1 - self.e0 - self.halo, self.y1 - self.e0)

    def recv_down(self) -> slice:
        """Held-row slice filled by the rank below."""
        return slice(0, self.y0 - self.e0)

    def recv_up(self) -> slice:
        """Held-row slice filled by the rank above."""
        return slice(self.y1 - self.e0, self.e1 - self.e0)


def slab_rows(ny: int, world: int, halo: int = HALO) -> list[tuple[int, int]]:
    """Owned rows [y0, y1) of each rank: ny split as evenly as possible, the
    first ny % world ranks one row taller; every slab at least `halo` rows, so
    that a halo comes from a single neighbour."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if ny < halo * world:
        raise ValueError(f"{ny} rows cannot give {world} slabs of at least {halo} rows")
    base, extra = divmod(ny, world)
    out, y = [], 0
    for r in range(world):
        h = base + (1 if r < extra else 0)
        out.append((y, y + h))
        y += h
    return out


def slab(ny: int, world: int, rank: int, halo: int = HALO) -> Slab:
    """The slab of `rank`: owned rows, held rows (with `halo` rows on each
    side that has a neighbour) and neighbours. The owned rows do not depend on
    the halo width, as long as every slab has at least `halo` rows."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    y0, y1 = slab_rows(ny, world, halo)[rank]
    down = rank - 1 if rank > 0 else None
    up = rank + 1 if rank < world - 1 else None
    e0 = y0 - halo if down is not None else y0
    e1 = y1 + halo if up is not None else y1
    return Slab(rank, world, y0, y1, e0, e1, down, up, halo)
