"""Plain model of the smart-container coherence protocol -- TEST INFRASTRUCTURE ONLY.

Sec. IV of the paper: a smart container tracks in which memory units valid
copies of its payload exist, reuses a valid copy close to the executing unit,
never lets a stale copy be read, and starts a transfer only when the unit that
accesses the data holds no valid copy ("lazy memory copying").

Two memory units here: host (H) and device (D).  State = set of units holding
a valid copy; a new container holds none (its contents are undefined).  For an
access by unit U with mode m:
  * a read (m in {R, RW}) of U when U is not valid and the other unit is
    valid copies other -> U (one transfer) and adds U to the valid set;
  * a read when nothing is valid copies nothing and leaves the set empty
    (the contents stay undefined until some unit writes);
  * a write (m in {W, RW}) leaves U as the only valid unit.
Whole-operand granularity (one transfer moves the whole container).
"""
from __future__ import annotations

HOST, DEVICE = 1, 2          # bits of the valid set
READ, WRITE, READWRITE = 1, 2, 3
NONE, H2D, D2H = 0, 1, 2


def step(valid: int, unit: int, mode: int) -> tuple[int, int]:
    """Returns (new valid set, transfer) for one access."""
    other = DEVICE if unit == HOST else HOST
    transfer = NONE
    if mode & READ:
        if not (valid & unit) and (valid & other):
            transfer = H2D if unit == DEVICE else D2H
            valid |= unit
    if mode & WRITE:
        valid = unit
    return valid, transfer


class Model:
    """Replays a sequence of accesses and counts transfers."""

    def __init__(self, valid: int = 0):
        self.valid = valid
        self.h2d = 0
        self.d2h = 0

    def access(self, unit: int, mode: int) -> int:
        self.valid, t = step(self.valid, unit, mode)
        self.h2d += t == H2D
        self.d2h += t == D2H
        return t
