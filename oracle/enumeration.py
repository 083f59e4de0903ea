"""Index enumerations of Alg. 1 and Alg. 2 (Sec. 2.1.1).

TEST INFRASTRUCTURE ONLY.  These generate the amplitude pairs a single-qubit
(Alg. 1) or controlled single-qubit (Alg. 2) gate updates.  They exist so the
tests can check the enumeration itself (the pairs partition the touched
subspace exactly) and its readings:

* the low mask of Alg. 1 at q_offset = 0 is read as (1 << q_offset) - 1 (the
  printed right shift by the full bit width is undefined in C);
* Alg. 2 inserts a zero bit at every sorted control/target offset, which the
  paper expresses with n+1 "gap" masks from getMasks; the combine step is read
  as a bitwise AND of k with the lowest gap mask;
* control bits are then set to the prescribed values (default all 1).
"""

from __future__ import annotations

from typing import Iterator, List, Sequence, Tuple


def insert_zero(k: int, pos: int) -> int:
    """Spread k so that bit ``pos`` of the result is 0 (bits at and above shift up)."""
    low = k & ((1 << pos) - 1)
    return ((k >> pos) << (pos + 1)) | low


def single_qubit_pairs(n: int, q: int) -> Iterator[Tuple[int, int]]:
    """Alg. 1: the 2^(n-1) disjoint pairs (i0, i1) a gate on wire q updates."""
    off = n - q - 1
    stride = 1 << off
    for k in range(1 << (n - 1)):
        i0 = insert_zero(k, off)
        yield i0, i0 | stride


def gap_masks(offsets: Sequence[int], width: int = 64) -> List[int]:
    """The len(offsets)+1 masks of the bit ranges strictly between sorted offsets."""
    bits = sorted(offsets)
    full = (1 << width) - 1
    masks = [(1 << bits[0]) - 1]
    for i in range(1, len(bits)):
        masks.append(((1 << bits[i]) - 1) & ~((1 << (bits[i - 1] + 1)) - 1))
    masks.append(full & ~((1 << (bits[-1] + 1)) - 1))
    return masks


def controlled_pairs(n: int, target: int, controls: Sequence[int],
                     control_values: Sequence[int] | None = None) -> Iterator[Tuple[int, int]]:
    """Alg. 2: pairs of a controlled single-qubit gate, 2^(n-1-len(controls)) of them."""
    vals = list(control_values) if control_values else [1] * len(controls)
    t_off = n - target - 1
    c_offs = [n - c - 1 for c in controls]
    masks = gap_masks(c_offs + [t_off])
    m = len(c_offs) + 1
    set_bits = 0
    for off, v in zip(c_offs, vals):
        if v:
            set_bits |= 1 << off
    for k in range(1 << (n - 1 - len(controls))):
        i0 = 0
        for i in range(m + 1):
            i0 |= (k << i) & masks[i]
        i0 |= set_bits
        yield i0, i0 | (1 << t_off)


def controlled_pairs_by_insertion(n: int, target: int, controls: Sequence[int],
                                  control_values: Sequence[int] | None = None):
    """Same pairs via one zero insertion per sorted offset (cross-check of the masks)."""
    vals = list(control_values) if control_values else [1] * len(controls)
    offs = sorted([n - c - 1 for c in controls] + [n - target - 1])
    for k in range(1 << (n - 1 - len(controls))):
        i0 = k
        for off in offs:
            i0 = insert_zero(i0, off)
        for c, v in zip(controls, vals):
            if v:
                i0 |= 1 << (n - c - 1)
        yield i0, i0 | (1 << (n - target - 1))
