"""Index maps of the row-slab decomposition of one image over ranks.

The paper divides its transform among 2^l processes, each computing a share
before they exchange results (Sec. 2).  The library divides one image of the
Sec. 5 pipeline by rows instead (include/gbfft.h, fft2_slab_*): rank r owns
the row pairs (p, N - p), p in [r P, (r + 1) P), P = N / (2 R), and the
half-spectrum columns [r C, (r + 1) C), C = M / (2 R), for R ranks of an
N x M image.  The row pass stores a rank's spectra as [M/2][L], L = N / R
(its slots of every column); an all-to-all of R equal chunks then hands rank
q the chunks [R][C][L] of its columns, and the same all-to-all brings them
back.  This module states those maps in plain Python (no library, no GPU) so
that the exchange can be checked on CPU ranks; the kernels implement the same
maps (layout.cuh: slot order, Slab, ColSlab).
"""

from __future__ import annotations


def pairs_per_block(cols: int) -> int:
    """Row pairs per block of the row pass (512 threads: 512 / (cols / 16), at least 2)."""
    t = max(1, cols // 16) if cols >= 16 else 1
    return max(2, 512 // t)


def check(rows: int, cols: int, nranks: int) -> None:
    def pow2(n):
        return n >= 1 and n & (n - 1) == 0

    if not (pow2(rows) and pow2(cols) and pow2(nranks)) or rows < 2 or cols < 4:
        raise ValueError("rows, cols and nranks must be powers of two (rows >= 2, cols >= 4)")
    g = min(pairs_per_block(cols), rows // 2)
    p = rows // (2 * nranks)
    if p < g or p % g or cols // (2 * nranks) < 1:
        raise ValueError(f"{nranks} ranks: each needs a multiple of {g} row pairs and at least one column")


def rows_of_pair(p: int, rows: int) -> tuple[int, int]:
    return p, (rows // 2 if p == 0 else rows - p)


def pair_range(rows: int, nranks: int, rank: int) -> range:
    P = rows // (2 * nranks)
    return range(rank * P, (rank + 1) * P)


def slab_rows(rows: int, nranks: int, rank: int) -> list[int]:
    """The image rows rank `rank` reads and writes: its pairs' first rows, then their mirrors."""
    pr = pair_range(rows, nranks, rank)
    return [rows_of_pair(p, rows)[0] for p in pr] + [rows_of_pair(p, rows)[1] for p in pr]


def column_block(cols: int, nranks: int, rank: int) -> tuple[int, int]:
    """(first global half-spectrum column, number of columns) of rank `rank`."""
    C = cols // (2 * nranks)
    return rank * C, C


def slot_of_row(x: int, rows: int, log2g: int) -> int:
    """Slot of image row x within a half-spectrum column (layout.cuh, slot order)."""
    h = rows // 2
    if x < h:
        p, side = x, 0
    elif x == h:
        p, side = 0, 1
    else:
        p, side = rows - x, 1
    return ((p >> log2g) << (log2g + 1)) + (side << log2g) + (p & ((1 << log2g) - 1))


def send_offset(k: int, local_slot: int, rows: int, nranks: int) -> int:
    """Element of global column k, local slot s in a rank's send (and back) buffer [M/2][L]."""
    return k * (rows // nranks) + local_slot


def recv_offset(kl: int, slot: int, rows: int, cols: int, nranks: int) -> int:
    """Element of local column kl, GLOBAL slot s in the received buffer [R][C][L]
    (chunk s // L from rank s // L): the address the column pass reads."""
    L = rows // nranks
    C = cols // (2 * nranks)
    return ((slot // L) * C + kl) * L + slot % L


def exchange(src, dst, group=None) -> None:
    """One exchange of the decomposition: chunk q of this rank's `src`
    (complex64, R equal contiguous chunks) to rank q, the chunks from every
    rank into `dst` in rank order (torch.distributed all_to_all_single)."""
    import torch
    import torch.distributed as dist

    dist.all_to_all_single(torch.view_as_real(dst), torch.view_as_real(src), group=group)
