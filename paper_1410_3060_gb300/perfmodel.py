"""Performance models: bytes and flops per lattice update (LUP), the paper's
CPU code-balance and cache-block-size models, and roofline arithmetic.

Paper models (arXiv 1410.3060):

* code balance B_C of the naive sweep in bytes/LUP (Sect. 3.3), with the CPU write-allocate transfer counted unless non-temporal
  stores are used;
* roofline P = b_S / B_C (Sect. 3.3);
* cache block size of one wavefront-diamond tile (Sect. 5.3, the equations
  for R = 1 and general R), with W_w the wavefront width.

GPU model: a GPU store does not allocate, so the plain one-step sweep moves
exactly one read of every input stream and one write of the output per
update; a sweep that applies b time levels per pass ideally moves that
amount once per b levels.
"""
from __future__ import annotations

J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA = 1, 2, 3, 4, 5, 6

# number of domain-sized streams read per update besides the stencil field
_COEFF_ARRAYS = {J7_CONST: 0, J7_VAR: 7, W25_CONST: 0, W25_VAR: 13, J25_VAR: 13, W25_ALPHA: 1}
_SECOND_ORDER = {J7_CONST: False, J7_VAR: False, W25_CONST: True, W25_VAR: True,
                 J25_VAR: False, W25_ALPHA: True}

# flops per update (FMA = 2) and the minimum FP instructions per update,
# after folding constant factors: see the kernel descriptions.
FLOPS_PER_LUP = {J7_CONST: 8, J7_VAR: 13, W25_CONST: 30, W25_VAR: 40, J25_VAR: 37, W25_ALPHA: 31}
FP_INSTR_PER_LUP = {J7_CONST: 7, J7_VAR: 7, W25_CONST: 25, W25_VAR: 26, J25_VAR: 25, W25_ALPHA: 26}


def cpu_code_balance(kind: int, word: int = 8, write_allocate: bool = True) -> float:
    """Minimum bytes/LUP of the naive sweep on a CPU (paper Sect. 3.3).

    First-order kinds read u and the coefficient streams and write u'; the
    write to a separate array costs a write-allocate read unless streaming
    stores are used.  Second-order kinds overwrite u^{t-1} by u^{t+1} in
    place: the line was already read, so no write-allocate is added.
    """
    reads = 1 + _COEFF_ARRAYS[kind] + (1 if _SECOND_ORDER[kind] else 0)
    wa = 1 if (write_allocate and not _SECOND_ORDER[kind]) else 0
    return float(word * (reads + 1 + wa))


def gpu_bytes_per_lup(kind: int, word: int) -> float:
    """Algorithmic bytes/LUP of one plain sweep on the GPU (no write-allocate)."""
    reads = 1 + _COEFF_ARRAYS[kind] + (1 if _SECOND_ORDER[kind] else 0)
    return float(word * (reads + 1))


def gpu_bytes_per_pass(kind: int, word: int, n_points: int, trace_plane: int = 0) -> float:
    """Algorithmic bytes of one pass that reads the state and coefficients once
    and writes the state once (any number of time levels per pass)."""
    return gpu_bytes_per_lup(kind, word) * n_points


def roofline(bandwidth: float, code_balance: float) -> float:
    """P = b_S / B_C (updates/s for bandwidth in bytes/s), Sect. 3.3."""
    return bandwidth / code_balance


def wavefront_width(Dw: int, NF: int, R: int = 1) -> int:
    """W_w = D_w - 2R + N_F + 1 (for R = 1: D_w + N_F - 1), paper Sect. 5.3."""
    return Dw - 2 * R + NF + 1


def cache_block_bytes(Dw: int, NF: int, Nxb: float, ND: int = 1, R: int = 1) -> float:
    """Cache block size of one extruded diamond, paper Sect. 5.3:
    N_xb [N_D D_w (D_w/2 - R + N_F + 1) + 2R (D_w + W_w)]; for R = 1 this is
    N_xb [N_D (D_w^2/2 + D_w N_F) + 2 (D_w + W_w)]."""
    Ww = wavefront_width(Dw, NF, R)
    return Nxb * (ND * Dw * (Dw / 2.0 - R + NF + 1) + 2 * R * (Dw + Ww))
