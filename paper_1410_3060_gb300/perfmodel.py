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


# ---------------------------------------------------------------- GPU block model
# The GPU counterpart of the cache block of Sect. 5.3.  There a wavefront tile
# of D_w x W_w cells (in y-z) times the untiled x extent must fit the shared
# L3 cache with its N_D domain-sized streams; the auto-tuner (Sect. 5.1)
# searches only the tile sizes that fit.  Here one CTA marches a tile through
# z; what must fit is its on-chip working set:
#   shared memory  the staged level-0 planes, the y-edge rows every level
#                  exchanges between warps and, for the coefficient streams,
#                  the planes level 1 keeps for the levels above it,
#                  <= 227 KB per CTA;
#   registers      the 2R+1-plane z ring of every level (the counterpart of
#                  the wavefront width W_w) for the thread's points, <= 255
#                  per thread and <= 64 K per SM;
# and the overlapped halo of a depth-B pass (B R columns and rows on each
# side, the counterpart of the diamond slopes) makes a CTA compute more
# points than it owns.  HBM bytes: each stream is read once per pass and the
# result written once (the halo re-reads hit L2: measured 2.66 B per update
# against 2.67 algorithmic for the depth-3 7-point constant pass).

SMEM_PER_CTA = 227 * 1024
REGS_PER_SM = 65536
MAX_REGS_PER_THREAD = 255

# register wavefront tile variants: (V points per thread along x, NR rows
# per thread, WY warps); variant 12 keeps 2 rows per thread at depth 4,
# variant 17 (FP32) takes 8 warps at depth 4
_WF_TILES = {10: (2, 4, 8), 11: (2, 2, 16), 12: (2, 4, 16), 17: (4, 2, 16)}
WF_VARIANTS = (10, 11, 12, 17)
WF_VARIANTS_WIDE = (17,)               # FP32 only: 4 points per thread row


def wavefront_tile(variant: int, B: int):
    """(V, NR, WY) of a register wavefront tile variant (0 = variant 10)."""
    if variant == 12 and B > 3:
        return (2, 2, 16)
    if variant == 17 and B > 3:
        return (4, 2, 8)
    return _WF_TILES.get(variant, _WF_TILES[10])


def wavefront_block(kind: int, word: int, B: int, variant: int) -> dict:
    """On-chip working set of one CTA of the register wavefront (7-point
    kinds, R = 1) at depth B: shared bytes, threads, computed / owned tile
    extents, the lower bound of registers per thread (the level rings and
    the result plane; 8-byte values take two registers), whether it fits,
    and the computed / owned ratio of the overlapped tile."""
    R = 1
    V, NR, WY = wavefront_tile(variant, B)
    TXE, TYE = 32 * V, WY * NR
    BR = B * R
    AX = -(-BR // V) * V
    SX = (TXE - BR - AX) // V * V
    SY = TYE - 2 * BR
    ring = 2 * R + 1
    NS = 4                                         # level-0 slots (2 planes in flight)
    base = word * (NS * TYE * TXE + ring * B * WY * 2 * R * TXE)
    NA = _COEFF_ARRAYS[kind]
    cring = 0
    if NA and B >= 2:
        c = word * (B - 1) * NA * TYE * TXE
        cring = c if base + c <= SMEM_PER_CTA else 0
    smem = base + cring
    threads = 32 * WY
    per_reg = word // 4
    regs_min = per_reg * NR * V * (B * ring + 1 + (NA if NA else 2))
    regs_cap = min(MAX_REGS_PER_THREAD, REGS_PER_SM // threads)
    fits = SX > 0 and SY > 0 and smem <= SMEM_PER_CTA and regs_min <= regs_cap
    return {"smem_bytes": smem, "threads": threads, "computed": (TXE, TYE), "owned": (SX, SY),
            "regs_min": regs_min, "regs_cap": regs_cap, "fits": fits,
            "redundancy": (TXE * TYE) / float(max(SX * SY, 1)), "coef_ring": cring > 0}


def vector_sweep_block(kind: int, word: int, variant: int) -> dict:
    """On-chip working set of one CTA of the vectorised one-level sweep
    (tile variants 13-16; 15, 16 staged by TMA): shared bytes, threads, tile
    extents.  16-byte vectors along x, a ring of R + 1 + PD plane slots (PD
    planes in flight, 3 where the TMA-staged forward of the constant and
    alpha-array waves fits it) with the u^{t-1} and alpha planes staged beside
    the field plane, one mbarrier per slot, an abort word, alignment slack."""
    R = 4 if kind in (W25_CONST, W25_VAR, J25_VAR, W25_ALPHA) else 1
    V = 16 // word
    big, tma = variant in (14, 16), variant >= 15
    if kind in (W25_VAR, J25_VAR):
        WY = 4 if big else 8
    else:
        WY = 16 if big else 8
    TX = 32 * V
    RH = -(-R // V) * V
    SW, SH = TX + 2 * RH, WY + 2 * R
    SP = -(-(SW * SH * word) // 128) * 128 // word
    NPS = (1 if _SECOND_ORDER[kind] else 0) + (1 if _COEFF_ARRAYS[kind] == 1 else 0)
    PP = TX * WY

    def smem_of(pd):
        slots = R + 1 + pd
        return word * (slots * SP + slots * NPS * PP) + 8 * slots + 16 + 128

    deep = tma and _COEFF_ARRAYS[kind] <= 1 and _SECOND_ORDER[kind]
    PD = 3 if deep and smem_of(3) <= SMEM_PER_CTA else 2
    return {"smem_bytes": smem_of(PD), "threads": 32 * WY, "computed": (TX, WY), "owned": (TX, WY),
            "fits": smem_of(PD) <= SMEM_PER_CTA, "redundancy": 1.0, "planes_in_flight": PD}


def dram_bytes_per_lup(kind: int, word: int, B: int = 1) -> float:
    """Modelled HBM bytes per lattice update of a pass of B levels: the plain
    sweep's streams once per pass (halo re-reads served by L2)."""
    return gpu_bytes_per_lup(kind, word) / B


def two_level_block(kind: int) -> dict:
    """On-chip working set of one CTA of the two-level pass of the 13-array
    kinds (scheme 4, FP32): an owned 64 x 16 tile, level 1 on it with an
    R = 4 halo (72 x 24, one 4-point vector per thread of 14 warps), level
    2 on the owned tile (8 warps), level 0 with a 2R halo (80 x 32).  Level
    2 runs one plane behind level 1's output, so the rings hold 2R + 2 + PD
    level-0 planes (PD in flight: 1, 2 for the constant wave), 2R + 2
    level-1 planes and, for the wave kinds, PD + 1 planes of u^{t-1} beside
    level 0; one mbarrier per level-0 slot, the abort word, alignment
    slack."""
    R, word = 4, 4
    TXO, TYO = 64, 16
    P1 = (TXO + 2 * R) * (TYO + 2 * R)
    P0 = (TXO + 4 * R) * (TYO + 4 * R)
    pd = 2 if kind == W25_CONST else 1             # level-0 planes in flight
    ns0 = 2 * R + 2 + pd
    wave = _SECOND_ORDER[kind]
    smem = word * (ns0 * P0 + ((pd + 1) * P1 if wave else 0) + (2 * R + 2) * P1) + 8 * ns0 + 16 + 128
    threads = 32 * (-(-((TXO + 2 * R) // 4 * (TYO + 2 * R)) // 32) + TXO // 4 * TYO // 32)
    return {"smem_bytes": smem, "threads": threads, "computed": (TXO + 2 * R, TYO + 2 * R), "owned": (TXO, TYO),
            "fits": smem <= SMEM_PER_CTA, "redundancy": ((TXO + 2 * R) * (TYO + 2 * R) + TXO * TYO) / (2.0 * TXO * TYO)}
