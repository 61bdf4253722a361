"""Algorithmic work of one generator launch, for the ALU roofline.

The generators are bound by FP32/INT32 issue on the CUDA cores (no dense
contraction, and the only DRAM traffic is one output write per sample).  The
work unit is a lane operation (one FP32 or INT32 arithmetic/logic operation of
one thread).  The counts below follow the kernels' dataflow, counted from
their formulas (never from compiled code); loads, stores, address arithmetic,
loop control and barriers are overhead and are NOT counted, so the achieved
fraction of the issue peak measures how little overhead and stall the kernels
add on top of the arithmetic they must do.

Per 2D tile of 64 x 64 samples, 128 threads, each thread a run of RW columns
in RR rows (RW x RR = 8 x 4 or 16 x 2, the thread shape), with d = 3 (C1), 5
(C2), 4 (Perlin-S3), 6 (Perlin-S5) and nrun = octaves whose cells are at least
RW samples wide ("run" octaves):
  basis tables: nrun x ((64/RW)(d+1) + 64) entries x (5 coordinate + basis
                ops: C1 7, C2 14, Perlin-S5 9, Perlin-S3 8);
  corners:      per staged corner 15 for pcg3d, 3 a hash word used (shift
                and add to a float in [2, 4), one FMA for amplitude and the
                -3 offset; three words for the Hermite cells, two for Perlin,
                one for the zero-gradient model) and 4 for the grid index:
                28, 25 and 22; the corners of cells of 2 samples are hashed
                a warp a corner row with x's LCG step taken once per lane and
                y's once per row (pcg3d 12 + 2 for the row word, grid index 1:
                24, 21 and 15 -- the zero-gradient model needs word 0 alone,
                whose last cross steps of y and z are not taken);
  run octaves, per thread and octave: prep + NR rows x (row reduction + one
                add of the row's V0 + (eval - 1) at each of the d+1 node
                columns); once per thread NR x (d+1) adds of the rows' V0 sums
                to the nodes, (RR - NR) rows x (d+1) node columns x (d+1) FMA
                of interpolation along y and RR rows x (RW - d - 1) columns x
                (d+1) FMA along x.  NR = rows a thread evaluates: RR, or 2 of
                its 4 with degree 3 and runs of 8 (node rows: a thread pair's
                8 x 8 block at rows 0, 2, 5, 7);
  tile octaves (cells >= 64 samples, when summed at the tile nodes): per tile
                (d+1)^2 nodes x nt x (2 (coordinate + basis) + prep + row + eval)
                and (lanes a node - 1) adds a node; degree 3: per tile the
                tile polynomial at 64 rows x 4 node columns (4 FMA each), per
                thread NR x (d+1)^2 FMA to its node columns; other degrees:
                per thread RR x (d+1)^2 FMA to the thread's rows and
                RR x (d+1)^2 to its node columns; no basis tables for these
                octaves;
  cells of CW < RW samples (CW = 8 for RW 16; 4, 2), per thread: RW/CW cells
                along the run, each with prep + one row reduction per row
                (row 0 of a cell, where the row is the corner data, costs 1),
                (CW - 1) evaluations per row and 1 accumulate of column 0; a
                thread whose RR rows are fewer than CW evaluates its two row
                bases at run time (2 + basis ops each).  (prep, row, eval) =
                (4, 9, 4) for the Hermite cells and Perlin, (4, 4, 3) for the
                zero-gradient model and (25, 8, 4) for the paper's D2M1N3
                coefficients;
  lattice octave: per sample 13 -- pcg3d word 0 of (x, y, key) with the
                row-invariant words' LCG steps and the x-word addend y*z
                hoisted out of the row: x's LCG step 1 (it advances by a
                per-octave constant along the run), y and z multiply-adds 2,
                three xorshifts 6, the final multiply-add 1; word->float 2;
                FMA 1 (the -3 offsets of all lattice octaves start the rows'
                V0 sums, no work a sample).  Perlin's lattice octaves are zero,
                no work.
3D tiles of 32 x 16 x 8 (each thread 8 x 4 x 1): the same regimes, with a
reduction along z of the cell's four corner columns (32 ops) before each cell
is used, and each run octave's rows summing their V0 once; C1 evaluates 2 of
its 4 rows (node rows, as in 2D: 2 x 16 FMA of interpolation along y); for C1
with four or more octaves of cells >= 32 samples, those are tile octaves: 64
nodes x nt x (3 x (coordinate + basis) + 32 + 9 + 4 + 1) + 64 a tile, the
nodes reduced along z for each of the 8 planes (8 x 16 x 4 FMA a tile) and
2 x 16 FMA of interpolation a thread and evaluated row, no basis tables; basis tables of n8 x (4 (d+1) + 24)
entries, corners 38 (pcg4d 20, four words 12, index 6; Perlin three words:
35; cells of 2 samples, hashed two rows a warp with the LCG steps of x per
lane and of y, z per row: 31 and 28) and lattice samples 14 (pcg4d word 0
with the row-invariant terms hoisted: 1 + 3 multiply-adds + 3 xorshifts (6) +
1, word->float 2, FMA 1; the offsets start the sums).
OpenSimplex-style (2D, dyadic steps): per sample and octave, the column's
offset and in-cell base (product, floor, convert, two adds: 5; redone for each
of the thread's rows), the row's share of its own (5 per 8 samples), the
stretched position and vertex (22: sum, split product and its error, floors,
fractions, converts and the integer vertex), the branch-free vertex choice (17)
and 4 vertices x (displacement and squish 6, kernel (2 - r^2)^4 (g . d) 9,
gradient: from the staged box 5 (index, clamp) or hashed 22 (vertex 2, pcg3d
15, two word maps 5)), the sum of the four terms and the amplitude FMA (4); a
staged octave adds 25 a box vertex a tile (index 4, pcg3d 15, word maps 4,
address 2), with box sides 64 step + 6 vertices (step = lattice units a
sample, staged while step <= 1).
3D OpenSimplex-style (tiles of 32 x 16 x 8): per sample and octave 40
(stretched position 20, reflection 12, squish 4, amplitude 4) + 19 candidate
vertices x 14 (displacement 3, r^2 3, kernel 4, g . d 3, accumulate 1); a
hashed octave adds 19 x 32 per sample (vertex 3, pcg4d 20, three
word->float maps 9); a staged one adds 29 per box vertex and tile.  Nineteen
candidates are evaluated where on average 5.9 (at most 8) are within range.
"""
from __future__ import annotations

import math

BASIS_OPS = {"c1": 7, "c2": 14, "perlin_s5": 9, "perlin_s3": 8, "zero_grad": 4, "paper_gauge": 0}
COORD_OPS = 5


def _staged(spc: int, octaves: int):
    """(octave index, samples per cell) of the staged octaves."""
    s = spc.bit_length() - 1
    return [(i, spc >> i) for i in range(min(octaves, s))]


DEG = {"c1": 3, "c2": 5, "perlin_s3": 4, "perlin_s5": 6, "paper_gauge": 3, "zero_grad": 3}
# (cell preparation, row collapse, per-sample evaluation) operations per model
MODEL_OPS = {"c1": (4, 9, 4), "c2": (4, 9, 4), "perlin_s3": (4, 9, 4), "perlin_s5": (4, 9, 4),
             "zero_grad": (4, 4, 3), "paper_gauge": (25, 8, 4)}


def small_cell_ops(kind: str, rw: int, cw: int) -> int:
    """Lane operations of one thread for one octave of cw-sample cells."""
    rr = 32 // rw
    prep, row, smp = MODEL_OPS[kind]
    ncx = rw // cw
    rpc = min(rr, cw)
    ncy = rr // rpc
    const_rows = rr >= cw
    per_cell = prep + (1 + (rpc - 1) * row if const_rows else rpc * row) + rpc * ((cw - 1) * smp + 1)
    ops = ncx * ncy * per_cell
    if not const_rows:
        ops += rpc * (2 + BASIS_OPS[kind])
    return ops


def lane_ops_2d(kind: str, size, spc: int, octaves: int, rw: int = 8, nt: int = 0) -> dict:
    w, h = size
    tiles = ((w + 63) // 64) * ((h + 63) // 64)
    threads = tiles * 128
    samples_padded = tiles * 64 * 64
    if kind == "opensimplex":
        tot = 0.0
        for i in range(octaves):
            step = 2.0 ** i / spc
            staged = step <= 1.0
            per = 5 + 5 / 8 + 22 + 17 + 4 * (6 + 9 + (5 if staged else 22)) + 4
            tot += samples_padded * per
            if staged:
                tot += tiles * (64 * step + 6) ** 2 * 25
        return dict(total=float(tot), per_sample=tot / (w * h))
    rr = 32 // rw
    d = DEG[kind]
    nr = 2 if (d == 3 and rw == 8) else rr  # rows a thread evaluates (node rows)
    st = _staged(spc, octaves)
    nrun = sum(1 for _, spci in st if spci >= rw) - nt
    lut = tiles * nrun * ((64 // rw) * (d + 1) + 64) * (COORD_OPS + BASIS_OPS[kind])
    corners = 0
    evalops = threads * rr * (rw - d - 1) * (d + 1) + threads * nr * (d + 1) + threads * (rr - nr) * (d + 1) * (d + 1)
    prep, row, smp = MODEL_OPS[kind]
    if nt:
        nodes = (d + 1) ** 2
        parts = 8 if nodes <= 16 else (4 if nodes <= 32 else 2)
        evalops += tiles * nodes * nt * (2 * (COORD_OPS + BASIS_OPS[kind]) + prep + row + smp)
        evalops += tiles * nodes * (parts - 1)  # adds across the lanes of a node
        if d == 3:
            evalops += tiles * 64 * (d + 1) * (d + 1) + threads * nr * (d + 1) ** 2
        else:
            evalops += threads * 2 * rr * (d + 1) ** 2
    for i, spci in st:
        k = spci.bit_length() - 1
        ncx = (63 >> min(k, 31)) + 2
        if spci == 2:
            per = {"zero_grad": 15, "perlin_s5": 21, "perlin_s3": 21}.get(kind, 24)
        else:
            per = {"zero_grad": 22, "perlin_s5": 25, "perlin_s3": 25}.get(kind, 28)
        corners += tiles * ncx * ncx * per
        if i < nt:
            continue
        if spci >= rw:
            evalops += threads * (prep + nr * (row + 1 + (smp - 1) * (d + 1)))
        else:
            evalops += threads * small_cell_ops(kind, rw, spci)
    n_lattice = octaves - len(st)
    lattice = 0 if kind.startswith("perlin") or n_lattice == 0 else samples_padded * n_lattice * 13
    tot = lut + corners + evalops + lattice
    return dict(total=float(tot), per_sample=tot / (w * h), lut=lut, corners=corners, eval=evalops,
                lattice=lattice)


def simplex3_box(step: float):
    """Vertices of the staged gradient box of a 3D OpenSimplex octave with
    `step` lattice units per sample, or 0 if that octave is hashed."""
    if step >= 1.0:
        return 0
    L = [31 * step, 15 * step, 7 * step]
    n = 1
    for k in range(3):
        n *= int(math.floor((5 * L[k] + (sum(L) - L[k])) / 6 + 1e-4)) + 5
    return n if n <= 4096 else 0


def lane_ops_3d(kind: str, size, spc: int, octaves: int, f: float = 2.0) -> dict:
    w, h, dd = size
    tiles = ((w + 31) // 32) * ((h + 15) // 16) * ((dd + 7) // 8)
    threads = tiles * 128
    samples_padded = tiles * 32 * 16 * 8
    if kind == "opensimplex":
        tot = 0
        for i in range(octaves):
            box = simplex3_box(f ** i / spc)
            tot += samples_padded * (40 + 19 * 14) + (tiles * box * 29 if box else samples_padded * 19 * 32)
        return dict(total=float(tot), per_sample=tot / (w * h * dd))
    d = DEG[kind]
    st = _staged(spc, octaves)
    n8 = sum(1 for _, spci in st if spci >= 8)
    # C1 tile octaves (cells >= 32 samples) when there are four or more
    nt = sum(1 for _, spci in st if spci >= 32) if kind == "c1" else 0
    nt = nt if nt >= 4 else 0
    lut = tiles * (n8 - nt) * (4 * (d + 1) + 24) * (COORD_OPS + BASIS_OPS[kind])
    corners = 0
    nr = 2 if d == 3 else 4  # rows a thread evaluates (node rows), of its 4
    evalops = threads * 4 * (7 - d) * (d + 1) + threads * nr * (d + 1) + threads * (4 - nr) * (d + 1) * (d + 1)
    if nt:
        # 64 nodes x nt octaves x (3 axes of coordinate + basis, z reduction 32,
        # row 9, evaluation 4, accumulate 1), one shuffle-add a node; the nodes
        # reduced along z for 8 planes (8 x 16 x 4 FMA); per thread and
        # evaluated row 2 x 16 FMA of interpolation (y, x)
        evalops += tiles * (64 * nt * (3 * (COORD_OPS + BASIS_OPS[kind]) + 32 + 9 + 4 + 1) + 64 + 8 * 16 * 4)
        evalops += threads * nr * 32
    for i, spci in st:
        k = spci.bit_length() - 1
        nc = ((31 >> min(k, 31)) + 2) * ((15 >> min(k, 31)) + 2) * ((7 >> min(k, 31)) + 2)
        if spci == 2:
            per = 28 if kind.startswith("perlin") else 31
        else:
            per = 35 if kind.startswith("perlin") else 38
        corners += tiles * nc * per
        if i < nt:
            continue
        if spci >= 8:
            evalops += threads * (32 + 4 + nr * (9 + 1 + 3 * (d + 1)))
        elif spci == 4:
            evalops += threads * (2 * (32 + 4 + 1 + 3 * 9) + 24 * 4 + 8)
        else:
            evalops += threads * (8 * (32 + 4 + 1 + 9) + 80)
    nl = octaves - len(st)
    lattice = 0 if kind.startswith("perlin") or nl == 0 else samples_padded * nl * 14
    tot = lut + corners + evalops + lattice
    return dict(total=float(tot), per_sample=tot / (w * h * dd), lut=lut, corners=corners, eval=evalops,
                lattice=lattice)


# Kernel-independent lower bound ("bound" lane operations): the work any
# implementation of the method with this corner hash must execute, whatever its
# tiling, staging or evaluation scheme:
#   - every distinct lattice corner of every octave whose cells span two or more
#     samples is hashed once: pcg3d (three LCG steps, six cross multiply-adds,
#     three xorshifts of two operations = 15; pcg4d 20) plus, per hash word the
#     model uses, its map to a float (1) and its amplitude scaling (1): 21 for
#     the Hermite cells and the paper's D2M1N3 (three words), 19 for Perlin
#     (two), 14 for the zero-gradient model (word 0 alone: 3 + 3 + 6 + 1 + 2);
#     3D: 20 + 2 per word (four words, Perlin three);
#   - every sample of an octave whose cells are one sample wide or narrower sits
#     on a lattice point and needs word 0 of its own corner hash: with the
#     row-invariant words hoisted out of a run of samples, 10 operations (2D;
#     3D 11) plus the word's map (1) and its accumulation into the sum (1);
#     Perlin's lattice octaves are zero and cost nothing;
#   - per sample, combining the octave sum: octaves whose cells are wider than
#     d + 1 samples along a row add up to one polynomial of degree d there,
#     which forward differences evaluate with d additions a sample; each octave
#     whose cells are d + 1 samples wide or narrower (but wider than one sample)
#     adds at least one operation a sample.
# Loads, stores, index arithmetic, node-to-sample interpolation beyond the d
# additions and every other part of the kernels' own design are not counted,
# so bound / time / issue peak is the fraction of the machine that the
# method's irreducible arithmetic would occupy at the measured speed.
BOUND_CORNER_2D = {"c1": 21, "c2": 21, "paper_gauge": 21, "zero_grad": 14, "perlin_s5": 19, "perlin_s3": 19}
BOUND_CORNER_3D = {"c1": 28, "c2": 28, "perlin_s5": 26, "perlin_s3": 26}


def bound_ops(kind: str, size, spc: int, octaves: int) -> dict:
    """Lower bound of the lane operations of one field (2D or 3D, fused
    generators: spc a power of two, frequency ratio 2); see above."""
    dims = len(size)
    samples = 1
    for v in size:
        samples *= v
    d = DEG[kind]
    st = _staged(spc, octaves)
    corners = 0
    for i, spci in st:
        n = 1
        for v in size:
            n *= (v + spci - 1) // spci + 1  # distinct corners of the field at this octave
        corners += n * (BOUND_CORNER_2D if dims == 2 else BOUND_CORNER_3D)[kind]
    nl = octaves - len(st)
    lattice = 0 if kind.startswith("perlin") else samples * nl * (12 if dims == 2 else 13)
    wide = any(spci > d + 1 for _, spci in st)
    narrow = sum(1 for _, spci in st if spci <= d + 1)
    combine = samples * ((d if wide else 0) + narrow)
    tot = corners + lattice + combine
    return dict(total=float(tot), per_sample=tot / samples, corners=corners, lattice=lattice, combine=combine)


def alu_peak(num_sms: int, clock_mhz: float, lanes_per_sm: int = 128) -> float:
    """Issue peak in lane operations per second: SMs x 128 FP32/INT32 lanes
    x clock (one warp instruction per cycle on each of four SM partitions)."""
    return num_sms * lanes_per_sm * clock_mhz * 1e6
