"""Convolution in the oracle: the plain definition, the slot layout, and the
homomorphic layer of Sec. 3.1 (padded convolution + Walsh-Hadamard output
packing) with the rotations of Sec. 2.3 hoisted.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings of the paper:
  * Layout (Sec. 2.4 pads the input; Sec. 3.1 packs c_n channels per
    ciphertext).  A slot row (N/2 slots) holds whole zero-padded halo
    tiles ("blocks") of (T_h + 2P) x (T_w + 2P) slots, row-major with width
    W_b = T_w + 2P.  Tap (dy, dx) is then a left rotation by dy*W_b + dx.
    With c_n = 2, row 0 of input ciphertext j carries channel 2j and row 1
    channel 2j+1; with c_n = 1 both rows carry channel j for different tiles.
  * c_n = 4 (Sec. 3.1 generalises the pair to the 4 x 4 Walsh-Hadamard
    basis without fixing which slots form the four parts): channel 4j + c
    of input ciphertext j sits in row c >> 1 at the slots of parity c & 1,
    so a block position pos is slot 2 pos + (c & 1) of its row and a row
    holds N/4 positions.  The four +-1 patterns of H_4 over these classes
    (row sign, slot parity and their product) encode to sparse plaintexts,
    where contiguous quarter rows would give dense ones.  A left rotation
    by 2o keeps each class and shifts by o positions; one by 2m + 1 moves
    parity 1 at offset m into parity 0 and parity 0 at offset m + 1 into
    parity 1.
  * Hadamard scalars (Eq. 1) are used without the 1/2: s0 = v0 + v1,
    s1 = v0 - v1, so the output decrypts to 2k * conv (k from Sec. 3.2.1).
    With c_n = 4, s_b = sum_c H4[b][c] v_c and the output decrypts to
    4 k4 * conv, k4 chosen for the three patterns together (k4_select).
  * Output-channel alignment (Sec. 3.1 rotates partial sums) is applied on
    the input side: the row swap is composed with every tap rotation
    (diagonal d = 1), which gives the same slots.
  * Stride S > 1 computes the stride-1 result on tiles whose origins are
    multiples of S and keeps every S-th position at decode.
  * Channel counts are padded with zero channels to a multiple of c_n.
"""
from __future__ import annotations

import os
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from . import bfv
from .params import Params


def conv_plain(act: np.ndarray, weights: np.ndarray, stride: int, pad: int, depthwise: bool, t: int) -> np.ndarray:
    """The definition the layer must reproduce: cross-correlation, no bias,
    zero padding, out[i][o][y][x] = sum_{c,dy,dx} w[o][c][dy][dx] *
    in[i][c][y*S + dy - P][x*S + dx - P], reduced mod t into [0, t)."""
    I, C, H, W = act.shape
    O, Cw, kh, kw = weights.shape
    Ho = (H + 2 * pad - kh) // stride + 1
    Wo = (W + 2 * pad - kw) // stride + 1
    x = np.zeros((I, C, H + 2 * pad, W + 2 * pad), dtype=np.int64)
    x[:, :, pad:pad + H, pad:pad + W] = act
    out = np.zeros((I, O, Ho, Wo), dtype=np.int64)
    for dy in range(kh):
        for dx in range(kw):
            win = x[:, :, dy:dy + stride * (Ho - 1) + 1:stride, dx:dx + stride * (Wo - 1) + 1:stride]
            if depthwise:
                out += win * weights[:, 0, dy, dx].reshape(1, O, 1, 1)
            else:
                out += np.einsum("icyx,oc->ioyx", win, weights[:, :, dy, dx])
            out %= t
    return out % t


@dataclass
class Layout:
    N: int
    C_in: int
    C_out: int
    H: int
    W: int
    kh: int
    stride: int
    depthwise: bool
    n_images: int
    c_n: int
    tile_h: int = 0
    tile_w: int = 0
    P: int = 0
    T_h: int = 0
    T_w: int = 0

    def __post_init__(self):
        if self.kh % 2 != 1:
            raise ValueError("odd square kernels only")
        if self.depthwise and self.C_in != self.C_out:
            raise ValueError("depthwise needs C_in == C_out")
        if self.c_n not in (1, 2, 4):
            raise ValueError("c_n must be 1, 2 or 4")
        self.P = (self.kh - 1) // 2
        if self.tile_h or self.tile_w:
            # a caller-chosen tile: any size whose padded block fits one slot row, with tile
            # origins on the stride grid (sides a multiple of S unless one tile spans the image)
            th, tw, S = self.tile_h, self.tile_w, self.stride
            if not (0 < th <= self.H and 0 < tw <= self.W):
                raise ValueError("tile must lie within the image, in both directions")
            if (th % S and th != self.H) or (tw % S and tw != self.W):
                raise ValueError("tile sides must be multiples of the stride")
            if (th + 2 * self.P) * (tw + 2 * self.P) > self.row_positions:
                raise ValueError("padded tile does not fit one slot row")
            self.T_h, self.T_w = th, tw
        else:
            self.T_h, self.T_w = choose_tile(self.row_positions, self.H, self.W, self.P, self.stride)

    # geometry -------------------------------------------------------------
    @property
    def row_positions(self):
        """block positions a slot row holds: N/2, or N/4 with c_n = 4 (two parities per position)"""
        return self.N // 4 if self.c_n == 4 else self.N // 2

    @property
    def W_b(self):
        return self.T_w + 2 * self.P

    @property
    def block_slots(self):
        return (self.T_h + 2 * self.P) * self.W_b

    @property
    def blocks_per_row(self):
        return self.row_positions // self.block_slots

    @property
    def n_ty(self):
        return -(-self.H // self.T_h)

    @property
    def n_tx(self):
        return -(-self.W // self.T_w)

    @property
    def units(self):
        return self.n_images * self.n_ty * self.n_tx

    @property
    def units_per_ct(self):
        """blocks of distinct tiles per ciphertext: one row's worth (c_n = 2) or both rows (c_n = 1)"""
        return self.blocks_per_row * (2 if self.c_n == 1 else 1)

    @property
    def row_units(self):
        return -(-self.units // self.units_per_ct)

    @property
    def in_groups(self):
        return -(-self.C_in // self.c_n)

    @property
    def out_groups(self):
        return -(-self.C_out // self.c_n)

    @property
    def n_ct_in(self):
        return self.row_units * self.in_groups

    @property
    def n_ct_out(self):
        return self.row_units * self.out_groups

    @property
    def Ho(self):
        return (self.H - 1) // self.stride + 1

    @property
    def Wo(self):
        return (self.W - 1) // self.stride + 1

    def taps(self):
        """(dy, dx) offsets, row-major over the kernel window."""
        return [(dy, dx) for dy in range(-self.P, self.P + 1) for dx in range(-self.P, self.P + 1)]

    # slot placement -------------------------------------------------------
    def slot_of(self, u_local: int, yl: int, xl: int) -> tuple[int, int]:
        """(row, position within the row) of block-local position (yl, xl)
        of the u_local-th tile held by a ciphertext."""
        B = self.blocks_per_row
        row, b = (u_local // B, u_local % B) if self.c_n == 1 else (0, u_local)
        return row, b * self.block_slots + yl * self.W_b + xl

    def flat_slot(self, row: int, pos: int, r: int) -> int:
        """Flat slot index of channel r (0 .. c_n - 1) of a ciphertext at (row, pos) from slot_of:
        c_n = 1 uses the row; c_n = 2 puts channel r in row r; c_n = 4 in row r >> 1 at parity r & 1."""
        half = self.N // 2
        if self.c_n == 1:
            return row * half + pos
        if self.c_n == 2:
            return r * half + pos
        return (r >> 1) * half + 2 * pos + (r & 1)

    def unit_coords(self, unit: int) -> tuple[int, int, int]:
        img, rest = divmod(unit, self.n_ty * self.n_tx)
        ty, tx = divmod(rest, self.n_tx)
        return img, ty, tx


def choose_tile(half: int, H: int, W: int, P: int, S: int) -> tuple[int, int]:
    """Interior tile size (T_h, T_w) whose padded block fits one slot row of `half` positions.
    Whole image if it fits; else full-width strips of a multiple of S rows;
    else square-ish tiles with sides a multiple of S."""
    if (H + 2 * P) * (W + 2 * P) <= half:
        return H, W
    if (W + 2 * P) * (S + 2 * P) <= half:
        Th = ((half // (W + 2 * P) - 2 * P) // S) * S
        return min(Th, H), W
    Tw = S
    while Tw + S <= W and (Tw + S + 2 * P) ** 2 <= half:
        Tw += S
    Th = ((half // (Tw + 2 * P) - 2 * P) // S) * S
    if Th < S or (Tw + 2 * P) * (S + 2 * P) > half:
        raise ValueError("kernel too large for the ring degree")
    return min(Th, H), Tw


def pack_slots(lay: Layout, act: np.ndarray, row_units=None) -> np.ndarray:
    """Input activations [I][C_in][H][W] -> slot vectors [n_ct_in][N].
    `row_units` (optional) fills only the ciphertexts of those row-units."""
    N, P = lay.N, lay.P
    out = np.zeros((lay.n_ct_in, N), dtype=np.int64)
    for unit in range(lay.units):
        ru, u_local = divmod(unit, lay.units_per_ct)
        if row_units is not None and ru not in row_units:
            continue
        img, ty, tx = lay.unit_coords(unit)
        for j in range(lay.in_groups):
            ct = ru * lay.in_groups + j
            for yl in range(lay.T_h + 2 * P):
                Y = ty * lay.T_h + yl - P
                if Y < 0 or Y >= lay.H:
                    continue
                for xl in range(lay.W_b):
                    X = tx * lay.T_w + xl - P
                    if X < 0 or X >= lay.W:
                        continue
                    row, pos = lay.slot_of(u_local, yl, xl)
                    for r in range(lay.c_n):
                        c = lay.c_n * j + r
                        if c < lay.C_in:
                            out[ct, lay.flat_slot(row, pos, r)] = act[img, c, Y, X]
    return out


def unpack_slots(lay: Layout, slots: np.ndarray) -> np.ndarray:
    """Output slot vectors [n_ct_out][N] -> [I][C_out][Ho][Wo] (valid positions only)."""
    P, S = lay.P, lay.stride
    out = np.zeros((lay.n_images, lay.C_out, lay.Ho, lay.Wo), dtype=np.int64)
    for unit in range(lay.units):
        ru, u_local = divmod(unit, lay.units_per_ct)
        img, ty, tx = lay.unit_coords(unit)
        for g in range(lay.out_groups):
            ct = ru * lay.out_groups + g
            for yl in range(P, P + lay.T_h):
                Y = ty * lay.T_h + yl - P
                if Y >= lay.H or Y % S:
                    continue
                for xl in range(P, P + lay.T_w):
                    X = tx * lay.T_w + xl - P
                    if X >= lay.W or X % S:
                        continue
                    row, pos = lay.slot_of(u_local, yl, xl)
                    for r in range(lay.c_n):
                        c = lay.c_n * g + r
                        if c < lay.C_out:
                            out[img, c, Y // S, X // S] = slots[ct, lay.flat_slot(row, pos, r)]
    return out


def ct_positions(lay: Layout, c: int) -> list[tuple[int, int, int, int, int]]:
    """Valid outputs carried by output ciphertext c: (image, channel, y, x, flat slot) tuples,
    the same placement as unpack_slots, for checking one ciphertext of a large layer."""
    P, S = lay.P, lay.stride
    ru, g = divmod(c, lay.out_groups)
    res = []
    for u_local in range(lay.units_per_ct):
        unit = ru * lay.units_per_ct + u_local
        if unit >= lay.units:
            break
        img, ty, tx = lay.unit_coords(unit)
        for yl in range(P, P + lay.T_h):
            Y = ty * lay.T_h + yl - P
            if Y >= lay.H or Y % S:
                continue
            for xl in range(P, P + lay.T_w):
                X = tx * lay.T_w + xl - P
                if X >= lay.W or X % S:
                    continue
                row, pos = lay.slot_of(u_local, yl, xl)
                for r in range(lay.c_n):
                    if lay.c_n * g + r < lay.C_out:
                        res.append((img, lay.c_n * g + r, Y // S, X // S, lay.flat_slot(row, pos, r)))
    return res


# ---------------------------------------------------------------- polyphase stride 2
# Reading of Sec. 2.4 for stride 2 (the paper is silent on stride): a 3x3 stride-2 convolution with
# zero padding 1 is a stride-1 convolution over the four phase planes of its input,
#   plane (a, b)[u][v] = in[2u + a][2v + b],  a, b in {0, 1},
# because tap (dy, dx) of output (y, x) reads in[2y + dy][2x + dx] = plane (dy mod 2, dx mod 2) at
# (y + floor(dy / 2), x + floor(dx / 2)): plane a = 0 only at row offset 0 (dy = 0), plane a = 1 at
# row offsets -1 (dy = -1) and 0 (dy = +1), likewise for columns.  The derived layer has 4 Cp input
# channels c' = (2a + b) Cp + c (Cp = C_in rounded up to c_n), planes of ceil(H/2) x ceil(W/2),
# a 3x3 kernel whose taps at offset +1 are zero, stride 1, and its output is the stride-2 output.
# A depthwise layer becomes a dense derived layer in which output channel o reads the four planes
# of channel o only.

def polyphase_planes(act: np.ndarray, c_n: int) -> np.ndarray:
    """[I][C][H][W] -> [I][4 Cp][ceil(H/2)][ceil(W/2)] phase planes, channel (2a + b) Cp + c."""
    I, C, H, W = act.shape
    Cp = -(-C // c_n) * c_n
    Hh, Wh = -(-H // 2), -(-W // 2)
    out = np.zeros((I, 4 * Cp, Hh, Wh), dtype=np.int64)
    for a in range(2):
        for b in range(2):
            plane = act[:, :, a::2, b::2]
            out[:, (2 * a + b) * Cp:(2 * a + b) * Cp + C, :plane.shape[2], :plane.shape[3]] = plane
    return out


def polyphase_weights(weights: np.ndarray, C_in: int, c_n: int, depthwise: bool) -> np.ndarray:
    """[O][C_in or 1][3][3] stride-2 weights -> [O][4 Cp][3][3] weights of the derived stride-1
    layer: tap (dy', dx') of plane (a, b) is tap (2 dy' + a, 2 dx' + b) of the original, zero where
    that tap lies outside [-1, 1]."""
    O = weights.shape[0]
    Cp = -(-C_in // c_n) * c_n
    out = np.zeros((O, 4 * Cp, 3, 3), dtype=np.int64)
    for a in range(2):
        for b in range(2):
            for dyp in (-1, 0, 1):
                for dxp in (-1, 0, 1):
                    dy, dx = 2 * dyp + a, 2 * dxp + b
                    if not (-1 <= dy <= 1 and -1 <= dx <= 1):
                        continue
                    for o in range(O):
                        if depthwise:
                            if o < C_in:
                                out[o, (2 * a + b) * Cp + o, dyp + 1, dxp + 1] = weights[o, 0, dy + 1, dx + 1]
                        else:
                            out[o, (2 * a + b) * Cp:(2 * a + b) * Cp + C_in, dyp + 1, dxp + 1] = \
                                weights[o, :, dy + 1, dx + 1]
    return out


def polyphase_spec(spec: dict) -> dict:
    """The derived stride-1 layer of a 3x3 stride-2 layer (a Layout spec)."""
    if spec["stride"] != 2 or spec["kh"] != 3:
        raise ValueError("polyphase packing is for 3x3 stride-2 layers")
    c_n = spec["c_n"]
    if c_n not in (1, 2):
        raise ValueError("polyphase packing is built for c_n 1 and 2")
    Cp = -(-spec["C_in"] // c_n) * c_n
    d = dict(spec, C_in=4 * Cp, H=-(-spec["H"] // 2), W=-(-spec["W"] // 2), stride=1, depthwise=False)
    d.pop("polyphase", None)
    return d


# ---------------------------------------------------------------- keys used
def rotation_steps4(lay: Layout) -> list[int]:
    """Left-rotation steps of a c_n = 4 layer, ascending: 2o for every tap offset o = dy W_b + dx
    and, unless the layer is depthwise (an output class then reads only its own class), the
    parity-changing steps 2o - 1 and 2o + 1."""
    offs = [dy * lay.W_b + dx for dy, dx in lay.taps()]
    steps = {2 * o for o in offs}
    if not lay.depthwise:
        steps |= {2 * o + e for o in offs for e in (-1, 1)}
    return sorted(steps)


def rotation_plan(P: Params, lay: Layout):
    """List of (key, d, Galois element) for every rotated copy of an input ciphertext; Galois
    element 1 is the identity (no key switch).  key is the tap index for c_n = 1, 2 and the
    rotation step (rotation_steps4) for c_n = 4; d = 1 composes the row swap."""
    rows = []
    diag = (0, 1) if (lay.c_n in (2, 4) and not lay.depthwise) else (0,)
    if lay.c_n == 4:
        for step in rotation_steps4(lay):
            g_step = bfv.rotation_element(P, step)
            for d in diag:
                g = g_step if d == 0 else (g_step * bfv.row_swap_element(P)) % (2 * P.N)
                rows.append((step, d, g))
        return rows
    for ti, (dy, dx) in enumerate(lay.taps()):
        g_tap = bfv.rotation_element(P, dy * lay.W_b + dx)
        for d in diag:
            g = g_tap if d == 0 else (g_tap * bfv.row_swap_element(P)) % (2 * P.N)
            rows.append((ti, d, g))
    return rows


def galois_elements(P: Params, lay: Layout) -> list[int]:
    return sorted({g for _, _, g in rotation_plan(P, lay) if g != 1})


# ---------------------------------------------------------------- the layer
def hadamard_scalars(lay: Layout, weights: np.ndarray, g: int, j: int, ti: int, d: int) -> tuple[int, int]:
    """(s0, s1) = (v0 + v1, v0 - v1) for output pair g, input pair j, tap ti,
    diagonal d (Eq. 1 without the 1/2).  Row 0 of the output is channel 2g,
    row 1 is 2g+1; diagonal d = 1 sees the input rows swapped."""
    kw = lay.kh
    dy, dx = divmod(ti, kw)

    def w(o, i):
        if o >= lay.C_out or i >= lay.C_in:
            return 0
        if lay.depthwise:
            return int(weights[o, 0, dy, dx]) if o == i else 0
        return int(weights[o, i, dy, dx])

    if d == 0:
        v0, v1 = w(2 * g, 2 * j), w(2 * g + 1, 2 * j + 1)
    else:
        v0, v1 = w(2 * g, 2 * j + 1), w(2 * g + 1, 2 * j)
    return v0 + v1, v0 - v1


# the 4 x 4 Walsh-Hadamard basis of Sec. 3.1, row b over the slot classes c = 0..3
H4 = ((1, 1, 1, 1), (1, -1, 1, -1), (1, 1, -1, -1), (1, -1, -1, 1))
# search range of k4: [1, min(t - 1, K4_MAX)]
K4_MAX = 1 << 20


def hadamard4_scalars(lay: Layout, weights: np.ndarray, g: int, j: int, step: int, d: int) -> list[int]:
    """(s_0, .., s_3) = H4 v for output group g, input group j and the rotated copy (step, d)
    of a c_n = 4 layer, v_c the weight the copy carries into output class c (Sec. 3.1 with the
    4 x 4 basis, without the 1/4).  Output class c = 2 r + e sits in row r at parity e; the copy
    brings the input of row r ^ d, parity e' = (e + step) mod 2, from offset o = (e + step - e') / 2
    positions away, which is tap (dy, dx) if dy W_b + dx = o with |dy|, |dx| <= P and no tap
    otherwise (unique because W_b > 2P)."""
    taps = {dy * lay.W_b + dx: (dy, dx) for dy, dx in lay.taps()}
    v = [0, 0, 0, 0]
    for c in range(4):
        e = c & 1
        e_src = (e + step) & 1
        tap = taps.get((e + step - e_src) // 2)
        if tap is None:
            continue
        o, i = 4 * g + c, 4 * j + 2 * ((c >> 1) ^ d) + e_src
        if o >= lay.C_out or i >= lay.C_in:
            continue
        dy, dx = tap[0] + lay.P, tap[1] + lay.P
        if lay.depthwise:
            v[c] = int(weights[o, 0, dy, dx]) if o == i else 0
        else:
            v[c] = int(weights[o, i, dy, dx])
    return [sum(H4[b][c] * v[c] for c in range(4)) for b in range(4)]


def hadamard4_patterns(P: Params) -> list[np.ndarray]:
    """Centred coefficients of the plaintexts whose slot of class c (row r, index i: c = 2r +
    (i mod 2)) holds H4[b][c], for b = 1, 2, 3 (slot parity, row, their product)."""
    half = P.N // 2
    cls = np.array([2 * r + (i & 1) for r in range(2) for i in range(half)])
    out = []
    for b in (1, 2, 3):
        m = bfv.encode(P, np.array(H4[b], dtype=np.int64)[cls]).astype(np.int64)
        out.append(np.where(m > P.t // 2, m - P.t, m))
    return out


_K4_CACHE: dict = {}


def k4_select(P: Params) -> int:
    """The k of c_n = 4 (reading of Sec. 3.2.1 for three PMult plaintexts): the k in
    [1, min(t - 1, K4_MAX)] minimising k + sum of |[k a]_t| over the non-zero coefficients a of
    the three patterns (the bound on the noise growth of CMult by k plus the three PMults by the
    k-scaled patterns); ties go to the smallest k."""
    key = (P.N, P.t, P.zeta)
    if key not in _K4_CACHE:
        coeffs = [int(a) % P.t for pat in hadamard4_patterns(P) for a in pat if a]
        ks = np.arange(1, min(P.t - 1, K4_MAX) + 1, dtype=np.int64)
        G = ks.copy()
        for a in coeffs:
            v = (ks * a) % P.t
            G += np.minimum(v, P.t - v)
        _K4_CACHE[key] = int(ks[int(np.argmin(G))])
    return _K4_CACHE[key]


def hadamard4_plaintexts(P: Params) -> tuple[int, list[np.ndarray]]:
    """(k4, [k4 x pattern b, centred, for b = 1, 2, 3])."""
    k4 = k4_select(P)
    out = []
    for pat in hadamard4_patterns(P):
        m = (pat * k4) % P.t
        out.append(np.where(m > P.t // 2, m - P.t, m))
    return k4, out


def output_scale(P: Params, lay: Layout) -> int:
    """The factor the layer's output carries: 2k with pair packing, 4 k4 with c_n = 4, 1 without."""
    if lay.c_n == 4:
        return (4 * k4_select(P)) % P.t
    return (2 * P.k) % P.t if lay.c_n == 2 else 1


def oracle_threads() -> int:
    """Threads the oracle runs on: every host core (HYENA_ORACLE_THREADS overrides)."""
    v = os.environ.get("HYENA_ORACLE_THREADS", "")
    return max(1, int(v)) if v.isdigit() else (os.cpu_count() or 1)


def he_conv(P: Params, lay: Layout, weights: np.ndarray, cts_in: np.ndarray, ksk: dict,
            out_cts: list[int] | None = None, threads: int | None = None,
            timings: dict | None = None) -> np.ndarray:
    """Homomorphic convolution of one layer.

    For every input ciphertext: decompose once, then one hoisted rotation per
    (tap, diagonal).  For every output ciphertext: CMult by the integer
    scalars and HAdd over input ciphertexts, taps and diagonals (reduced
    eagerly: the residues equal those of the lazy form), then with packing
    out = k * A0 + PMult(A1, [k, -k]) (Sec. 3.1, Sec. 3.2.1).

    `out_cts` restricts the work to a subset of output ciphertexts (the
    others are left zero), for sampled comparisons at full size.

    The rotations of different input ciphertexts and the sums of different
    output ciphertexts are independent; they run on `threads` threads (default:
    every host core).  Each job is the same plain code as the one-thread form
    and writes only its own results, so the words do not depend on the count.
    `timings` (optional dict) receives the wall seconds of the two phases,
    "rotations" and "sums" (for the CPU baseline's timing)."""
    plan = rotation_plan(P, lay)
    n_out = lay.n_ct_out
    todo = range(n_out) if out_cts is None else sorted(set(out_cts))
    if any(c < 0 or c >= n_out for c in todo):
        raise ValueError(f"output ciphertext index out of range [0, {n_out})")
    need_ru = sorted({c // lay.out_groups for c in todo})
    out = np.zeros((n_out, 2, P.L, P.N), dtype=np.uint64)
    pk = bfv.hadamard_plaintext(P) if lay.c_n == 2 else (hadamard4_plaintexts(P) if lay.c_n == 4 else None)
    pool = ThreadPoolExecutor(max_workers=threads or oracle_threads())

    def rotations_of(ru: int, j: int) -> dict:
        ct = cts_in[ru * lay.in_groups + j]
        digits = bfv.decompose(P, ct)
        return {(j, ti, d): ct.copy() if g == 1 else bfv.rotate_hoisted(P, ct, digits, ksk[g], g)
                for ti, d, g in plan}

    try:
        for ru in need_ru:
            # rotated copies of this row-unit's input ciphertexts
            rot = {}
            needed_j = range(lay.in_groups)
            if lay.depthwise:
                needed_j = sorted({c % lay.out_groups for c in todo if c // lay.out_groups == ru})
            t0 = time.perf_counter()
            for part in pool.map(lambda j: rotations_of(ru, j), needed_j):
                rot.update(part)
            t1 = time.perf_counter()
            mine = [c for c in todo if c // lay.out_groups == ru]
            for c, res in zip(mine, pool.map(lambda c: _output_ct(P, lay, weights, plan, rot, pk, c), mine)):
                out[c] = res
            if timings is not None:
                timings["rotations"] = timings.get("rotations", 0.0) + t1 - t0
                timings["sums"] = timings.get("sums", 0.0) + time.perf_counter() - t1
    finally:
        pool.shutdown()
    return out


def _output_ct(P: Params, lay: Layout, weights: np.ndarray, plan, rot: dict, pk, c: int) -> np.ndarray:
    """Output ciphertext c of the layer from the rotated copies of its row-unit's inputs."""
    g_out = c % lay.out_groups
    if lay.c_n == 4:
        # four sums A_b = sum s_b x, then out = k4 A_0 + sum_b PMult(A_b, k4 pattern_b)
        A = np.zeros((4, 2, P.L, P.N), dtype=np.uint64)
        js = [g_out] if lay.depthwise else range(lay.in_groups)
        for j in js:
            for step, d, _ in plan:
                sv = hadamard4_scalars(lay, weights, g_out, j, step, d)
                for b in range(4):
                    if sv[b]:
                        bfv.cmult_add(P, A[b], rot[(j, step, d)], sv[b])
        k4, pks = pk
        res = bfv.cmult(P, A[0], k4)
        for b in range(1, 4):
            res = bfv.hadd(P, res, bfv.pmult(P, A[b], pks[b - 1]))
    elif lay.c_n == 2:
        A0 = np.zeros((2, P.L, P.N), dtype=np.uint64)
        A1 = np.zeros((2, P.L, P.N), dtype=np.uint64)
        js = [g_out] if lay.depthwise else range(lay.in_groups)
        for j in js:
            for ti, d, _ in plan:
                s0, s1 = hadamard_scalars(lay, weights, g_out, j, ti, d)
                if s0:
                    bfv.cmult_add(P, A0, rot[(j, ti, d)], s0)
                if s1:
                    bfv.cmult_add(P, A1, rot[(j, ti, d)], s1)
        res = bfv.cmult(P, A0, P.k)
        res = bfv.hadd(P, res, bfv.pmult(P, A1, pk))
    else:
        res = np.zeros((2, P.L, P.N), dtype=np.uint64)
        js = [g_out] if lay.depthwise else range(lay.in_groups)
        for j in js:
            for ti, _, _ in plan:
                dy, dx = divmod(ti, lay.kh)
                f = int(weights[g_out, 0 if lay.depthwise else j, dy, dx]) \
                    if (g_out < lay.C_out and j < lay.C_in) else 0
                if f:
                    bfv.cmult_add(P, res, rot[(j, ti, 0)], f)
    return res


# ------------------------------------------------------------ client helpers
def encrypt_image(P: Params, lay: Layout, s: np.ndarray, act: np.ndarray, seed: int, only=None,
                  threads: int | None = None) -> np.ndarray:
    """Input ciphertexts [n_ct_in][2][L][N] of a layer; ciphertext c uses the random streams of index c.
    `only` (optional): encrypt just these ciphertext indices and leave the others zero."""
    idx = range(lay.n_ct_in) if only is None else sorted(set(only))
    ru_set = None if only is None else {c // lay.in_groups for c in idx}
    slots = pack_slots(lay, act, ru_set)
    out = np.zeros((lay.n_ct_in, 2, P.L, P.N), dtype=np.uint64)
    with ThreadPoolExecutor(max_workers=threads or oracle_threads()) as pool:
        for c, ct in zip(idx, pool.map(lambda c: bfv.encrypt(P, s, bfv.encode(P, slots[c]), seed, c), idx)):
            out[c] = ct
    return out


def decrypt_image(P: Params, lay: Layout, s: np.ndarray, cts_out: np.ndarray, unscale: bool = True) -> np.ndarray:
    slots = np.stack([bfv.decode(P, bfv.decrypt(P, s, cts_out[c])) for c in range(lay.n_ct_out)])
    out = unpack_slots(lay, slots)
    if unscale:
        inv = pow(output_scale(P, lay), -1, P.t)
        out = (out * inv) % P.t
    return out
