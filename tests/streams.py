"""Test helpers: numpy brick extraction, the mode pyramid, golden fixtures and an enumerator of
legal operation streams for tiny bricks.

These are written from the definitions independently of the oracle's C code, so that the oracle
can be checked against them.
"""
from __future__ import annotations

import os
import random

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

OP_PARENT, OP_NX, OP_NY, OP_NZ, OP_ADV, OP_LAST, OP_DELTA = range(7)


def padded_brick(V: np.ndarray, b: int, brick_id: int) -> np.ndarray:
    """The b^3 voxels of brick `brick_id` (x-fastest ids), clamp-to-edge beyond the volume."""
    dz, dy, dx = V.shape
    nbx, nby = -(-dx // b), -(-dy // b)
    bx, by, bz = brick_id % nbx, (brick_id // nbx) % nby, brick_id // (nbx * nby)
    zs = np.minimum(np.arange(bz * b, bz * b + b), dz - 1)
    ys = np.minimum(np.arange(by * b, by * b + b), dy - 1)
    xs = np.minimum(np.arange(bx * b, bx * b + b), dx - 1)
    return V[np.ix_(zs, ys, xs)]


def mode_down(g: np.ndarray) -> np.ndarray:
    """One level of the mode pyramid: each 2^3 block -> its most frequent label, ties -> smallest."""
    n = g.shape[0] // 2
    c = g.reshape(n, 2, n, 2, n, 2).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 8).astype(np.int64)
    counts = (c[:, :, None] == c[:, None, :]).sum(axis=2)
    key = counts * (1 << 33) + ((1 << 32) - 1 - c)
    pick = np.argmax(key, axis=1)
    return c[np.arange(c.shape[0]), pick].astype(np.uint32).reshape(n, n, n)


def mode_pyramid(brick: np.ndarray) -> list:
    """[level 0 (1^3), ..., level L (the brick)] as (z, y, x) arrays."""
    levels = [brick]
    while levels[0].shape[0] > 1:
        levels.insert(0, mode_down(levels[0]))
    return levels


def uniform_pyramid(brick: np.ndarray) -> list:
    """Per level: True where every voxel below the node has one label."""
    n = brick.shape[0]
    L = n.bit_length() - 1
    out = []
    for l in range(L + 1):
        s = n >> l
        m = 1 << l
        blk = brick.reshape(m, s, m, s, m, s).transpose(0, 2, 4, 1, 3, 5).reshape(m, m, m, -1)
        out.append((blk == blk[..., :1]).all(axis=-1))
    return out


def morton_to_xyz(m: int, bits: int):
    x = y = z = 0
    for i in range(bits):
        x |= ((m >> (3 * i)) & 1) << i
        y |= ((m >> (3 * i + 1)) & 1) << i
        z |= ((m >> (3 * i + 2)) & 1) << i
    return x, y, z


def load_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            out[key] = rest.split()
    return out


def golden_volume(g: dict) -> np.ndarray:
    dx, dy, dz = (int(v) for v in g["dims"])
    rule = g["rule"][0]
    z, y, x = np.meshgrid(np.arange(dz), np.arange(dy), np.arange(dx), indexing="ij")
    if rule.startswith("corner:"):
        _, a, c = rule.split(":")
        V = np.full((dz, dy, dx), int(a), dtype=np.uint32)
        V[dz - 1, dy - 1, dx - 1] = int(c)
        return V
    thr = int(rule.split("<")[1].split(":")[0])
    lo, hi = int(g["rule"][0].split(":")[1]), int(g["rule"][1].split(":")[1])
    return np.where(x < thr, lo, hi).astype(np.uint32)


def octal_digits(d: int) -> list:
    return [int(c) for c in oct(d)[2:]]


class StreamEnumerator:
    """All (or randomly sampled) legal operation streams that decode a tiny brick to its voxels.

    Coarse nodes take their mode-pyramid labels; each emitted node may use any enabled operation
    that yields its label: parent, a neighbour copy (coordinate even and > 0), last, any delta
    1 <= d <= k pointing at the label, or a palette advance (always legal, duplicates included).
    A node whose subtree is constant may set its stop bit or not.
    """

    def __init__(self, brick: np.ndarray, op_mask: int = 0x7F, allow_stop: bool = True):
        self.brick = brick
        self.n = brick.shape[0]
        self.L = self.n.bit_length() - 1
        self.lab = mode_pyramid(brick)
        self.uni = uniform_pyramid(brick)
        self.op_mask = op_mask
        self.allow_stop = allow_stop

    def _options(self, l, c, dec, pal):
        x, y, z = c
        t = int(self.lab[l][z, y, x])
        k = len(pal)
        opts = []
        en = lambda o: (self.op_mask >> o) & 1
        if l > 0 and en(OP_PARENT) and int(dec[l - 1][(x >> 1, y >> 1, z >> 1)]) == t:
            opts.append((OP_PARENT, 0))
        for a, op in ((0, OP_NX), (1, OP_NY), (2, OP_NZ)):
            if not en(op) or c[a] == 0 or c[a] & 1:
                continue
            q = list(c)
            q[a] -= 1
            if int(dec[l][tuple(q)]) == t:
                opts.append((op, 0))
        if en(OP_LAST) and k >= 1 and pal[k - 1] == t:
            opts.append((OP_LAST, 0))
        if en(OP_DELTA):
            for d in range(1, k + 1):
                if pal[k - d] == t:
                    opts.append((OP_DELTA, d))
        opts.append((OP_ADV, 0))
        stops = [0]
        if l < self.L and self.allow_stop and bool(self.uni[l][z, y, x]):
            stops = [0, 1]
        return t, opts, stops

    def _walk(self, chooser):
        """Replays one stream; chooser(options) picks. Yields (symbols, palette, n_delta)."""
        L = self.L
        dec = [dict() for _ in range(L + 1)]
        expanded = [dict() for _ in range(L + 1)]
        pal, sym, nd = [], [], 0
        for l in range(L + 1):
            m_count = 1 << (3 * l)
            for m in range(m_count):
                c = morton_to_xyz(m, l)
                pc = (c[0] >> 1, c[1] >> 1, c[2] >> 1)
                if l > 0 and not expanded[l - 1][pc]:
                    dec[l][c] = dec[l - 1][pc]
                    expanded[l][c] = False
                    continue
                t, opts, stops = self._options(l, c, dec, pal)
                (op, d), stop = chooser(opts, stops)
                if op == OP_ADV:
                    pal.append(t)
                sym.append(op | (stop << 3))
                if op == OP_DELTA:
                    digits = octal_digits(d)
                    for i, g in enumerate(digits):
                        sym.append(g | (8 if i + 1 < len(digits) else 0))
                    nd += 1
                dec[l][c] = t
                expanded[l][c] = (l < L) and not stop
        return sym, pal, nd

    def sample(self, rng: random.Random):
        return self._walk(lambda opts, stops: (rng.choice(opts), rng.choice(stops)))

    def canonical_first(self):
        return self._walk(lambda opts, stops: (opts[0], stops[-1]))

    def count_and_enumerate(self, limit: int):
        """Exhaustive DFS over all choices; returns the list of streams, or None past `limit`."""
        out = []
        choices = []

        def run():
            idx = [0]

            def chooser(opts, stops):
                flat = [(o, s) for o in opts for s in stops]
                i = idx[0]
                idx[0] += 1
                if i == len(choices):
                    choices.append([0, len(flat)])
                return flat[choices[i][0]]

            return self._walk(chooser)

        while True:
            out.append(run())
            if len(out) > limit:
                return None
            # advance the mixed-radix counter from the deepest decision
            while choices and choices[-1][0] + 1 >= choices[-1][1]:
                choices.pop()
            if not choices:
                return out
            choices[-1][0] += 1
