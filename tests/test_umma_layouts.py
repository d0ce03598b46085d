"""Host checks of the order-sized tcgen05 kernel's shared-memory layout table
(kGenLayouts in csrc/ax_umma.cuh): for every order and operand width, the
three operand buffers' core matrices (8 rows x 16 bytes) do not overlap,
every staging and MMA access stays inside its buffer and 16-byte aligned,
the exchange rows fit their k pitch, a CTA's shared memory fits, and a
bank-conflict model of the kernel's shared-memory accesses counts no more
wavefronts per tile than for dense layouts (the table came from a search
over that model).  The tile geometry is restated here from the kernel's
definitions: EPB = 128 / N1^2 elements (one above N1 = 11), one thread per
MMA row, K padded to whole instructions."""
import os
import re
from collections import defaultdict

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "paper_2504_07042_gb300", "csrc", "ax_umma.cuh")


def table():
    text = open(SRC).read()
    body = text[text.index("constexpr GenLayout kGenLayouts[] = {"):]
    body = body[:body.index("};")]
    rows = [tuple(int(v) for v in m.groups()) for m in re.finditer(r"\{(\d+), (\d+), " + ", ".join([r"(\d+)"] * 8) + r"\}", body)]
    return {(r[0], r[1]): r[2:] for r in rows}


class Shape:
    def __init__(self, N1, op, layout):
        self.N1, self.F = N1, N1 * N1
        self.EPB = 1 if self.F > 128 else 128 // self.F
        self.ROWS, self.N3 = self.EPB * self.F, N1 ** 3
        self.MB = (self.ROWS + 127) // 128
        self.ESZ = 4 if op == 0 else 2
        self.PER = 16 // self.ESZ
        self.KI = 8 if op == 0 else 16
        self.NI = (N1 + self.KI - 1) // self.KI
        self.NC = self.NI * self.KI // self.PER
        self.NCD = (N1 + self.PER - 1) // self.PER
        self.PJ, self.XK, lr, sr, ls, ss, lt, st = layout
        self.L = [(lr, sr), (ls, ss), (lt, st)]
        self.XE = N1 * self.XK

    def span(self, b):
        lbo, sbo = self.L[b]
        return (16 * self.MB - 1) * sbo + (self.NC - 1) * lbo + 128

    def cm(self, b, row, k):
        lbo, sbo = self.L[b]
        return (row >> 3) * sbo + (k // self.PER) * lbo + (row & 7) * 16 + (k % self.PER) * self.ESZ

    def lab(self, t):
        return t % self.N1, (t // self.N1) % self.N1, t // self.F

    def xpos(self, e, i, j, k):
        return e * self.XE + k * self.XK + j * self.PJ + i


def wavefronts(addrs, width):
    """Shared-memory wavefronts of one warp access: 32 banks of 4 bytes; a
    16-byte access is served in quarter-warp phases."""
    if not addrs:
        return 0
    per = 32 if width <= 4 else 128 // width
    total = 0
    lanes = sorted(addrs)
    for p in range(0, 32, per):
        banks = defaultdict(set)
        for lane in lanes:
            if p <= lane < p + per:
                a = addrs[lane]
                for w in range(max(1, width // 4)):
                    banks[((a // 4) + w) % 32].add(a // 4 + w)
        if banks:
            total += max(len(v) for v in banks.values())
    return total


def tile_wavefronts(s):
    """Wavefronts per tile of the kernel's shared-memory accesses: staging and
    r, s stores (per value), the t row in 16-byte stores, the two exchange
    writes and the owners' reads (x and Y passes)."""
    N1, F = s.N1, s.F
    tot = 0
    for w in range(s.MB * 4):
        rows = [t for t in range(32 * w, 32 * w + 32) if t < s.ROWS]
        if not rows:
            continue
        for k in range(N1):
            ar = {t - 32 * w: s.cm(0, s.lab(t)[1] + N1 * k + F * s.lab(t)[2], s.lab(t)[0]) for t in rows}
            as_ = {t - 32 * w: s.cm(1, s.lab(t)[0] + N1 * k + F * s.lab(t)[2], s.lab(t)[1]) for t in rows}
            tot += 2 * (wavefronts(ar, s.ESZ) + wavefronts(as_, s.ESZ))
        for c in range(s.NCD):
            tot += 2 * wavefronts({t - 32 * w: s.cm(2, t, c * s.PER) for t in rows}, 16)
        for q in range(N1):
            a0 = {t - 32 * w: 4 * s.xpos(s.lab(t)[2], q, s.lab(t)[0], s.lab(t)[1]) for t in rows}
            a1 = {t - 32 * w: 4 * s.xpos(s.lab(t)[2], s.lab(t)[0], q, s.lab(t)[1]) for t in rows}
            tot += 2 * (wavefronts(a0, 4) + wavefronts(a1, 4))
        for k in range(N1):
            a = {t - 32 * w: 4 * s.xpos(s.lab(t)[2], s.lab(t)[0], s.lab(t)[1], k) for t in rows}
            tot += 4 * wavefronts(a, 4)
    return tot


TABLE = table()


def test_table_covers_every_order():
    # every order but 7 (its own kernel), both operand widths
    assert set(TABLE) == {(n1, op) for n1 in range(2, 17) if n1 != 8 for op in (0, 1)}


@pytest.mark.parametrize("key", sorted(TABLE))
def test_layout_is_sound(key):
    N1, op = key
    s = Shape(N1, op, TABLE[key])
    for b in range(3):
        lbo, sbo = s.L[b]
        assert lbo % 16 == 0 and sbo % 16 == 0 and lbo >= 16 and sbo >= 16
        # the core matrices of the buffer are disjoint
        pos = sorted(g * sbo + c * lbo for g in range(16 * s.MB) for c in range(s.NC))
        assert all(q - p >= 128 for p, q in zip(pos, pos[1:]))
        # each MMA instruction's K slice of each 128-row block lies inside
        for mb in range(s.MB):
            for q in range(s.NI):
                first = mb * 16 * sbo + q * (s.KI // s.PER) * lbo
                assert first % 16 == 0
                assert first + 15 * sbo + (s.KI // s.PER - 1) * lbo + 128 <= s.span(b)
    assert s.span(2) % 16 == 0
    for t in range(s.ROWS):
        la, lb, le = s.lab(t)
        for k in range(N1):
            assert s.cm(0, lb + N1 * k + s.F * le, la) + s.ESZ <= s.span(0)
            assert s.cm(1, la + N1 * k + s.F * le, lb) + s.ESZ <= s.span(1)
        for c in range(s.NCD):
            o = s.cm(2, t, c * s.PER)
            assert o % 16 == 0 and o + 16 <= s.span(2)
    # exchange rows inside the k pitch, the buffer inside EPB elements
    assert (N1 - 1) * s.PJ + N1 <= s.XK
    xf = s.EPB * s.XE
    for t in range(s.ROWS):
        la, lb, le = s.lab(t)
        assert s.xpos(le, N1 - 1, la, lb) < xf and s.xpos(le, la, N1 - 1, lb) < xf and s.xpos(le, la, lb, N1 - 1) < xf
    # shared memory of a CTA: operand buffers, two exchange buffers, two B
    # buffers, the geometry records and barriers
    a16 = lambda v: (v + 15) // 16 * 16
    bbytes = ((16 if N1 > 8 else 24) // 8) * s.NC * 128
    total = sum(s.span(b) for b in range(3)) + 2 * a16(4 * xf) + 2 * bbytes + s.EPB * 96 + 64
    assert total <= 227 * 1024


@pytest.mark.parametrize("key", sorted(TABLE))
def test_layout_no_worse_than_dense(key):
    N1, op = key
    s = Shape(N1, op, TABLE[key])
    dense_layout = (N1, N1 * N1 + (4 if (N1 * N1) % 32 == 16 else 0)) + (128, s.NC * 128 + 16) * 3
    dense = Shape(N1, op, dense_layout)
    assert tile_wavefronts(s) <= tile_wavefronts(dense)


def _consts(block):
    return {k: int(eval(v)) for k, v in re.findall(r"(k\w+) = ([0-9 *]+)[,;]", block)}


def _fmt_blocks():
    text = open(SRC).read()
    f0 = text[text.index("struct Fmt<0> {"):]
    f0 = f0[:f0.index("};")]
    f16 = text[text.index("struct Fmt16 {"):]
    f16 = f16[:f16.index("};")]
    return _consts(f0), _consts(f16)


@pytest.mark.parametrize("which", ["tf32", "16-bit"])
def test_order7_layouts_are_sound(which):
    # the order-7 kernel's hand-tuned operand layouts: 128 rows (16 row
    # groups) of K = 8 values; TF32 fills two 16-byte K cores, the 16-bit
    # formats one (its second K half is the first again, LBO = 0, against a
    # zero second K half of the B buffers)
    c = _fmt_blocks()[0 if which == "tf32" else 1]
    esz = 4 if which == "tf32" else 2
    ncols = 8 * esz // 16  # K cores holding the 8 values of a row
    for buf in "RST":
        lbo, sbo, nbytes = c["kLbo" + buf], c["kSbo" + buf], c["kBytes" + buf]
        assert lbo % 16 == 0 and sbo % 16 == 0 and nbytes % 16 == 0
        pos = sorted(g * sbo + col * lbo for g in range(16) for col in range(ncols))
        assert all(q - p >= 128 for p, q in zip(pos, pos[1:]))
        assert pos[-1] + 128 <= nbytes
        if ncols == 1:
            assert lbo == 0  # the MMA's second K half reads the first again
    # B buffers: 24 rows (3 row groups) of two K cores (TF32) or of one K core
    # and the zero second K half (16-bit)
    lbo, sbo, nbytes = c["kLboB"], c["kSboB"], c["kBytesB"]
    pos = sorted(g * sbo + col * lbo for g in range(3) for col in range(2))
    assert all(q - p >= 128 for p, q in zip(pos, pos[1:]))
    assert pos[-1] + 128 <= nbytes
