"""The swizzled operand layouts of the tensor-core convolution, checked on the host.

The producer stages input pixel px, channel ch of a row at
    slot + px * RB + ((ch // 8) ^ f(px)) * 16 + (ch % 8) * 2,
RB = 64 bytes and f(px) = (px >> 1) & 3 for 32 channels (64-byte swizzle), RB = 32 and
f(px) = (px >> 2) & 1 for 16 channels (32-byte swizzle), and the weights likewise with the B row
r = (2 - dy) * 32 + co in place of px.  The MMA of horizontal tap dx and channel step kc starts
its descriptor dx * RB + kc * 32 bytes into the slot; the tensor core reads row i, element k at
the logical address start + i * RB + 2 k with address bits 4-5 (64-byte) or bit 4 (32-byte)
XORed with bits 7-8 or bit 7 -- a swizzle of absolute shared-memory addresses, which a GPU test
(a layer against a CPU convolution, row by row) confirmed.  Here every (tap, step, row,
element) is mapped both ways for both layouts, with the slot sizes and the weight block size
read from the kernel source, which must keep every slot on the swizzle pattern's boundary."""
import pathlib
import re

import pytest

SRC = (pathlib.Path(__file__).resolve().parents[1] / "paper_2312_06827_gb300" / "csrc" / "svgf_kpn.cu").read_text()


def constant(name):
    m = re.search(rf"constexpr\s+\w+\s+{name}\s*=\s*([^;]+);", SRC)
    assert m, name
    return int(eval(m.group(1), {}))          # e.g. "17 * 512"


K_RING = constant("kRing")
HP = constant("HP") if re.search(r"constexpr int HP = \d+;", SRC) else constant("M") + 2


def swizzle(addr, rb):
    if rb == 64:
        return addr ^ (((addr >> 7) & 3) << 4)
    return addr ^ (((addr >> 7) & 1) << 4)


def staged(slot, px, ch, rb):
    f = ((px >> 1) & 3) if rb == 64 else ((px >> 2) & 1)
    return slot + px * rb + (((ch // 8) ^ f) << 4) + (ch % 8) * 2


@pytest.mark.parametrize("ci", [32, 16])
def test_a_operand_addresses(ci):
    rb = 2 * ci
    row_bytes = constant("kRowSw64Bytes") if ci == 32 else constant("kRowSw32Bytes")
    pattern = 512 if ci == 32 else 256
    w_bytes = 9 * (ci // 8) * 32 * 16
    assert row_bytes % pattern == 0 and row_bytes >= HP * rb
    assert w_bytes % pattern == 0                 # the ring starts after the weights
    for sl in range(K_RING):
        slot = w_bytes + sl * row_bytes           # shared memory is 1024-byte aligned
        assert slot % pattern == 0
        for dx in range(3):
            for kc in range(ci // 16):
                start = slot + dx * rb + kc * 32
                for i in range(128):
                    for k in range(16):
                        logical = start + i * rb + 2 * k
                        assert swizzle(logical, rb) == staged(slot, dx + i, kc * 16 + k, rb)
                        assert slot <= swizzle(logical, rb) < slot + row_bytes


@pytest.mark.parametrize("ci", [32, 16])
def test_b_operand_addresses(ci):
    """Weights: per dx the 96 rows (2 - dy) * 32 + co; an MMA over output blocks blk0.. starts
    dx * 96 * RB + blk0 * 32 * RB + kc * 32 bytes in."""
    rb = 2 * ci
    w_bytes = 9 * (ci // 8) * 32 * 16
    assert 3 * 96 * rb == w_bytes
    for dx in range(3):
        for blk0 in range(3):
            for kc in range(ci // 16):
                start = dx * 96 * rb + blk0 * 32 * rb + kc * 32
                for n in range(32 * (3 - blk0)):
                    for k in range(16):
                        logical = start + n * rb + 2 * k
                        r = blk0 * 32 + n
                        assert swizzle(logical, rb) == staged(dx * 96 * rb, r, kc * 16 + k, rb)
                        assert swizzle(logical, rb) < w_bytes


def test_a_shift_in_the_plain_layout_would_not_hold():
    """The check is not vacuous: without the swizzle on the staging side, odd tap shifts land
    on the wrong chunks."""
    rb, slot = 64, 0
    bad = sum(swizzle(slot + dx * rb + i * rb, rb) != slot + (dx + i) * rb
              for dx in range(3) for i in range(128))
    assert bad > 0
