"""The barrier protocol of the tensor-core convolution (k_conv3x3_tc), modelled on the host.

The kernel's three roles -- the producer warp copying input rows into a ring (one TMA copy a
row, landing in any order), the warp issuing the MMAs of each input row, the epilogue warps
draining output rows -- meet only at mbarriers, and a parity wait is correct only when its barrier is at the awaited phase or the
one after it.  This model walks the same chunks and rows as the kernel, with the ring, slot and
barrier sizes read from the kernel source, under random interleavings of the three roles, and
checks that:
  - no role waits forever (every schedule finishes);
  - every parity wait finds its barrier at the awaited phase or the next one;
  - the issuer reads the row the producer staged for it, and only once it has landed;
  - an accumulator slot is first written only after its previous output row was drained, and
    the epilogue reads the slot of the output row it expects.
Image heights from 1 row to several chunks, and blocks walking several chunks, are covered."""
import pathlib
import random
import re

import pytest

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2312_06827_gb300" / "csrc" / "svgf_kpn.cu"


def constant(name):
    m = re.search(rf"constexpr\s+\w+\s+{name}\s*=\s*(\d+)\s*;", SRC.read_text())
    assert m, name
    return int(m.group(1))


K_RING = constant("kRing")
K_SLOTS, K_DONE = constant("kSlots"), constant("kDone")


class Barrier:
    def __init__(self, count=1):
        self.count, self.arrived, self.phase = count, 0, 0

    def arrive(self):
        self.arrived += 1
        if self.arrived == self.count:
            self.arrived, self.phase = 0, self.phase + 1

    def done(self, k):
        """Parity wait for phase k: complete, or not yet; anything else is a protocol error."""
        assert self.phase in (k, k + 1), f"parity wait for phase {k} at phase {self.phase}"
        return self.phase == k + 1


def simulate(H, chunks_per_block, seed, chunk=16, groups=2):
    rnd = random.Random(seed)
    chunks = [(y0, min(y0 + chunk, H)) for _ in range(chunks_per_block) for y0 in range(0, H, chunk)]
    done = [Barrier() for _ in range(K_DONE)]
    full = [Barrier(1) for _ in range(K_RING)]
    rfree = [Barrier() for _ in range(K_RING)]
    drained = [Barrier(128) for _ in range(K_SLOTS)]
    staged, acc = {}, {}

    copies = []                                 # TMA copies issued, not yet landed (slot)

    def producer():
        """Warp 5: one TMA copy a row, issued once the slot's previous row was read."""
        used, phase, rs = set(), [0] * K_RING, 0
        for ci, (y0, y1) in enumerate(chunks):
            for q in range(y0 - 1, y1 + 1):
                sl = rs % K_RING
                rs += 1
                if sl in used:
                    while not rfree[sl].done(phase[sl]):
                        yield
                    phase[sl] += 1
                used.add(sl)
                staged[sl] = ("in flight", ci, q)
                copies.append(sl)
                yield
        while copies:                            # its copies land before the block ends
            yield

    def copy_engine():
        """The copies land in any order, each completing its slot's barrier (expected bytes)."""
        while True:
            if copies:
                sl = copies.pop(rnd.randrange(len(copies)))
                staged[sl] = ("landed",) + staged[sl][1:]
                full[sl].arrive()
            yield

    def issuer():
        nb, obase = 0, 0
        fphase, dphase, dused = [0] * K_RING, [0] * K_SLOTS, set()
        for ci, (y0, y1) in enumerate(chunks):
            for r in range(y0 - 1, y1 + 1):
                sl = nb % K_RING
                while not full[sl].done(fphase[sl]):
                    yield
                fphase[sl] += 1
                assert staged[sl] == ("landed", ci, r), (staged[sl], ci, r)
                if r + 1 <= y1 - 1:                     # output row r + 1 starts here
                    ts = (obase + r + 1 - y0) % K_SLOTS
                    if ts in dused:
                        while not drained[ts].done(dphase[ts]):
                            yield
                        dphase[ts] += 1
                    dused.add(ts)
                    assert acc.get(ts, ("drained",))[0] == "drained", (ts, acc.get(ts))
                    acc[ts] = ("live", ci, r + 1)
                yield                                   # the MMAs run
                assert staged[sl] == ("landed", ci, r), ("restaged under the MMAs", staged[sl], ci, r)
                if r - 1 >= y0:
                    done[(obase + r - 1 - y0) % K_DONE].arrive()
                rfree[sl].arrive()
                nb += 1
            obase += y1 - y0

    def epilogue(g):
        """Warps 4g .. 4g + 3: the output rows whose running index is g modulo `groups`."""
        obase = 0
        for ci, (y0, y1) in enumerate(chunks):
            for o in range(y0, y1):
                oi = obase + o - y0
                if oi % groups != g:
                    continue
                while not done[oi % K_DONE].done(oi // K_DONE):
                    yield
                ts = oi % K_SLOTS
                assert acc.get(ts) == ("live", ci, o), (ts, acc.get(ts), ci, o)
                acc[ts] = ("drained",)
                for _ in range(128):
                    drained[ts].arrive()
                yield
            obase += y1 - y0

    roles = [copy_engine(), producer(), issuer()] + [epilogue(g) for g in range(groups)]
    alive = [True] * len(roles)
    # uneven speeds drawn per schedule, so that one role can run far ahead of another
    weights = [rnd.choice((1, 1, 4, 16)) for _ in roles]
    for _ in range(10 ** 6):
        if not any(alive[1:]):
            return
        i = rnd.choices(range(len(roles)), weights)[0]
        if alive[i]:
            try:
                next(roles[i])
            except StopIteration:
                alive[i] = False
    raise AssertionError(f"no progress: H={H}, {chunks_per_block} chunk rounds, seed {seed}")


def test_constants_satisfy_the_ring_bounds():
    assert K_RING >= 3                        # the three input rows of an output row fit the ring
    assert K_DONE >= K_SLOTS                 # the issuer completes at most K_SLOTS - 3 rows ahead
    assert K_SLOTS % 2 == 0 and K_DONE % 2 == 0   # with two drain groups each slot has one group


@pytest.mark.parametrize("H", [1, 2, 3, 5, 15, 16, 17, 33, 64, 135])
@pytest.mark.parametrize("rounds", [1, 3])
@pytest.mark.parametrize("groups", [1, 2])
def test_protocol_under_random_schedules(H, rounds, groups):
    for seed in range(12):
        simulate(H, rounds, seed, groups=groups)


def conv_chunk(B, H, W, sm_count=152):
    """The launcher's chunk length (svgf_kpn.cu, conv_chunk): at most one chunk a block."""
    cols = B * ((W + 127) // 128)
    cap = 2 * sm_count
    per = 1 if cols >= cap else cap // cols
    per = min(per, H)
    return (H + per - 1) // per


def test_chunk_choice_fills_the_grid_once():
    for B, H, W in ((1, 1080, 1920), (1, 2160, 3840), (16, 256, 256), (2, 24, 40), (51, 17, 257),
                    (1, 360, 640), (1, 120, 200), (3, 1, 1)):
        chunk = conv_chunk(B, H, W)
        assert 1 <= chunk <= H
        tiles = B * ((W + 127) // 128) * ((H + chunk - 1) // chunk)
        cols = B * ((W + 127) // 128)
        assert tiles <= max(304, cols)           # one chunk a block, unless the columns alone exceed the grid
    assert conv_chunk(1, 1080, 1920) == 54 and conv_chunk(1, 2160, 3840) == 216
    src = SRC.read_text()
    assert "long per = cols >= cap ? 1 : cap / cols;" in src and "if (per > H) per = H;" in src


@pytest.mark.parametrize("chunk", [1, 2, 3, 6, 29, 54])
@pytest.mark.parametrize("H", [1, 2, 7, 29, 54, 120])
def test_protocol_with_the_launch_chunk_lengths(chunk, H):
    for seed in range(6):
        simulate(H, 2, seed, chunk)


@pytest.mark.parametrize("old,new", [
    # the producer copies a row into a slot before the MMAs of its previous row completed
    ("while not rfree[sl].done(phase[sl]):", "while False:"),
    # the issuer starts an output row without waiting for its slot to be drained
    ("while not drained[ts].done(dphase[ts]):", "while False:"),
    # the producer and the issuer number the ring slots differently (per chunk and running)
    ("sl = nb % K_RING", "sl = (r + 1) % K_RING"),
    # both drain groups take every output row
    ("                if oi % groups != g:\n                    continue\n", ""),
])
def test_model_catches_planted_protocol_mistakes(old, new):
    """The model is not vacuous: each planted mistake makes some schedule stall or trip a check."""
    import inspect
    src = inspect.getsource(simulate)
    assert src.count(old) == 1, old
    ns = dict(globals())
    exec(src.replace(old, new), ns)
    failures = 0
    for seed in range(24):
        try:
            ns["simulate"](17, 3, seed)
        except AssertionError:
            failures += 1
    assert failures > 0