"""The barrier protocol of the two-layer tensor-core kernels (k_kpn_pair), modelled on the host.

A block runs two layers.  Warp 16 stages the input rows into the first ring (a fixed number of
rows ahead) and issues the first layer's MMAs; warp 17 issues the second layer's.  The tensor
core completes each warp's MMAs in that warp's issue order (a commit arrives once all of that
warp's earlier MMAs have completed; the two warps' streams interleave arbitrarily).  Each layer's
output rows are drained by two groups of four warps, the rows of even and of odd running index;
the first layer's rows go into the second layer's ring.  The model takes the ring, slot,
barrier and look-ahead sizes from the kernel source and runs random interleavings, checking that:
  - every schedule finishes (no role waits forever);
  - every parity wait finds its barrier at the awaited phase or the one after it;
  - an MMA reads the row it expects from a ring slot, from issue until it completes;
  - an accumulator slot is first written only after its previous output row was drained, and
    each group drains the output row it expects, with all three input rows accumulated.
Heights from one row to several chunks, and blocks walking several chunks, are covered."""
import inspect
import pathlib
import random
import re

import pytest

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2312_06827_gb300" / "csrc" / "svgf_kpn.cu"


def constant(name):
    m = re.search(rf"\b{name}\s*=\s*(\d+)\s*[;,]", SRC.read_text())
    assert m, name
    return int(m.group(1))


RING_IN, AHEAD = constant("kPairRingIn"), constant("kPairAhead")
RING, SLOTS, DONE = constant("kPairRing"), constant("kPairSlots"), constant("kPairDone")


class Barrier:
    def __init__(self, count=1):
        self.count, self.arrived, self.phase = count, 0, 0

    def arrive(self):
        self.arrived += 1
        if self.arrived == self.count:
            self.arrived, self.phase = 0, self.phase + 1

    def done(self, k):
        assert self.phase in (k, k + 1), f"parity wait for phase {k} at phase {self.phase}"
        return self.phase == k + 1


def simulate(H, chunk, rounds, seed, ahead=AHEAD, ring=RING, slots=SLOTS, max_moves=10 ** 6):
    rnd = random.Random(seed)
    chunks = [(y0, min(y0 + chunk, H)) for _ in range(rounds) for y0 in range(0, H, chunk)]
    rfree_in = [Barrier() for _ in range(RING_IN)]
    full = [Barrier(128) for _ in range(ring)]
    rfree = [Barrier() for _ in range(ring)]
    done = [[Barrier() for _ in range(DONE)] for _ in range(2)]
    drained = [[Barrier(128) for _ in range(slots)] for _ in range(2)]
    rin, rmid = {}, {}
    acc = [{}, {}]
    tensor = [[], []]

    def nin(rows, j):
        return rows + 4 - 2 * j

    in_rows = [(ci, k) for ci, (y0, y1) in enumerate(chunks) for k in range(nin(y1 - y0, 0))]

    def issuer(j):
        nb, ob, dused = 0, 0, set()
        fphase, dphase = [0] * ring, [0] * slots
        staged, used0, phase0 = 0, set(), [0] * RING_IN
        for ci, (y0, y1) in enumerate(chunks):
            rows = y1 - y0
            n_in = nin(rows, j)
            nout = n_in - 2
            for k in range(n_in):
                if j == 0:
                    sl = nb % RING_IN
                    while staged < nb + 1 + ahead and staged < len(in_rows):
                        s0 = staged % RING_IN
                        if s0 in used0:
                            while not rfree_in[s0].done(phase0[s0]):
                                yield
                            phase0[s0] += 1
                        used0.add(s0)
                        rin[s0] = ("in flight",) + in_rows[staged]
                        staged += 1
                        yield
                    rin[sl] = ("landed",) + rin[sl][1:]
                    assert rin[sl] == ("landed", ci, k), (rin[sl], ci, k)
                else:
                    sl = nb % ring
                    while not full[sl].done(fphase[sl]):
                        yield
                    fphase[sl] += 1
                    assert rmid.get(sl) == (ci, k), (sl, rmid.get(sl), ci, k)
                if k < nout:
                    ts = (ob + k) % slots
                    if ts in dused:
                        while not drained[j][ts].done(dphase[ts]):
                            yield
                        dphase[ts] += 1
                    dused.add(ts)
                    assert acc[j].get(ts, ["drained"])[0] == "drained", (j, ts, acc[j].get(ts))
                    acc[j][ts] = ["live", ci, k, 0]
                lo, hi = max(k - 2, 0), min(k, nout - 1)
                outs = []
                for o in range(lo, hi + 1):
                    ts = (ob + o) % slots
                    assert acc[j][ts][:3] == ["live", ci, o], (j, ts, acc[j][ts], ci, o)
                    outs.append(ts)
                yield
                commits = [("done", (ob + k - 2) % DONE)] if k >= 2 else []
                commits.append(("rfree", sl))
                tensor[j].append((sl, ci, k, outs, commits))
                nb += 1
            ob += nout

    def tensor_core():
        while True:
            busy = [j for j in (0, 1) if tensor[j]]
            if not busy:
                yield
                continue
            j = rnd.choice(busy)
            sl, ci, k, outs, commits = tensor[j][0]
            if j == 0:
                assert rin[sl] == ("landed", ci, k), ("restaged under the MMAs", rin[sl], ci, k)
            else:
                assert rmid.get(sl) == (ci, k), ("rewritten under the MMAs", sl)
            for ts in outs:
                acc[j][ts][3] += 1
            tensor[j].pop(0)
            for kind, idx in commits:
                (done[j][idx] if kind == "done" else (rfree_in[idx] if j == 0 else rfree[idx])).arrive()
            yield

    def drain(j, par):
        """Warps 4g .. 4g + 3, g = 2j + par: layer j's rows of running parity par, in order."""
        ob = 0
        rphase, rused = [0] * ring, set()
        for ci, (y0, y1) in enumerate(chunks):
            nout = nin(y1 - y0, j) - 2
            for o in range(nout):
                oi = ob + o
                if oi % 2 != par:
                    continue
                while not done[j][oi % DONE].done(oi // DONE):
                    yield
                q = oi % ring
                if j == 0:
                    if q in rused:
                        while not rfree[q].done(rphase[q]):
                            yield
                        rphase[q] += 1
                    rused.add(q)
                ts = oi % slots
                assert acc[j].get(ts) == ["live", ci, o, 3], (j, ts, acc[j].get(ts), ci, o)
                acc[j][ts] = ["drained"]
                for _ in range(128):
                    drained[j][ts].arrive()
                yield
                if j == 0:
                    rmid[q] = (ci, o)
                    for _ in range(128):
                        full[q].arrive()
            ob += nout

    roles = [tensor_core(), issuer(0), issuer(1)] + [drain(j, p) for j in (0, 1) for p in (0, 1)]
    alive = [True] * len(roles)
    # uneven speeds: each role moves with a weight drawn per schedule, so that some roles run far
    # ahead of others (a drain group lagging by a whole slot ring, say)
    weights = [rnd.choice((1, 1, 4, 16)) for _ in roles]
    for _ in range(max_moves):
        if not any(alive[1:]):
            assert not any(tensor)
            return
        i = rnd.choices(range(len(roles)), weights)[0]
        if alive[i]:
            try:
                next(roles[i])
            except StopIteration:
                alive[i] = False
    raise AssertionError(f"no progress: H={H}, chunk {chunk}, {rounds} rounds, seed {seed}")


def test_constants_satisfy_the_ring_bounds():
    assert RING % 2 == 0 and SLOTS % 2 == 0 and DONE % 2 == 0   # one parity owns each slot / barrier
    assert SLOTS >= 3 and DONE >= SLOTS
    assert RING_IN > AHEAD
    assert 2 * 32 * SLOTS <= 512


@pytest.mark.parametrize("H,chunk", [(1, 1), (2, 1), (3, 2), (5, 5), (9, 4), (17, 17), (40, 13)])
@pytest.mark.parametrize("rounds", [1, 2])
def test_protocol_under_random_schedules(H, chunk, rounds):
    for seed in range(6):
        simulate(H, chunk, rounds, seed)


def pair_chunk(B, H, W, sm_count=152):
    """The launcher's chunk length (svgf_kpn.cu, pair_chunk): at most one chunk a block."""
    cols = B * ((W + 125) // 126)
    per = 1 if cols >= sm_count else sm_count // cols
    per = min(per, H)
    return (H + per - 1) // per


def test_chunk_choice_gives_each_block_at_most_one_chunk():
    for B, H, W in ((1, 1080, 1920), (1, 2160, 3840), (1, 120, 200), (3, 1, 1), (2, 40, 300)):
        chunk = pair_chunk(B, H, W)
        cols = B * ((W + 125) // 126)
        assert 1 <= chunk <= H and cols * ((H + chunk - 1) // chunk) <= max(152, cols)
    assert "constexpr int kPairSeg = 126;" in SRC.read_text()


def _mutated(old, new):
    src = inspect.getsource(simulate)
    assert src.count(old) == 1, old
    ns = dict(globals())
    exec(src.replace(old, new), ns)
    return ns["simulate"]


@pytest.mark.parametrize("old,new", [
    ("while not rfree[q].done(rphase[q]):", "while False:"),
    ("while not drained[j][ts].done(dphase[ts]):", "while False:"),
    ("while not rfree_in[s0].done(phase0[s0]):", "while False:"),
    ("                if oi % 2 != par:\n", "                if o % 2 != par:\n"),
    ("            ob += nout\n\n    def tensor_core", "            pass\n\n    def tensor_core"),
])
def test_model_catches_planted_protocol_mistakes(old, new):
    """Each planted mistake makes some schedule stall or trip a check (the fourth: the groups
    split rows by their parity within the chunk, so an odd-length chunk hands a row's slot to the
    other group)."""
    sim = _mutated(old, new)
    for seed in range(16):
        try:
            sim(9, 4, 3, seed, max_moves=2 * 10 ** 5)
        except AssertionError:
            return
    raise AssertionError("the planted mistake went unnoticed")
