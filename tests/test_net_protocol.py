"""The barrier protocol of the four-layer tensor-core kernel (k_kpn_net), modelled on the host.

The roles meet at mbarriers: one warp a layer issuing its MMAs input row by input row (layer
0's warp also stages the feature rows into ring 0, a fixed number of rows ahead), the tensor
core completing each warp's MMAs in that warp's issue order (a commit arrives once all of that
warp's earlier MMAs have completed; the warps' streams interleave arbitrarily), and one
epilogue group a layer draining its output rows in order into the next layer's ring.  The model takes the ring, slot, barrier and look-ahead
sizes from the kernel source and runs random interleavings of the roles, checking that:
  - every schedule finishes (no role waits forever);
  - every parity wait finds its barrier at the awaited phase or the one after it;
  - an MMA reads the row it expects from a ring slot, from issue until it completes (the slot
    is neither restaged nor rewritten by the epilogue before then);
  - an accumulator slot is first written only after its previous output row was drained, and
    the epilogue drains the output row it expects, with all three input rows accumulated.
Heights from one row to several chunks, and blocks walking several chunks, are covered."""
import pathlib
import random
import re

import pytest

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2312_06827_gb300" / "csrc" / "svgf_kpn.cu"


def constant(name):
    m = re.search(rf"constexpr\s+\w+\s+{name}\s*=\s*(\d+)\s*[;,]", SRC.read_text())
    if not m:
        m = re.search(rf"\b{name}\s*=\s*(\d+)\s*[;,]", SRC.read_text())
    assert m, name
    return int(m.group(1))


RING0, AHEAD = constant("kNetRing0"), constant("kNetAhead")
RING, SLOTS, DONE = constant("kNetRing"), constant("kNetSlots"), constant("kNetDone")


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
    rfree0 = [Barrier() for _ in range(RING0)]
    full = [[Barrier(128) for _ in range(ring)] for _ in range(3)]
    rfree = [[Barrier() for _ in range(ring)] for _ in range(3)]
    done = [[Barrier() for _ in range(DONE)] for _ in range(4)]
    drained = [[Barrier(128) for _ in range(slots)] for _ in range(4)]
    ring0 = {}                                   # slot -> (state, chunk, layer-0 input row)
    rings = [{} for _ in range(3)]               # ring of layer l + 1: slot -> (chunk, row index)
    acc = [{} for _ in range(4)]                 # layer -> slot -> [chunk, output row, contributions]
    tensor = [[] for _ in range(4)]              # per issuing thread: issued, not yet completed

    def nin(rows, l):
        return rows + 8 - 2 * l

    feature_rows = [(ci, k) for ci, (y0, y1) in enumerate(chunks) for k in range(nin(y1 - y0, 0))]

    def issuer(l):
        """Warp 16 + l: layer l's input rows in order; warp 16 stages the feature rows too."""
        nb, ob, dused = 0, 0, set()
        fphase, dphase = [0] * ring, [0] * slots
        staged, used0, phase0 = 0, set(), [0] * RING0
        for ci, (y0, y1) in enumerate(chunks):
            rows = y1 - y0
            n_in = nin(rows, l)
            nout = n_in - 2
            for k in range(n_in):
                if l == 0:
                    sl = nb % RING0
                    while staged < nb + 1 + ahead and staged < len(feature_rows):
                        s0 = staged % RING0
                        if s0 in used0:                       # the slot's previous row's MMAs
                            while not rfree0[s0].done(phase0[s0]):
                                yield
                            phase0[s0] += 1
                        used0.add(s0)
                        ring0[s0] = ("in flight",) + feature_rows[staged]
                        staged += 1
                        yield
                    ring0[sl] = ("landed",) + ring0[sl][1:]   # its copies waited for
                else:
                    sl = nb % ring
                    while not full[l - 1][sl].done(fphase[sl]):
                        yield
                    fphase[sl] += 1
                if l == 0:
                    assert ring0[sl] == ("landed", ci, k), (ring0[sl], ci, k)
                else:
                    assert rings[l - 1].get(sl) == (ci, k), (l, sl, rings[l - 1].get(sl), ci, k)
                if k < nout:                                      # output k starts here
                    ts = (ob + k) % slots
                    if ts in dused:
                        while not drained[l][ts].done(dphase[ts]):
                            yield
                        dphase[ts] += 1
                    dused.add(ts)
                    assert acc[l].get(ts, ["drained"])[0] == "drained", (l, ts, acc[l].get(ts))
                    acc[l][ts] = ["live", ci, k, 0]
                lo, hi = max(k - 2, 0), min(k, nout - 1)
                outs = []
                for o in range(lo, hi + 1):
                    ts = (ob + o) % slots
                    assert acc[l][ts][:3] == ["live", ci, o], (l, ts, acc[l][ts], ci, o)
                    outs.append(ts)
                yield                                             # the MMAs are issued
                commits = []
                if k >= 2:
                    commits.append(("done", l, (ob + k - 2) % DONE))
                commits.append(("rfree", l, sl))
                tensor[l].append((l, sl, ci, k, outs, commits))
                nb += 1
            ob += nout

    def tensor_core():
        """Each issuing thread's MMAs complete in its issue order (a commit arrives once all of
        that thread's earlier MMAs have); the threads' streams interleave arbitrarily."""
        while True:
            busy = [q for q in tensor if q]
            if not busy:
                yield
                continue
            q = rnd.choice(busy)
            l, sl, ci, k, outs, commits = q[0]
            # the operands are still the row the MMAs were issued for
            if l == 0:
                assert ring0[sl] == ("landed", ci, k), ("restaged under the MMAs", ring0[sl], ci, k)
            else:
                assert rings[l - 1].get(sl) == (ci, k), ("rewritten under the MMAs", l, sl)
            for ts in outs:
                acc[l][ts][3] += 1
            q.pop(0)
            for kind, ll, idx in commits:
                (done[ll][idx] if kind == "done" else (rfree0[idx] if ll == 0 else rfree[ll - 1][idx])).arrive()
            yield

    eob = [0] * 4
    rphase, rused = [[0] * ring for _ in range(3)], [set() for _ in range(3)]

    def item(l, ci, o):
        """Output row o of layer l (chunk ci): wait for its MMAs and the next ring slot, drain."""
        oi = eob[l] + o
        while not done[l][oi % DONE].done(oi // DONE):
            yield
        q = oi % ring
        if l < 3:
            if q in rused[l]:
                while not rfree[l][q].done(rphase[l][q]):
                    yield
                rphase[l][q] += 1
            rused[l].add(q)
        ts = oi % slots
        assert acc[l].get(ts) == ["live", ci, o, 3], (l, ts, acc[l].get(ts), ci, o)
        acc[l][ts] = ["drained"]
        for _ in range(128):
            drained[l][ts].arrive()
        yield
        if l < 3:
            rings[l][q] = (ci, o)
            for _ in range(128):
                full[l][q].arrive()

    def epilogue_group(l):
        """Warps 4l .. 4l + 3: layer l's output rows in order."""
        for ci, (y0, y1) in enumerate(chunks):
            nout = nin(y1 - y0, l) - 2
            for o in range(nout):
                yield from item(l, ci, o)
            eob[l] += nout

    roles = [tensor_core()] + [issuer(l) for l in range(4)] + [epilogue_group(l) for l in range(4)]
    alive = [True] * len(roles)
    for _ in range(max_moves):
        if not any(alive[1:]):
            assert not any(tensor)
            return
        i = rnd.randrange(len(roles))
        if alive[i]:
            try:
                next(roles[i])
            except StopIteration:
                alive[i] = False
    raise AssertionError(f"no progress: H={H}, chunk {chunk}, {rounds} rounds, seed {seed}")


def test_constants_satisfy_the_schedule_bounds():
    assert RING >= 2
    assert SLOTS >= 3 and DONE >= SLOTS      # a triple of output rows fits the slot ring
    assert RING0 > AHEAD
    assert 4 * 32 * SLOTS <= 512             # the tensor memory of one SM


@pytest.mark.parametrize("H,chunk", [(1, 1), (2, 1), (3, 2), (5, 5), (9, 4), (17, 17), (40, 13)])
@pytest.mark.parametrize("rounds", [1, 2])
def test_protocol_under_random_schedules(H, chunk, rounds):
    for seed in range(6):
        simulate(H, chunk, rounds, seed)


def net_chunk(B, H, W, sm_count=152):
    """The launcher's chunk length (svgf_kpn.cu, net_chunk): at most one chunk a block."""
    cols = B * ((W + 121) // 122)
    per = 1 if cols >= sm_count else sm_count // cols
    per = min(per, H)
    return (H + per - 1) // per


def test_chunk_choice_gives_each_block_at_most_one_chunk():
    for B, H, W in ((1, 1080, 1920), (1, 2160, 3840), (1, 120, 200), (3, 1, 1), (2, 40, 300), (1, 7, 5000)):
        chunk = net_chunk(B, H, W)
        assert 1 <= chunk <= H
        cols = B * ((W + 121) // 122)
        assert cols * ((H + chunk - 1) // chunk) <= max(152, cols)
    assert net_chunk(1, 1080, 1920) == 120
    src = SRC.read_text()
    assert "long per = cols >= sm_count ? 1 : sm_count / cols;" in src and "constexpr int kNetSeg = 122;" in src


def _mutated(old, new):
    import inspect
    src = inspect.getsource(simulate)
    assert src.count(old) == 1, old
    ns = dict(globals())
    exec(src.replace(old, new), ns)
    return ns["simulate"]


@pytest.mark.parametrize("old,new", [
    # the epilogue writes the next layer's ring slot before the MMAs of its previous row completed
    ("while not rfree[l][q].done(rphase[l][q]):", "while False:"),
    # the epilogue numbers the next layer's ring rows per chunk, the issuer across chunks
    ("        q = oi % ring\n", "        q = o % ring\n"),
    # the issuer starts an output row without waiting for the slot's previous row to be drained
    ("while not drained[l][ts].done(dphase[ts]):", "while False:"),
    # layer 0's warp restages a feature row before the MMAs of the slot's previous row completed
    ("while not rfree0[s0].done(phase0[s0]):", "while False:"),
    # an issuer counts its output rows per chunk instead of running on
    ("            ob += nout\n\n    def tensor_core", "            pass\n\n    def tensor_core"),
    # an epilogue group counts its output rows per chunk
    ("            eob[l] += nout\n", "            pass\n"),
    # layer 0's warp stages as far ahead as its ring holds (a slot restaged under its MMAs' wait)
    ("while staged < nb + 1 + ahead and", "while staged < nb + 1 + RING0 and"),
])
def test_model_catches_planted_protocol_mistakes(old, new):
    """The model is not vacuous: each planted mistake makes some schedule stall or trip a check."""
    sim = _mutated(old, new)
    for seed in range(16):
        try:
            sim(9, 4, 3, seed, max_moves=2 * 10 ** 5)
        except AssertionError:
            return
    raise AssertionError("the planted mistake went unnoticed")


def test_smaller_rings_and_less_look_ahead_are_still_safe():
    """One-slot rings and no look-ahead only serialise the roles; the waits keep them correct."""
    for kw in ({"ahead": 0}, {"ring": 1}, {"ahead": 1, "ring": 2}):
        for seed in range(4):
            simulate(9, 4, 2, seed, **kw)
