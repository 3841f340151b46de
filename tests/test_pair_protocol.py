"""Host model of the synchronisation of the fused step (no GPU).

The single-CTA kernel (M = 64, 128, 256) and, above all, the 512-bead one:
at M = 512 a tile runs on a cluster of two CTAs.  Each CTA keeps half of the
bonds and modes in TMEM, runs all 48 K blocks of a step, writes the A operand
of the blocks it owns and bulk-copies it into the same stage of the other CTA.
This test runs both CTAs' roles (TMA producer, MMA issuer and the copies its
polling loop sends, compute warps, noise warps with their epilogue share) as
coroutines under random interleavings, with asynchronous TMA loads, copies
and in-order MMA commits, and checks on every run:
  * no deadlock;
  * every mbarrier parity wait targets the barrier's current phase or the one
    before it (a wait two phases ahead would pass on the wrong phase);
  * no region of a stage (R staging, A, B) is overwritten while its content
    still has a consumer (split, MMA, outbound copy, epilogue);
  * every MMA reads the A and B operands of its own block;
  * when both CTAs pass the final cluster barrier, no copy or commit is still
    in flight towards either of them.
A negative control replaces the compute warps' release-counter waits by plain
parity waits and must be caught.  In the single-CTA kernel the producer moves
each stage's part of the epilogue's R tile in as soon as the last MMA of the
step that reads that stage has retired.  The block order is the kernel's
(inverse / noise blocks interleaved, then force / noise pairs; FILL noise
blocks moved to the end of phase 1), modelled here at block granularity."""
import random

import pytest

def decode(fill, blk, KB=16):
    """(kind, index) of block blk of a step of KB K blocks per contraction:
    kind 0 inverse, 1 noise, 2 force."""
    h = KB // 2
    p = min(fill, h)
    if blk < 3 * h:
        m, r = divmod(blk, 3)
        return (1 if r == 1 else 0), (2 * m if r == 0 else m if r == 1 else 2 * m + 1)
    if blk < 3 * h + p:
        return 1, h + (blk - 3 * h)
    b = blk - 3 * h - p
    if b < 2 * (h - p):
        return (1, h + p + (b >> 1)) if b & 1 else (2, b >> 1)
    return 2, b - (h - p)


class ProtocolError(Exception):
    pass


class Barrier:
    def __init__(self, name, count):
        self.name, self.count, self.pending, self.tx, self.phase = name, count, count, 0, 0

    def _complete(self):
        if self.pending < 0:
            raise ProtocolError(f"{self.name}: more arrivals than the phase expects")
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self, n=1, tx=0):
        self.tx += tx
        self.pending -= n
        self._complete()

    def complete_tx(self, n):
        self.tx -= n                      # may go negative before the expect_tx
        if self.pending == 0:
            self._complete()


class Pair:
    """pair: two CTAs at M = 512 (KB = 16), else one CTA with KB K blocks;
    epi_stages: the stages the epilogue's R tile covers."""

    def __init__(self, fill, stages, steps, seed, counter_waits=True, tf32=False, pair=True, KB=16,
                 epi_stages=2):
        self.fill, self.st, self.steps = fill, stages, steps
        self.rng = random.Random(seed)
        # how eagerly asynchronous work (TMA loads, copies, MMA retirement) runs:
        # uniform among all options, or only now and then, so that it lags
        self.lag = (None, 0.2, 0.03)[seed % 3]
        self.counter_waits, self.tf32 = counter_waits, tf32
        self.pair, self.KB, self.epi_stages = pair, KB, epi_stages
        self.NBLK = 3 * KB
        self.KBL = KB // 2 if pair else KB
        self.ncta = 2 if pair else 1
        self.bar = []
        for r in range(self.ncta):
            d = {}
            for s in range(stages):
                d["full", s] = Barrier(f"{r}.full{s}", 1)
                d["ready", s] = Barrier(f"{r}.ready{s}", 1)
                d["empty", s] = Barrier(f"{r}.empty{s}", self.ncta)   # every CTA's MMAs
            for k, c in (("u_done", 1), ("inc_done", 1), ("epi_done", 2), ("r_blk", 1), ("both_done", 2),
                         ("peer_epi", 1)):
                d[k] = Barrier(f"{r}.{k}", c)
            self.bar.append(d)
        self.freed = [-1, -1]             # the producers' release counters
        self.region = {}                  # (cta, stage, region) -> [tag, consumers]
        self.events = []                  # asynchronous work: (target cta, action, label)
        self.pipe = [[] for _ in range(self.ncta)]   # MMAs and commits of each CTA, in order
        self.left = False

    # -- stage regions
    def put(self, r, s, reg, tag, consumers):
        cur = self.region.get((r, s, reg))
        if cur and cur[1]:
            raise ProtocolError(f"CTA {r} stage {s} {reg}: {tag} over {cur[0]} still used by {cur[1]}")
        self.region[r, s, reg] = [tag, set(consumers)]

    def take(self, r, s, reg, who, tag):
        cur = self.region.get((r, s, reg))
        if not cur or cur[0] != tag or who not in cur[1]:
            raise ProtocolError(f"CTA {r} stage {s} {reg}: {who} wants {tag}, finds {cur}")
        cur[1].discard(who)

    def holds(self, r, s, reg, tag):
        cur = self.region.get((r, s, reg))
        if not cur or cur[0] != tag:
            raise ProtocolError(f"CTA {r} stage {s} {reg}: MMA wants {tag}, finds {cur}")

    # -- waits: predicates polled by the scheduler
    def parity(self, r, key, x):
        bar = self.bar[r][key]

        def done():
            if bar.phase < x and (bar.phase & 1) != (x & 1):
                raise ProtocolError(f"{bar.name} at phase {bar.phase}: a wait for phase {x} would pass")
            if bar.phase > x + 1:
                raise ProtocolError(f"{bar.name} at phase {bar.phase}: a wait for phase {x} would hang")
            return bar.phase > x
        return done

    def counter(self, r, b):
        return lambda: self.freed[r] >= b

    def block(self, kind, idx):
        return next(x for x in range(self.NBLK) if self.dec(x) == (kind, idx))

    def dec(self, blk):
        return decode(self.fill, blk, self.KB)

    def own(self, idx, r):
        return (idx & 1) == r if self.pair else True

    def owned(self, r):
        """indices of the blocks of each kind that CTA r writes, in order"""
        return [2 * i + r for i in range(self.KBL)] if self.pair else list(range(self.KBL))

    # -- roles
    def producer(self, r):
        bar, st, nblk = self.bar[r], self.st, self.NBLK
        for sp in range(self.steps):
            if sp > 0:
                yield self.parity(r, "epi_done", sp - 1)
                if self.pair:
                    self.bar[r ^ 1]["peer_epi"].arrive()
                    yield self.parity(r, "peer_epi", sp - 1)
            for blk in range(nblk):
                b, s = sp * nblk + blk, (sp * nblk + blk) % st
                if b >= st:
                    yield self.parity(r, ("empty", s), b // st - 1)
                self.freed[r] = b
                kind, idx = self.dec(blk)
                own = self.own(idx, r)
                loads_r = kind == 0 and own
                bar["full", s].arrive(1, tx=1 + loads_r + (not own))
                self.events.append((r, self.load_b(r, s, b), "B load"))
                if loads_r:
                    self.events.append((r, self.load_r(r, s, b), "R load"))
                if not own:
                    bar["ready", s].arrive()
                yield None
            if self.pair:
                yield self.parity(r, "inc_done", sp)
                yield self.parity(r, "both_done", sp)
                for s in range(self.epi_stages):    # the epilogue's R tile fills the first stages
                    for reg in ("R", "A", "B"):
                        self.put(r, s, reg, ("epilogue", sp), {"compute", "noise"})
            else:
                # single CTA: each of the first stages takes its part of the R tile
                # as soon as the last MMA of this step that reads it has retired
                for s in range(self.epi_stages):
                    last = max(b for b in range(sp * nblk, (sp + 1) * nblk) if b % st == s)
                    yield self.parity(r, ("empty", s), last // st)
                    for reg in ("R", "A", "B"):
                        self.put(r, s, reg, ("epilogue", sp), {"compute", "noise"})
            self.events.append((r, lambda r=r: self.bar[r]["r_blk"].arrive(), "R reload"))
        if self.pair:
            total = self.steps * nblk
            for s in range(min(st, total)):
                last = s + st * ((total - 1 - s) // st)
                yield self.parity(r, ("empty", s), last // st)

    def load_b(self, r, s, b):
        def act():
            self.put(r, s, "B", b, {"mma"})
            self.bar[r]["full", s].complete_tx(1)
        return act

    def load_r(self, r, s, b):
        def act():
            self.put(r, s, "A" if self.tf32 else "R", b, {"split"})
            self.bar[r]["full", s].complete_tx(1)
        return act

    def copy(self, r, s, b):
        def act():
            self.take(r, s, "A", "copy", b)
            self.put(r ^ 1, s, "A", b, {"mma"})
            self.bar[r ^ 1]["full", s].complete_tx(1)
        return act

    def mma(self, r):
        st, nblk = self.st, self.NBLK
        for sp in range(self.steps):
            for blk in range(nblk):
                b, s = sp * nblk + blk, (sp * nblk + blk) % st
                kind, idx = self.dec(blk)
                yield self.parity(r, ("full", s), b // st)
                yield self.parity(r, ("ready", s), b // st)
                self.holds(r, s, "A", b)
                self.holds(r, s, "B", b)
                self.pipe[r] += [("mma", s, b), ("commit all", ("empty", s))]
                if kind == 0 and idx == self.KB - 1:
                    self.pipe[r].append(("commit", "u_done"))
                yield None
            self.pipe[r].append(("commit", "inc_done"))
            if self.pair:
                self.pipe[r].append(("commit all", "both_done"))

    def sender(self, r):
        """The copies of the MMA thread's polling loop: each block this CTA owns,
        in order, once the release counter has reached it and its writers are done."""
        st, nblk = self.st, self.NBLK
        for sp in range(self.steps):
            for blk in range(nblk):
                kind, idx = self.dec(blk)
                if not self.own(idx, r):
                    continue
                b, s = sp * nblk + blk, (sp * nblk + blk) % st
                yield self.counter(r, b)
                yield self.parity(r, ("ready", s), b // st)
                self.take(r, s, "A", "to copy", b)
                self.region[r, s, "A"][1].add("copy")
                self.events.append((r ^ 1, self.copy(r, s, b), "copy"))
                yield None

    def retire(self, r):
        item = self.pipe[r].pop(0)
        if item[0] == "mma":
            self.take(r, item[1], "A", "mma", item[2])
            self.take(r, item[1], "B", "mma", item[2])
        elif item[0] == "commit":
            self.bar[r][item[1]].arrive()
        else:
            for t in range(self.ncta):
                self.bar[t][item[1]].arrive()

    def write_block(self, r, kind, idx, sp):
        b = sp * self.NBLK + self.block(kind, idx)
        s = b % self.st
        if self.counter_waits or kind == 1:
            yield self.counter(r, b)
        if kind == 0:
            yield self.parity(r, ("full", s), b // self.st)
            self.take(r, s, "A" if self.tf32 else "R", "split", b)
        elif kind == 2 and not self.counter_waits:
            yield self.parity(r, ("empty", s), b // self.st - 1)
        self.put(r, s, "A", b, {"mma", "to copy"} if self.pair else {"mma"})
        self.bar[r]["ready", s].arrive()
        yield None

    def epilogue(self, r, sp, who):
        yield self.parity(r, "inc_done", sp)
        yield self.parity(r, "r_blk", sp)
        for s in range(self.epi_stages):
            for reg in ("R", "A", "B"):
                self.take(r, s, reg, who, ("epilogue", sp))
        self.bar[r]["epi_done"].arrive()
        yield None

    def compute(self, r):
        for sp in range(self.steps):
            for idx in self.owned(r):
                yield from self.write_block(r, 0, idx, sp)
            yield self.parity(r, "u_done", sp)
            for idx in self.owned(r):
                yield from self.write_block(r, 2, idx, sp)
            yield from self.epilogue(r, sp, "compute")

    def noise(self, r):
        for sp in range(self.steps):
            for idx in self.owned(r):
                yield from self.write_block(r, 1, idx, sp)
            yield from self.epilogue(r, sp, "noise")

    def run(self):
        roles = []
        for r in range(self.ncta):
            gens = [self.producer(r), self.mma(r), self.compute(r), self.noise(r)]
            if self.pair:
                gens.append(self.sender(r))
            roles += [[r, g, None, False] for g in gens]
        while True:
            options = [("role", i) for i, (r, g, ready, done) in enumerate(roles)
                       if not done and (ready is None or ready())]
            later = [("event", i) for i in range(len(self.events))]
            later += [("pipe", r) for r in range(self.ncta) if self.pipe[r]]
            if self.lag is None or not options or (later and self.rng.random() < self.lag):
                options += later
            if not options:
                if not all(x[3] for x in roles):
                    raise ProtocolError("deadlock")
                return
            kind, i = self.rng.choice(options)
            if kind == "role":
                try:
                    roles[i][2] = next(roles[i][1])
                except StopIteration:
                    roles[i][3] = True
            elif kind == "event":
                if self.left:
                    raise ProtocolError(f"{self.events[i][2]} after the CTAs left")
                self.events.pop(i)[1]()
            else:
                if self.left:
                    raise ProtocolError("a commit after the CTAs left")
                self.retire(i)
            if all(x[3] for x in roles) and not self.left:
                if self.events or any(self.pipe):
                    raise ProtocolError("the CTAs leave with copies or commits in flight")
                self.left = True


# The 512-bead kernel: BF16 four stages of 48 KB (the epilogue's R tile, 8 x 16
# KB, covers three), four noise blocks in phase 1's tail; TF32 two stages of
# 96 KB (the tile covers both) and one.  Also BF16 with none, the first design.
CONFIGS = [pytest.param(4, 4, False, 3, id="bf16"), pytest.param(1, 2, True, 2, id="tf32"),
           pytest.param(0, 4, False, 3, id="bf16-fill0")]


@pytest.mark.parametrize("fill,stages,tf32,epi", CONFIGS)
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_pair_protocol_under_random_interleavings(fill, stages, tf32, epi, steps):
    for seed in range(40):
        Pair(fill, stages, steps, seed, tf32=tf32, epi_stages=epi).run()


@pytest.mark.parametrize("fill,stages,tf32,epi", CONFIGS)
def test_plain_parity_waits_are_caught(fill, stages, tf32, epi):
    """Negative control: with parity waits where the stage's previous uses
    belong to the other CTA's blocks, a wait can run two phases ahead."""
    caught = 0
    for seed in range(10):
        try:
            Pair(fill, stages, 1, seed, counter_waits=False, tf32=tf32, epi_stages=epi).run()
        except ProtocolError:
            caught += 1
    assert caught == 10


# The single-CTA kernel: (K blocks, BF16 stages / TF32 stages, R-tile stages).
SINGLE = [pytest.param(8, 0, 4, False, 3, id="256bp-bf16"), pytest.param(8, 1, 2, True, 2, id="256bp-tf32"),
          pytest.param(4, 0, 4, False, 2, id="128bp-bf16"), pytest.param(4, 1, 3, True, 2, id="128bp-tf32"),
          pytest.param(2, 0, 4, False, 2, id="64bp-bf16"), pytest.param(2, 1, 4, True, 1, id="64bp-tf32")]


@pytest.mark.parametrize("KB,fill,stages,tf32,epi", SINGLE)
@pytest.mark.parametrize("steps", [1, 3])
def test_single_cta_protocol_under_random_interleavings(KB, fill, stages, tf32, epi, steps):
    for seed in range(30):
        Pair(fill, stages, steps, seed, tf32=tf32, pair=False, KB=KB, epi_stages=epi).run()
