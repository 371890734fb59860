"""Model check of the x-edge exchange between the two CTAs of a cluster that
share every row (n = 2048 at depth 8), on the CPU.

The fused kernel's protocol, restated as a small event simulation:
- A CTA runs global steps g = 0, 1, ...; step i of a segment sits at ring
  position K = i mod 12 (segments start at a multiple of 12).
- Each CTA has two end threads.  Thread 0 pushes its left-edge entry into the
  partner's edge buffer K & 1 at the offset its own store would use; the
  partner's thread NT-1 reads it at its next step from buffer (K & 1) ^ 1.
  Thread NT-1 pushes its right-edge entry to the partner's thread 0 the same
  way.  A push lands some time after it is issued and then completes 16 bytes
  per part on the receiver's mbarrier (g & 1, receiving end, part).
- At the start of step g (g > 0) a receiving end thread waits for the phase
  ((g-1) >> 1) & 1 of mbarrier ((g-1) & 1, its end, part) and re-arms it (one
  arrival with 16 expected bytes); its reads come after that wait, its pushes
  at the end of the step.  All threads of a CTA meet at one barrier per step.

With segments of an even number of steps (what the kernel uses), random
interleavings and landing delays never make a wait hang, never let an
mbarrier run two phases ahead of its waiter, and every read inside a segment
(i >= 1) sees the partner's entry of the previous step.  With odd segments,
consecutive steps across a segment boundary reuse one buffer, and a late
landing push can leave a stale entry: the model finds it.
"""
import random

KU = 12
PARTS = 2


class MBar:
    """Transaction mbarrier with an expected arrival count of 1."""

    def __init__(self):
        self.phase = 0        # completed phases
        self.pending = 1
        self.tx = 0

    def _check(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = 1

    def arm(self, nbytes=16):           # mbarrier.arrive.expect_tx
        self.tx += nbytes
        self.pending -= 1
        assert self.pending >= 0
        self._check()

    def complete(self, nbytes=16):      # complete_tx of a landed push
        self.tx -= nbytes
        self._check()

    def done(self, parity):             # try_wait.parity
        return self.phase % 2 != parity


class Violation(AssertionError):
    pass


def run(segments, seed):
    """Simulate both CTAs over the given segment lengths; raise Violation on
    a stale read, an overwrite before the read or a runaway phase."""
    rng = random.Random(seed)
    steps = [(i, i % KU, sg) for sg, n in enumerate(segments) for i in range(n)]
    G = len(steps)
    # per CTA: edge entries [buf][entry] -> (writer step, segment); entry e is
    # read by end thread e (0: thread 0, 1: thread NT-1)
    xbuf = [[[None, None] for _ in range(2)] for _ in range(2)]
    bars = [[[[MBar() for _ in range(PARTS)] for _ in range(2)] for _ in range(2)] for _ in range(2)]
    for c in range(2):
        for b in range(2):
            for e in range(2):
                for q in range(PARTS):
                    bars[c][b][e][q].arm()      # armed for the partner's steps 0 and 1
    read_done = set()
    in_flight = []       # (land time, cta, buf, entry, writer step, segment, barrier b)
    state = [{"g": 0, "phase": "wait", "ends": [False, False]} for _ in range(2)]
    now = 0
    while any(s["g"] < G for s in state) or in_flight:
        now += 1
        if now > 400 * G + 10_000:
            raise Violation("no progress: a wait never ends")
        rng.shuffle(in_flight)
        keep = []
        for ev in in_flight:
            if ev[0] <= now and rng.random() < 0.7:
                _, c, buf, entry, wstep, seg, b = ev
                old = xbuf[c][buf][entry]
                if old is not None:
                    ow = old[0]
                    if ow + 1 < G and steps[ow + 1][0] >= 1 and (c, buf, entry, ow) not in read_done:
                        raise Violation(f"entry of step {ow} overwritten before its read")
                xbuf[c][buf][entry] = (wstep, seg)
                for q in range(PARTS):
                    bars[c][b][entry][q].complete()
            else:
                keep.append(ev)
        in_flight = keep
        for c in rng.sample(range(2), 2):
            st = state[c]
            g = st["g"]
            if g >= G:
                continue
            i, K, seg = steps[g]
            if st["phase"] == "wait":
                for e in range(2):
                    if st["ends"][e]:
                        continue
                    if g > 0:
                        mb = [bars[c][(g - 1) & 1][e][q] for q in range(PARTS)]
                        if any(m.phase > (g - 1) // 2 + 1 for m in mb):
                            raise Violation("an mbarrier ran two phases ahead of its waiter")
                        if not all(m.done(((g - 1) >> 1) & 1) for m in mb):
                            continue
                        for m in mb:
                            m.arm()
                    buf = (K & 1) ^ 1
                    if i >= 1:
                        if xbuf[c][buf][e] != (g - 1, seg):
                            raise Violation(f"step {g} read {xbuf[c][buf][e]}, not step {g - 1}")
                        read_done.add((c, buf, e, g - 1))
                    st["ends"][e] = True
                if all(st["ends"]):
                    st["phase"] = "push"
            elif st["phase"] == "push":
                # thread 0 fills the partner's entry 1, thread NT-1 its entry 0
                for entry in (1, 0):
                    in_flight.append((now + rng.randint(1, 30), c ^ 1, K & 1, entry, g, seg, g & 1))
                st["phase"] = "barrier"
            else:   # the CTA barrier closes the step
                st.update(g=g + 1, phase="wait", ends=[False, False])
    return G


def test_exchange_protocol_model_even_segments():
    for seed in range(300):
        rng = random.Random(seed)
        segments = [2 * rng.randint(9, 40) for _ in range(rng.randint(1, 4))]
        assert run(segments, seed) == sum(segments)


def test_model_catches_odd_segments():
    failures = 0
    for seed in range(300):
        rng = random.Random(10_000 + seed)
        segments = [2 * rng.randint(9, 20) + 1 for _ in range(3)]
        try:
            run(segments, 10_000 + seed)
        except Violation:
            failures += 1
    assert failures > 0
