"""Model check of the fused 2D kernel's static shared-memory rings, on the CPU.

The kernel's schedule, restated:
- A CTA walks segments of H rows with an L-row halo on both sides:
  nload = H + 2L rows are loaded, niter = H + L + B steps run (B levels per
  pass; for cluster rows niter is rounded up to even).  A segment starts at
  ring position pos, a multiple of 12, and the next one at the multiple of
  12 that follows pos + niter.
- Row rho of the segment goes to deep slot (pos + rho) mod 12 (kappa, D0)
  and shallow slot (pos + rho) mod 6 (u_hi, u_t, residual).  Rows 0 and 1
  are requested before step 0, row i + 2 at step i.
- Each deep slot has one mbarrier (one arrival per phase plus the copy's
  bytes).  Positions that receive no copy (drain and padding) get a plain
  arrival when the segment ends, so slot s completes phase j at position
  12 j + s, and step i waits on its row's slot with the parity of the ring
  lap, ((pos + i) / 12) mod 2.
- Level l at step i advances row i - 1 - l: row r's deep slot is read at
  steps r .. r + B (its kappa at step r, its D0 written at r + 1, both read
  by the levels up to step r + B), its shallow slot at steps r and r + 1.
  One CTA barrier separates steps.

Checked for random segment mixes and depths 4, 8 and 9: every wait finds
its row's copy complete in exactly the phase it expects (never an older or
a newer one), and no slot is refilled while a step that still reads it has
not finished.
"""
import random

from tests._shipped import header_constant

# the ring sizes and the prefetch distance of the shipped kernel
KU, KRS, KPRE = (header_constant("tb2d_kernels.cuh", k) for k in ("kU", "kRS", "kPre"))


def run(segments, B, even=False):
    """segments: list of (H, L).  Raises AssertionError on a schedule error."""
    phase = [0] * KU           # completed phases per deep slot
    pending = [None] * KU      # position whose copy is in flight in each slot
    deep_owner = [None] * KU   # (position, last step that reads it)
    shal_owner = [None] * KRS
    pos = 0
    step_clock = 0             # global step counter (the barrier order)

    def issue(q, at):
        """Request row position q at the start of the step with clock `at`
        (after the barrier that closed every step with a smaller clock)."""
        s = q % KU
        # the slot's previous row must be finished with: its last reader ran
        # at an earlier step
        if deep_owner[s] is not None:
            assert deep_owner[s][1] < at, ("deep slot refilled early", q, deep_owner[s])
        if shal_owner[q % KRS] is not None:
            assert shal_owner[q % KRS][1] < at, ("shallow slot refilled early", q)
        assert pending[s] is None
        pending[s] = q

    def land(q):                       # the copy's bytes and arrival complete the phase
        s = q % KU
        assert pending[s] == q
        pending[s] = None
        assert phase[s] == q // KU, ("phase out of step", q, phase[s])
        phase[s] += 1

    for H, L in segments:
        assert pos % KU == 0
        nload = H + 2 * L
        niter = H + L + B
        if even:
            niter += niter & 1
        for rho in range(min(KPRE, nload)):     # before step 0, after the last barrier
            issue(pos + rho, step_clock + 1)
            land(pos + rho)
        seg_end = step_clock + niter       # reads stop with the segment's last step
        for i in range(niter):
            step_clock += 1
            q = pos + i
            if i + KPRE < nload:
                issue(q + KPRE, step_clock)
                land(q + KPRE)
            if i < nload:
                s = q % KU
                par = (q // KU) & 1
                # try_wait.parity(par): the phase of parity par has completed,
                # and it is this lap's (not the next lap's) phase
                assert phase[s] % 2 != par, ("wait would block forever", q)
                assert phase[s] == q // KU + 1, ("wait sees another lap", q, phase[s])
                deep_owner[s] = (q, min(step_clock + B, seg_end))          # read up to step r + B
                shal_owner[q % KRS] = (q, min(step_clock + 1, seg_end))    # read at steps r, r + 1
        nxt = -(-(pos + niter) // KU) * KU
        for q in range(pos + nload, nxt):                    # plain arrivals
            s = q % KU
            assert pending[s] is None
            assert phase[s] == q // KU, ("padding phase out of step", q)
            phase[s] += 1
        pos = nxt
    return pos


def test_ring_schedule_whole_rows():
    rng = random.Random(1905)
    for B in (4, 8, 9):
        for _ in range(400):
            segs = []
            for _ in range(rng.randint(1, 5)):
                L = B if rng.random() < 0.7 else rng.randint(1, B)
                segs.append((rng.randint(1, 300), L))
            run(segs, B)
            run(segs, B, even=True)


def test_ring_schedule_edge_cases():
    for B in (4, 8, 9):
        run([(1, B)], B)                   # one output row
        run([(1, 1)] * 7, B)               # many tiny segments back to back
        run([(1024, B), (1, B), (1024, B)], B)


def test_model_catches_a_short_ring():
    """With a 10-row deep ring instead of 12, depth 9 would refill a slot
    that a level still reads: the model must say so."""
    global KU
    saved = KU
    try:
        KU = 10
        failed = False
        try:
            run([(200, 9)], 9)
        except AssertionError:
            failed = True
        assert failed
    finally:
        KU = saved
