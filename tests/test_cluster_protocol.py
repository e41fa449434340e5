"""A host-side model of the synchronisation of the clustered tensor-core pass 2.

Each CTA of a cluster of G runs three roles: a producer that reserves slots of a
7-deep shared-memory ring (TMA tiles, and slots into which the other CTAs send their
weight tiles), an MMA issuer that consumes the ring in the same order, and an epilogue
that turns the logits of its own observation block into a weight tile and sends it to
the slots the other CTAs reserved for it (announced through an 8-row mailbox).  The
model runs the roles as coroutines under random schedules, with the kernel's slot
order, and reports a deadlock when no role can move.  It checks the order the kernel
uses, and that the model does catch the order that deadlocks (all weight slots of a
round reserved before any Y'^T tile)."""
import random

import pytest

SLOTS, MBOX = 7, 8


class MailboxRace(Exception):
    """An epilogue read a mailbox row whose entries belong to different rounds."""


def run(G, units, order, seed=0, nk=16, cvalid=None, mbox=MBOX):
    """units: observation blocks per work unit (every CTA of the cluster walks the same
    units).  order: 'lookahead' (the kernel's) or 'weights_first'.  Returns True when
    every role finishes, False on a deadlock."""
    rnd = random.Random(seed)
    st = [dict(free=[0] * SLOTS, full=[0] * SLOTS, sfull=[0, 0], sempty=[0, 0], zfull=0,
               zempty=0, mfull=[0] * mbox, mbox=[[None] * G for _ in range(mbox)],
               rounds=[[None] * G for _ in range(mbox)])
          for _ in range(G)]
    valid = cvalid or [True] * G

    def producer(r):
        it = 0
        sent = [0] * G

        def reserve():
            nonlocal it
            s, need = it % SLOTS, it // SLOTS
            yield lambda: st[r]["free"][s] >= need
            it += 1
            return s

        def reserve_w(kq):  # a slot for CTA kq's weight tile, announced in its mailbox
            s = yield from reserve()
            row = sent[kq] % mbox
            st[kq]["mbox"][row][r] = s
            st[kq]["rounds"][row][r] = sent[kq]  # which use of the row this entry is for
            st[kq]["mfull"][row] += 1
            sent[kq] += 1

        def tile():  # a TMA tile: it lands at once
            s = yield from reserve()
            st[r]["full"][s] += 1

        for nb in units:
            rounds = -(-nb // G)
            for j in range(rounds + 1):
                nq = min(G, nb - j * G) if j < rounds else 0
                if r < nq:
                    for _ in range(2 * nk):  # logits: (A hi+lo, Y hi+lo) per k-block
                        yield from tile()
                nqp = min(G, nb - (j - 1) * G) if j >= 1 else 0
                if order == "lookahead":
                    if nqp:
                        yield from reserve_w(0)
                    for kq in range(nqp):
                        if kq + 1 < nqp:
                            yield from reserve_w(kq + 1)
                        if valid[r]:
                            yield from tile()
                            yield from tile()
                else:
                    for kq in range(nqp):
                        yield from reserve_w(kq)
                    for kq in range(nqp):
                        if valid[r]:
                            yield from tile()
                            yield from tile()

    def mma(r):
        it = sc = uc = 0

        def wait_slot():
            nonlocal it
            s, need = it % SLOTS, it // SLOTS + 1
            yield lambda: st[r]["full"][s] >= need
            it += 1
            return s

        def z_block(stP, first):
            if valid[r]:
                if first:
                    yield lambda u=uc: st[r]["zempty"] >= u
                for _ in range(2):
                    t = yield from wait_slot()
                    st[r]["free"][t] += 1
            st[r]["free"][stP] += 1

        for nb in units:
            rounds = -(-nb // G)
            first = True
            for j in range(rounds + 1):
                nq = min(G, nb - j * G) if j < rounds else 0
                if r < nq:
                    b, need = sc & 1, sc >> 1
                    yield lambda b=b, need=need: st[r]["sempty"][b] >= need
                    for _ in range(2 * nk):
                        s = yield from wait_slot()
                        st[r]["free"][s] += 1
                    st[r]["sfull"][b] += 1
                    sc += 1
                nqp = min(G, nb - (j - 1) * G) if j >= 1 else 0
                stP = [None] * nqp
                if order == "lookahead":
                    if nqp:
                        stP[0] = yield from wait_slot()
                    for kq in range(nqp):
                        if kq + 1 < nqp:
                            stP[kq + 1] = yield from wait_slot()
                        yield from z_block(stP[kq], first)
                        first = first and not valid[r]
                else:
                    for kq in range(nqp):
                        stP[kq] = yield from wait_slot()
                    for kq in range(nqp):
                        yield from z_block(stP[kq], first)
                        first = first and not valid[r]
            if valid[r]:
                st[r]["zfull"] += 1
                uc += 1

    def epilogue(r):
        sc = mr = uc = 0
        for nb in units:
            for r0 in range(0, nb, G):
                if r >= min(G, nb - r0):
                    continue
                b, need = sc & 1, (sc >> 1) + 1
                yield lambda b=b, need=need: st[r]["sfull"][b] >= need
                st[r]["sempty"][b] += 1  # weights computed; logits released
                row, mneed = mr % mbox, G * (mr // mbox + 1)
                yield lambda row=row, mneed=mneed: st[r]["mfull"][row] >= mneed
                if st[r]["rounds"][row] != [mr] * G:
                    raise MailboxRace((r, mr, st[r]["rounds"][row]))
                slots = list(st[r]["mbox"][row])
                for j in range(G):  # own slot written, copies land in the others'
                    st[j]["full"][slots[j]] += 1
                sc += 1
                mr += 1
            if valid[r]:
                yield lambda u=uc: st[r]["zfull"] >= u + 1
                st[r]["zempty"] += 1
                uc += 1

    roles = []
    for r in range(G):
        for f in (producer, mma, epilogue):
            g = f(r)
            roles.append([g, next(g, None)])
    while True:
        live = [ro for ro in roles if ro[1] is not None]
        if not live:
            return True
        ready = [ro for ro in live if ro[1]()]
        if not ready:
            return False
        ro = rnd.choice(ready)
        ro[1] = next(ro[0], None)


UNITS = [[24] * 4, [23] * 4, [24, 23, 24, 23], [6], [2], [5, 3], [1], [7, 1, 9], [13] * 3,
         [16] * 2, [40], [9, 7], [1] * 10, [2, 1, 1, 1, 1, 1, 1, 3]]


def cvalid_patterns(G):
    """Which CTAs of the cluster own a pixel chunk: all, all but one, one (a last chunk
    group with a single chunk), and about half."""
    return [None, [True] * (G - 1) + [False], [True] + [False] * (G - 1),
            [k < (G + 1) // 2 for k in range(G)]]


@pytest.mark.parametrize("G", [2, 3, 4, 5, 6, 7, 8, 9, 12, 13, 16])
def test_kernel_slot_order_never_deadlocks(G):
    for units in UNITS:
        for cvalid in cvalid_patterns(G):
            for seed in range(3):
                assert run(G, units, "lookahead", seed=seed, cvalid=cvalid, nk=8), (units, cvalid)


def test_model_catches_a_mailbox_shallower_than_the_ring():
    """A producer may lead a peer's epilogue by one mailbox row per ring slot it holds
    for that peer (at most 7); with rows for only 4 uses, CTAs that own no pixel chunk
    in a run of one-block units (one ring slot per unit) overwrite rows not yet read."""
    with pytest.raises(MailboxRace):
        for seed in range(6):
            run(4, [1] * 10, "lookahead", seed=seed, cvalid=[True, False, False, False], nk=8,
                mbox=4)


def test_model_catches_the_weights_first_order():
    assert not run(4, [6], "weights_first")
    assert not run(4, [24] * 2, "weights_first", seed=1)
