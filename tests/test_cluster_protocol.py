"""Host-side models of the synchronisation of the clustered tensor-core pass 2, in its
two forms.

Staged form (clusters of 5 to 16).  Each CTA of a cluster of G runs four roles:
- a producer that reserves slots of a 6-deep shared-memory ring, for TMA tiles and for
  the weight tiles the other CTAs send it, and announces each weight slot in the
  sender's mailbox (an 8-row table of tagged entries, one row per use of a tile);
- an MMA issuer that consumes the ring in the same order, and its own weight tile from a
  staging slot;
- an epilogue that turns the logits of its own observation block into the staged
  weight tile, once the previous tile has been consumed and copied;
- a sender that copies the staged tile into each chunk-owning peer's announced slot as
  soon as that peer's announcement arrives.

A CTA takes the blocks of a round in its own order: its own block first, then the next
ranks cyclically.  The model runs the roles as coroutines under random schedules, with
the kernel's order, and reports a deadlock when no role can move, or a mailbox race when
a sender finds a row already overwritten by a later use.  It checks the kernel's order,
and that the model catches a weight slot reserved two blocks ahead (a deadlock in a
6-slot ring), a mailbox too shallow to hold the announcements in flight, and skipped
uses left uncounted.

Ring form (clusters up to 4).  Every weight tile, the owner's included, goes through a
7-slot ring; each producer reserves a slot for every tile of the round in block order
and announces it on a counting barrier per mailbox row, and an owner sends its tile
once all G reservations are in.  The model checks the kernel's order (weight slots one
block ahead of their Y'^T tiles), and that it catches the order that reserves all weight
slots of a round first (a deadlock) and a mailbox with fewer rows than ring slots."""
import random

import pytest

SLOTS, RING_SLOTS, MBOX = 6, 7, 8


class MailboxRace(Exception):
    """A sender read a mailbox entry that a later use of the row had overwritten."""


def block_order(r, n):
    """The blocks 0..n-1 of a round in CTA r's order (own first when r < n)."""
    return [(r % n + i) % n for i in range(n)] if n else []


def run_staged(G, units, seed=0, nk=8, cvalid=None, mbox=MBOX, lookahead=1, count_skipped=True):
    """units: observation blocks per work unit (every CTA of the cluster walks the same
    units).  cvalid: which CTAs own a pixel chunk, one pattern for all units or a list of
    patterns cycled over the units (ownership changes with the unit's chunk group).
    lookahead: how many blocks ahead a weight slot is reserved (the kernel: 1).
    count_skipped: a CTA without a chunk still counts the uses of the peers' tiles it
    does not take (the kernel does).  Returns True when every role finishes, False on a
    deadlock."""
    rnd = random.Random(seed)
    st = [dict(free=[0] * SLOTS, full=[0] * SLOTS, sfull=[0, 0], sempty=[0, 0], zfull=0,
               zempty=0, wfull=0, wfree=0, cdone=0, mbox=[[(0, 0)] * G for _ in range(mbox)])
          for _ in range(G)]
    pats = [[True] * G] if cvalid is None else (
        cvalid if isinstance(cvalid[0], (list, tuple)) else [cvalid])

    def valid_in(u):  # ownership pattern of unit u
        return pats[u % len(pats)]

    def own_rounds(r, nb):
        return [r0 for r0 in range(0, nb, G) if r < min(G, nb - r0)]

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
            st[kq]["mbox"][row] = (st[kq]["mbox"][row][:r] + [(sent[kq] + 1, s)]
                                   + st[kq]["mbox"][row][r + 1:])
            sent[kq] += 1

        def tile():  # a TMA tile: it lands at once
            s = yield from reserve()
            st[r]["full"][s] += 1

        for u, nb in enumerate(units):
            valid = valid_in(u)
            rounds = -(-nb // G)
            for j in range(rounds + 1):
                nq = min(G, nb - j * G) if j < rounds else 0
                if r < nq:
                    for _ in range(2 * nk):  # logits: (A hi+lo, Y hi+lo) per k-block
                        yield from tile()
                ks = block_order(r, min(G, nb - (j - 1) * G) if j >= 1 else 0)
                if not valid[r]:
                    if count_skipped:
                        for kq in ks:
                            if kq != r:
                                sent[kq] += 1
                    continue
                for i in range(min(lookahead, len(ks))):
                    if ks[i] != r:
                        yield from reserve_w(ks[i])
                for i in range(len(ks)):
                    if i + lookahead < len(ks) and ks[i + lookahead] != r:
                        yield from reserve_w(ks[i + lookahead])
                    yield from tile()
                    yield from tile()

    def mma(r):
        it = sc = uc = ow = 0

        def wait_slot():
            nonlocal it
            s, need = it % SLOTS, it // SLOTS + 1
            yield lambda: st[r]["full"][s] >= need
            it += 1
            return s

        for u, nb in enumerate(units):
            valid = valid_in(u)
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
                ks = block_order(r, min(G, nb - (j - 1) * G) if j >= 1 else 0)
                stP = {}
                for i in range(min(lookahead, len(ks))):
                    if valid[r] and ks[i] != r:
                        stP[i] = yield from wait_slot()
                for i, kq in enumerate(ks):
                    if valid[r] and i + lookahead < len(ks) and ks[i + lookahead] != r:
                        stP[i + lookahead] = yield from wait_slot()
                    if kq == r:
                        yield lambda o=ow: st[r]["wfull"] >= o + 1
                    if valid[r]:
                        if first:
                            yield lambda u=uc: st[r]["zempty"] >= u
                        for _ in range(2):
                            t = yield from wait_slot()
                            st[r]["free"][t] += 1
                        first = False
                    if kq == r:
                        st[r]["wfree"] += 1
                        ow += 1
                    elif valid[r]:
                        st[r]["free"][stP[i]] += 1
            if valid[r]:
                st[r]["zfull"] += 1
                uc += 1

    def epilogue(r):
        sc = m = uc = 0
        for u, nb in enumerate(units):
            valid = valid_in(u)
            for _ in own_rounds(r, nb):
                b, need = sc & 1, (sc >> 1) + 1
                yield lambda b=b, need=need: st[r]["sfull"][b] >= need
                st[r]["sempty"][b] += 1  # weights computed; logits released
                sc += 1
                yield lambda m=m: st[r]["wfree"] >= m and st[r]["cdone"] >= m
                st[r]["wfull"] += 1  # the tile is staged
                m += 1
            if valid[r]:
                yield lambda u=uc: st[r]["zfull"] >= u + 1
                st[r]["zempty"] += 1
                uc += 1

    def sender(r):
        m = 0
        for u, nb in enumerate(units):
            valid = valid_in(u)
            for _ in own_rounds(r, nb):
                yield lambda m=m: st[r]["wfull"] >= m + 1
                row, pending = m % mbox, {k for k in range(G) if k != r and valid[k]}

                def announced(row=row, m=m):
                    hits = []
                    for k in pending:
                        tag, s = st[r]["mbox"][row][k]
                        if tag > m + 1:
                            raise MailboxRace((r, m, k, tag))
                        if tag == m + 1:
                            hits.append((k, s))
                    return hits

                while pending:
                    yield lambda: bool(announced())
                    for k, s in announced():
                        st[k]["full"][s] += 1  # the copy lands in the peer's slot
                        pending.discard(k)
                st[r]["cdone"] += 1
                m += 1

    roles = []
    for r in range(G):
        for f in (producer, mma, epilogue, sender):
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


def run_ring(G, units, order, seed=0, nk=16, cvalid=None, mbox=MBOX):
    """The ring form (clusters up to 4): every weight tile, the owner's included, goes
    through the 7-slot ring, and an owner sends its tile once all G reservations for it
    are announced (one counting barrier per mailbox row).  units: observation blocks per
    work unit.  order: 'lookahead' (the kernel's) or 'weights_first'.  Returns True when
    every role finishes, False on a deadlock."""
    rnd = random.Random(seed)
    st = [dict(free=[0] * RING_SLOTS, full=[0] * RING_SLOTS, sfull=[0, 0], sempty=[0, 0], zfull=0,
               zempty=0, mfull=[0] * mbox, mbox=[[None] * G for _ in range(mbox)],
               rounds=[[None] * G for _ in range(mbox)])
          for _ in range(G)]
    valid = cvalid or [True] * G

    def producer(r):
        it = 0
        sent = [0] * G

        def reserve():
            nonlocal it
            s, need = it % RING_SLOTS, it // RING_SLOTS
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
            s, need = it % RING_SLOTS, it // RING_SLOTS + 1
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
    group with a single chunk), about half; and ownership that changes from unit to unit
    (a full chunk group, then a last group with some CTAs idle)."""
    full = [True] * G
    half = [k < (G + 1) // 2 for k in range(G)]
    one = [True] + [False] * (G - 1)
    return [None, [True] * (G - 1) + [False], one, half, [full, half], [half, full, one]]


def test_block_order():
    assert block_order(2, 5) == [2, 3, 4, 0, 1]
    assert block_order(0, 3) == [0, 1, 2]
    assert block_order(6, 4) == [2, 3, 0, 1]  # no own block: start at rank mod n
    assert block_order(1, 0) == []


@pytest.mark.parametrize("G", [5, 6, 7, 8, 9, 12, 13, 16])
def test_staged_form_order_never_deadlocks(G):
    for units in UNITS:
        for cvalid in cvalid_patterns(G):
            for seed in range(3):
                assert run_staged(G, units, seed=seed, cvalid=cvalid, nk=8), (units, cvalid)


def test_staged_model_catches_a_shallow_mailbox():
    """With a single mailbox row, a producer's announcement for the next use of a tile
    overwrites the row before the sender has read it."""
    with pytest.raises(MailboxRace):
        for seed in range(4):
            run_staged(2, [24] * 4, seed=seed, nk=1, mbox=1)


def test_staged_model_catches_uncounted_skipped_uses():
    """A CTA without a pixel chunk takes none of the peers' tiles; if it did not count
    those uses, its later announcements would carry stale tags and the senders would
    wait for them forever."""
    G = 4
    half = [True, True, False, False]
    assert not run_staged(G, [8, 8, 8], cvalid=[[True] * G, half], count_skipped=False)
    assert run_staged(G, [8, 8, 8], cvalid=[[True] * G, half])


def test_staged_model_catches_a_weight_slot_two_blocks_ahead():
    """Reserving weight slots two blocks ahead puts a Y'^T tile 7 places after its weight
    slot, which a 6-slot ring cannot hold: the fill waits for the slot that only its own
    products free."""
    assert not any(run_staged(4, [24] * 2, seed=s, lookahead=2) for s in range(3))


@pytest.mark.parametrize("G", [2, 3, 4])
def test_ring_form_order_never_deadlocks(G):
    for units in UNITS:
        for cvalid in cvalid_patterns(G)[:4]:
            for seed in range(3):
                assert run_ring(G, units, "lookahead", seed=seed, cvalid=cvalid, nk=8), \
                    (units, cvalid)


def test_ring_model_catches_a_mailbox_shallower_than_the_ring():
    """A producer may lead a peer's epilogue by one mailbox row per ring slot it holds
    for that peer (at most 7); with rows for only 4 uses, CTAs that own no pixel chunk
    in a run of one-block units (one ring slot per unit) overwrite rows not yet read."""
    with pytest.raises(MailboxRace):
        for seed in range(6):
            run_ring(4, [1] * 10, "lookahead", seed=seed, cvalid=[True, False, False, False],
                     nk=8, mbox=4)


def test_ring_model_catches_the_weights_first_order():
    assert not run_ring(4, [6], "weights_first")
    assert not run_ring(4, [24] * 2, "weights_first", seed=1)
