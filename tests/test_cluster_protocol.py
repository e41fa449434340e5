"""Host-side models of the synchronisation of the clustered tensor-core pass 2, in its
two forms.

Interleaved form (clusters of 5 to 16).  Each CTA of a cluster of G runs five roles:
- a producer that fills a 4-slot main ring with the logit operands of its own block and
  the Y'^T tiles of its chunk, in the MMA's order: the Z' blocks of round j - 1 between
  the logit k-blocks of round j;
- a weight producer that reserves slots of a 2-slot weight ring for the peers' tiles and
  announces each in the tile owner's mailbox (an 8-row table of tagged entries, one row
  per use of a tile), once the main producer has begun the round;
- an MMA issuer that consumes both rings in the same orders, and its own weight tile from
  a staging slot;
- an epilogue that turns the logits of its own observation block into the staged
  weight tile, once the previous tile has been consumed and copied;
- a sender that copies the staged tile into each chunk-owning peer's announced slot as
  soon as that peer's announcement arrives.

A CTA takes the blocks of a round in its own order: its own block first, then the next
ranks cyclically.  The model runs the roles as coroutines under random schedules, with
the kernel's orders, and reports a deadlock when no role can move, or a mailbox race when
a sender finds a row already overwritten by a later use.  It checks the kernel's orders,
with chunk ownership fixed and changing from unit to unit, and that the model catches a
weight producer that is not held to the main producer's round, a mailbox too shallow
for the announcements in flight, and skipped uses left uncounted.

Ring form (clusters up to 4).  Every weight tile, the owner's included, goes through a
7-slot ring; each producer reserves a slot for every tile of the round in block order
and announces it on a counting barrier per mailbox row, and an owner sends its tile
once all G reservations are in.  The model checks the kernel's order (weight slots one
block ahead of their Y'^T tiles), and that it catches the order that reserves all weight
slots of a round first (a deadlock) and a mailbox with fewer rows than ring slots.

Pair form (clusters of G pairs of CTAs issuing 2-CTA MMAs).  The ring protocol among
the CTAs of one parity, with one Y'^T fill per weight tile (128 observations x 128
pixels): all weight slots of a round are reserved first, and the MMA thread takes each
tile's Y'^T fill right after the tile.  The model checks that order with ring-sized and
small numbers of k-blocks, and that it deadlocks with two fills per tile."""
import random

import pytest

MAIN_SLOTS, W_SLOTS, RING_SLOTS, MBOX = 4, 2, 7, 8


class MailboxRace(Exception):
    """A sender read a mailbox entry that a later use of the row had overwritten."""


def block_order(r, n):
    """The blocks 0..n-1 of a round in CTA r's order (own first when r < n)."""
    return [(r % n + i) % n for i in range(n)] if n else []


def zpos(i, nqp, nk):
    """k-block of round j after which Z' block i of round j - 1 is issued."""
    return ((i + 1) * nk) // (nqp + 1) - 1 if nk >= nqp + 1 else nk - 1


def run_interleaved(G, units, seed=0, nk=8, cvalid=None, mslots=MAIN_SLOTS, wslots=W_SLOTS,
                    mbox=MBOX, count_skipped=True, gate=True):
    """The interleaved form (clusters of 5 to 16).  units: observation blocks per work unit
    (every CTA of the cluster walks the same units).  cvalid: which CTAs own a pixel chunk,
    one pattern for all units or a list of patterns cycled over the units.  gate: the
    weight producer announces the slots of round j - 1 only once the main producer has
    begun round j (the kernel does).  count_skipped: a CTA without a chunk still counts
    the uses of the peers' tiles it does not take (the kernel does).  Returns True when
    every role finishes, False on a deadlock."""
    rnd = random.Random(seed)
    st = [dict(free_m=[0] * mslots, full_m=[0] * mslots, free_w=[0] * wslots, full_w=[0] * wslots,
               sfull=[0, 0], sempty=[0, 0], zfull=0, zempty=0, wfull=0, wfree=0, cdone=0,
               rstart=0,
               mbox=[[(0, 0)] * G for _ in range(mbox)]) for _ in range(G)]
    pats = [[True] * G] if cvalid is None else (
        cvalid if isinstance(cvalid[0], (list, tuple)) else [cvalid])

    def valid_in(u):
        return pats[u % len(pats)]

    def own_rounds(r, nb):
        return [r0 for r0 in range(0, nb, G) if r < min(G, nb - r0)]

    def schedule(r, nb, j):
        """The main-ring sequence of round j: ('L', kb) logit k-blocks, ('Z', i) Z blocks."""
        rounds = -(-nb // G)
        nq = min(G, nb - j * G) if j < rounds else 0
        nqp = min(G, nb - (j - 1) * G) if j >= 1 else 0
        seq = []
        done = 0
        if r < nq:
            for kb in range(nk):
                seq.append(('L', kb))
                while done < nqp and zpos(done, nqp, nk) == kb:
                    seq.append(('Z', done))
                    done += 1
        while done < nqp:
            seq.append(('Z', done))
            done += 1
        return seq, nq, nqp

    def producer(r):
        it = 0

        def fill():
            nonlocal it
            s, need = it % mslots, it // mslots
            yield lambda: st[r]["free_m"][s] >= need
            it += 1
            st[r]["full_m"][s] += 1

        for u, nb in enumerate(units):
            valid = valid_in(u)
            rounds = -(-nb // G)
            for j in range(rounds + 1):
                seq, nq, nqp = schedule(r, nb, j)
                st[r]["rstart"] += 1  # round (u, j) started
                for kind, _ in seq:
                    if kind == 'L':
                        yield from fill()
                        yield from fill()
                    elif valid[r]:
                        yield from fill()
                        yield from fill()

    def wprod(r):
        itw = 0
        sent = [0] * G
        g = 0  # rounds (u, j) passed, in the producer's count
        for u, nb in enumerate(units):
            valid = valid_in(u)
            rounds = -(-nb // G)
            g += 1  # round j = 0 of the unit carries no Z' blocks
            for j in range(1, rounds + 1):
                g += 1
                if gate:
                    yield lambda g=g: st[r]["rstart"] >= g
                nqp = min(G, nb - (j - 1) * G)
                ks = block_order(r, nqp)
                for kq in ks:
                    if kq == r:
                        continue
                    if not valid[r]:
                        if count_skipped:
                            sent[kq] += 1
                        continue
                    s, need = itw % wslots, itw // wslots
                    yield lambda s=s, need=need: st[r]["free_w"][s] >= need
                    itw += 1
                    row = sent[kq] % mbox
                    st[kq]["mbox"][row] = (st[kq]["mbox"][row][:r] + [(sent[kq] + 1, s)]
                                           + st[kq]["mbox"][row][r + 1:])
                    sent[kq] += 1

    def mma(r):
        it = itw = sc = uc = ow = 0

        def take_m():
            nonlocal it
            s, need = it % mslots, it // mslots + 1
            yield lambda: st[r]["full_m"][s] >= need
            it += 1
            return s

        for u, nb in enumerate(units):
            valid = valid_in(u)
            rounds = -(-nb // G)
            first = True
            for j in range(rounds + 1):
                seq, nq, nqp = schedule(r, nb, j)
                ks = block_order(r, nqp)
                if r < nq:
                    b, need = sc & 1, sc >> 1
                    yield lambda b=b, need=need: st[r]["sempty"][b] >= need
                for kind, idx in seq:
                    if kind == 'L':
                        for _ in range(2):
                            s = yield from take_m()
                            st[r]["free_m"][s] += 1
                        if idx == nk - 1:
                            st[r]["sfull"][sc & 1] += 1
                            sc += 1
                        continue
                    kq = ks[idx]
                    sw = None
                    if kq == r:
                        yield lambda o=ow: st[r]["wfull"] >= o + 1
                    elif valid[r]:
                        sw, need = itw % wslots, itw // wslots + 1
                        yield lambda sw=sw, need=need: st[r]["full_w"][sw] >= need
                        itw += 1
                    if valid[r]:
                        if first:
                            yield lambda u=uc: st[r]["zempty"] >= u
                        for _ in range(2):
                            s = yield from take_m()
                            st[r]["free_m"][s] += 1
                        first = False
                    if kq == r:
                        st[r]["wfree"] += 1
                        ow += 1
                    elif valid[r]:
                        st[r]["free_w"][sw] += 1
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
                st[r]["sempty"][b] += 1
                sc += 1
                yield lambda m=m: st[r]["wfree"] >= m and st[r]["cdone"] >= m
                st[r]["wfull"] += 1
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
                        st[k]["full_w"][s] += 1
                        pending.discard(k)
                st[r]["cdone"] += 1
                m += 1

    roles = []
    for r in range(G):
        for f in (producer, wprod, mma, epilogue, sender):
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


def run_pair(G, units, seed=0, nk=16, cvalid=None, mbox=MBOX, t_per_w=1):
    """The pair form (clusters of G pairs): each CTA's ring, seen from one parity (the
    two CTAs of a pair fill the same slots in step, and the even CTA's MMA thread takes a
    fill once it has landed in both, so one parity's CTAs carry the whole dependency
    structure).  Per round: the logit fills of the pair's block (two template fills and
    one observation fill per two k-blocks), then for round j - 1 a slot for every weight
    tile (announced to its owner, which sends once all G reservations are in) followed by
    t_per_w Y'^T fills per tile; the MMA thread takes weight tile i, then its Y'^T fills,
    out of the ring order.  Returns True when every role finishes, False on a deadlock."""
    rnd = random.Random(seed)
    st = [dict(free=[0] * RING_SLOTS, full=[0] * RING_SLOTS, sfull=[0, 0], sempty=[0, 0], zfull=0,
               zempty=0, mfull=[0] * mbox, mbox=[[None] * G for _ in range(mbox)],
               rounds=[[None] * G for _ in range(mbox)])
          for _ in range(G)]
    valid = cvalid or [True] * G

    def logit_fills():
        return sum(min(2, nk - kb) + 1 for kb in range(0, nk, 2))

    def producer(r):
        it = 0
        sent = [0] * G

        def reserve():
            nonlocal it
            s, need = it % RING_SLOTS, it // RING_SLOTS
            yield lambda: st[r]["free"][s] >= need
            it += 1
            return s

        for nb in units:
            rounds = -(-nb // G)
            for j in range(rounds + 1):
                nq = min(G, nb - j * G) if j < rounds else 0
                if r < nq:
                    for _ in range(logit_fills()):
                        s = yield from reserve()
                        st[r]["full"][s] += 1
                nqp = min(G, nb - (j - 1) * G) if j >= 1 else 0
                for kq in range(nqp):
                    s = yield from reserve()
                    row = sent[kq] % mbox
                    st[kq]["mbox"][row][r] = s
                    st[kq]["rounds"][row][r] = sent[kq]
                    st[kq]["mfull"][row] += 1
                    sent[kq] += 1
                if valid[r]:
                    for _ in range(nqp * t_per_w):
                        s = yield from reserve()
                        st[r]["full"][s] += 1

    def mma(r):
        it = sc = uc = 0

        def take(k):
            s, need = k % RING_SLOTS, k // RING_SLOTS + 1
            yield lambda: st[r]["full"][s] >= need
            return s

        for nb in units:
            rounds = -(-nb // G)
            first = True
            for j in range(rounds + 1):
                nq = min(G, nb - j * G) if j < rounds else 0
                if r < nq:
                    b, need = sc & 1, sc >> 1
                    yield lambda b=b, need=need: st[r]["sempty"][b] >= need
                    for _ in range(logit_fills()):
                        s = yield from take(it)
                        it += 1
                        st[r]["free"][s] += 1
                    st[r]["sfull"][b] += 1
                    sc += 1
                nqp = min(G, nb - (j - 1) * G) if j >= 1 else 0
                base = it
                it += nqp + (nqp * t_per_w if valid[r] else 0)
                for i in range(nqp):
                    sw = yield from take(base + i)
                    if valid[r]:
                        if first:
                            yield lambda u=uc: st[r]["zempty"] >= u
                        for t in range(t_per_w):
                            s = yield from take(base + nqp + i * t_per_w + t)
                            st[r]["free"][s] += 1
                        first = False
                    st[r]["free"][sw] += 1
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
                st[r]["sempty"][b] += 1
                row, mneed = mr % mbox, G * (mr // mbox + 1)
                yield lambda row=row, mneed=mneed: st[r]["mfull"][row] >= mneed
                if st[r]["rounds"][row] != [mr] * G:
                    raise MailboxRace((r, mr, st[r]["rounds"][row]))
                slots = list(st[r]["mbox"][row])
                for j in range(G):
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
def test_interleaved_form_order_never_deadlocks(G):
    for units in UNITS:
        for cvalid in cvalid_patterns(G):
            for seed in range(2):
                assert run_interleaved(G, units, seed=seed, cvalid=cvalid, nk=8), \
                    (units, cvalid)


def test_interleaved_form_with_few_k_blocks():
    """Fewer k-blocks than Z' blocks per round: all Z' blocks after the last k-block."""
    for G in (5, 9):
        for units in ([12] * 3, [7, 1, 9]):
            assert run_interleaved(G, units, nk=2, cvalid=cvalid_patterns(G)[4])


def test_interleaved_model_catches_an_ungated_weight_producer():
    """Without the gate, the weight producer runs through a unit where its CTA owns no
    chunk (counting, not taking, the peers' tiles) and announces a later use into a
    mailbox row the peer's sender has not read yet."""
    with pytest.raises(MailboxRace):
        for seed in range(2):
            run_interleaved(2, [13] * 3, seed=seed, cvalid=[[True, True], [True, False]],
                            gate=False)


def test_interleaved_model_catches_a_shallow_mailbox():
    """With 3 mailbox rows a weight producer's announcement can overwrite a row whose
    use the sender has not reached (the kernel has 8)."""
    with pytest.raises(MailboxRace):
        for seed in range(2):
            run_interleaved(2, [1] * 10, seed=seed, nk=4, mbox=3,
                            cvalid=[[True, False], [True, True], [True, False]])


def test_interleaved_model_catches_uncounted_skipped_uses():
    """Uncounted skipped uses leave later announcements with stale tags: the senders
    wait for them forever."""
    G = 4
    half = [True, True, False, False]
    assert not run_interleaved(G, [8, 8, 8], cvalid=[[True] * G, half], count_skipped=False)
    assert run_interleaved(G, [8, 8, 8], cvalid=[[True] * G, half])


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


@pytest.mark.parametrize("G", [1, 2, 3, 4])
def test_pair_form_order_never_deadlocks(G):
    for units in UNITS:
        for cvalid in cvalid_patterns(G)[:4]:
            for nk in (16, 9, 2, 1):
                for seed in range(2):
                    assert run_pair(G, units, seed=seed, cvalid=cvalid, nk=nk), \
                        (units, cvalid, nk)


def test_pair_model_catches_too_many_fills_per_weight_tile():
    """Reserving all weight slots of a round first is safe only while each tile's Y'^T
    fills lie within the ring: with two 64-observation fills per tile (the single-CTA
    layout) the last tile's fills wait for slots that only its own products release."""
    assert not run_pair(4, [24] * 2, t_per_w=2, nk=8)
