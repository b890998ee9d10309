"""Host-side model of the four-warp diagonal-block step's schedule
(csrc/msts_diagw.cu): the per-warp sequence of rescales, AXPYs, productions of
x_i and named-barrier operations, written out from the kernel's loop
structure, run for every lane width and both directions of the cyclic row
layout and for the chunk-pair layouts of solves with four lanes (upper and
conjugate-transposed).

It checks what the kernel's correctness rests on: (1) every row value sees the
same operations in the same order as in the serial substitution (the rescale of
row i before x_i is formed and before x_i's AXPY, AXPYs in row order), which is
why the layouts agree bit for bit; (2) every row's barrier is met by all four
warps, one arrive and three waits, and the warps can always progress (no
deadlock); (3) a barrier id is never reused while an earlier row with the same
id is still open."""
import random

import pytest

NB = 32


def warp_program(w, L, conj, rescale_rows):
    """The ops warp w issues, in order: ('rescale', slot, i), ('axpy', slot, i),
    ('produce', slot, i), ('arrive', i), ('sync', i)."""
    RPT, SLOT = NB // (4 * L), 4 * L
    ops = []
    i0 = 0 if conj else NB - 1
    if w == (i0 & 3):
        if rescale_rows.get(i0):
            ops += [("rescale", q, i0) for q in range(RPT)]
        ops += [("produce", 0 if conj else RPT - 1, i0), ("arrive", i0)]
    ahead = w == (i0 & 3)
    for s_ in range(RPT):
        qs = s_ if conj else RPT - 1 - s_
        for u_ in range(SLOT):
            k = u_ if conj else SLOT - 1 - u_
            i = SLOT * qs + k
            last = i == (NB - 1 if conj else 0)
            nxt = i + 1 if conj else i - 1
            if rescale_rows.get(i) and not ahead:
                ops += [("rescale", q, i) for q in range(RPT)]
            if w != (i & 3):
                ops.append(("sync", i))
            ahead = False
            if not last and w == (nxt & 3):
                same = k < SLOT - 1 if conj else k > 0
                qn = qs if same else qs + (1 if conj else -1)
                assert 0 <= qn < RPT
                ops.append(("axpy", qn, i))
                if rescale_rows.get(nxt):
                    ops.append(("rescale", qn, nxt))
                ops += [("produce", qn, nxt), ("arrive", nxt)]
                for q in range(RPT):
                    if q != qn:
                        ops.append(("axpy", q, i))
                        if rescale_rows.get(nxt):
                            ops.append(("rescale", q, nxt))
                ahead = True
            else:
                ops += [("axpy", q, i) for q in range(RPT)]
    return ops


def chunk_program(w, rescale_rows):
    """The chunk-pair layout (upper, L = 4): warp w holds chunk w (slot 0) and
    chunk 7 - w (slot 1), four consecutive rows each; chunk c is owned by warp
    7 - c (c >= 4) or c; an owner of a chunk c >= 4 defers its slot 0's
    operations of the chunk to the chunk's last row."""
    ops = []
    kk = rescale_rows.get

    def produce(q, i):
        if kk(i):
            ops.append(("rescale", q, i))
        ops.extend([("produce", q, i), ("arrive", i)])

    ahead = False
    if w == 0:
        if kk(NB - 1):
            ops.extend(("rescale", q, NB - 1) for q in range(2))
        ops.extend([("produce", 1, NB - 1), ("arrive", NB - 1)])   # no rescale inside
        ahead = True
    for c in range(7, 3, -1):
        own = w == 7 - c
        for k in range(3, -1, -1):
            i = 4 * c + k
            if kk(i) and not ahead:
                ops.extend(("rescale", q, i) for q in range(2))
            if not own:
                ops.append(("sync", i))
            ahead = False
            if own:
                if k > 0:
                    ops.append(("axpy", 1, i))
                    produce(1, i - 1)
                    ahead = True
                else:
                    for d in (2, 1, 0):
                        ops.append(("axpy", 0, 4 * c + d + 1))
                        if kk(4 * c + d):
                            ops.append(("rescale", 0, 4 * c + d))
                    ops.append(("axpy", 0, i))
                    if c == 4:
                        produce(0, i - 1)
                        if kk(i - 1):
                            ops.append(("rescale", 1, i - 1))
                        ahead = True
            elif k == 0 and w == 8 - c:
                ops.append(("axpy", 1, i))
                produce(1, i - 1)
                ops.append(("axpy", 0, i))
                if kk(i - 1):
                    ops.append(("rescale", 0, i - 1))
                ahead = True
            else:
                ops.append(("axpy", 0, i))
                if w > 7 - c:
                    ops.append(("axpy", 1, i))
    for c in range(3, -1, -1):
        own = w == c
        for k in range(3, -1, -1):
            i = 4 * c + k
            if kk(i) and not ahead:
                ops.extend(("rescale", q, i) for q in range(2))
            if not own:
                ops.append(("sync", i))
            ahead = False
            if (own and k > 0) or (not own and k == 0 and w == c - 1):
                ops.append(("axpy", 0, i))
                produce(0, i - 1)
                if kk(i - 1):
                    ops.append(("rescale", 1, i - 1))
                ahead = True
            elif w < c:
                ops.append(("axpy", 0, i))
    return ops


def chunkg_program(w, L, conj, rescale_rows):
    """The general chunk-pair loop (the kernel's conjugate L = 4 solves; also
    modelled at L = 2, which the kernel keeps cyclic): chunks
    of L consecutive rows, warp w holding chunks 8 b + w (slot 2 b) and
    8 b + 7 - w (slot 2 b + 1); the cyclic layout's loop with this ownership,
    the owner of a chunk leaving its other slots' share of the chunk's x_i (and
    the rescales after them) until it has produced the chunk's last row."""
    RPT = NB // (4 * L)
    kk = rescale_rows.get

    def chunk_of(q):
        return 8 * (q >> 1) + (7 - w if q & 1 else w)

    def owner_of(c):
        t = c & 7
        return t if t < 4 else 7 - t

    def slot_of(c):
        return 2 * (c >> 3) + (1 if (c & 7) >= 4 else 0)

    def pending(q, i):
        r0 = L * chunk_of(q)
        return r0 + L - 1 > i if conj else r0 < i

    ops = []
    i0 = 0 if conj else NB - 1
    ahead = False
    if w == owner_of(i0 // L):
        if kk(i0):
            ops.extend(("rescale", q, i0) for q in range(RPT))
        ops.extend([("produce", slot_of(i0 // L), i0), ("arrive", i0)])
        ahead = True
    for n in range(NB):
        i = n if conj else NB - 1 - n
        last = n == NB - 1
        nxt = i + 1 if conj else i - 1
        kc = (L - 1 - i % L) if conj else i % L          # rows after this one in its chunk
        own = w == owner_of(i // L)
        if kk(i) and not ahead:
            ops.extend(("rescale", q, i) for q in range(RPT))
        if not own:
            ops.append(("sync", i))
        ahead = False
        if own and kc > 0:                                # defer the other slots' share
            qn = slot_of(i // L)
            ops.append(("axpy", qn, i))
            if kk(nxt):
                ops.append(("rescale", qn, nxt))
            ops.extend([("produce", qn, nxt), ("arrive", nxt)])
            ahead = True
            continue
        if own and L > 1:                                 # the chunk's last row: replay
            qo = slot_of(i // L)
            for d in range(L - 1, 0, -1):
                rd = i - d if conj else i + d
                for q in range(RPT):
                    if q != qo and pending(q, rd):
                        ops.append(("axpy", q, rd))
                rn = rd + 1 if conj else rd - 1           # the rescale taken at the next row
                if kk(rn):
                    ops.extend(("rescale", q, rn) for q in range(RPT) if q != qo)
        if not last and w == owner_of(nxt // L):
            qn = slot_of(nxt // L)
            ops.append(("axpy", qn, i))
            if kk(nxt):
                ops.append(("rescale", qn, nxt))
            ops.extend([("produce", qn, nxt), ("arrive", nxt)])
            for q in range(RPT):
                if q != qn:
                    if pending(q, i):
                        ops.append(("axpy", q, i))
                    if kk(nxt):
                        ops.append(("rescale", q, nxt))
            ahead = True
        else:
            ops.extend(("axpy", q, i) for q in range(RPT) if pending(q, i))
    return ops


def program(layout, w, L, conj, rescale_rows):
    if layout == "chunk":
        return chunk_program(w, rescale_rows)
    if layout == "chunkg":
        return chunkg_program(w, L, conj, rescale_rows)
    return warp_program(w, L, conj, rescale_rows)


def rows_of(w, L, q, layout="cyclic"):
    if layout == "chunk":
        return [4 * (w if q == 0 else 7 - w) + h for h in range(4)]
    if layout == "chunkg":
        c = 8 * (q >> 1) + (7 - w if q & 1 else w)
        return [L * c + h for h in range(L)]
    return [w + 4 * (h + L * q) for h in range(L)]


# every layout the kernel runs (cyclic at L = 1, 2; chunk-pair at L = 4, the
# upper form with deferral and the conjugate one on the general loop), the
# cyclic L = 4 it used before, and the general loop at L = 2, which the kernel
# does not use (it measured slower) but which the model still checks
LAYOUTS = ([("cyclic", L, conj) for L in (1, 2, 4) for conj in (False, True)] + [("chunk", 4, False)]
           + [("chunkg", 2, False), ("chunkg", 2, True), ("chunkg", 4, True)])


def test_slot_multiply_adds_per_warp():
    """Slot multiply-adds each warp issues per block (counting only those with a
    row to update): equal for all warps in the chunk-pair layouts, and below
    the busiest warp's count in the cyclic layout, which bounds its block."""
    def count(layout, L, conj, w):        # multiply-adds with at least one row to update
        return sum(1 for op in program(layout, w, L, conj, {}) if op[0] == "axpy"
                   and any((r > op[2]) if conj else (r < op[2]) for r in rows_of(w, L, op[1], layout)))
    for L, conj in ((2, False), (2, True), (4, True)):
        got = {count("chunkg", L, conj, w) for w in range(4)}
        assert len(got) == 1, (L, conj, got)
        assert got.pop() < max(count("cyclic", L, conj, w) for w in range(4))
    assert {count("chunk", 4, False, w) for w in range(4)} == {34}


def test_layouts_cover_every_row_once():
    for layout, L, conj in LAYOUTS:
        RPT = NB // (4 * L)
        rows = sorted(r for w in range(4) for q in range(RPT) for r in rows_of(w, L, q, layout))
        assert rows == list(range(NB)), (layout, L)


@pytest.mark.parametrize("layout,L,conj", LAYOUTS)
def test_every_value_sees_the_serial_order(layout, L, conj):
    rng = random.Random(17 + L + 10 * conj + 100 * (layout == "chunk"))
    order = list(range(NB)) if conj else list(range(NB - 1, -1, -1))
    for _ in range(40):
        resc = {i: rng.random() < 0.25 for i in range(NB)}
        seen = {r: [] for r in range(NB)}
        for w in range(4):
            for op in program(layout, w, L, conj, resc):
                if op[0] in ("rescale", "axpy", "produce"):
                    _, q, i = op
                    for r in rows_of(w, L, q, layout):
                        if op[0] == "rescale":
                            seen[r].append(("R", i))
                        elif op[0] == "axpy" and (r > i if conj else r < i):
                            seen[r].append(("A", i))
                        elif op[0] == "produce" and r == i:
                            seen[r].append(("P", i))
        for r in range(NB):
            want = []
            for i in order:
                if resc[i]:
                    want.append(("R", i))
                if i == r:
                    want.append(("P", i))
                elif (r > i) if conj else (r < i):
                    want.append(("A", i))
            assert seen[r] == want, (L, conj, r)


@pytest.mark.parametrize("layout,L,conj", LAYOUTS)
def test_barriers_complete_without_deadlock_or_id_reuse(layout, L, conj):
    order = list(range(NB)) if conj else list(range(NB - 1, -1, -1))
    pos = {r: n for n, r in enumerate(order)}
    progs = {w: [op for op in program(layout, w, L, conj, {}) if op[0] in ("arrive", "sync")] for w in range(4)}
    for w in range(4):
        assert [op[1] for op in progs[w]] == order      # one barrier operation per row, in row order
    pc = {w: 0 for w in range(4)}
    reached, waiting = {}, set()
    while any(pc[w] < len(progs[w]) for w in range(4)):
        progressed = False
        for w in range(4):
            if pc[w] >= len(progs[w]):
                continue
            kind, r = progs[w][pc[w]]
            for r2 in order[:pos[r]]:                    # id (row & 7) reused only after the row closed
                assert (r2 & 7) != (r & 7) or reached.get(r2, 0) == 4
            if kind == "arrive":
                reached[r] = reached.get(r, 0) + 1
                pc[w] += 1
                progressed = True
            else:
                if (w, r) not in waiting:
                    waiting.add((w, r))
                    reached[r] = reached.get(r, 0) + 1
                if reached[r] == 4:
                    pc[w] += 1
                    progressed = True
        assert progressed, "deadlock"
    assert all(reached[r] == 4 for r in range(NB))
