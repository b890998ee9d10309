"""Host-side model of the four-warp diagonal-block step's schedule
(csrc/msts_diagw.cu): the per-warp sequence of rescales, AXPYs, productions of
x_i and named-barrier operations, written out from the kernel's loop
structure, run for every lane width and both directions of the cyclic row
layout and for the chunk-pair layout of upper solves with four lanes.

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


def program(layout, w, L, conj, rescale_rows):
    return chunk_program(w, rescale_rows) if layout == "chunk" else warp_program(w, L, conj, rescale_rows)


def rows_of(w, L, q, layout="cyclic"):
    if layout == "chunk":
        return [4 * (w if q == 0 else 7 - w) + h for h in range(4)]
    return [w + 4 * (h + L * q) for h in range(L)]


LAYOUTS = [("cyclic", L, conj) for L in (1, 2, 4) for conj in (False, True)] + [("chunk", 4, False)]


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
