"""Host-side model of the four-warp diagonal-block step's schedule
(csrc/msts_diagw.cu): the per-warp sequence of rescales, AXPYs, productions of
x_i and named-barrier operations, written out from the kernel's loop
structure, run for every lane width and both directions.

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


def rows_of(w, L, q):
    return [w + 4 * (h + L * q) for h in range(L)]


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("conj", [False, True])
def test_every_value_sees_the_serial_order(L, conj):
    rng = random.Random(17 + L + 10 * conj)
    order = list(range(NB)) if conj else list(range(NB - 1, -1, -1))
    for _ in range(40):
        resc = {i: rng.random() < 0.25 for i in range(NB)}
        seen = {r: [] for r in range(NB)}
        for w in range(4):
            for op in warp_program(w, L, conj, resc):
                if op[0] in ("rescale", "axpy", "produce"):
                    _, q, i = op
                    for r in rows_of(w, L, q):
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


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("conj", [False, True])
def test_barriers_complete_without_deadlock_or_id_reuse(L, conj):
    order = list(range(NB)) if conj else list(range(NB - 1, -1, -1))
    pos = {r: n for n, r in enumerate(order)}
    progs = {w: [op for op in warp_program(w, L, conj, {}) if op[0] in ("arrive", "sync")] for w in range(4)}
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
