"""rt_check_triples (host only, no GPU): the structural contract of a block
product's triple list.  Lists built here from the definition of the truncated
product (for output block (i,j) of P_C, one triple per k with (i,k) in P_A and
(k,j) in P_B, k ascending; the A operand is the stored block (i,k), or (k,i)
for A^dagger; the B operand (k,j), or (j,k) for B^dagger) pass for every op
combination and for upper-only outputs; each planted defect (a missing or
extra triple, k out of order, an operand index out of range or in the wrong
row or column, an output block with two writers or none, an upper-only list
with a lower block, a bad ptr, an asymmetric pattern) is caught."""
import itertools

import numpy as np
import pytest

import oracle
import synth

rt = pytest.importorskip("paper_1404_5776_gb300")


@pytest.fixture(scope="module")
def lib():
    try:
        rt.load()
    except RuntimeError:
        rt.build()
        rt.load()
    return rt


@pytest.fixture(scope="module")
def pats():
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    return s.n_atoms, {r: oracle.pattern(s.pos, s.cell, r) for r in (4.0, 5.0, 6.0)}


def _index(p):
    return {(i, int(p.col[q])): q for i in range(len(p.rowptr) - 1) for q in range(p.rowptr[i], p.rowptr[i + 1])}


def _build(n, pa, ad, pb, bd, pc, upper):
    ia, ib = _index(pa), _index(pb)
    items, ptr, ab = [], [0], []
    for i in range(n):
        row_a = set(int(k) for k in pa.col[pa.rowptr[i]:pa.rowptr[i + 1]])
        for q in range(pc.rowptr[i], pc.rowptr[i + 1]):
            j = int(pc.col[q])
            if upper and j < i:
                continue
            row_b = set(int(k) for k in pb.col[pb.rowptr[j]:pb.rowptr[j + 1]])
            for k in sorted(row_a & row_b):
                ab.append((ia[(k, i)] if ad else ia[(i, k)], ib[(j, k)] if bd else ib[(k, j)]))
            items.append(q)
            ptr.append(len(ab))
    return (np.array(items, np.int32), np.array(ptr, np.int64),
            np.array(ab, np.int32).reshape(-1, 2))


def _run(lib, n, pa, ad, pb, bd, pc, upper, items, ptr, ab):
    return lib.rt_check_triples(n, pa.rowptr, pa.col, ad, pb.rowptr, pb.col, bd, pc.rowptr, pc.col, upper,
                                items, ptr, ab)


@pytest.mark.parametrize("ad,bd,upper", list(itertools.product([0, 1], [0, 1], [0, 1])))
def test_lists_from_the_definition_pass(lib, pats, ad, bd, upper):
    n, P = pats
    for ra, rb, rc in ((5.0, 6.0, 4.0), (4.0, 5.0, 6.0), (6.0, 6.0, 6.0)):
        pa, pb, pc = P[ra], P[rb], P[rc]
        items, ptr, ab = _build(n, pa, ad, pb, bd, pc, upper)
        st, bad = _run(lib, n, pa, ad, pb, bd, pc, upper, items, ptr, ab)
        assert st == rt.RT_OK and bad == -1, (ra, rb, rc)
        # the same list read with the other convention for op(A) is rejected
        # (its A operands are off-diagonal blocks stored the other way round)
        st, _ = _run(lib, n, pa, 1 - ad, pb, bd, pc, upper, items, ptr, ab)
        assert st == rt.RT_EINTERNAL, (ra, rb, rc)


def test_planted_defects_are_caught(lib, pats):
    n, P = pats
    pa, pb, pc = P[5.0], P[6.0], P[5.0]
    items, ptr, ab = _build(n, pa, 0, pb, 1, pc, 1)
    assert _run(lib, n, pa, 0, pb, 1, pc, 1, items, ptr, ab)[0] == rt.RT_OK
    t = 7  # an item with several triples
    assert ptr[t + 1] - ptr[t] >= 3

    def expect_fail(items_, ptr_, ab_, upper=1, pa_=pa, item=None):
        st, bad = _run(lib, n, pa_, 0, pb, 1, pc, upper, items_, ptr_, ab_)
        assert st == rt.RT_EINTERNAL
        if item is not None:
            assert bad == item

    # a triple dropped (ptr shifted after it)
    ab2 = np.delete(ab, ptr[t], axis=0)
    ptr2 = ptr.copy()
    ptr2[t + 1:] -= 1
    expect_fail(items, ptr2, ab2, item=t)
    # a triple duplicated
    ab2 = np.insert(ab, ptr[t], ab[ptr[t]], axis=0)
    ptr2 = ptr.copy()
    ptr2[t + 1:] += 1
    expect_fail(items, ptr2, ab2, item=t)
    # k out of order within the item
    ab2 = ab.copy()
    ab2[[ptr[t], ptr[t] + 1]] = ab2[[ptr[t] + 1, ptr[t]]]
    expect_fail(items, ptr, ab2, item=t)
    # operand indices out of range
    for col, limit in ((0, pa.rowptr[-1]), (1, pb.rowptr[-1])):
        ab2 = ab.copy()
        ab2[ptr[t], col] = limit
        expect_fail(items, ptr, ab2, item=t)
        ab2[ptr[t], col] = -1
        expect_fail(items, ptr, ab2, item=t)
    # the B operand of another output column
    ab2 = ab.copy()
    ab2[ptr[t], 1] = (ab2[ptr[t], 1] + 1) % pb.rowptr[-1]
    expect_fail(items, ptr, ab2, item=t)
    # two writers for one output block, and an output block without a writer
    items2 = items.copy()
    items2[t + 1] = items2[t]
    expect_fail(items2, ptr, ab)
    expect_fail(items[:-1], ptr[:-1], ab[:ptr[-2]])
    # an upper-only list that carries a lower block (its mirror would race)
    full_items, full_ptr, full_ab = _build(n, pa, 0, pb, 1, pc, 0)
    expect_fail(full_items, full_ptr, full_ab, upper=1)
    # ptr not ending at the triple count
    ptr2 = ptr.copy()
    ptr2[-1] += 1
    expect_fail(items, ptr2, ab)
    # an asymmetric operand pattern: block (0, j0) dropped from row 0 while
    # (j0, 0) stays
    j0 = int(pa.col[pa.rowptr[0] + 1])
    assert j0 != 0
    keep = np.ones(pa.col.size, bool)
    keep[pa.rowptr[0] + 1] = False
    rowptr = pa.rowptr.copy()
    rowptr[1:] -= 1
    pa_asym = oracle.Pattern(rowptr, pa.col[keep].copy())
    st, bad = _run(lib, n, pa_asym, 0, pb, 1, pc, 1, items, ptr, ab)
    assert st == rt.RT_EINTERNAL and bad == -1


def test_empty_product(lib, pats):
    n, P = pats
    pa = P[4.0]
    empty = oracle.Pattern(np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
    st, bad = lib.rt_check_triples(n, pa.rowptr, pa.col, 0, pa.rowptr, pa.col, 0, empty.rowptr, empty.col, 0,
                                   np.zeros(0, np.int32), np.zeros(1, np.int64), np.zeros((0, 2), np.int32))
    assert st == rt.RT_OK and bad == -1
