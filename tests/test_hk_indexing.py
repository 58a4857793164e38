"""Held-Karp table indexing, restated on the CPU: the subset a thread unranks, the next
subset in colex order by Gosper's step, and the table word each transition reads and
writes.  Plane c holds h(S, c) for the subsets S that contain c, indexed by T = S - c with
c's bit squeezed out, first by |T| (blocks of C(k - 1, l) words) and then by the colex
rank of T.  The kernel reaches every rank by prefix sums of binomial terms over the bits
of S; here each is checked against a direct count over all subsets (the dynamic programme
over subsets follows Held and Karp's recurrence on the pick sequence of Sec. 2.4)."""
import itertools
import math

import pytest


def colex_rank(bits):
    """Rank of a set of bit positions among the sets of its size in colex order (numeric
    order of the bitmasks), by counting the smaller ones."""
    bits = sorted(bits)
    return sum(math.comb(b, t + 1) for t, b in enumerate(bits))


def unrank(rr, L, k):
    """The kernel's unranking: bits from the top, each the largest c below the previous one
    with C(c, i) <= rr; the same pass sums pb = C(b_t - 1, t + 1) and pc = C(b_t - 1, t)."""
    def binx(n, r):  # C(n, r) with C(-1, r) = 0
        return math.comb(n, r) if n >= 0 else 0
    s, pb, pc, c = 0, 0, 0, k - 1
    for i in range(L, 0, -1):
        while binx(c, i) > rr:
            c -= 1
        s |= 1 << c
        rr -= binx(c, i)
        pb += binx(c - 1, i)
        pc += binx(c - 1, i - 1)
        c -= 1
    return s, pb, pc


def gosper(s):
    u = s & -s
    v = s + u
    return v | (((v ^ s) >> 2) >> (u.bit_length() - 1))


def squeeze(bits, j):
    return [b if b < j else b - 1 for b in bits if b != j]


@pytest.mark.parametrize("k", [4, 7, 9])
def test_unrank_gosper_and_ranks(k):
    for L in range(1, k + 1):
        subsets = sorted(sum(1 << b for b in comb) for comb in itertools.combinations(range(k), L))
        for w, s_true in enumerate(subsets):
            s, pb, pc = unrank(w, L, k)
            assert s == s_true, (k, L, w)
            bits = [b for b in range(k) if s >> b & 1]
            assert pb == sum(math.comb(b - 1, t + 1) if b else 0 for t, b in enumerate(bits))
            assert pc == sum(math.comb(b - 1, t) if b else 0 for t, b in enumerate(bits))
            if w + 1 < len(subsets):
                assert gosper(s) == subsets[w + 1]
            # successor h(S + j, j) for each j outside S: the word the kernel reads in plane j,
            # block |S|, is pb + the sum over the bits of S below j of C(b - 1, t) (Pascal)
            pcr, m = 0, 0
            for j in range(k):
                if s >> j & 1:
                    pcr += math.comb(j - 1, m) if j else 0
                    m += 1
                else:
                    assert pb + pcr == colex_rank(squeeze(bits, j)), (k, L, w, j)
            # stores h(S, c) for c in S: plane c, block |S| - 1, rank of S - c squeezed at c
            pa, pcs = 0, 0
            for t, c in enumerate(bits):
                cc = math.comb(c - 1, t) if c else 0
                assert pa + pc - pcs - cc == colex_rank(squeeze(bits, c)), (k, L, w, c)
                pa += math.comb(c, t + 1)
                pcs += cc
