"""The enumeration's unit schemes, restated on the CPU: every unit's sequences get the
lexicographic ranks the kernel gives them, and the units of an order cover its k! ranks
once each.  Prefix units fix the first k - 7 picks by the factorial digits of the unit
index and hold 5040 sequences; set units (orders of 11 and 12 picks in a call with enough
of them) are a set Q of the first k - 7 picks, the next pick x and, for k = 12, Q's first
pick, and walk every ordering of (the rest of) Q before x and the 720 orderings of the
other six.  The rank of a sequence is its position among the k! orderings of the picks
1..k in lexicographic order (Sec. 4.6 enumerates them all; the tie rule keeps the first).
"""
import itertools
import math

import pytest


def nth_bit(m, n):
    for _ in range(n):
        m &= m - 1
    return (m & -m).bit_length() - 1


def lex_rank(seq, k):
    """Position of seq among the orderings of 1..k in lexicographic order, by counting."""
    avail = list(range(1, k + 1))
    r = 0
    for i, p in enumerate(seq):
        r += avail.index(p) * math.factorial(k - 1 - i)
        avail.remove(p)
    return r


def orderings_table(n):
    """The kernel's table of the orderings of n <= 4 items: per position the item and how
    many items before it are smaller."""
    out = []
    for perm in itertools.permutations(range(n)):
        out.append([(p, sum(1 for q in perm[:i] if q < p)) for i, p in enumerate(perm)])
    return out


def set_unit_sequences(k, u):
    """(rank the kernel computes, the sequence) for each walked prefix ordering of unit u,
    the six picks after x in increasing order (rank of the part's first sequence)."""
    q = k - 7
    nf = 5 if q == 5 else 1
    qr = 4 if q == 5 else q
    fi, t = u % nf, u // nf
    xi, t = t % 7, t // 7
    Q, rr, c = 0, t, k - 1
    for i in range(q, 0, -1):  # colex unranking, bits from the top
        while math.comb(c, i) > rr:
            c -= 1
        Q |= 2 << c
        rr -= math.comb(c, i)
        c -= 1
    allp = ((1 << k) - 1) << 1
    rest = allp & ~Q
    x = nth_bit(rest, xi)
    f, base = 0, xi * 720
    if q == 5:
        f = nth_bit(Q, fi)
        Q &= ~(1 << f)
        base += (f - 1) * math.factorial(k - 1)
    qs = [b for b in range(16) if Q >> b & 1]
    six = [b for b in range(16) if (rest & ~(1 << x)) >> b & 1]
    out = []
    for pattern in (orderings_table(qr) if qr else [[]]):
        rank, seq = base, ([f] if f else [])
        for i, (pos, earlier) in enumerate(pattern):
            p = qs[pos]
            digit = (p - 1) - earlier - (1 if f and f < p else 0)
            rank += digit * math.factorial(k - 1 - (1 if q == 5 else 0) - i)
            seq.append(p)
        out.append((rank, seq + [x] + six))
    return out


def set_units(k):
    q = k - 7
    return math.comb(k, q) * 7 * (5 if q == 5 else 1)


@pytest.mark.parametrize("k", [7, 8, 9, 10, 11])
def test_set_units_cover_every_rank_once(k):
    ranks = set()
    for u in range(set_units(k)):
        for rank, seq in set_unit_sequences(k, u):
            assert sorted(seq) == list(range(1, k + 1))
            assert rank == lex_rank(seq, k), (k, u, seq)
            assert rank % 720 == 0 and rank not in ranks
            ranks.add(rank)
    assert len(ranks) * 720 == math.factorial(k)


def test_set_units_twelve_picks_sampled():
    """k = 12: 27,720 units of 24 orderings; every 97th unit checked against the counted rank,
    and the unit count times the sequences per unit is 12!."""
    assert set_units(12) * 24 * 720 == math.factorial(12)
    seen = set()
    for u in range(0, set_units(12), 97):
        for rank, seq in set_unit_sequences(12, u):
            assert rank == lex_rank(seq, 12)
            assert rank not in seen
            seen.add(rank)


@pytest.mark.parametrize("k", [7, 8, 9])
def test_prefix_units_cover_every_rank_once(k):
    """Prefix unit u: the first k - 7 picks from u's factorial digits (radix k - i at
    position i), then part j takes the j-th of the other seven next; the part's first
    sequence has rank (7 u + j) x 720."""
    q = k - 7
    ranks = set()
    for u in range(math.factorial(k) // 5040):
        digits, v = [0] * q, u
        for i in range(q - 1, -1, -1):
            digits[i] = v % (k - i)
            v //= k - i
        avail = list(range(1, k + 1))
        prefix = []
        for d in digits:
            prefix.append(avail.pop(d))
        for j, x in enumerate(avail):
            seq = prefix + [x] + [p for p in avail if p != x]
            rank = (7 * u + j) * 720
            assert rank == lex_rank(seq, k)
            ranks.add(rank)
    assert len(ranks) * 720 == math.factorial(k)
