"""The carry-lookahead identity the multi-lane Montgomery code relies on.

With an operation sliced over T lanes, lane r generates a carry (bit G_r) or
propagates an incoming one (bit P_r: its slice is all ones), never both.  The
kernels take the carries into the lanes from one integer sum: the carry into
lane r is bit r of (G + (G | P)) xor G xor (G | P).  Here that identity is
checked against ripple-carry for every G, P pattern of 2, 4 and 8 lanes.
"""
import pytest


def lookahead(G, P):
    Y = G | P
    return (G + Y) ^ G ^ Y


def ripple(G, P, T):
    carries, c = 0, 0
    for r in range(T):
        carries |= c << r
        c = 1 if (G >> r) & 1 or ((P >> r) & 1 and c) else 0
    return carries | (c << T)


@pytest.mark.parametrize("T", [2, 4, 8])
def test_lookahead_equals_ripple(T):
    for G in range(1 << T):
        for P in range(1 << T):
            if G & P:
                continue                      # a lane cannot both generate and propagate
            assert lookahead(G, P) & ((1 << (T + 1)) - 1) == ripple(G, P, T), (G, P)
