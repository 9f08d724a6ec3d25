"""Reference costs for binomial checkpointing (TEST INFRASTRUCTURE ONLY).

The paper's optimal checkpointing (Sec. 2.1, ManageWavefieldChk with the
Checkpoint class; Griewank and Walther's revolve) stores selected forward
states and recomputes the rest.  Convention used throughout: reversing l
steps starting from a state that is held and restorable at will, with s
additional free snapshot slots, costs C(l, s) forward steps.

* ``dp_cost`` is the brute-force minimum over every split of the recursive
  schedule (advance j steps, store, reverse the right part with s-1 slots,
  restore, reverse the left part with s slots).
* ``binomial_cost`` is the closed form of Griewank and Walther for s+1
  snapshots (the held start state counts as one): with beta(a, t) =
  (a+t)! / (a! t!) and t the least integer such that beta(s+1, t) >= l,
  C(l, s) = t l - beta(s+2, t-1).
"""
from functools import lru_cache
from math import comb


@lru_cache(maxsize=None)
def dp_cost(l: int, s: int) -> int:
    if l <= 1:
        return 0
    if s == 0:
        return l * (l - 1) // 2
    return min(j + dp_cost(l - j, s - 1) + dp_cost(j, s) for j in range(1, l))


def binomial_cost(l: int, s: int) -> int:
    if l <= 1:
        return 0
    t = 0
    while comb(s + 1 + t, t) < l:
        t += 1
    return t * l - comb(s + 2 + t - 1, t - 1)
