"""Pin of the checkpointing reference costs: the brute-force minimum over
all recursive split schedules equals Griewank and Walther's binomial closed
form (revolve, the optimal checkpointing of Sec. 2.1)."""
from oracle import revolve


def test_dp_equals_binomial_closed_form():
    for s in range(0, 7):
        for l in range(1, 61):
            assert revolve.dp_cost(l, s) == revolve.binomial_cost(l, s), (l, s)


def test_known_small_values():
    # one free slot: l=4 needs advance 2, store, (reverse 2 with 0 slots: 1),
    # restore, reverse 2 with 1 slot: 1  -> 4
    assert revolve.dp_cost(4, 1) == 4
    assert revolve.dp_cost(3, 0) == 3
    assert revolve.dp_cost(10, 9) == 9
