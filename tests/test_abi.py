"""Host-side checks of the C ABI (no GPU needed): the library builds and
exports every function include/mamute.h declares; the checkpoint planner is
optimal and executable; the CFL bound matches the von Neumann analysis."""
import numpy as np
import pytest

from oracle import revolve as rref


@pytest.fixture(scope="module")
def lib():
    from paper_2502_12350_gb300 import build, mamute
    build.build()
    return mamute


def test_exports_every_declared_symbol(lib):
    names = lib.header_symbols()
    assert len(names) >= 10
    so = lib.load()
    for n in names:
        assert hasattr(so, n), n


def test_cfl_limit_matches_symbol(lib, oracle):
    c = oracle.fd_coeffs()
    th = np.linspace(0, np.pi, 400001)
    sym = -(c[0] + 2 * sum(c[j] * np.cos(j * th) for j in range(1, 5)))
    assert abs(lib.cfl_limit() - 2 / np.sqrt(3 * sym.max())) < 1e-8


def _simulate(nt, acts, slots):
    """Executes a plan symbolically: returns the reversal order and the
    forward-step count, checking every restore / reverse sees the right
    state."""
    cur = 0
    store = {}
    order = []
    nfwd = 0
    for kind, a, b in acts:
        if kind == 0:
            assert cur == a and b > a
            nfwd += b - a
            cur = b
        elif kind == 1:
            assert 0 <= a < slots and cur == b
            store[a] = b
        elif kind == 2:
            assert (a == -1 and b == 0) or store.get(a) == b
            cur = b
        elif kind == 3:
            assert cur == a
            order.append(a)
    return order, nfwd + 1


@pytest.mark.parametrize("nt,s", [(1, 0), (2, 0), (7, 0), (10, 1), (37, 3), (60, 6), (100, 2),
                                  (500, 16), (2000, 64), (4000, 8)])
def test_revolve_plan_is_optimal_and_valid(lib, nt, s):
    nf, acts = lib.revolve_plan(nt, s)
    order, counted = _simulate(nt, acts, s)
    assert order == list(range(nt - 1, -1, -1))
    assert counted == nf
    assert nf == rref.binomial_cost(nt, min(s, nt)) + 1
    if nt <= 60 and s <= 6:
        assert nf == rref.dp_cost(nt, s) + 1


def test_revolve_rejects_bad_arguments(lib):
    with pytest.raises(lib.MamuteError):
        lib.revolve_plan(0, 3)
