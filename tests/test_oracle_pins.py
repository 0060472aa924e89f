"""CPU-only pins of the oracle (no GPU): golden cases, brute force, invariants, closed
forms, adjoint and error codes.  See tests/pins.py for what each check compares."""
import pytest

import oracle
import pins
from paper_2309_07337_gb300 import patterns as pt


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(lib, check):
    check(lib)


def test_closed_form_config1(lib):
    """2D 5-point halo, 256^2 grid over 4x4 ranks, 4 ranks per node: every count follows
    from the geometry (4 ranks with 2 neighbours, 8 with 3, 4 with 4; 64-point edges)."""
    st = oracle.locality_stats(pt.config1(), lib=lib)
    assert st["E"] == 48 and st["V"] == 48 * 64
    assert st["V_direct"] == 1536 and st["V_inter"] == 1536
    assert st["msgs_inter"] == 24 and st["node_pairs"] == 6 and st["U"] == 1536


@pytest.mark.slow
def test_closed_form_config5(lib):
    """512^3 27-point stencil over 16^3 ranks, 64 per node: the oracle's counts equal the
    geometric recount (per-direction products and boundary-type unions)."""
    p = pt.config5()
    want = pins.stencil_counts((16, 16, 16), (32, 32, 32), 64, "all")
    st = oracle.locality_stats(pins.bytes1(p), lib=lib)
    for k, v in want.items():
        assert st[k] == v, (k, st[k], v)
    assert st["V"] == 25_002_360 and st["E"] == 93_240
    assert st["V_direct"] == 14_524_416 and st["V_inter"] == 10_477_944
    assert st["msgs_inter"] == 67_896 and st["node_pairs"] == 396 and st["U"] == 9_529_344
