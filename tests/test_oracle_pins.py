"""The CPU oracle against facts fixed by the paper and by mathematics."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    assert pin() == []


def test_fig1_printed_facts_are_all_checked():
    names, rows, facts = pins.load_fig1()
    assert names == ["A", "B", "C", "D"]
    kinds = sorted({f[0] for f in facts})
    assert kinds == ["absent", "inline", "overlap", "size"]
