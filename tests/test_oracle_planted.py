"""Each planted mistake in the oracle (a dropped term, a wrong sign, a wrong
base, a transposed operand, a wrong rounding) must be caught by some pin."""
import pytest

import oracle
import oracle_pins as P

PLANTS = {1: "texp drops the x1 term", 2: "tlog correction has the wrong sign",
          3: "tlog1p correction uses the wrong base", 4: "main part rounded toward zero",
          5: "tmul drops a cross term", 6: "tadd error term with transposed operands",
          7: "texp rounds x0 + x1 to double first", 8: "chain product drops the operand tail",
          9: "chain condition sum ignores the gains", 10: "float main part rounded toward zero"}


@pytest.mark.parametrize("k", sorted(PLANTS), ids=lambda k: PLANTS[k].replace(" ", "_"))
def test_planted_mistake_is_caught(k):
    path = oracle.build(force=True, defines=(f"TFO_PLANT={k}",), name=f"libtforacle_plant{k}.so")
    lib = oracle.load(path)
    caught = []
    for pin in P.ALL_PINS:
        if pin(lib):
            caught.append(pin.__name__)
            break
    assert caught, f"planted mistake {k} ({PLANTS[k]}) passed every pin"


PY_PLANTS = {11: "re-decision shifts the deviation the wrong way", 12: "re-decision rounds toward zero"}


@pytest.mark.parametrize("k", sorted(PY_PLANTS), ids=lambda k: PY_PLANTS[k].replace(" ", "_"))
def test_planted_redecision_mistake_is_caught(k, monkeypatch):
    """Mistakes planted in the oracle's decimal re-decision of main parts near a
    rounding midpoint: the near-midpoint pin family catches them, and it is the
    only family that reaches that code with a main part to change."""
    lib = oracle.load()
    monkeypatch.setattr(oracle, "_PLANT", k)
    caught = [pin.__name__ for pin in P.ALL_PINS if pin(lib)]
    assert caught == ["pin_near_midpoint"], f"planted mistake {k} ({PY_PLANTS[k]}) caught by {caught}"
