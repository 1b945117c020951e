"""The oracle reproduces its committed regression fixtures (tests/golden)."""
import json
import os

import numpy as np
import pytest

import oracle
from tests.golden.make_golden import cases

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name,model,system", list(cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_oracle_matches_golden(name, model, system):
    with open(os.path.join(HERE, f"{name}.json")) as f:
        g = json.load(f)
    r = oracle.compute(model, system)
    assert r.energy == pytest.approx(g["energy"], rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(r.virial_total, g["virial_total"], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(r.site_energy[:8], g["site_energy_first8"], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(r.force[:, :8], g["force_first8"], rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(r.virial[:, :4], g["virial_first4"], rtol=1e-10, atol=1e-13)
