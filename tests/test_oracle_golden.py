"""The oracle against hand-derived 2x2 examples (tests/golden/n2_worked_examples.json).

The paper prints no worked example with values; these cases were worked out
by hand from Eq. 3 (with F_c of Sec. II), Eq. 5, Eq. 4 and Eq. 6, and each
case in the fixture carries its derivation."""
import json
import os

import numpy as np
import pytest

from oracle import dm

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "n2_worked_examples.json")) as f:
    GOLDEN = json.load(f)


def cx(a):
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("case", GOLDEN["cases"], ids=[c["name"] for c in GOLDEN["cases"]])
def test_hand_derived_example(case):
    probe = cx(case["probe"])
    obj = cx(case["object"])
    inten = np.asarray(case["intensity"], np.float64)[None]
    pos = np.array([[0, 0]], np.int32)
    psi = dm.init_exit_waves(probe, obj, pos)
    psi1, p1, o1, m = dm.dm_iteration(psi, probe, obj, pos, inten, beta=case["beta"],
                                       delta_rel=case["delta_rel"])
    np.testing.assert_allclose(psi1[0], cx(case["psi_out"]), atol=1e-15)
    np.testing.assert_allclose(o1, cx(case["object_out"]), atol=1e-15)
    np.testing.assert_allclose(p1, cx(case["probe_out"]), atol=1e-15)
    assert m["eps_obj"] == pytest.approx(case["eps_obj"], rel=1e-14)
    assert m["fourier_err"] == pytest.approx(case["fourier_err"], rel=1e-14)
    np.testing.assert_allclose(m["eps_probe"], case["eps_probe"], atol=1e-15)
