"""The oracle against its pins (CPU only)."""
import numpy as np
import pytest

import oracle_pins as P
from oracle import bse_oracle as O


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(O)


def test_hermitian_and_pd_c1():
    import bse_inputs as bi
    p = bi.make_problem("c1")
    A, B = O.build_A_B(p)
    assert np.abs(A - A.conj().T).max() < 1e-13
    assert np.abs(B - B.conj().T).max() < 1e-13
    assert np.linalg.eigvalsh(A - B).min() > 0 and np.linalg.eigvalsh(A + B).min() > 0


def test_golden_c1():
    """The oracle against its stored c1 outputs (written by tests/golden/make_golden.py)."""
    import json
    import os
    import bse_inputs as bi
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_oracle.json")))
    p = bi.make_problem("c1")
    A, B = O.build_A_B(p)
    e, osc, eps = O.spectrum(A, B, p)
    assert np.allclose(e, g["E_full_eV"], rtol=1e-12)
    assert np.allclose(osc, g["osc_full"], rtol=1e-9, atol=1e-15)
    assert np.allclose(eps.real[::50], g["eps_re"], rtol=1e-10)
    assert np.allclose(eps.imag[::50], g["eps_im"], rtol=1e-10, atol=1e-12)


def test_spin_factor_table():
    """Table tab:approx: the IP row removes all interaction, RPA keeps exchange only."""
    import os
    import bse_inputs as bi
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "spin_factors.txt")):
        if line.strip() and not line.startswith("#"):
            name, gx, gc = line.split()
            rows[name] = (float(gx), float(gc))
    p = bi.make_problem("c1")
    e = O.transition_energies(p["e_v"], p["e_c"])
    A, B = O.build_A_B(p, *rows["IP"])
    assert np.allclose(A, np.diag(e)) and np.abs(B).max() == 0.0
    A_t, B_t = O.build_A_B(p, *rows["triplet"])
    A_r, B_r = O.build_A_B(p, *rows["RPA"])
    A_s, B_s = O.build_A_B(p, *rows["singlet"])
    # singlet = triplet + exchange part of RPA
    assert np.allclose(A_s, A_t + (A_r - np.diag(e)), atol=1e-13)
    assert np.allclose(B_s, B_t + B_r, atol=1e-13)
