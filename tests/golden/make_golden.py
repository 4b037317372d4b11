"""Writes tests/golden/c1_oracle.json from the CPU oracle only.

The 2x2x2-grid, 2x2-band, NG = 59 problem (seed 20190411) is built, reduced
and solved by oracle/bse_oracle.py; the exciton energies, oscillator
strengths and eps_M on every 50th frequency are stored so that later changes
to the oracle's arithmetic show up as a diff.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import bse_inputs as bi  # noqa: E402
from oracle import bse_oracle as O  # noqa: E402


def main():
    p = bi.make_problem("c1")
    A, B = O.build_A_B(p)
    e, osc, eps = O.spectrum(A, B, p)
    et, _, _ = O.spectrum(A, B, p, coupling=False)
    out = {
        "source": "oracle/bse_oracle.py on bse_inputs.make_problem('c1'), seed 20190411",
        "E_full_eV": e.tolist(),
        "E_tda_eV": sorted(et.tolist()),
        "osc_full": osc.tolist(),
        "omega_idx": list(range(0, len(p["omega"]), 50)),
        "eps_re": eps.real[::50].tolist(),
        "eps_im": eps.imag[::50].tolist(),
        "A_fro": float((abs(A) ** 2).sum() ** 0.5),
        "B_fro": float((abs(B) ** 2).sum() ** 0.5),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
