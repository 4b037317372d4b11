"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check
that at least one pin fails for each: the pins are not blind to them."""
import importlib.util
import os
import types

import pytest

import oracle_pins as P

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "bse_oracle.py")

MUTANTS = {
    "exchange_factor_1": ("2.0 * gamma_x * V - gamma_c * Wrr", "1.0 * gamma_x * V - gamma_c * Wrr"),
    "exchange_conj_second": ("((np.conj(m) * v_bar[None, :]) @ m.T)", "((m * v_bar[None, :]) @ np.conj(m).T)"),
    "direct_sign": ("+ 2.0 * gamma_x * V - gamma_c * Wrr", "+ 2.0 * gamma_x * V + gamma_c * Wrr"),
    "wrr_vv_transposed": ('np.einsum("avg,cdg->acvd", np.conj(m_vv[k, kp])',
                          'np.einsum("vag,cdg->acvd", np.conj(m_vv[k, kp])'),
    "wrr_cc_transposed": ('np.einsum("gh,cdh->cdg", wq, m_cc[k, kp]', 'np.einsum("gh,dch->cdg", wq, m_cc[k, kp]'),
    "wrr_w_transposed": ('np.einsum("gh,cdh->cdg", wq,', 'np.einsum("hg,cdh->cdg", wq,'),
    "wrr_conj_on_cc": ('np.conj(m_vv[k, kp]), inner', 'm_vv[k, kp], np.conj(inner)'),
    "wrr_qplus": ("wq = w[q_minus[k, kp]]", "wq = w[q_minus[kp, k]]"),
    "wra_no_pair_swap": ("first = np.conj(n_vc[kp, k])", "first = np.conj(n_vc[k, kp])"),
    "wra_sign": ("B = 2.0 * gamma_x * V - gamma_c * Wra", "B = 2.0 * gamma_x * V + gamma_c * Wra"),
    "wra_conj_on_second": ("first = np.conj(n_vc[kp, k])          # [v', c, G]\n"
                           "            second = n_vc[k, kp]",
                           "first = n_vc[kp, k]          # [v', c, G]\n"
                           "            second = np.conj(n_vc[k, kp])"),
    "wra_w_transposed": ('inner = np.einsum("gh,vyh->vyg", wq, second',
                         'inner = np.einsum("hg,vyh->vyg", wq, second'),
    "kappa_no_nk": ("HARTREE_EV / (nk * omega_cell)", "HARTREE_EV / omega_cell"),
    "energy_sign": ("e[k, v, c] = e_c[k, c] - e_v[k, v]", "e[k, v, c] = e_v[k, v] - e_c[k, c]"),
    "xpy_power": ("xpy = (r @ z) / np.sqrt(e)[None, :]", "xpy = (r @ z) * np.sqrt(e)[None, :]"),
    "reduce_order": ("s = r @ (A + B) @ r", "s = r @ (A - B) @ r"),
    "osc_no_vc": ("np.conj(rho)) / np.sqrt(vc)", "np.conj(rho))"),
    "eps_antiresonant_sign": ("1.0 / (-w - e - 1j * delta)", "1.0 / (w + e + 1j * delta)"),
    "eps_no_hartree": ("c_q * HARTREE_EV * np.sum", "c_q * np.sum"),
}


def _mutant(old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    mod = types.ModuleType("bse_oracle_mutant")
    exec(compile(src.replace(old, new), "bse_oracle_mutant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    mod = _mutant(*MUTANTS[name])
    caught = []
    for pin in P.ALL_PINS:
        try:
            pin(mod)
        except (AssertionError, Exception) as exc:   # LinAlgError counts as caught too
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"
