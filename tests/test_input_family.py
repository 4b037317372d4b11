"""A family of problems along Q (bse_inputs.make_problem(draws_of=j)) for
exciton-dispersion checks: every random array comes from the streams of one
Q index, so only v(G+Q), c_Q and Q itself change along the line; without
draws_of nothing changes from the default recipe."""
import numpy as np

import bse_inputs as bi

CFG = bi.BSEConfig("family", grid=2, nv=2, nc=2, ng=27, q_abs=(0.1, 0.3, 0.5), w_scale=0.1)
RANDOM = ("e_v", "e_c", "m_x", "m_vv", "m_cc", "n_vc", "w")


def test_family_shares_random_arrays():
    ps = [bi.make_problem(CFG, q_index=q, draws_of=0) for q in range(3)]
    for key in RANDOM:
        for p in ps[1:]:
            assert np.array_equal(p[key], ps[0][key]), key
    # v(G+Q) follows Q
    assert not np.allclose(ps[0]["v_bar"], ps[2]["v_bar"])
    assert ps[0]["q_vec"][0] == 0.1 and ps[2]["q_vec"][0] == 0.5


def test_default_draws_unchanged():
    a = bi.make_problem(CFG, q_index=1)
    b = bi.make_problem(CFG, q_index=1, draws_of=1)
    c = bi.make_problem(CFG, q_index=1, draws_of=0)
    for key in RANDOM:
        assert np.array_equal(a[key], b[key]), key
    assert not np.array_equal(a["m_x"], c["m_x"])
