"""Seeded input generators (no method arithmetic): layouts they promise."""
import numpy as np

from paper_2310_01881_gb300 import scenes as S


def test_with_biases_touches_exactly_the_bias_entries():
    width, hidden, lx, ld = 32, 3, 10, 4
    P0 = S.xavier_weights(1, np.array([2.0, 0.5]), width, hidden, lx, ld)
    P = S.with_biases(P0, 1, width, hidden, lx, ld, scale=0.25)
    per = S.params_per_leaf(width, hidden, lx, ld)
    k0 = S.mlp_input_width(lx, ld)
    is_bias = np.zeros(per, bool)
    off = 0
    for fi, fo in [(k0, width)] + [(width, width)] * (hidden - 1) + [(width, 4)]:
        off += fi * fo
        is_bias[off:off + fo] = True
        off += fo
    assert off == per
    changed = (P != P0).reshape(-1, per)
    assert not changed[:, ~is_bias].any()
    assert changed[:, is_bias].mean() > 0.99
    delta = (P - P0).reshape(-1, per)[:, is_bias]
    assert np.abs(delta).max() <= 0.25
