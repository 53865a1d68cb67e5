"""Pins of the Rao-Blackwellised estimator (oracle/rb.py) against what the
mathematics fixes: its exact expectation over all spanning trees of G*
(enumerated) equals Omega[v, v] from the dense inverse, its exact variance
is at most the indicator's, leaves take the closed form 1 / (1 + alpha
d_w(v)), and sampled trees give an unbiased average."""
import numpy as np
import pytest

import synth
from oracle import dense, native, rb
from oracle.enumerate import spanning_trees


def _tiny_graphs():
    return [
        ("path4", synth.path(4), 0.7),
        ("K4w", synth.complete(4, weight=1.5), 1.3),
        ("two_parts", synth.from_edges(5, [0, 1, 3], [1, 2, 4], [2.0, 0.5, 3.0]), 0.4),
        ("cycle5", synth.cycle(5), 2.0),
        ("star5", synth.star(5), 0.9),
        ("isolated", synth.from_edges(4, [0], [1], None), 1.0),
    ]


@pytest.mark.parametrize("name,g,alpha", _tiny_graphs(), ids=[t[0] for t in _tiny_graphs()])
def test_exact_expectation_and_variance_by_enumeration(name, g, alpha):
    om = np.diag(dense.forest_matrix(g, alpha))
    total = 0.0
    m1 = np.zeros(g.n)
    m2 = np.zeros(g.n)
    ind1 = np.zeros(g.n)
    for par, wt in spanning_trees(g, alpha):
        val = rb.rb_values(g, alpha, par)
        total += wt
        m1 += wt * val
        m2 += wt * val * val
        ind1 += wt * (par == g.n)
    m1 /= total
    m2 /= total
    ind1 /= total
    np.testing.assert_allclose(ind1, om, rtol=0, atol=1e-12)  # Prop. 1 on the same enumeration
    np.testing.assert_allclose(m1, om, rtol=0, atol=1e-12)    # unbiased
    var_rb = m2 - m1 * m1
    assert np.all(var_rb <= om * (1 - om) + 1e-12)             # Rao-Blackwell


def test_leaf_and_root_closed_forms():
    g = synth.barabasi_albert(60, 2, 3, weighted=True)
    alpha = 0.8
    out = native.wilson(g, alpha, seed=4, tau=5, want_parents=True)
    dw = np.array([g.w[g.rowptr[v]:g.rowptr[v + 1]].astype(np.float64).sum() for v in range(g.n)])
    for par in out["parents"]:
        val = rb.rb_values(g, alpha, par)
        has_child = np.zeros(g.n, bool)
        has_child[par[par < g.n]] = True
        leaves = ~has_child
        np.testing.assert_allclose(val[leaves], 1.0 / (1.0 + alpha * dw[leaves]), rtol=1e-15)
        tin, size = rb.subtree_intervals(par, g.n)
        assert np.sum(size[par == g.n]) == g.n  # the roots' subtrees cover V
        assert np.all(val > 0) and np.all(val <= 1)


def test_fixed_point_rounding_is_exact():
    v = np.array([1.0, 0.5, 1.0 / 3.0, 2.0 ** -48, 0.0])
    q = rb.to_fixed(v)
    assert q[0] == 1 << 48 and q[1] == 1 << 47 and q[3] == 1 and q[4] == 0
    assert q[2] == round((1 << 48) / 3)


def test_sampled_average_is_unbiased_and_tighter_than_frequency():
    g = synth.erdos_renyi(120, 5, 8)
    alpha, tau = 1.0, 400
    om = np.diag(dense.forest_matrix(g, alpha))
    out = native.wilson(g, alpha, seed=11, tau=tau, want_parents=True)
    est = rb.diag_from_fixed(rb.accumulate(g, alpha, out["parents"]), tau)
    plain = out["R"] / tau
    # unbiased: the standardised mean error over vertices is small
    err_rb = est - om
    assert abs(err_rb.mean()) < 4 * err_rb.std() / np.sqrt(g.n) + 1e-3
    # and much tighter than the frequency on the same trees
    assert np.sqrt(np.mean(err_rb ** 2)) < 0.5 * np.sqrt(np.mean((plain - om) ** 2))
