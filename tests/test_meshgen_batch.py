"""The batched input (disjoint union of cases) is a faithful copy of its cases:
the oracle's operators on the union equal those on each case alone."""
import numpy as np

import oracle as O
from paper_2603_15920_b300 import meshgen as mg


def test_batch_union_reproduces_each_case():
    ms = [mg.kuhn_cube(3, 0.2, 1), mg.shuffle(mg.kuhn_cube(4, 0.2, 2), 3), mg.channel_2d(8, 4, seed=1)]
    u, cs = mg.batch(ms)
    assert list(cs) == [0] + list(np.cumsum([m.n_cells for m in ms]))
    assert u.n_internal == sum(m.n_internal for m in ms)
    assert u.n_patches == sum(m.n_patches for m in ms)
    ou = O.OMesh.from_mesh(u)
    rng = np.random.default_rng(0)
    phi = [rng.normal(size=m.n_cells) for m in ms]
    phib = [rng.normal(size=m.n_boundary) for m in ms]
    gu = O.grad_gauss(ou, ou.bc_U(), np.concatenate(phi)[None], np.concatenate(phib)[None])
    for k, m in enumerate(ms):
        om = O.OMesh.from_mesh(m)
        g = O.grad_gauss(om, om.bc_U(), phi[k][None], phib[k][None])
        np.testing.assert_array_equal(gu[..., cs[k]:cs[k + 1]], g)
