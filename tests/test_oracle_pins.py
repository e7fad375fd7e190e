"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import pytest

import _pins


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin()


def test_alg1_equals_counting_on_config_sized_soup():
    """Literal Algorithm 1 (markers, scans, GlobalCoords, stable sort, RLE)
    and the counting placement agree on a 100k-triangle uniform soup."""
    import numpy as np
    import oracle
    import scenes
    s = scenes.uniform_soup()
    a = oracle.build_grid(s.verts, s.tris, s.lam, method="alg1")
    c = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
    assert a.NO == c.NO and np.array_equal(a.G, c.G) and np.array_equal(a.refs, c.refs)


def test_empty_scene():
    import numpy as np
    import oracle
    g = oracle.build_grid(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), 4.0)
    assert g.NO == 0 and list(g.G) == [0, 0] and g.refs.shape == (0,)
