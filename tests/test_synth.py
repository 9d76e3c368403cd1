"""Input generators: the forked cell-average path equals the serial one, and the
periodised Gaussian pulse equals its 27-image sum written out."""
import numpy as np

import synth


def test_forked_cell_average_equals_serial():
    m = synth.hexprism_mesh(8, 0.2, 3)
    a = synth.cell_average(m, synth.gaussian3d, q=2)
    b = synth.cell_average(m, synth.gaussian3d, q=2, workers=3)
    assert np.abs(a - b).max() <= 1e-15


def test_gaussian_is_the_image_sum():
    p = np.random.default_rng(0).uniform(size=(500, 3))
    want = np.zeros(500)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for c in (-1, 0, 1):
                d = p - (np.array([0.5, 0.5, 0.5]) + np.array([a, b, c]))
                want += np.exp(-0.5 * (d * d).sum(axis=1) / 0.01)
    assert np.abs(synth.gaussian3d(p) - want).max() < 1e-14


def test_cell_average_of_a_linear_field_is_its_centroid_value():
    """A linear field's average is its value at the cell's centroid, which for a
    simplex is the vertex mean: check on a tetrahedral mesh of 5-tet hexes."""
    m = synth.tet_mesh(4, 0.15, 3)
    f = lambda p: 1.0 + 2.0 * p[:, 0] - 0.5 * p[:, 1] + 0.25 * p[:, 2]
    avg = synth.cell_average(m, f, q=2)
    ones = synth.cell_average(m, lambda p: np.ones(p.shape[0]), q=2)
    assert np.abs(ones - 1.0).max() < 1e-13
    # centroid from first moments of the coordinates
    xc = np.stack([synth.cell_average(m, lambda p, k=k: p[:, k], q=2) for k in range(3)], axis=1)
    assert np.abs(avg - f(xc)).max() < 1e-12


def test_blasius_profile_constants():
    """The Blasius solution behind the boundary-layer inputs: wall curvature
    f''(0) = 0.33206 and displacement eta - f -> 1.7208 (classical values), u rising
    from 0 at the wall to 1 outside the layer."""
    from synth import fields
    eta, f, fp, fpp, s = fields._blasius_table()
    assert abs(s - 0.33206) < 2e-5
    assert abs((eta[-1] - f[-1]) - 1.7208) < 2e-4
    uv = fields.blasius(np.array([[1.0, 0.0], [1.0, 0.02], [1.0, 0.4]]))
    assert uv[0, 0] == 0.0 and 0.0 < uv[1, 0] < 1.0 and abs(uv[2, 0] - 1.0) < 1e-9
