"""Host logic of the inverse-rendering loop: object labels and vertex
normals used to set up the rigid-object variant and to split the vertex
error into its normal and tangential parts (CPU only)."""
import numpy as np

from paper_1904_12228_gb300 import inverse
from paper_1904_12228_gb300 import scenegen as sg


def test_components_of_the_procedural_scene():
    sc = sg.procedural(1237, n_target=20_000, width=32, height=32)
    lab = inverse.components(sc.verts, sc.tris)
    assert lab.shape == (len(sc.verts),)
    sizes = np.bincount(lab)
    # objects: icospheres (642 vertices), boxes (6 sheets of 5x5 welded at
    # their borders: 150 vertices), the ground and the two lights (4 each)
    assert set(sizes.tolist()) <= {642, 150, 4}
    assert (sizes == 4).sum() == 3
    n_tri = (sizes == 642).sum() * 1280 + (sizes == 150).sum() * 192 + 3 * 2
    assert n_tri == len(sc.tris)
    # every triangle lies in one object
    t = np.asarray(sc.tris)
    assert np.all(lab[t[:, 0]] == lab[t[:, 1]]) and np.all(lab[t[:, 0]] == lab[t[:, 2]])


def test_vertex_normals_of_a_box_point_outward():
    v, f = sg.subdivided_box()
    n = inverse.vertex_normals(v, f)
    c = v.mean(0)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0)
    # each sheet is flat: the normal of a vertex inside a face is the face's axis
    assert np.all(((v - c) * n).sum(1) > 0)
