"""Host-side logic of the efficiency / fake-rate study (no GPU): the matching
of reconstructed tracks to reference lines, tan theta and its binning, the
reference selection, and the planted-line truth the generator records."""
import numpy as np

from paper_1311_5334_gb300 import efficiency as E
from paper_1311_5334_gb300 import synth


def _ref(p, d):
    d = np.asarray(d, dtype=float)
    return np.concatenate([p, d / np.linalg.norm(d)])


def test_match_tolerances():
    truth = np.array([_ref([10, 20, 5], [1, 0, 1]), _ref([100, 100, 25], [0, 0, 1])])
    d0 = np.array([1, 0, 1]) / np.sqrt(2)
    # on the line, any point along it, either orientation
    assert E.match(truth, [[10 + 7, 20, 5 + 7]], [d0]).tolist() == [True, False]
    assert E.match(truth, [[10, 20, 5]], [-d0]).tolist() == [True, False]
    # 0.9 um off the line: matched; 1.1 um: not
    n = np.array([1, 0, -1]) / np.sqrt(2)
    assert E.match(truth, [np.array([10, 20, 5]) + 0.9 * n], [d0])[0]
    assert not E.match(truth, [np.array([10, 20, 5]) + 1.1 * n], [d0])[0]
    # direction 0.02 rad off: matched; 0.05 rad: not
    for ang, ok in [(0.02, True), (0.05, False)]:
        u = [np.sin(ang), 0, np.cos(ang)]
        assert E.match(truth, [[100, 100, 25]], [u])[1] == ok
    assert E.match(truth, np.zeros((0, 3)), np.zeros((0, 3))).tolist() == [False, False]


def test_tan_theta_and_bins():
    t = E.tan_theta([[0, 0, 1], [1, 0, 1], [3, 4, 5], [1, 0, 0]])
    assert np.allclose(t[:3], [0, 1, 1]) and np.isinf(t[3])
    rows = E.binned(np.array([True, False, True, True]), np.array([0.1, 0.7, 0.8, np.inf]))
    assert [(r[2], r[3]) for r in rows] == [(1, 1.0), (2, 0.5), (0, None), (0, None), (1, 1.0)]


def test_generator_truth_lines_pass_through_their_grains():
    v = synth.make_view(3, n_fog=100, n_through=12, n_short=3)
    assert v.truth.shape == (15, 6)
    for k in range(v.n_tracks):
        g = v.xyz[v.label == k] / synth.UM
        p, d = v.truth[k, :3], v.truth[k, 3:]
        assert abs(np.linalg.norm(d) - 1) < 1e-12
        rel = g - p
        dist = np.linalg.norm(rel - np.outer(rel @ d, d), axis=1)
        assert (dist < 2.0).all()   # jitter 0.05 / 0.3 um, clamping at the faces
    ref = E.reference_mask(v, 10)
    assert ref.shape == (15,) and ref.dtype == bool
