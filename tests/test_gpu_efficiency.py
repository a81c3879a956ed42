"""The efficiency / fake-rate study on the GPU path (Section 3 analogue): on
clean synthetic views nearly every reference track is found, tracks of another
view (displaced data) almost never match, and fog alone gives few tracks."""
import pytest

pytestmark = pytest.mark.gpu


def test_small_study():
    from paper_1311_5334_gb300 import efficiency as E
    from paper_1311_5334_gb300 import et
    with et.Context(0) as ctx:
        rep = E.study(ctx, n_views=8, seed=5, n_fog=10000, n_tracks=40)
    assert rep["references"] > 200
    assert rep["efficiency"] >= 0.95
    assert rep["displaced_fake_rate"] <= 0.02
    assert rep["fog_only_tracks_per_view"] <= 1.0
    assert sum(b["n"] for b in rep["efficiency_by_tan_theta"]) == rep["references"]
