"""The library's scoring (host C++ in libgeonet.so) against the oracle's
(pinned to scikit-learn in test_estimator_oracle.py); runs without a GPU."""
import numpy as np
import pytest

from oracle import estimator as est
from paper_0908_3934_b300 import build, geonet


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_auroc_f1_and_threshold_match_the_oracle(seed):
    rng = np.random.default_rng(seed)
    n = 5000
    s = rng.normal(size=n).astype(np.float32)
    if seed == 2:
        s = np.round(s, 1)  # heavy ties
    y = (s + rng.normal(size=n) > 0).astype(np.uint8)
    assert geonet.gn_score_auroc(s, y) == pytest.approx(est.auroc(s, y), abs=1e-12)
    for thr in (-1.0, 0.0, 0.5):
        assert geonet.gn_score_f1(s, y, thr) == pytest.approx(est.f1_at(s, y, thr), abs=1e-12)
    t_lib, f_lib = geonet.gn_score_best_f1(s, y)
    t_orc, f_orc = est.best_threshold(s, y)
    assert f_lib == pytest.approx(f_orc, abs=1e-12) and t_lib == pytest.approx(t_orc)


def test_scoring_special_cases():
    assert geonet.gn_score_auroc(np.array([1, 2, 3, 4], np.float32), [0, 0, 1, 1]) == 1.0
    assert geonet.gn_score_auroc(np.array([4, 3, 2, 1], np.float32), [0, 0, 1, 1]) == 0.0
    assert geonet.gn_score_auroc(np.array([5, 5, 5, 5], np.float32), [0, 1, 0, 1]) == 0.5
    assert np.isnan(geonet.gn_score_auroc(np.array([1, 2], np.float32), [1, 1]))
    with pytest.raises(geonet.GeonetError):
        geonet.gn_score_auroc(np.array([1, np.nan], np.float32), [0, 1])
