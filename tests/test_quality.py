"""DVH figures from histogram counts (host arithmetic), by hand: 100 voxels,
10 bins of width 0.1 over [0, 1)."""
import numpy as np
import pytest

from paper_1005_4396_b300 import quality


def test_dvh_metrics_by_hand():
    c = np.zeros((1, 10), np.int64)
    c[0, 2] = 10   # doses in [0.2, 0.3)
    c[0, 9] = 90   # doses in [0.9, 1.0) or above
    m = quality.dvh_metrics(c, 1.0, ["target"], rx=0.9)["target"]
    assert m["voxels"] == 100
    assert m["mean"] == pytest.approx(0.1 * 0.25 + 0.9 * 0.95)
    # 95% of the volume receives at least 0.2 (bins 2..9 hold 100%); 5% at least 0.9
    assert m["D95"] == pytest.approx(0.2) and m["D5"] == pytest.approx(0.9)
    assert m["V_rx"] == pytest.approx(0.9)
    assert quality.dvh_metrics(np.zeros((1, 10), np.int64), 1.0, ["empty"], rx=0.5) == {}
