"""The Eq. 5 similarity study (Sec. 3.2-3.4) end to end on a 4^3 = 64 signal grid: features
through the library (Eq. 4 transform, time average, mu-log), K-NN regression and Isomap run,
and give finite results; carrier frequency, the parameter every representation recovers in the
paper, is regressed within 25 % for most examples."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build, manifold
    build.build()
    torch.cuda.set_device(0)
    return manifold


def test_small_grid_study(M):
    res = M.run(count=4, K=8)
    assert res["signals"] == 64
    for name in ("f_c", "f_m", "gamma"):
        r = res["knn_error_ratio"][name]
        assert np.isfinite(r["median"]) and r["p10"] <= r["median"] <= r["p90"]
        assert 0.0 <= res["isomap_alignment"][name]["rho"] <= 1.0
    assert res["knn_error_ratio"]["f_c"]["within_0.75_1.5"] > 0.5
