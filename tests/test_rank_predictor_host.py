"""Host side of the rank predictor: parameter layout and the model file."""
import numpy as np

from paper_2603_09381_gb300 import rank_predictor as rp


def test_parameter_layout_and_initialisation():
    th = rp.init_params(seed=3)
    assert th.dtype == np.float32 and th.size == rp.NPARAM == 64 * 8 + 64 + 64 * 64 + 64 + 2 * 64 + 2
    b1 = th[512:576]
    b2 = th[576 + 4096:576 + 4096 + 64]
    b3 = th[-2:]
    assert not b1.any() and not b2.any() and not b3.any()          # zero biases
    W2 = th[576:576 + 4096]
    assert 0.5 < np.std(W2) * 8 < 2.0                               # ~ N(0, 1/64)
    assert np.array_equal(th, rp.init_params(seed=3)) and not np.array_equal(th, rp.init_params(seed=4))


def test_committed_model_file():
    m = rp.load_model()
    assert m is not None and m.dtype == np.float32 and m.size == rp.NPARAM + 16
    assert np.all(np.isfinite(m))
    assert np.all(m[-8:] > 0)                                       # feature scales


def test_save_and_load_round_trip(tmp_path):
    m = np.arange(rp.NPARAM + 16, dtype=np.float64) * 0.5
    p = str(tmp_path / "sub" / "model.npy")
    rp.save(m, p)
    back = rp.load_model(p)
    assert back.dtype == np.float32 and np.array_equal(back, m.astype(np.float32))
    assert rp.load_model(str(tmp_path / "missing.npy")) is None
