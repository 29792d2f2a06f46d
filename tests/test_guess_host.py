"""Host logic of the learned guess (paper_1208_2643_gb300/guess.py) on the CPU: the
parameter blob's layout, its initialisation, the packaged model and the input and
target scales."""
import numpy as np
import pytest

from paper_1208_2643_gb300 import guess

torch = pytest.importorskip("torch")


def test_blob_layout_covers_every_parameter_once():
    """Four normalisation scales, then per layer 9*cin*cout weights and cout biases, in
    order, with nothing left over (3-32-32-32-32-1: 28 933 parameters)."""
    assert guess.PARAM_COUNT == 28933
    off = 4
    for (ws, bs), (ci, co) in zip(guess.layer_slices(), guess.LAYERS):
        assert (ws.start, ws.stop) == (off, off + 9 * ci * co)
        assert (bs.start, bs.stop) == (ws.stop, ws.stop + co)
        off = bs.stop
    assert off == guess.PARAM_COUNT


def test_initial_network_leaves_the_extrapolation_unchanged():
    """Unit scales, zero biases, He-scaled hidden weights, and a zero last layer, so the
    untrained network predicts a zero correction."""
    b = guess.init_params(3)
    assert b.dtype == np.float32 and b.size == guess.PARAM_COUNT
    np.testing.assert_array_equal(b[:4], 1.0)
    sl = guess.layer_slices()
    for i, ((ws, bs), (ci, co)) in enumerate(zip(sl, guess.LAYERS)):
        np.testing.assert_array_equal(b[bs], 0.0)
        if i < 4:
            assert abs(float(np.std(b[ws])) / np.sqrt(2.0 / (9 * ci)) - 1.0) < 0.15
        else:
            np.testing.assert_array_equal(b[ws], 0.0)
    np.testing.assert_array_equal(guess.init_params(3), b)


def test_packaged_model_has_the_blob_layout():
    m = guess.load()
    assert m.size == guess.PARAM_COUNT and np.all(np.isfinite(m))
    assert np.all(m[:4] > 0)          # trained RMS scales of the three inputs and the target


def test_norms_of_a_linear_trajectory():
    """phi_k = phi_0 + k d: the first difference has the RMS of d, the second difference
    and the extrapolation error vanish, and the first channel is phi's spread."""
    rng = np.random.default_rng(1)
    phi0 = rng.uniform(-1, 1, (16, 16))
    d = 0.01 * rng.uniform(-1, 1, (16, 16))
    tr = torch.from_numpy(np.stack([phi0 + k * d for k in range(12)]))
    n = guess.compute_norms([tr], samples=16, seed=0)
    assert n[0] == pytest.approx(np.sqrt(np.mean((phi0 - phi0.mean()) ** 2)), rel=0.2)
    assert n[1] == pytest.approx(np.sqrt(np.mean(d ** 2)), rel=1e-5)
    assert n[2] < 1e-12 and n[3] < 1e-12
