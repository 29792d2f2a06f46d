"""The seeded input generator that both the oracle and the CUDA path read
(paper_1208_2643_gb300/inputs.py), pinned to the published SplitMix64 generator."""
import numpy as np

from paper_1208_2643_gb300 import inputs

_MASK = (1 << 64) - 1


def _splitmix64_sequential(state, count):
    """SplitMix64 as published (Steele, Lea and Flood, 2014): advance the state by the
    golden gamma, then mix it with two xor-shift-multiply rounds and a final xor-shift."""
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out.append(z ^ (z >> 31))
    return out


def test_first_outputs_from_state_zero():
    """The generator's widely quoted first outputs from state 0."""
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
            0x1B39896A51A8749B]
    assert [int(x) for x in inputs.splitmix64(0, 5)] == want


def test_counter_form_equals_the_sequential_generator():
    """Output k of seed s is the sequential generator started at state s * gamma."""
    for seed in (1, 3, 20):
        start = (seed * 0x9E3779B97F4A7C15) & _MASK
        assert [int(x) for x in inputs.splitmix64(seed, 40)] == _splitmix64_sequential(start, 40)


def test_offsets_address_the_same_stream():
    full = inputs.splitmix64(7, 100)
    np.testing.assert_array_equal(inputs.splitmix64(7, 60, offset=40), full[40:])


def test_uniform_range_and_moments():
    u = inputs.uniform(11, 200000, -1.0, 1.0)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01


def test_cell_centres_and_field_shapes():
    """Arrays are (n, m), row j = y, column i = x, centres at (i + 1/2) h (App. A)."""
    X, Y = inputs.cell_centres(6, 4, 0.5)
    assert X.shape == (4, 6) and Y.shape == (4, 6)
    assert X[0, 0] == 0.25 and X[0, 5] == 2.75 and Y[3, 0] == 1.75
    f = inputs.noise_field(6, 4, 0.07, 0.05, 1)
    assert f.shape == (4, 6) and np.all(np.abs(f - 0.07) <= 0.05)


def test_patch_and_device_generators_give_the_field_bits():
    """noise_at (values at given rows and columns, with wrap-around indices) and
    noise_field_torch (built by torch, here on the CPU, in small chunks) hold exactly
    the values of noise_field."""
    torch = __import__("pytest").importorskip("torch")
    f = inputs.noise_field(96, 40, 0.07, 0.05, 8)
    t = inputs.noise_field_torch(96, 40, 0.07, 0.05, 8, device="cpu", chunk=1000)
    assert t.dtype == torch.float64 and tuple(t.shape) == (40, 96)
    np.testing.assert_array_equal(t.numpy(), f)
    rows, cols = [39, 0, 1, 17], [95, 0, 1, 50, 94]
    np.testing.assert_array_equal(inputs.noise_at(96, 0.07, 0.05, 8, rows, cols), f[np.ix_(rows, cols)])
    big = (1 << 15) * (1 << 15) - 5   # indices past 2^30 address the same stream
    np.testing.assert_array_equal(inputs.uniform_at(3, [big, big + 4]), inputs.uniform(3, 5, offset=big)[[0, 4]])
