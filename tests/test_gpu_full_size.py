"""Parity at the full sizes of the workload list, in the launch configurations the
benchmark times.  Where the oracle solves the whole problem in seconds it does (the
512^2 second-order run in lockstep; one 2048^2 step against the mixed-precision
form); the 64-instance ensemble is checked instance by instance against the
single-instance solver (itself in lockstep with the oracle); the 1024^2 tcgen05
convolution is checked on sampled outputs computed one by one in FP64; the learned
guess at 1024^2 must leave the converged step unchanged."""
import math

import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2643_gb300 import mpfc
    mpfc.load()
    return mpfc


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_second_order_512_crystallites_lockstep(mp, oracle_mod):
    """512^2, scheme 2, h = pi/4, eps = 0.25, beta = 0.9, mean -0.285, s = 0.05, three
    crystallites of radius 20h with 1e-3 noise (seed 2): lockstep, every cell."""
    m, h, s = 512, math.pi / 4, 0.05
    phi0 = inputs.crystallite_field(m, m, h, -0.285, 0.25, count=3, radius_cells=20, noise=1e-3, seed=2)
    g = mp.Solver(mp.default_params(m=m, n=m, h=h, dt=s, epsilon=0.25, beta=0.9))
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s, eps=0.25, beta=0.9))
    o.set_state(phi0)
    for k in range(2):
        ro = o.step(2, tol=1e-10, guess=1)
        assert ro["status"] == 0
        assert g.step_cycles(2, ro["cycles"])["status"] == 0
        assert relerr(g.get_state()[0], o.get_state()[0]) <= 1e-10, k


def test_mixed_precision_2048_step(mp, oracle_mod):
    """2048^2, scheme 1, h = 0.5, eps = 0.025, beta = 0.9, s = 0.02, noise data: one
    FP32-inner step against the oracle's step solved to 1e-13, every cell."""
    m, h, s = 2048, 0.5, 0.02
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 3)
    g = mp.Solver(mp.default_params(m=m, n=m, h=h, dt=s, precision=mp.MPFC_FP32_INNER))
    g.set_state(phi0)
    info = g.step(1, 1)[0]
    assert info["status"] == 0 and info["res"] <= 1e-10
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s))
    o.set_state(phi0)
    assert o.step(1, tol=1e-13, guess=1)["status"] == 0
    assert relerr(g.get_state()[0], o.get_state()[0]) <= 1e-8


@pytest.mark.parametrize("scheme", [1, 2])
def test_ensemble_64_first_steps(mp, scheme):
    """The 64-instance batched workload (sizes 128^2 .. 1024^2): every instance's
    steps equal the single-instance solver's, with the same V-cycle counts."""
    ens = inputs.ensemble_instances(64, seed=4)
    ps = [mp.default_params(m=e["m"], n=e["n"], h=e["h"], dt=e["dt"], epsilon=e["epsilon"], beta=e["beta"])
          for e in ens]
    b = mp.BatchSolver(ps)
    for i, e in enumerate(ens):
        b.set_state(i, e["phi0"])
    rc, st, cy = b.step(scheme, 2)
    assert rc == 0 and all(x == 0 for x in st)
    for i, (e, p) in enumerate(zip(ens, ps)):
        g = mp.Solver(p)
        g.set_state(e["phi0"])
        infos = g.step(scheme, 2)
        assert cy[i] == sum(x["cycles"] for x in infos), i
        ref = g.get_state()[0]
        assert np.abs(b.get_state(i)[0] - ref).max() <= 1e-12 * np.abs(ref).max(), i
        g.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_conv32_1024_sampled(mode):
    """The benchmark's 32 -> 32 convolution launch at 1 x 1024 x 1024 x 32 (tcgen05
    path), checked on 400 sampled pixels (all 32 channels) against an FP64 evaluation
    of the periodic convolution with the same BF16 inputs and weights."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2643_gb300 import guess as gmod
    lib = gmod._lib()
    lib.mpfc_cnn_set_tensor_path(1)
    size = 1024
    s = torch.cuda.current_stream().cuda_stream
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(1, size, size, 32, device="cuda", generator=g).bfloat16()
    wt = torch.randn(9, 32, 32, device="cuda", generator=g) * 0.1
    bias = torch.randn(32, device="cuda", generator=g) * 0.1
    wk = torch.empty(32 * 288, dtype=torch.bfloat16, device="cuda")
    assert lib.mpfc_cnn_pack_weights(wt.data_ptr(), 32, 32, 32, 32, 0, wk.data_ptr(), s) == 0
    if mode == 0:
        y = torch.empty(1, size, size, 32, dtype=torch.bfloat16, device="cuda")
        assert lib.mpfc_cnn_conv_forward(x.data_ptr(), 1, size, size, 32, wk.data_ptr(), bias.data_ptr(), 32, 32, 0,
                                         y.data_ptr(), None, None, s) == 0
    else:
        y = torch.empty(1, size, size, 32, dtype=torch.float32, device="cuda")
        assert lib.mpfc_cnn_conv_forward(x.data_ptr(), 1, size, size, 32, wk.data_ptr(), bias.data_ptr(), 32, 32, 1,
                                         None, y.data_ptr(), None, s) == 0
    torch.cuda.synchronize()
    assert lib.mpfc_cnn_tensor_path_status() == 0
    xs = x.float().cpu().numpy().astype(np.float64)[0]
    wr = wt.bfloat16().float().cpu().numpy().astype(np.float64)
    br = bias.cpu().numpy().astype(np.float64)
    got = y.float().cpu().numpy().astype(np.float64)[0]
    rng = np.random.default_rng(1)
    pts = np.concatenate([rng.integers(0, size, size=(392, 2)),
                          np.array([[0, 0], [0, size - 1], [size - 1, 0], [size - 1, size - 1],
                                    [0, 127], [5, 128], [1023, 640], [512, 1023]])])
    ref = np.empty((len(pts), 32))
    for k, (yy, xx) in enumerate(pts):
        acc = br.copy()
        for tap in range(9):
            dy, dx = tap // 3 - 1, tap % 3 - 1
            acc += xs[(yy + dy) % size, (xx + dx) % size] @ wr[tap]
        ref[k] = acc
    out = np.array([got[yy, xx] for yy, xx in pts])
    if mode == 1:
        assert np.abs(out - ref).max() <= 1e-4 * np.abs(ref).max()
    else:
        erf = np.vectorize(math.erf)
        gel = 0.5 * ref * (1.0 + erf(ref / math.sqrt(2.0)))
        assert np.abs(out - gel).max() <= 1e-2 * np.abs(gel).max()


def test_learned_guess_1024_keeps_the_solution(mp):
    """With the packaged network at 1024^2 every step still reaches tol, and the
    converged fields equal those of the extrapolated guess to the solve tolerance."""
    from paper_1208_2643_gb300 import guess as gmod
    m = 1024
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    a = mp.Solver(mp.default_params(m=m, n=m, guess=mp.MPFC_GUESS_LEARNED))
    gmod.attach(a, gmod.load())
    b = mp.Solver(mp.default_params(m=m, n=m, guess=mp.MPFC_GUESS_EXTRAP))
    for g in (a, b):
        g.set_state(phi0)
    for k in range(4):
        ia, ib = a.step(1, 1)[0], b.step(1, 1)[0]
        assert ia["status"] == 0 and ia["res"] <= 1e-10 and ib["status"] == 0
        assert relerr(a.get_state()[0], b.get_state()[0]) <= 1e-8, k
