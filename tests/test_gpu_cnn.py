"""The learned guess's kernels against the FP64 numpy oracle (oracle/cnn.py), fed the
same BF16-rounded inputs and weights, and the gain of a trained network.

Tolerances: FP32 outputs 1e-4 relative to their maximum (FP32 accumulation of exact
BF16 products); BF16 outputs 1e-2 (one BF16 rounding)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2643_gb300 import guess
    guess._lib()
    return guess


def bf16(a):
    """BF16-rounded copy (torch on the CPU) as float64 numpy, and the device bf16 tensor."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.float().double().numpy(), t.cuda()


def pad_ch(a, cp):
    out = np.zeros(a.shape[:-1] + (cp,))
    out[..., :a.shape[-1]] = a
    return out


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("ci,co,cip,cop,H,W", [(32, 32, 32, 32, 8, 40), (3, 32, 4, 32, 12, 32), (32, 1, 32, 8, 5, 70)])
def test_conv_forward_linear(G, oracle_mod, ci, co, cip, cop, H, W):
    from oracle import cnn
    lib = G._lib()
    rng = np.random.default_rng(0)
    B = 2
    xr, xd = bf16(pad_ch(rng.normal(size=(B, H, W, ci)), cip))
    w = rng.normal(scale=0.2, size=(9, ci, co)).astype(np.float32)
    wr = torch.from_numpy(w).bfloat16().float().double().numpy()
    bias = rng.normal(size=co).astype(np.float32)
    wd = torch.from_numpy(w).cuda()
    K = (9 * cip + 15) // 16 * 16
    wk = torch.empty(cop * K, dtype=torch.bfloat16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.mpfc_cnn_pack_weights(wd.data_ptr(), ci, co, cip, cop, 0, wk.data_ptr(), s) == 0
    y = torch.empty((B, H, W, cop), dtype=torch.float32, device="cuda")
    bd = torch.from_numpy(bias).cuda()
    assert lib.mpfc_cnn_conv_forward(xd.data_ptr(), B, H, W, cip, wk.data_ptr(), bd.data_ptr(), co, cop, 1, None,
                                     y.data_ptr(), None, s) == 0
    torch.cuda.synchronize()
    ref = cnn.conv3x3(xr[..., :ci], wr, bias.astype(np.float64))
    got = y.cpu().numpy()
    assert rel(got[..., :co], ref) < 1e-4
    assert np.all(got[..., co:] == 0)


def test_conv_forward_gelu_and_saved_preactivation(G):
    from oracle import cnn
    lib = G._lib()
    rng = np.random.default_rng(1)
    B, H, W, ci, co = 1, 8, 64, 32, 32
    xr, xd = bf16(rng.normal(size=(B, H, W, ci)))
    w = rng.normal(scale=0.2, size=(9, ci, co)).astype(np.float32)
    wr = torch.from_numpy(w).bfloat16().float().double().numpy()
    wk = torch.empty(32 * 288, dtype=torch.bfloat16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.mpfc_cnn_pack_weights(torch.from_numpy(w).cuda().data_ptr(), ci, co, 32, 32, 0, wk.data_ptr(), s) == 0
    yb = torch.empty((B, H, W, 32), dtype=torch.bfloat16, device="cuda")
    z = torch.empty((B, H, W, 32), dtype=torch.float32, device="cuda")
    assert lib.mpfc_cnn_conv_forward(xd.data_ptr(), B, H, W, 32, wk.data_ptr(), None, co, 32, 0, yb.data_ptr(), None,
                                     z.data_ptr(), s) == 0
    torch.cuda.synchronize()
    zr = cnn.conv3x3(xr, wr)
    assert rel(z.cpu().numpy(), zr) < 1e-4
    assert rel(yb.float().cpu().numpy(), cnn.gelu(zr)) < 1e-2


@pytest.mark.parametrize("cin,cout_p,H,W", [(32, 32, 8, 40), (32, 4, 6, 32)])
def test_conv_backward_data(G, cin, cout_p, H, W):
    from oracle import cnn
    lib = G._lib()
    rng = np.random.default_rng(2)
    B = 2
    cout = 1 if cout_p == 4 else 32
    dzr, dzd = bf16(pad_ch(rng.normal(size=(B, H, W, cout)), cout_p))
    w = rng.normal(scale=0.2, size=(9, cin, cout)).astype(np.float32)
    wr = torch.from_numpy(w).bfloat16().float().double().numpy()
    K = (9 * cout_p + 15) // 16 * 16
    wkt = torch.empty(32 * K, dtype=torch.bfloat16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.mpfc_cnn_pack_weights(torch.from_numpy(w).cuda().data_ptr(), cin, cout, 32, cout_p, 1,
                                     wkt.data_ptr(), s) == 0
    zp = rng.normal(size=(B, H, W, 32)).astype(np.float32)
    zpd = torch.from_numpy(zp).cuda()
    ob = torch.empty((B, H, W, 32), dtype=torch.bfloat16, device="cuda")
    of = torch.empty((B, H, W, 32), dtype=torch.float32, device="cuda")
    assert lib.mpfc_cnn_conv_backward_data(dzd.data_ptr(), B, H, W, cout_p, wkt.data_ptr(), cin, 32, zpd.data_ptr(),
                                           ob.data_ptr(), of.data_ptr(), s) == 0
    torch.cuda.synchronize()
    ref = cnn.conv3x3_grad_input(dzr[..., :cout], wr) * cnn.gelu_grad(zp.astype(np.float64))
    assert rel(of.cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("cin,cin_p,cout,cout_p,B,H,W", [(32, 32, 32, 32, 2, 24, 40), (32, 32, 32, 32, 2, 37, 200),
                                                         (3, 4, 32, 32, 2, 24, 40), (32, 32, 1, 4, 2, 24, 40)])
def test_conv_backward_weight(G, cin, cin_p, cout, cout_p, B, H, W):
    """dW[tap][ci][co] = sum_p x[p + off(tap)][ci] dz[p][co] and db.  The 32 -> 32 layers
    run on tensor cores with dz rounded to BF16 (both operands BF16, FP32 accumulation):
    they are compared with the oracle fed the same BF16 operands (1e-4), and with the
    FP32-dz oracle within the BF16 rounding of dz (2^-8 of sum |x dz|).  The other
    layers keep FP32 dz on CUDA cores (1e-4 against the FP32-dz oracle).  db sums the
    FP32 dz on both paths.  The second shape has ragged pixel segments and row chunks."""
    from oracle import cnn
    lib = G._lib()
    rng = np.random.default_rng(3)
    xr, xd = bf16(pad_ch(rng.normal(size=(B, H, W, cin)), cin_p))
    dz = pad_ch(rng.normal(size=(B, H, W, cout)), cout_p).astype(np.float32)
    dzd = torch.from_numpy(dz).cuda()
    dw = torch.empty(9 * cin * cout, dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    scratch = torch.empty(int(lib.mpfc_cnn_wgrad_scratch_bytes(B, H, W)), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.mpfc_cnn_conv_backward_weight(xd.data_ptr(), B, H, W, cin, cin_p, dzd.data_ptr(), cout, cout_p,
                                             dw.data_ptr(), db.data_ptr(), scratch.data_ptr(), s) == 0
    torch.cuda.synchronize()
    got = dw.cpu().numpy().reshape(9, cin, cout)
    gw, gb = cnn.conv3x3_grad_weight(xr[..., :cin], dz[..., :cout].astype(np.float64))
    if cin == 32 and cin_p == 32 and cout_p == 32:
        dzr, _ = bf16(dz)
        gw_b, _ = cnn.conv3x3_grad_weight(xr[..., :cin], dzr[..., :cout])
        assert rel(got, gw_b) < 1e-4
        gabs, _ = cnn.conv3x3_grad_weight(np.abs(xr[..., :cin]), np.abs(dz[..., :cout].astype(np.float64)))
        assert np.all(np.abs(got - gw) <= 2.0 ** -8 * gabs + 1e-4 * np.abs(gw).max())
    else:
        assert rel(got, gw) < 1e-4
    assert rel(db.cpu().numpy(), gb) < 1e-4


def test_adam_matches_oracle(G):
    from oracle import cnn
    lib = G._lib()
    rng = np.random.default_rng(4)
    p, g = rng.normal(size=1000), rng.normal(size=1000)
    m, v = np.zeros(1000), np.zeros(1000)
    pd, gd = torch.tensor(p, dtype=torch.float32, device="cuda"), torch.tensor(g, dtype=torch.float32, device="cuda")
    md, vd = torch.zeros_like(pd), torch.zeros_like(pd)
    s = torch.cuda.current_stream().cuda_stream
    for t in (1, 2, 3):
        assert lib.mpfc_cnn_adam(pd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), 1000, 1e-2, 0.9, 0.999,
                                 1e-8, t, s) == 0
        p, m, v = cnn.adam(p, g, m, v, t, lr=1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(pd.cpu().numpy(), p, rtol=1e-5, atol=1e-6)


def test_learned_guess_trains_and_lowers_res0(G):
    """A network trained briefly on solver trajectories (generation, features, forward,
    backward and Adam all on the library's kernels) lowers the residual of the initial
    guess against the linear extrapolation on a held-out trajectory, takes no more
    V-cycles, and the solver still converges to the same tolerance."""
    from paper_1208_2643_gb300 import inputs, mpfc
    trajs = G.generate_trajectories(n_traj=2, steps=300, size=64, seed=11)
    blob = G.train(trajs, epochs=3, batch=8, lr=3e-3, seed=0)
    m = 64
    phi0 = inputs.noise_field(m, m, 0.08, 0.05, 99)
    res = {}
    for gs in (mpfc.MPFC_GUESS_EXTRAP, mpfc.MPFC_GUESS_LEARNED):
        g = mpfc.Solver(mpfc.default_params(m=m, n=m, guess=gs))
        if gs == mpfc.MPFC_GUESS_LEARNED:
            G.attach(g, blob)
            g.set_guess_gate(0.0)   # the network on every step: this tests the network
        g.set_state(phi0)
        g.step(1, 20)
        infos = g.step(1, 40)
        assert all(i["status"] == 0 and i["res"] <= 1e-10 for i in infos)
        res[gs] = (np.mean([i["res0"] for i in infos]), np.mean([i["cycles"] for i in infos]))
    assert res[mpfc.MPFC_GUESS_LEARNED][0] < 0.8 * res[mpfc.MPFC_GUESS_EXTRAP][0], res
    assert res[mpfc.MPFC_GUESS_LEARNED][1] <= res[mpfc.MPFC_GUESS_EXTRAP][1], res


def test_learned_guess_saves_vcycles_early_in_the_headline_run(G):
    """The packaged model on the benchmark's workload (1024^2, noise initial data), steps
    11-110: fewer V-cycles per step than the extrapolated guess at the same tolerance (the
    regime where the extrapolation error is large; later in the run the extrapolation
    becomes accurate enough that the network's own BF16 error floor costs as much as it
    saves, and over 1000 steps the two take the same cycles)."""
    from paper_1208_2643_gb300 import inputs, mpfc
    blob = G.load()
    m = 1024
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    cyc = {}
    for gs in (mpfc.MPFC_GUESS_EXTRAP, mpfc.MPFC_GUESS_LEARNED):
        g = mpfc.Solver(mpfc.default_params(m=m, n=m, guess=gs))
        if gs == mpfc.MPFC_GUESS_LEARNED:
            G.attach(g, blob)
        g.set_state(phi0)
        g.step(1, 10)
        infos = g.step(1, 100)
        assert all(i["status"] == 0 and i["res"] <= 1e-10 for i in infos)
        cyc[gs] = np.mean([i["cycles"] for i in infos])
        g.close()
    assert cyc[mpfc.MPFC_GUESS_LEARNED] <= cyc[mpfc.MPFC_GUESS_EXTRAP] - 0.2, cyc


def test_learned_guess_gate(G):
    """The gate of the learned guess on the benchmark's workload (1024^2): steps whose
    extrapolated guess has a scaled residual below the threshold are the extrapolated
    guess's steps bit for bit; a threshold below every residual gives the ungated
    network's steps bit for bit; in graph and stream launch modes alike.  Over steps
    11-110 the gated guess takes no more V-cycles than the extrapolated one."""
    from paper_1208_2643_gb300 import inputs, mpfc
    blob = G.load()
    m = 1024
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)

    def run(gs, gate=None, stream=False, steps=12):
        g = mpfc.Solver(mpfc.default_params(m=m, n=m, guess=gs))
        if gs == mpfc.MPFC_GUESS_LEARNED:
            G.attach(g, blob)
            if gate is not None:
                g.set_guess_gate(gate)
        if stream:
            g.set_launch_mode(mpfc.MPFC_LAUNCH_STREAM)
        g.set_state(phi0)
        infos = g.step(1, steps)
        st = g.get_state()
        g.close()
        return infos, st

    ext, st_ext = run(mpfc.MPFC_GUESS_EXTRAP)
    never, st_never = run(mpfc.MPFC_GUESS_LEARNED, gate=1e30)
    assert [i["cycles"] for i in never] == [i["cycles"] for i in ext]
    for a, b in zip(st_never, st_ext):
        assert np.array_equal(a, b)
    always, st_always = run(mpfc.MPFC_GUESS_LEARNED, gate=0.0)
    tiny, st_tiny = run(mpfc.MPFC_GUESS_LEARNED, gate=1e-300)
    assert [i["res0"] for i in tiny] == [i["res0"] for i in always]
    for a, b in zip(st_tiny, st_always):
        assert np.array_equal(a, b)
    dflt, st_d = run(mpfc.MPFC_GUESS_LEARNED)
    dflt_s, st_ds = run(mpfc.MPFC_GUESS_LEARNED, stream=True)
    assert [i["cycles"] for i in dflt] == [i["cycles"] for i in dflt_s]
    for a, b in zip(st_d, st_ds):
        assert np.array_equal(a, b)
    # until the network first runs, the default gate's steps are the extrapolated guess's
    gate = 2.6e4 * 1e-10
    for i, e in zip(dflt, ext):
        if e["res0"] >= gate:
            break
        assert i["res0"] == e["res0"] and i["cycles"] == e["cycles"]
    cyc = {}
    for name in ("extrap", "gated"):
        gs = mpfc.MPFC_GUESS_EXTRAP if name == "extrap" else mpfc.MPFC_GUESS_LEARNED
        infos, _ = run(gs, steps=110)
        cyc[name] = np.mean([i["cycles"] for i in infos[10:]])
    assert cyc["gated"] <= cyc["extrap"], cyc
    with pytest.raises(mpfc.MPFCError):
        g = mpfc.Solver(mpfc.default_params(m=64, n=64))
        g.set_guess_gate(1.0)


def test_learned_guess_gate_scheme2(G):
    """The gate's two bitwise limits for the second-order scheme (whose step also
    restricts phi^k to the coarse levels) at 256^2: a gate above every residual gives
    the extrapolated guess's steps, one below every residual the ungated network's."""
    from paper_1208_2643_gb300 import inputs, mpfc
    blob = G.load()
    m = 256
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 3)

    def run(gs, gate=None):
        g = mpfc.Solver(mpfc.default_params(m=m, n=m, h=0.5, dt=0.05, guess=gs))
        if gs == mpfc.MPFC_GUESS_LEARNED:
            G.attach(g, blob)
            g.set_guess_gate(gate)
        g.set_state(phi0)
        infos = g.step(2, 4)
        assert all(i["status"] == 0 for i in infos)
        st = g.get_state()
        g.close()
        return [(i["cycles"], i["res0"]) for i in infos], st

    for (a, sa), (b, sb) in ((run(mpfc.MPFC_GUESS_LEARNED, 1e30), run(mpfc.MPFC_GUESS_EXTRAP)),
                             (run(mpfc.MPFC_GUESS_LEARNED, 1e-300), run(mpfc.MPFC_GUESS_LEARNED, 0.0))):
        assert a == b
        for x, y in zip(sa, sb):
            assert np.array_equal(x, y)


@pytest.fixture
def tensor_path(G):
    """Yields a setter of the 32 -> 32 convolutions' tensor-core path; restores tcgen05."""
    lib = G._lib()
    yield lambda use_tc: lib.mpfc_cnn_set_tensor_path(use_tc)
    lib.mpfc_cnn_set_tensor_path(1)


@pytest.mark.parametrize("H,W", [(3, 128), (5, 256)])
@pytest.mark.parametrize("use_tc", [1, 0])
def test_conv32_both_tensor_paths_match_oracle(G, tensor_path, use_tc, H, W):
    """Forward (linear, and GELU with the saved pre-activation) and data gradient of a
    32 -> 32 layer on widths that take the tcgen05 kernel, on both tensor-core paths;
    fewer real output channels (cout 20) than padded ones check the zero fill."""
    from oracle import cnn
    lib = G._lib()
    tensor_path(use_tc)
    rng = np.random.default_rng(7)
    B = 2
    s = torch.cuda.current_stream().cuda_stream
    xr, xd = bf16(rng.normal(size=(B, H, W, 32)))
    for co in (32, 20):
        w = rng.normal(scale=0.2, size=(9, 32, co)).astype(np.float32)
        wr = torch.from_numpy(w).bfloat16().float().double().numpy()
        bias = rng.normal(size=co).astype(np.float32)
        wk = torch.empty(32 * 288, dtype=torch.bfloat16, device="cuda")
        assert lib.mpfc_cnn_pack_weights(torch.from_numpy(w).cuda().data_ptr(), 32, co, 32, 32, 0, wk.data_ptr(),
                                         s) == 0
        bd = torch.from_numpy(bias).cuda()
        y = torch.full((B, H, W, 32), 7.0, dtype=torch.float32, device="cuda")
        assert lib.mpfc_cnn_conv_forward(xd.data_ptr(), B, H, W, 32, wk.data_ptr(), bd.data_ptr(), co, 32, 1, None,
                                         y.data_ptr(), None, s) == 0
        yb = torch.empty((B, H, W, 32), dtype=torch.bfloat16, device="cuda")
        z = torch.empty((B, H, W, 32), dtype=torch.float32, device="cuda")
        assert lib.mpfc_cnn_conv_forward(xd.data_ptr(), B, H, W, 32, wk.data_ptr(), bd.data_ptr(), co, 32, 0,
                                         yb.data_ptr(), None, z.data_ptr(), s) == 0
        torch.cuda.synchronize()
        assert lib.mpfc_cnn_tensor_path_status() == 0
        ref = cnn.conv3x3(xr, wr, bias.astype(np.float64))
        got = y.cpu().numpy()
        assert rel(got[..., :co], ref) < 1e-4
        assert np.all(got[..., co:] == 0)
        assert rel(z.cpu().numpy()[..., :co], ref) < 1e-4
        gb = yb.float().cpu().numpy()
        assert rel(gb[..., :co], cnn.gelu(ref)) < 1e-2
        assert np.all(gb[..., co:] == 0)
    # data gradient through a 32 -> 32 layer
    dzr, dzd = bf16(rng.normal(size=(B, H, W, 32)))
    w = rng.normal(scale=0.2, size=(9, 32, 32)).astype(np.float32)
    wr = torch.from_numpy(w).bfloat16().float().double().numpy()
    wkt = torch.empty(32 * 288, dtype=torch.bfloat16, device="cuda")
    assert lib.mpfc_cnn_pack_weights(torch.from_numpy(w).cuda().data_ptr(), 32, 32, 32, 32, 1, wkt.data_ptr(),
                                     s) == 0
    zp = rng.normal(size=(B, H, W, 32)).astype(np.float32)
    zpd = torch.from_numpy(zp).cuda()
    ob = torch.empty((B, H, W, 32), dtype=torch.bfloat16, device="cuda")
    of = torch.empty((B, H, W, 32), dtype=torch.float32, device="cuda")
    assert lib.mpfc_cnn_conv_backward_data(dzd.data_ptr(), B, H, W, 32, wkt.data_ptr(), 32, 32, zpd.data_ptr(),
                                           ob.data_ptr(), of.data_ptr(), s) == 0
    torch.cuda.synchronize()
    assert lib.mpfc_cnn_tensor_path_status() == 0
    ref = cnn.conv3x3_grad_input(dzr, wr) * cnn.gelu_grad(zp.astype(np.float64))
    assert rel(of.cpu().numpy(), ref) < 1e-4
    assert rel(ob.float().cpu().numpy(), ref) < 1e-2


def test_tensor_path_wait_timeout_is_reported_and_recovers(G, tensor_path):
    """The tcgen05 convolution's waits are bounded.  Through the test hook the first CTA
    withholds the tensor copy of its first input row (no out-of-bounds access): the MMA
    issuer's wait runs out after 2e6 clock cycles, the CTA drains the copies and MMAs it
    issued, frees its tensor memory and returns; the status call reports the timeout once.
    The next launch, with the hook off, matches the oracle and reports no failure."""
    import ctypes
    from oracle import cnn
    lib = G._lib()
    lib.mpfc_cnn_test_withhold_load.argtypes = [ctypes.c_int, ctypes.c_longlong]
    tensor_path(1)
    rng = np.random.default_rng(9)
    B, H, W = 1, 6, 256
    s = torch.cuda.current_stream().cuda_stream
    xr, xd = bf16(rng.normal(size=(B, H, W, 32)))
    w = rng.normal(scale=0.2, size=(9, 32, 32)).astype(np.float32)
    wr = torch.from_numpy(w).bfloat16().float().double().numpy()
    bias = rng.normal(size=32).astype(np.float32)
    wk = torch.empty(32 * 288, dtype=torch.bfloat16, device="cuda")
    assert lib.mpfc_cnn_pack_weights(torch.from_numpy(w).cuda().data_ptr(), 32, 32, 32, 32, 0, wk.data_ptr(), s) == 0
    bd = torch.from_numpy(bias).cuda()
    y = torch.full((B, H, W, 32), 7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    assert lib.mpfc_cnn_tensor_path_status() == 0
    try:
        assert lib.mpfc_cnn_test_withhold_load(1, 2000000) == 0
        assert lib.mpfc_cnn_conv_forward(xd.data_ptr(), B, H, W, 32, wk.data_ptr(), bd.data_ptr(), 32, 32, 1, None,
                                         y.data_ptr(), None, s) == 0
        torch.cuda.synchronize()
    finally:
        assert lib.mpfc_cnn_test_withhold_load(0, 0) == 0
    assert lib.mpfc_cnn_tensor_path_status() == -4      # MPFC_ERR_NOT_CONVERGED: a wait gave up
    assert lib.mpfc_cnn_tensor_path_status() == 0       # reported once
    ref = cnn.conv3x3(xr, wr, bias.astype(np.float64))
    assert np.all(y.cpu().numpy()[0, 0, :128] == 7.0)   # the aborted CTA's tile stays unwritten
    y.fill_(7.0)
    assert lib.mpfc_cnn_conv_forward(xd.data_ptr(), B, H, W, 32, wk.data_ptr(), bd.data_ptr(), 32, 32, 1, None,
                                     y.data_ptr(), None, s) == 0
    torch.cuda.synchronize()
    assert lib.mpfc_cnn_tensor_path_status() == 0
    assert rel(y.cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("m,n", [(96, 160), (256, 64)])
def test_guess_inference_matches_network_definition(G, m, n):
    """The solver's inference of the packaged model (features and first layer fused in
    one kernel, the 32 -> 32 layers on tcgen05 (width 256) or mma.sync (width 96), the
    output layer added into an FP64 field) against the oracle's network on the same
    state, with the network's bf16 roundings (features, weights, activations) applied
    on the oracle side too: within 1e-2 of the largest correction (bf16 ties that FP32
    accumulation order or the GELU approximation flip)."""
    import ctypes
    from oracle import cnn
    from paper_1208_2643_gb300 import inputs, mpfc
    lib = G._lib()
    blob = G.load()
    g = mpfc.Solver(mpfc.default_params(m=m, n=n, guess=mpfc.MPFC_GUESS_LEARNED))
    G.attach(g, blob)
    g.set_state(inputs.noise_field(m, n, 0.08, 0.05, 21))
    g.step(1, 1)
    phi_km2 = g.get_state()[1]
    g.step(1, 1)
    phik, phikm1, _ = g.get_state()
    out = torch.empty((n, m), dtype=torch.float64, device="cuda")
    assert lib.mpfc_guess_correction(g.h, out.data_ptr()) == 0
    torch.cuda.synchronize()

    def r(a):
        return torch.from_numpy(np.asarray(a, dtype=np.float32)).bfloat16().float().double().numpy()

    norms, layers = cnn.unpack(blob)
    a = r(cnn.features(phik, phikm1, phi_km2, norms))[None]
    for i, (w, b) in enumerate(layers):
        z = cnn.conv3x3(a, r(w), b)
        a = r(cnn.gelu(z)) if i < 4 else z
    ref = a[0, ..., 0] * norms[3]
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-2 * np.abs(ref).max(), (np.abs(got - ref).max(), np.abs(ref).max())


def test_learned_guess_same_on_both_tensor_paths(G, tensor_path):
    """The packaged 256 x 256 model gives the same initial residual (to FP32 accumulation
    order) whichever tensor-core path runs its 32 -> 32 layers."""
    from paper_1208_2643_gb300 import inputs, mpfc
    m = 256
    phi0 = inputs.noise_field(m, m, 0.08, 0.05, 5)
    out = {}
    for use_tc in (1, 0):
        tensor_path(use_tc)
        g = mpfc.Solver(mpfc.default_params(m=m, n=m, guess=mpfc.MPFC_GUESS_LEARNED))
        G.attach(g, G.load())
        g.set_guess_gate(0.0)
        g.set_state(phi0)
        g.step(1, 3)
        infos = g.step(1, 3)
        assert all(i["status"] == 0 for i in infos)
        out[use_tc] = np.array([i["res0"] for i in infos])
        assert G._lib().mpfc_cnn_tensor_path_status() == 0
    np.testing.assert_allclose(out[1], out[0], rtol=1e-3)


def test_gelu_matches_exact_erf(G):
    """The kernels' GELU and GELU' (erf after Abramowitz & Stegun 7.1.26) against the
    exact functions in float64, over the range activations take and far tails."""
    import ctypes
    import math
    lib = G._lib()
    lib.mpfc_probe_gelu.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    z = np.concatenate([np.linspace(-12, 12, 200001), [0.0, -0.0, 1e-30, -1e-30, 50.0, -50.0, 1e4, -1e4]])
    z = z.astype(np.float32)
    zd = torch.from_numpy(z).cuda()
    g, dg = torch.empty_like(zd), torch.empty_like(zd)
    assert lib.mpfc_probe_gelu(zd.data_ptr(), g.data_ptr(), dg.data_ptr(), z.size, None) == 0
    torch.cuda.synchronize()
    zz = z.astype(np.float64)
    erf = np.array([math.erf(v / math.sqrt(2.0)) for v in zz])
    g_ref = 0.5 * zz * (1.0 + erf)
    dg_ref = 0.5 * (1.0 + erf) + zz * np.exp(-0.5 * zz * zz) / math.sqrt(2.0 * math.pi)
    gg, dd = g.cpu().numpy().astype(np.float64), dg.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gg - g_ref) <= 4e-7 * np.abs(zz) + 4e-7 * np.abs(g_ref) + 1e-37)
    assert np.all(np.abs(dd - dg_ref) <= 1e-6 * (1.0 + np.abs(zz)))
    # the 8-wide form (shared reciprocal), with mixed magnitudes inside each group of 8
    lib.mpfc_probe_gelu8.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int, ctypes.c_void_p]
    perm = np.random.default_rng(3).permutation(z.size)
    zp = np.ascontiguousarray(z[perm])
    zpd = torch.from_numpy(zp).cuda()
    g8 = torch.empty_like(zpd)
    assert lib.mpfc_probe_gelu8(zpd.data_ptr(), g8.data_ptr(), zp.size, None) == 0
    torch.cuda.synchronize()
    gr = g_ref[perm]
    got8 = g8.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got8 - gr) <= 4e-7 * np.abs(zz[perm]) + 4e-7 * np.abs(gr) + 1e-37)


def test_features_match_oracle(G):
    """Network input and training target of mpfc_cnn_features against the oracle's
    features() (and the extrapolation error for the target), on two samples."""
    from oracle import cnn
    lib = G._lib()
    rng = np.random.default_rng(8)
    B, H, W = 2, 24, 40
    f = [rng.normal(0.07, 0.05, size=(B, H, W)) for _ in range(4)]   # phi^k, phi^{k-1}, phi^{k-2}, phi^{k+1}
    norms = np.array([0.05, 2e-3, 3e-4, 1e-4], dtype=np.float32)
    fd = [torch.from_numpy(a).cuda() for a in f]
    nd = torch.from_numpy(norms).cuda()
    means = torch.empty(B * 129, dtype=torch.float64, device="cuda")
    x = torch.empty((B, H, W, 4), dtype=torch.bfloat16, device="cuda")
    y = torch.empty((B, H, W), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.mpfc_cnn_features(fd[0].data_ptr(), fd[1].data_ptr(), fd[2].data_ptr(), fd[3].data_ptr(), B, H, W,
                                 nd.data_ptr(), means.data_ptr(), x.data_ptr(), y.data_ptr(), s) == 0
    torch.cuda.synchronize()
    got = x.float().cpu().numpy().astype(np.float64)
    for b in range(B):
        ref = cnn.features(f[0][b], f[1][b], f[2][b], norms.astype(np.float64))
        # one bf16 rounding (8 significant bits) of each feature
        assert np.all(np.abs(got[b, ..., :3] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-30)
        assert np.all(got[b, ..., 3] == 0)
        tgt = (f[3][b] - 2 * f[0][b] + f[1][b]) / float(norms[3])
        np.testing.assert_allclose(y.cpu().numpy()[b], tgt, rtol=1e-6, atol=1e-6 * np.abs(tgt).max())
