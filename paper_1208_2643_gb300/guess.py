"""Learned initial guess: model parameters, data generation and training.

Everything here drives the library's own kernels (include/mpfc_cnn.h and the solver)
through the C ABI; PyTorch only holds device buffers.  The network (5 periodic 3x3
convolutions, 3 -> 32 -> 32 -> 32 -> 32 -> 1, GELU after the first four, BF16 weights
and activations, FP32 accumulation) predicts, from phi^k, phi^{k-1}, phi^{k-2}, the
error phi^{k+1} - (2 phi^k - phi^{k-1}) of the linear extrapolation; the solver adds
the prediction to its initial guess (MPFC_GUESS_LEARNED).

Training data are time steps the solver itself produces at 256^2 (scheme 1,
epsilon in [0.02, 0.1], random-noise and crystallite initial data).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import inputs, mpfc

LAYERS = [(3, 32), (32, 32), (32, 32), (32, 32), (32, 1)]
PADDED = [(4, 32), (32, 32), (32, 32), (32, 32), (32, 8)]     # (cin_p, cout_p) of the forward kernels
PARAM_COUNT = 4 + sum(9 * ci * co + co for ci, co in LAYERS)
DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "guess_cnn_256.npy")


def _lib():
    lib = mpfc.load()
    V, P = ctypes.c_void_p, ctypes.POINTER
    lib.mpfc_cnn_features.argtypes = [V, V, V, V, ctypes.c_int, ctypes.c_int, ctypes.c_int, V, V, V, V, V]
    lib.mpfc_cnn_pack_weights.argtypes = [V, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          V, V]
    lib.mpfc_cnn_conv_forward.argtypes = [V, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, V, V,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, V, V, V, V]
    lib.mpfc_cnn_conv_backward_data.argtypes = [V, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, V,
                                                ctypes.c_int, ctypes.c_int, V, V, V, V]
    lib.mpfc_cnn_wgrad_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.mpfc_cnn_wgrad_scratch_bytes.restype = ctypes.c_size_t
    lib.mpfc_cnn_conv_backward_weight.argtypes = [V, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, V, ctypes.c_int, ctypes.c_int, V, V, V, V]
    lib.mpfc_cnn_mse.argtypes = [V, ctypes.c_int, V, ctypes.c_longlong, V, V, ctypes.c_int, V, ctypes.c_int, V]
    lib.mpfc_cnn_adam.argtypes = [V, V, V, V, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_int, V]
    lib.mpfc_set_guess_model.argtypes = [V, V, ctypes.c_size_t]
    lib.mpfc_cnn_set_tensor_path.argtypes = [ctypes.c_int]
    lib.mpfc_cnn_tensor_path_status.argtypes = []
    return lib


def _ck(rc, where):
    if rc != 0:
        raise mpfc.MPFCError(rc, where)


def init_params(seed=0):
    """He-style initialisation; the last layer starts at zero so the untrained network
    leaves the extrapolation unchanged.  Normalisation scales default to 1."""
    rng = np.random.default_rng(seed)
    parts = [np.ones(4)]
    for i, (ci, co) in enumerate(LAYERS):
        std = math.sqrt(2.0 / (9 * ci))
        w = rng.normal(0.0, std, size=(9, ci, co)) if i < 4 else np.zeros((9, ci, co))
        parts += [w.ravel(), np.zeros(co)]
    blob = np.concatenate(parts).astype(np.float32)
    assert blob.size == PARAM_COUNT
    return blob


def layer_slices():
    """[(w_slice, b_slice)] of the five layers in the blob."""
    out, off = [], 4
    for ci, co in LAYERS:
        ws = slice(off, off + 9 * ci * co)
        off += 9 * ci * co
        bs = slice(off, off + co)
        off += co
        out.append((ws, bs))
    return out


# --------------------------------------------------------------------------- data
def generate_trajectories(n_traj=10, steps=2000, size=256, seed=5, stream=None):
    """Runs the FP64 solver (scheme 1, h = 0.5, s = 0.01, tol 1e-10) and returns a list of
    device tensors [steps+1, size, size] (fp64) of phi after every step."""
    import torch
    rng = np.random.default_rng(seed)
    trajs = []
    for t in range(n_traj):
        eps = float(rng.uniform(0.02, 0.1))
        p = mpfc.default_params(m=size, n=size, h=0.5, dt=0.01, epsilon=eps)
        g = mpfc.Solver(p, stream=stream)
        if t % 2 == 0:
            phi0 = inputs.noise_field(size, size, float(rng.uniform(0.05, 0.1)), 0.05, seed * 1000 + t)
        else:
            phi0 = inputs.crystallite_field(size, size, 0.5, float(rng.uniform(0.05, 0.1)), max(eps, 0.05), count=3,
                                            radius_cells=size / 8, noise=0.01, seed=seed * 1000 + t)
        g.set_state(phi0)
        out = torch.empty((steps + 1, size, size), dtype=torch.float64, device="cuda")
        out[0].copy_(torch.from_numpy(phi0))
        for k in range(steps):
            g.step(1, 1)
            out[k + 1].copy_(g.get_state(device=True)[0])
        trajs.append(out)
        g.close()
    return trajs


def compute_norms(trajs, samples=64, seed=0):
    """RMS scales of the three inputs and of the target over a sample of steps."""
    rng = np.random.default_rng(seed)
    acc = np.zeros(4)
    for _ in range(samples):
        tr = trajs[rng.integers(len(trajs))]
        k = int(rng.integers(2, tr.shape[0] - 1))
        a, b, c, d = [tr[k + o].cpu().numpy() for o in (0, -1, -2, 1)]
        acc += [np.mean((a - a.mean()) ** 2), np.mean((a - b) ** 2), np.mean((a - 2 * b + c) ** 2),
                np.mean((d - 2 * a + b) ** 2)]
    return np.sqrt(acc / samples).astype(np.float32)


# --------------------------------------------------------------------------- training
class Trainer:
    """Forward, backward and Adam for batches of (B, H, W) samples, all on the GPU."""

    def __init__(self, blob, B, H, W, stream=None, lr=1e-3):
        import torch
        self.t = torch
        self.lib = _lib()
        self.B, self.H, self.W = B, H, W
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.s = self.stream.cuda_stream
        dev = "cuda"
        self.params = torch.from_numpy(np.asarray(blob, dtype=np.float32)).to(dev)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_no = 0
        self.lr = lr
        N = B * H * W
        bf = torch.bfloat16
        self.x = torch.empty((N, 4), dtype=bf, device=dev)
        self.y = torch.empty(N, dtype=torch.float32, device=dev)
        self.means = torch.empty(B * 129, dtype=torch.float64, device=dev)
        self.a = [torch.empty((N, 32), dtype=bf, device=dev) for _ in range(4)]
        self.z = [torch.empty((N, 32), dtype=torch.float32, device=dev) for _ in range(4)]
        self.yhat = torch.empty((N, 8), dtype=torch.float32, device=dev)
        self.dy_f = torch.empty((N, 4), dtype=torch.float32, device=dev)
        self.dy_b = torch.empty((N, 4), dtype=bf, device=dev)
        self.dz_f = torch.empty((N, 32), dtype=torch.float32, device=dev)
        self.dz_b = torch.empty((N, 32), dtype=bf, device=dev)
        self.dz2_f = torch.empty((N, 32), dtype=torch.float32, device=dev)
        self.dz2_b = torch.empty((N, 32), dtype=bf, device=dev)
        self.wk = [torch.empty((co_p * ((9 * ci_p + 15) // 16 * 16),), dtype=bf, device=dev) for ci_p, co_p in PADDED]
        # data-gradient packing of layers 1..4: rows = cin_p (32), K = 9 x (dgrad input channels)
        self.wk_t = [None] + [torch.empty((32 * ((9 * (4 if l == 4 else 32) + 15) // 16 * 16),), dtype=bf,
                                          device=dev) for l in range(1, 5)]
        self.scratch = torch.empty(int(self.lib.mpfc_cnn_wgrad_scratch_bytes(B, H, W)), dtype=torch.uint8, device=dev)
        self.lpart = torch.empty(512, dtype=torch.float32, device=dev)
        self.slices = layer_slices()
        self.pack()

    def _p(self, x):
        return x.data_ptr()

    def pack(self):
        for l, ((ci, co), (ci_p, co_p)) in enumerate(zip(LAYERS, PADDED)):
            ws = self.slices[l][0]
            w = self.params[ws]
            _ck(self.lib.mpfc_cnn_pack_weights(self._p(w), ci, co, ci_p, co_p, 0, self._p(self.wk[l]), self.s), "pack")
            if l > 0:
                _ck(self.lib.mpfc_cnn_pack_weights(self._p(w), ci, co, ci_p, 4 if l == 4 else 32, 1,
                                                   self._p(self.wk_t[l]), self.s), "pack_t")

    def features(self, pk, pkm1, pkm2, pkp1):
        _ck(self.lib.mpfc_cnn_features(self._p(pk), self._p(pkm1), self._p(pkm2), self._p(pkp1), self.B, self.H,
                                       self.W, self._p(self.params), self._p(self.means), self._p(self.x),
                                       self._p(self.y), self.s), "features")

    def forward(self):
        lib, B, H, W, s = self.lib, self.B, self.H, self.W, self.s
        inp, cin_p = self.x, 4
        for l in range(4):
            bs = self.slices[l][1]
            _ck(lib.mpfc_cnn_conv_forward(self._p(inp), B, H, W, cin_p, self._p(self.wk[l]),
                                          self._p(self.params[bs]), 32, 32, 0, self._p(self.a[l]), None,
                                          self._p(self.z[l]), s), "fwd")
            inp, cin_p = self.a[l], 32
        bs = self.slices[4][1]
        _ck(lib.mpfc_cnn_conv_forward(self._p(inp), B, H, W, 32, self._p(self.wk[4]), self._p(self.params[bs]), 1,
                                      8, 1, None, self._p(self.yhat), None, s), "fwd5")

    def loss_and_grad(self):
        N = self.B * self.H * self.W
        nb = 512
        _ck(self.lib.mpfc_cnn_mse(self._p(self.yhat), 8, self._p(self.y), N, self._p(self.dy_f), self._p(self.dy_b), 4,
                                  self._p(self.lpart), nb, self.s), "mse")

    def backward(self):
        lib, B, H, W, s = self.lib, self.B, self.H, self.W, self.s
        g = self.grads
        # layer 5: weight gradient and data gradient into layer 4's GELU
        ws, bs = self.slices[4]
        _ck(lib.mpfc_cnn_conv_backward_weight(self._p(self.a[3]), B, H, W, 32, 32, self._p(self.dy_f), 1, 4,
                                              self._p(g[ws]), self._p(g[bs]), self._p(self.scratch), s), "wg5")
        _ck(lib.mpfc_cnn_conv_backward_data(self._p(self.dy_b), B, H, W, 4, self._p(self.wk_t[4]), 32, 32,
                                            self._p(self.z[3]), self._p(self.dz_b), self._p(self.dz_f), s), "dg5")
        cur_b, cur_f, nxt_b, nxt_f = self.dz_b, self.dz_f, self.dz2_b, self.dz2_f
        for l in (3, 2, 1):
            ws, bs = self.slices[l]
            _ck(lib.mpfc_cnn_conv_backward_weight(self._p(self.a[l - 1]), B, H, W, 32, 32, self._p(cur_f), 32, 32,
                                                  self._p(g[ws]), self._p(g[bs]), self._p(self.scratch), s), "wg")
            _ck(lib.mpfc_cnn_conv_backward_data(self._p(cur_b), B, H, W, 32, self._p(self.wk_t[l]), 32, 32,
                                                self._p(self.z[l - 1]), self._p(nxt_b), self._p(nxt_f), s), "dg")
            cur_b, cur_f, nxt_b, nxt_f = nxt_b, nxt_f, cur_b, cur_f
        ws, bs = self.slices[0]
        _ck(lib.mpfc_cnn_conv_backward_weight(self._p(self.x), B, H, W, 3, 4, self._p(cur_f), 32, 32,
                                              self._p(g[ws]), self._p(g[bs]), self._p(self.scratch), s), "wg1")

    def adam(self):
        self.step_no += 1
        n = self.params.numel() - 4
        _ck(self.lib.mpfc_cnn_adam(self._p(self.params[4:]), self._p(self.grads[4:]), self._p(self.m[4:]),
                                   self._p(self.v[4:]), n, self.lr, 0.9, 0.999, 1e-8, self.step_no, self.s), "adam")
        self.pack()

    def loss_value(self):
        self.stream.synchronize()
        return float(self.lpart.sum().item()) / (self.B * self.H * self.W)

    def train_step(self, pk, pkm1, pkm2, pkp1):
        self.features(pk, pkm1, pkm2, pkp1)
        self.forward()
        self.loss_and_grad()
        self.backward()
        self.adam()

    def blob(self):
        self.stream.synchronize()
        return self.params.detach().cpu().numpy().copy()


def train(trajs, epochs=2, batch=8, lr=2e-3, seed=0, log=None, max_steps=None):
    """Trains on every (k-2, k-1, k, k+1) window of the trajectories; returns the blob."""
    import torch
    H, W = trajs[0].shape[1:]
    blob = init_params(seed)
    blob[:4] = compute_norms(trajs)
    tr = Trainer(blob, batch, H, W, lr=lr)
    rng = np.random.default_rng(seed)
    index = [(i, k) for i, t in enumerate(trajs) for k in range(2, t.shape[0] - 1)]
    total = epochs * (len(index) // batch)
    if max_steps:
        total = min(total, max_steps)
    pk = torch.empty((batch, H, W), dtype=torch.float64, device="cuda")
    pkm1, pkm2, pkp1 = torch.empty_like(pk), torch.empty_like(pk), torch.empty_like(pk)
    for it in range(total):
        sel = rng.choice(len(index), size=batch, replace=False)
        for b, j in enumerate(sel):
            i, k = index[j]
            pk[b].copy_(trajs[i][k])
            pkm1[b].copy_(trajs[i][k - 1])
            pkm2[b].copy_(trajs[i][k - 2])
            pkp1[b].copy_(trajs[i][k + 1])
        tr.lr = lr * 0.5 * (1 + math.cos(math.pi * it / total))
        tr.train_step(pk, pkm1, pkm2, pkp1)
        if log and (it % 200 == 0 or it == total - 1):
            log(it, tr.loss_value())
    return tr.blob()


def save(blob, path=DEFAULT_PATH):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, np.asarray(blob, dtype=np.float32))


def load(path=DEFAULT_PATH):
    return np.load(path).astype(np.float32) if os.path.exists(path) else None


def attach(solver, blob):
    """Loads the model into a solver created with guess = MPFC_GUESS_LEARNED."""
    b = np.ascontiguousarray(blob, dtype=np.float32)
    _ck(_lib().mpfc_set_guess_model(solver.h, b.ctypes.data, b.size), "mpfc_set_guess_model")


def main(argv):
    """python -m paper_1208_2643_gb300.guess [n_traj steps epochs out_path]: generates the
    training trajectories at 256^2 and trains the model."""
    import time
    t0 = time.time()
    n_traj = int(argv[0]) if len(argv) > 0 else 40
    steps = int(argv[1]) if len(argv) > 1 else 500
    epochs = int(argv[2]) if len(argv) > 2 else 8
    out = argv[3] if len(argv) > 3 else DEFAULT_PATH
    trajs = generate_trajectories(n_traj, steps)
    print(f"data: {n_traj} x {steps} steps in {time.time() - t0:.1f} s", flush=True)
    blob = train(trajs, epochs=epochs, log=lambda i, l: print(f"step {i} loss {l:.4e}", flush=True))
    save(blob, out)
    print(f"saved {out} after {time.time() - t0:.1f} s")


if __name__ == "__main__":
    import sys
    main(sys.argv[1:])
