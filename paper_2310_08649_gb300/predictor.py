"""Learned Newton predictor for the van der Pol model: data from the solver,
training and inference through the C ABI (tvi_predictor_*).

The predictor maps a chunk's start state y_i, log10 mu and the log10 step sizes
of its c steps to per-step slopes s_1..s_c (2 c outputs); tvi_integrate forms
the guess dy_j = sum_{l <= j} dt_l s_l and uses it as Newton's starting point
where its FP64 residual beats dy = 0.  Newton then runs to the same tolerance,
so results are unchanged.  Slopes, unlike increments, do not scale with the
step sizes, which span six decades on the log-spaced grid.
"""
import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from .api import Model, Options, integrate


@dataclass(frozen=True)
class PredictorSpec:
    chunk: int = 100
    hidden: int = 256

    @property
    def n_in(self):
        return 3 + self.chunk

    @property
    def n_out(self):
        return 2 * self.chunk

    def size(self):
        n = _lib.load().tvi_predictor_size(self.n_in, self.hidden, self.n_out)
        if n < 0:
            raise ValueError(f"bad predictor sizes {self}")
        return n

    def offsets(self):
        i, h, o = self.n_in, self.hidden, self.n_out
        off = {"mean": 0, "std": i, "scale": 2 * i, "W1": 2 * i + o}
        off["b1"] = off["W1"] + h * i
        off["W2"] = off["b1"] + h
        off["b2"] = off["W2"] + h * h
        off["W3"] = off["b2"] + h
        off["b3"] = off["W3"] + o * h
        off["end"] = off["b3"] + o
        return off


def chunk_samples(y, times, mu, chunk, lengths=None):
    """(features [S][3 + c], targets [S][2 c]) of every full c-step chunk of solved
    van der Pol trajectories y [B][N+1][2] (host arrays).  Targets are the slopes
    (y_k - y_{k-1}) / dt_k, 0 on padding steps (dt = 0)."""
    B, Np1, _ = y.shape
    N = Np1 - 1
    xs, ts = [], []
    for i in range(0, N - chunk + 1, chunk):
        dt = np.diff(times[:, i:i + chunk + 1], axis=1)
        if lengths is not None:
            steps = np.arange(i + 1, i + chunk + 1)[None, :]
            dt = np.where(steps > lengths[:, None], 0.0, dt)
        feat = np.concatenate([y[:, i], np.log10(mu)[:, None],
                               np.log10(np.maximum(dt, 1e-30))], axis=1)
        inc = y[:, i + 1:i + chunk + 1] - y[:, i:i + chunk]
        slope = np.where(dt[:, :, None] > 0, inc / np.where(dt > 0, dt, 1.0)[:, :, None], 0.0)
        xs.append(feat)
        ts.append(slope.reshape(B, 2 * chunk))
    return np.concatenate(xs).astype(np.float32), np.concatenate(ts).astype(np.float32)


def solver_dataset(make_workload, seeds, spec, tol=1e-8, device="cuda"):
    """Run the chunked solver on the given seeded workloads (a callable seed ->
    workload dict) and collect its converged chunks as training samples."""
    xs, ts = [], []
    for seed in seeds:
        w = make_workload(seed)
        m = Model.from_spec(w["spec"])
        d = {k: torch.as_tensor(w[k], dtype=torch.float64, device=device)
             for k in ("y0", "times", "params")}
        o = Options(chunk=spec.chunk, tol_abs=tol, precision="fp32")
        y, _, _, _ = integrate(m, o, d["y0"], d["times"], d["params"])
        x, t = chunk_samples(y.cpu().numpy(), w["times"], w["params"][:, 0], spec.chunk)
        xs.append(x)
        ts.append(t)
    return np.concatenate(xs), np.concatenate(ts)


class Predictor:
    """Packed predictor weights on the GPU, with training and inference."""

    def __init__(self, spec=PredictorSpec(), seed=0, device="cuda"):
        self.spec, self.device = spec, torch.device(device)
        off = spec.offsets()
        g = np.random.Generator(np.random.PCG64(seed))
        p = np.zeros(spec.size(), dtype=np.float32)
        p[off["std"]:off["std"] + spec.n_in] = 1.0
        p[off["scale"]:off["scale"] + spec.n_out] = 1.0
        for (W, fan_in, fan_out) in (("W1", spec.n_in, spec.hidden),
                                     ("W2", spec.hidden, spec.hidden),
                                     ("W3", spec.hidden, spec.n_out)):
            a = np.sqrt(6.0 / (fan_in + fan_out))  # Xavier-uniform
            p[off[W]:off[W] + fan_in * fan_out] = g.uniform(-a, a, fan_in * fan_out)
        self.packed = torch.as_tensor(p, device=self.device)
        n_train = spec.size() - off["W1"]
        self.m = torch.zeros(n_train, dtype=torch.float32, device=self.device)
        self.v = torch.zeros_like(self.m)
        self.step = 0

    def set_normalisation(self, x, t):
        """Feature mean/std and output scales from training data (host arrays)."""
        off = self.spec.offsets()
        p = self.packed.cpu().numpy()
        p[off["mean"]:off["mean"] + self.spec.n_in] = x.mean(axis=0)
        p[off["std"]:off["std"] + self.spec.n_in] = np.maximum(x.std(axis=0), 1e-6)
        rms = np.sqrt(np.mean(np.square(t, dtype=np.float64), axis=0))
        p[off["scale"]:off["scale"] + self.spec.n_out] = np.maximum(rms, 1e-12)
        self.packed.copy_(torch.as_tensor(p))

    def options(self):
        return {"predictor": self.packed, "predictor_chunk": self.spec.chunk,
                "predictor_hidden": self.spec.hidden}

    def forward(self, x, stream=None):
        """x [M][n_in] raw features (CUDA float32) -> slopes [M][n_out]."""
        s = self.spec
        M = x.shape[0]
        y = torch.empty((M, s.n_out), dtype=torch.float32, device=self.device)
        st = stream if stream is not None else torch.cuda.current_stream()
        rc = _lib.load().tvi_predictor_forward(ctypes.c_void_p(self.packed.data_ptr()), s.n_in,
                                              s.hidden, s.n_out, M,
                                              ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(y.data_ptr()),
                                              ctypes.c_void_p(st.cuda_stream))
        if rc != 0:
            raise _lib.TviError(rc, "tvi_predictor_forward")
        return y

    def train_step(self, x, t, lr, rows=None, workspace=None, loss=None):
        """One Adam step.  x [S][n_in], t [S][n_out] CUDA float32; the batch is
        rows (CUDA int32 [M]) of them, or all S rows.  loss: a CUDA float32
        slot receiving the batch loss."""
        s = self.spec
        M = rows.numel() if rows is not None else x.shape[0]
        lib = _lib.load()
        if workspace is None:
            workspace = torch.empty(lib.tvi_predictor_workspace_bytes(s.n_in, s.hidden, s.n_out, M),
                                    dtype=torch.uint8, device=self.device)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=self.device)
        self.step += 1
        rc = lib.tvi_predictor_train_step(
            ctypes.c_void_p(self.packed.data_ptr()), ctypes.c_void_p(self.m.data_ptr()),
            ctypes.c_void_p(self.v.data_ptr()), s.n_in, s.hidden, s.n_out, M,
            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
            None if rows is None else ctypes.c_void_p(rows.data_ptr()), float(lr), self.step,
            ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(workspace.data_ptr()),
            workspace.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != 0:
            raise _lib.TviError(rc, "tvi_predictor_train_step")
        return loss

    def fit(self, x, t, epochs=20, batch=1024, lr=1e-3, lr_end=None, seed=0):
        """Minibatch Adam over host arrays (seeded shuffles); the step size decays
        from lr to lr_end on a cosine (constant when lr_end is None).  Returns the
        mean loss of each epoch."""
        xd = torch.as_tensor(x, device=self.device)
        td = torch.as_tensor(t, device=self.device)
        S = x.shape[0]
        nb = S // batch
        lib = _lib.load()
        s = self.spec
        ws = torch.empty(lib.tvi_predictor_workspace_bytes(s.n_in, s.hidden, s.n_out, batch),
                         dtype=torch.uint8, device=self.device)
        losses = torch.empty(epochs * nb, dtype=torch.float32, device=self.device)
        g = np.random.Generator(np.random.PCG64(seed))
        total = epochs * nb
        for e in range(epochs):
            perm = torch.as_tensor(g.permutation(S).astype(np.int32), device=self.device)
            for k in range(nb):
                q = e * nb + k
                rate = lr if lr_end is None else \
                    lr_end + 0.5 * (lr - lr_end) * (1.0 + np.cos(np.pi * q / total))
                self.train_step(xd, td, rate, perm[k * batch:(k + 1) * batch], ws,
                                losses[q:q + 1])
        return losses.cpu().numpy().reshape(epochs, nb).mean(axis=1).tolist()
