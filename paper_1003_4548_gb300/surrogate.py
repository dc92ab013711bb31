"""Training of the elliptic-relaxation surrogate on the method's own runs.

Harvest: elliptic-relaxation canyons of several aspect ratios W/H run with
the FE solve every step. Every few steps, each free node contributes its
features and the FE solution wp_ij / eps (pdf_surrogate_harvest).

Train: the C-ABI kernels standardise the columns and draw mini-batches. Adam
steps the FP32 parameters, with the network's own forward and backward
kernels on the tensor cores (pdf_mlp_loss_grad_bf16; the FP32 kernels of
pdf_mlp_loss_grad on request). The host only orders the calls and holds the
seeded batch permutation.

PyTorch supplies the device buffers and the stream; no step of the network
runs in it.
"""
from __future__ import annotations

import time

import numpy as np

from . import capi
from .workload import canyon_params

IN, OUT, NPARAM, NNORM = capi.MLP_IN, capi.MLP_OUT, capi.MLP_NPARAM, capi.MLP_NNORM
LAYERS = ((64, 10), (64, 64), (64, 64), (5, 64))


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases, in the C-ABI layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in LAYERS:
        a = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-a, a, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == NPARAM
    return p


def harvest(meshes, *, steps: int, every: int, per_element: int, dt_of, C0: float = 2.1, seed: int = 0,
            precision: str = "fp32", torch=None):
    """Run each mesh with the FE solve and collect (features, targets) every
    `every` steps (and after the initial estimate). Returns device tensors
    X[n][10], T[n][5] and the number of samples per mesh."""
    import torch as _torch
    torch = torch or _torch
    stream = torch.cuda.current_stream()
    chunks_x, chunks_t, counts = [], [], []
    for m_i, mesh in enumerate(meshes):
        p = canyon_params(mesh, wall_model="er", precision=precision, C0=C0, seed=seed + m_i)
        g = capi.Canyon(p, mesh, stream=stream.cuda_stream)
        g.seed_particles(per_element)
        g.estimate_stats()
        rows = g.surrogate_rows()
        nh = steps // every + 1
        X = torch.empty((nh * rows, IN), dtype=torch.float32, device="cuda")
        T = torch.empty((nh * rows, OUT), dtype=torch.float32, device="cuda")
        dt = dt_of(mesh)
        for h in range(nh):
            if h:
                g.step(dt, every)
            g.surrogate_harvest(X[h * rows].data_ptr(), T[h * rows].data_ptr())
        g.sync()
        g.close()
        chunks_x.append(X)
        chunks_t.append(T)
        counts.append(nh * rows)
    return torch.cat(chunks_x), torch.cat(chunks_t), counts


def train(X, T, *, epochs: int = 10, batch: int = 4096, lr: float = 2e-3, lr_final: float = 1e-4, seed: int = 0,
          params=None, torch=None, log=None, tensor_cores: bool = True):
    """Standardise, then Adam over seeded mini-batches. The loss gradient of a
    batch comes from the tensor-core kernels (bfloat16 operands, FP32
    accumulation and FP32 parameters; pdf_mlp_loss_grad_bf16), or with
    tensor_cores=False from the FP32 kernels (pdf_mlp_loss_grad). Returns
    (params, norm, history) with params/norm as float32 numpy arrays in the
    C-ABI layout and history a list of (epoch, mean batch loss)."""
    import torch as _torch
    torch = torch or _torch
    s = torch.cuda.current_stream().cuda_stream
    n = X.shape[0]
    Xs, Ts = X.clone(), T.clone()
    stats = torch.empty(NNORM, dtype=torch.float32, device="cuda")
    capi.mlp_column_stats(Xs.data_ptr(), n, IN, stats[0:].data_ptr(), stats[IN:].data_ptr(), s)
    capi.mlp_column_stats(Ts.data_ptr(), n, OUT, stats[2 * IN:].data_ptr(), stats[2 * IN + OUT:].data_ptr(), s)
    capi.mlp_standardize(Xs.data_ptr(), n, IN, stats[0:].data_ptr(), stats[IN:].data_ptr(), s)
    capi.mlp_standardize(Ts.data_ptr(), n, OUT, stats[2 * IN:].data_ptr(), stats[2 * IN + OUT:].data_ptr(), s)
    P = torch.from_numpy(init_params(seed) if params is None else np.asarray(params, np.float32)).cuda()
    G = torch.zeros(NPARAM, dtype=torch.float32, device="cuda")
    M = torch.zeros_like(G)
    V = torch.zeros_like(G)
    b = min(batch, n)
    work = torch.empty(capi.mlp_work_floats(b), dtype=torch.float32, device="cuda")
    xb = torch.empty((b, IN), dtype=torch.float32, device="cuda")
    tb = torch.empty((b, OUT), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grad_fn = capi.mlp_loss_grad_bf16 if tensor_cores else capi.mlp_loss_grad
    rng = np.random.default_rng(seed)
    nb = max(1, n // b)
    total = epochs * nb
    hist, t = [], 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
        acc = torch.zeros(1, dtype=torch.float32, device="cuda")
        for k in range(nb):
            idx = perm[k * b:(k + 1) * b]
            capi.mlp_gather_rows(Xs.data_ptr(), idx.data_ptr(), b, IN, xb.data_ptr(), s)
            capi.mlp_gather_rows(Ts.data_ptr(), idx.data_ptr(), b, OUT, tb.data_ptr(), s)
            grad_fn(P.data_ptr(), xb.data_ptr(), tb.data_ptr(), b, work.data_ptr(), G.data_ptr(), loss.data_ptr(), s)
            t += 1
            rate = lr * (lr_final / lr) ** (t / max(1, total))  # geometric decay
            capi.mlp_adam(P.data_ptr(), G.data_ptr(), M.data_ptr(), V.data_ptr(), t, rate, stream=s)
            acc += loss
        hist.append((ep, float(acc.item()) / nb))
        if log:
            log(f"epoch {ep}: loss {hist[-1][1]:.4e} ({time.perf_counter() - t0:.1f} s)")
    return P.cpu().numpy(), stats.cpu().numpy(), hist


def evaluate(params, norm, X, T, torch=None):
    """Mean-squared error of the bf16 network on raw (unstandardised) samples,
    in the standardised target units, through pdf_mlp_forward."""
    import torch as _torch
    torch = torch or _torch
    s = torch.cuda.current_stream().cuda_stream
    n = X.shape[0]
    q = torch.from_numpy(np.asarray(norm, np.float32)).cuda()
    Xs, Ts = X.clone(), T.clone()
    capi.mlp_standardize(Xs.data_ptr(), n, IN, q[0:].data_ptr(), q[IN:].data_ptr(), s)
    capi.mlp_standardize(Ts.data_ptr(), n, OUT, q[2 * IN:].data_ptr(), q[2 * IN + OUT:].data_ptr(), s)
    P = torch.from_numpy(np.asarray(params, np.float32)).cuda()
    Y = torch.empty((n, OUT), dtype=torch.float32, device="cuda")
    work = torch.empty(capi.mlp_work_floats(n), dtype=torch.float32, device="cuda")
    capi.mlp_forward(P.data_ptr(), Xs.data_ptr(), n, Y.data_ptr(), work.data_ptr(), True, s)
    torch.cuda.synchronize()
    e = (Y - Ts).double()
    return float((e * e).mean().item())


def calibrate(params, norm, mesh, *, steps: int, every: int, per_element: int, dt: float, seed: int = 99,
              precision: str = "fp32", C0: float = 2.1, torch=None):
    """Coarse FE residuals of the network's wp along a held-out run (its own
    seed; the network's wp is used without the check, mode 2). Returns the
    list of residuals (coarse, fine) at every `every` steps; a threshold for
    mode 1 is a stated multiple of their maximum."""
    import torch as _torch
    torch = torch or _torch
    p = canyon_params(mesh, wall_model="er", precision=precision, C0=C0, seed=seed)
    g = capi.Canyon(p, mesh, stream=torch.cuda.current_stream().cuda_stream)
    g.seed_particles(per_element)
    g.estimate_stats()
    g.set_surrogate(2, params, norm, 0.0)
    out = []
    for k in range(steps // every):
        g.step(dt, every)
        out.append(g.surrogate_stats()[2])
    g.close()
    return out
