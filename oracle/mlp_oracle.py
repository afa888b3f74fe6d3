"""Plain FP64 CPU oracle of the learned-trace multilayer perceptron.

TEST INFRASTRUCTURE.  Only the test suite may import it.  The perceptron is
not part of the paper; this module restates its definition so that the CUDA
forward/backward kernels can be checked: layers d_0 -> d_1 -> ... -> d_L,
h_{l+1} = tanh(h_l W_l + b_l) for hidden layers, identity output, loss
mean((y - t)^2).  With bf16=True the inputs of every product are rounded to
bfloat16 (round to nearest even) the way the kernels feed the tensor cores;
accumulation stays FP64 here.

Pin: tests/test_mlp_oracle.py checks the analytic gradient against central
finite differences of the loss in FP64.
"""
import numpy as np


def bf16_round(x):
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, dims):
    Ws, bs, o = [], [], 0
    for l in range(len(dims) - 1):
        n = dims[l] * dims[l + 1]
        Ws.append(np.asarray(params[o:o + n], dtype=np.float64).reshape(dims[l], dims[l + 1]))
        o += n
        bs.append(np.asarray(params[o:o + dims[l + 1]], dtype=np.float64))
        o += dims[l + 1]
    return Ws, bs


def forward(params, dims, x, bf16=False):
    Ws, bs = unpack(params, dims)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    hs = [np.asarray(x, dtype=np.float64)]
    L = len(Ws)
    for l in range(L):
        z = r(hs[-1]) @ r(Ws[l]) + bs[l]
        hs.append(np.tanh(z) if l < L - 1 else z)
    return hs


def loss_and_grad(params, dims, x, t, bf16=False):
    Ws, bs = unpack(params, dims)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    hs = forward(params, dims, x, bf16)
    y = hs[-1]
    n = y.size
    loss = float(np.mean((y - t) ** 2))
    dz = 2.0 * (y - t) / n
    grads = []
    L = len(Ws)
    for l in range(L - 1, -1, -1):
        dW = r(hs[l]).T @ r(dz)
        db = dz.sum(axis=0)
        grads.append((dW, db))
        if l > 0:
            dh = r(dz) @ r(Ws[l]).T
            dz = dh * (1.0 - hs[l] ** 2)
    grads.reverse()
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, flat
