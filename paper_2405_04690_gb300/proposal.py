"""Learned birth / in-model proposal: training data from the sampler's own cold chain and
the training loop over the library's tensor-core kernels.

The network and its mixture are defined in include/gbk.h (mdn_* and
gbk_sweep_set_proposal). Training pairs are (x, u): x the BF16 features of a band's
opened window (its cold residual with the band's own cold sources added back, whitened),
u the unit-box coordinates of one of those sources. A network trained on such pairs
proposes new sources where the cold chain has put them for similar residuals: the
amortised version of the paper's mixture fits to earlier sampler output (Sec. V.E,
App. G). Every arithmetic step, and the per-minibatch gather of training rows, runs in
libgbk; this module allocates device buffers, assembles the pair buffer and draws the
minibatch order.
"""
import math

import numpy as np
import torch

from . import _lib as L

N_IN, N_HID, N_COMP, N_DIM = 1024, 512, 16, 8
N_OUT = N_COMP * (1 + 2 * N_DIM)
LAYERS = ((N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID))

# Floating-point operations of one sample (multiply-add = 2):
# forward: every layer's matrix product; backward: the weight gradients of every layer
# and the input gradients of layers 2-4 (the features need none).
FLOPS_FORWARD = 2 * sum(o * i for o, i in LAYERS)
FLOPS_TRAIN = FLOPS_FORWARD + 2 * sum(o * i for o, i in LAYERS) + 2 * sum(o * i for o, i in LAYERS[1:])


def init_params(seed, scale=1.0, out_scale=0.1, width_bias=2.0):
    """Training start: He-normal hidden layers, the output layer scaled by out_scale, and
    width-logit biases at width_bias (widths e^(-10 + 10 sigmoid(2)) ~ 0.3: broad
    components, so the first losses are moderate). float32 [mdn_param_count()]."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for li, (o, i) in enumerate(LAYERS):
        sc = scale * (out_scale if li == len(LAYERS) - 1 else 1.0)
        out.append((g.standard_normal((o, i)) * sc * math.sqrt(2.0 / i)).ravel())
        b = np.zeros(o)
        if li == len(LAYERS) - 1:
            b.reshape(N_COMP, 1 + 2 * N_DIM)[:, 1 + N_DIM:] = width_bias
        out.append(b)
    p = np.concatenate(out).astype(np.float32)
    assert p.size == L.mdn_param_count()
    return p


class PairBuffer:
    """Device buffer of training pairs: x [capacity][1024] BF16, u [capacity][8] float32."""

    def __init__(self, capacity, device="cuda"):
        self.x = torch.empty((capacity, N_IN), dtype=torch.bfloat16, device=device)
        self.u = torch.empty((capacity, N_DIM), dtype=torch.float32, device=device)
        self.n = 0
        self.capacity = capacity

    def add_from_sweep(self, plan, params, exists, residual, psd):
        """Append one pair per present cold-chain source (features of its band's window)."""
        d = plan.desc
        x_all = torch.empty((d.n_walkers, d.n_bands, N_IN), dtype=torch.bfloat16, device=params.device)
        u_all = torch.empty((d.n_walkers, d.n_bands, d.n_max, N_DIM), dtype=torch.float32, device=params.device)
        L.gb_sweep_features(plan, params, exists, residual, psd, x_all, u_all)
        present = exists[0].reshape(d.n_walkers, d.n_bands, d.n_max).bool()
        rows = present.nonzero()                          # (w, b, slot)
        k = min(rows.shape[0], self.capacity - self.n)
        if k <= 0:
            return 0
        rows = rows[:k]
        self.x[self.n:self.n + k] = x_all[rows[:, 0], rows[:, 1]]
        self.u[self.n:self.n + k] = u_all[rows[:, 0], rows[:, 1], rows[:, 2]]
        self.n += k
        return k


class Trainer:
    """Adam training of the network on a PairBuffer (one mdn_train_epoch call per epoch)."""

    def __init__(self, net, params, lr=1e-3):
        self.net = net
        self.p = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.step = 0
        self.lr = lr
        self.loss = torch.zeros(1, dtype=torch.float64, device=params.device)
        L.mdn_set_params(net, params)

    @staticmethod
    def order(buf, batch, seed, max_steps=None):
        """The seeded random order of one epoch over the buffer (whole minibatches), on the device."""
        g = np.random.Generator(np.random.PCG64(seed))
        steps = buf.n // batch if max_steps is None else min(buf.n // batch, max_steps)
        return torch.from_numpy(g.permutation(buf.n)[:steps * batch].astype(np.int32)).to(buf.x.device)

    def epoch_ordered(self, buf, order, batch):
        """One epoch in a given order (from order()): the gathers and Adam steps run in one
        library call, stream-ordered, without waiting for the device."""
        L.mdn_train_epoch(self.net, self.p, self.m, self.v, buf.x[:buf.n], buf.u[:buf.n], order, batch, self.step,
                          self.lr, self.loss)
        self.step += order.numel() // batch

    def epoch(self, buf, batch, seed, max_steps=None):
        """One pass over the buffer in a seeded random order; returns the last minibatch loss."""
        self.epoch_ordered(buf, self.order(buf, batch, seed, max_steps), batch)
        return float(self.loss.item())

    def mean_loss(self, buf, batch=4096, limit=None):
        """Mean -ln q over (up to limit) pairs of a buffer, with the current parameters."""
        n = buf.n if limit is None else min(buf.n, limit)
        grad = torch.empty_like(self.p)
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            L.mdn_backward(self.net, buf.x[s:s + batch], buf.u[s:s + batch], grad, self.loss)
            tot += float(self.loss.item()) * batch
            cnt += batch
        return tot / max(cnt, 1)
